"""Pins of the oracle's per-node algebra against brute force (CPU only).

The basis matrices are rebuilt here with NumPy from their definitions
(D2Q9: Eq. 10, 12; D2Q5: Eq. 28, 29); central moments are computed by brute
force from Eq. 14 / 31; the relaxation that the cascaded collision must
realise is the definition of the method (post-collision central moments =
(1 - omega) pre-collision + omega Maxwellian, Sec. 2.2-2.4).  None of this
re-types the oracle's closed forms (Eq. 17, 27, 34, 42).
"""
import itertools

import numpy as np
import pytest

import oracle

EX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
EX5 = np.array([0, 1, 0, -1, 0], float)
EY5 = np.array([0, 0, 1, 0, -1], float)
CS2 = 1.0 / 3.0


def K_matrix():
    one = np.ones(9)
    cols = [one, EX9, EY9, 3 * (EX9**2 + EY9**2) - 4 * one, EX9**2 - EY9**2, EX9 * EY9,
            -3 * EX9**2 * EY9 + 2 * EY9, -3 * EX9 * EY9**2 + 2 * EX9,
            9 * EX9**2 * EY9**2 - 6 * (EX9**2 + EY9**2) + 4 * one]
    return np.stack(cols, axis=1)  # [alpha, beta]


def L_matrix():
    one = np.ones(5)
    cols = [one, EX5, EY5, 5 * (EX5**2 + EY5**2) - 4 * one, EX5**2 - EY5**2]
    return np.stack(cols, axis=1)


def central(f, ex, ey, ux, uy, m, n):
    return float(np.sum(f * (ex - ux) ** m * (ey - uy) ** n))


def raw(f, ex, ey, m, n):
    return float(np.sum(f * ex**m * ey**n))


def test_basis_orthogonal_and_paper_identities():
    K, L = K_matrix(), L_matrix()
    G = K.T @ K
    assert np.allclose(G, np.diag(np.diag(G))) and np.all(np.diag(G) > 0)
    H = L.T @ L
    assert np.allclose(H, np.diag(np.diag(H))) and np.all(np.diag(H) > 0)
    # Eq. 24-25: <K_b|1> = 9 delta_b0, <K_b|e_x> = 6 delta_b1, <K_b|e_y> = 6 delta_b2
    assert np.array_equal(K.T @ np.ones(9), [9, 0, 0, 0, 0, 0, 0, 0, 0])
    assert np.array_equal(K.T @ EX9, [0, 6, 0, 0, 0, 0, 0, 0, 0])
    assert np.array_equal(K.T @ EY9, [0, 0, 6, 0, 0, 0, 0, 0, 0])
    # text after Eq. 40: <L_b|1> = 5 delta_b0
    assert np.array_equal(L.T @ np.ones(5), [5, 0, 0, 0, 0])


def test_back_transform_equals_K_and_L_columns():
    """Eq. 27 / 42 written out equal f + K p-hat / g + L q-hat (exact integers)."""
    K, L = K_matrix(), L_matrix()
    for b in range(9):
        p = np.zeros(9)
        p[b] = 1.0
        assert np.array_equal(oracle.post_d2q9(np.zeros(9), p), K[:, b])
    for b in range(5):
        q = np.zeros(5)
        q[b] = 1.0
        assert np.array_equal(oracle.post_d2q5(np.zeros(5), q), L[:, b])
    rng = np.random.default_rng(3)
    f, p = rng.normal(size=9), rng.normal(size=9)
    assert np.allclose(oracle.post_d2q9(f, p), f + K @ p, rtol=0, atol=1e-14)
    g, q = rng.normal(size=5), rng.normal(size=5)
    assert np.allclose(oracle.post_d2q5(g, q), g + L @ q, rtol=0, atol=1e-14)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.08, -0.05), (0.97, -0.11, 0.07)])
def test_equilibria_have_maxwellian_central_moments(rho, ux, uy):
    feq = oracle.eq_d2q9(rho, ux, uy)
    want = {(0, 0): rho, (1, 0): 0, (0, 1): 0, (2, 0): CS2 * rho, (0, 2): CS2 * rho,
            (1, 1): 0, (2, 1): 0, (1, 2): 0, (2, 2): CS2 * CS2 * rho}
    for (m, n), v in want.items():
        assert central(feq, EX9, EY9, ux, uy, m, n) == pytest.approx(v, abs=1e-15)
    s = 0.7
    geq = oracle.eq_d2q5(s, ux, uy)
    want5 = {(0, 0): s, (1, 0): 0, (0, 1): 0, (2, 0): CS2 * s, (0, 2): CS2 * s}
    for (m, n), v in want5.items():
        assert central(geq, EX5, EY5, ux, uy, m, n) == pytest.approx(v, abs=1e-15)
    # the rest state weights: 4/9, 1/9, 1/36 and 1/3, 1/6
    w9 = oracle.eq_d2q9(1.0, 0.0, 0.0)
    assert np.allclose(w9, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-15)
    assert np.allclose(oracle.eq_d2q5(1.0, 0, 0), [1 / 3] + [1 / 6] * 4, rtol=0, atol=1e-15)


def _random_near_eq(rng, n, eq):
    return eq * (1.0 + 0.2 * rng.uniform(-1, 1, size=n))


@pytest.mark.parametrize("seed", range(6))
def test_d2q9_cascaded_collision_relaxes_central_moments(seed):
    """Post-collision central moments are relaxed towards the Maxwellian with
    omega_3 (trace), omega_4 (normal difference), omega_5 (shear), omega_6,7
    (third order) and omega_8 (fourth order), mass and momentum conserved."""
    rng = np.random.default_rng(seed)
    ux0, uy0 = rng.uniform(-0.1, 0.1, 2)
    f = _random_near_eq(rng, 9, oracle.eq_d2q9(1.0, ux0, uy0))
    rho = f.sum()
    ux, uy = f @ EX9 / rho, f @ EY9 / rho
    om = np.zeros(9)
    om[3:] = rng.uniform(0.3, 1.9, 6)
    ph = oracle.collide_d2q9(f, rho, ux, uy, om)
    assert np.all(ph[:3] == 0)
    fp = oracle.post_d2q9(f, ph)
    c = lambda d, m, n: central(d, EX9, EY9, ux, uy, m, n)
    assert fp.sum() == pytest.approx(rho, abs=1e-14)
    assert c(fp, 1, 0) == pytest.approx(0, abs=1e-14)
    assert c(fp, 0, 1) == pytest.approx(0, abs=1e-14)
    tr, trp = c(f, 2, 0) + c(f, 0, 2), c(fp, 2, 0) + c(fp, 0, 2)
    assert trp == pytest.approx((1 - om[3]) * tr + om[3] * 2 * CS2 * rho, abs=1e-14)
    d, dp = c(f, 2, 0) - c(f, 0, 2), c(fp, 2, 0) - c(fp, 0, 2)
    assert dp == pytest.approx((1 - om[4]) * d, abs=1e-14)
    assert c(fp, 1, 1) == pytest.approx((1 - om[5]) * c(f, 1, 1), abs=1e-14)
    assert c(fp, 2, 1) == pytest.approx((1 - om[6]) * c(f, 2, 1), abs=1e-14)
    assert c(fp, 1, 2) == pytest.approx((1 - om[7]) * c(f, 1, 2), abs=1e-14)
    assert c(fp, 2, 2) == pytest.approx((1 - om[8]) * c(f, 2, 2) + om[8] * CS2**2 * rho,
                                        abs=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_d2q5_cascaded_collision_relaxes_central_moments(seed):
    """Eq. 34 / 49 with the sign reading: first central moments relax with
    omega_1,2 towards 0, the trace with omega_3 towards 2 c^2 s and the
    normal difference with omega_4 towards 0; the scalar is conserved."""
    rng = np.random.default_rng(100 + seed)
    ux, uy = rng.uniform(-0.12, 0.12, 2)
    g = _random_near_eq(rng, 5, oracle.eq_d2q5(0.8, ux, uy))
    s = g.sum()
    om = np.zeros(5)
    om[1:] = rng.uniform(0.3, 1.9, 4)
    qh = oracle.collide_d2q5(g, s, ux, uy, om, 0)
    gp = oracle.post_d2q5(g, qh)
    c = lambda d, m, n: central(d, EX5, EY5, ux, uy, m, n)
    assert gp.sum() == pytest.approx(s, abs=1e-14)
    assert c(gp, 1, 0) == pytest.approx((1 - om[1]) * c(g, 1, 0), abs=1e-14)
    assert c(gp, 0, 1) == pytest.approx((1 - om[2]) * c(g, 0, 1), abs=1e-14)
    tr, trp = c(g, 2, 0) + c(g, 0, 2), c(gp, 2, 0) + c(gp, 0, 2)
    assert trp == pytest.approx((1 - om[3]) * tr + om[3] * 2 * CS2 * s, abs=1e-14)
    d, dp = c(g, 2, 0) - c(g, 0, 2), c(gp, 2, 0) - c(gp, 0, 2)
    assert dp == pytest.approx((1 - om[4]) * d, abs=1e-14)


def test_printed_d2q5_sign_breaks_the_fixed_point():
    """With the sign printed in Eq. 34 / 49 the equilibrium is not a fixed
    point; with the derived sign it is (the reason for the reading)."""
    ux, uy, s = 0.08, -0.05, 0.7
    geq = oracle.eq_d2q5(s, ux, uy)
    om = np.array([0, 1.2, 1.2, 1.0, 1.0])
    q_lit = oracle.collide_d2q5(geq, s, ux, uy, om, 1)
    q_der = oracle.collide_d2q5(geq, s, ux, uy, om, 0)
    assert np.max(np.abs(q_der)) < 1e-16
    # the printed bracket leaves 2 |u|^2 s behind: q3 = omega_3 / 4 * 2 |u|^2 s
    assert q_lit[3] == pytest.approx(om[3] / 4 * 2 * (ux * ux + uy * uy) * s, rel=1e-12)


def test_equilibrium_is_fixed_point_of_d2q9_collision():
    for rho, ux, uy in [(1.0, 0.05, 0.02), (0.95, -0.1, 0.09)]:
        feq = oracle.eq_d2q9(rho, ux, uy)
        om = np.array([0, 0, 0, 1.3, 1.7, 1.7, 1.0, 0.8, 1.1])
        assert np.max(np.abs(oracle.collide_d2q9(feq, rho, ux, uy, om))) < 1e-16


def test_source_moments_change_conserved_moments_by_the_source():
    """Eq. 23 / 25 / 26 and Eq. 40-41: with p0 = M/9, p1 = F_x/6, p2 = F_y/6
    and q0 = S/5 the post-collision zeroth and first moments change by exactly
    M, F and S (whatever the non-conserved moment changes are)."""
    rng = np.random.default_rng(7)
    f = oracle.eq_d2q9(1.0, 0.03, -0.02) * (1 + 0.1 * rng.uniform(-1, 1, 9))
    M, Fx, Fy = 3e-4, -2e-4, 5e-5
    ph = rng.normal(size=9) * 1e-3
    ph[0], ph[1], ph[2] = M / 9, Fx / 6, Fy / 6
    fp = oracle.post_d2q9(f, ph)
    assert fp.sum() - f.sum() == pytest.approx(M, abs=2e-15)
    assert fp @ EX9 - f @ EX9 == pytest.approx(Fx, abs=2e-15)
    assert fp @ EY9 - f @ EY9 == pytest.approx(Fy, abs=2e-15)
    g = oracle.eq_d2q5(0.4, 0.03, -0.02)
    qh = rng.normal(size=5) * 1e-3
    S = -7e-5
    qh[0] = S / 5
    gp = oracle.post_d2q5(g, qh)
    assert gp.sum() - g.sum() == pytest.approx(S, abs=2e-15)


def test_moment_matrix_brute_force_inverse():
    """Raw moments of the nine D2Q9 monomials form an invertible map; the
    oracle's equilibrium is the unique distribution with the Maxwellian's raw
    moments (solved here by inverting that map)."""
    mons = list(itertools.product(range(3), range(3)))
    Mm = np.array([[EX9[a] ** m * EY9[a] ** n for a in range(9)] for m, n in mons])
    assert abs(np.linalg.det(Mm)) > 1e-9
    rho, ux, uy = 1.02, 0.07, -0.04
    mx = [1.0, ux, CS2 + ux * ux]
    my = [1.0, uy, CS2 + uy * uy]
    target = np.array([rho * mx[m] * my[n] for m, n in mons])
    f = np.linalg.solve(Mm, target)
    assert np.allclose(f, oracle.eq_d2q9(rho, ux, uy), rtol=0, atol=1e-15)
