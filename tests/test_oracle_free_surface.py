"""Pins of the Czochralski (Wheeler) boundary family of Sec. 3.6 in the oracle:
a free surface on an end wall (no normal velocity, no shear: specular
reflection of f, zero-flux u_theta), a top split into an inner segment (the
crystal) and an outer one, and a surface temperature linear in r.

* symmetric extension: a lattice of height nz under a free surface equals the
  lower half of a lattice of height 2 nz whose upper half mirrors the lower
  one (walls, state) -- the discrete symmetry the specular rule, the
  zero-flux psi and T rules and the even u_y ghost must reproduce, corners
  with the axis and with moving lateral walls included;
* rigid rotation under a free surface persists (d u_theta / dz = 0, u_z = 0);
* a split top whose segments are equal is the unsplit top, bit for bit;
* the ramp holds the linear conduction profile of a planar box exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1806_10241_gb300 import workloads as W

# reversal of e_x: D2Q9 1<->3, 5<->6, 7<->8; D2Q5 1<->3
MIRX = [0, 3, 2, 1, 4, 6, 5, 8, 7, 9, 12, 11, 10, 13, 14, 17, 16, 15, 18]


def _random_dist(params, seed):
    rng = np.random.default_rng(seed)
    nz, nr = params["nz"], params["nr"]
    f = np.empty((5, nz, nr))
    f[0] = 1.0 + 0.01 * rng.uniform(-1, 1, (nz, nr))
    f[1] = 0.03 * rng.uniform(-1, 1, (nz, nr))
    f[2] = 0.03 * rng.uniform(-1, 1, (nz, nr))
    f[3] = 0.02 * rng.uniform(-1, 1, (nz, nr))
    f[4] = rng.uniform(0, 1, (nz, nr))
    o = oracle.Oracle(params)
    o.init_fields(f)
    d = o.get_dist()
    return d * (1.0 + 0.02 * rng.uniform(-1, 1, d.shape))


def _mirror_pair(nr, nz, r0, inner, outer, bottom):
    """The half lattice (free-surface top) and its doubled mirror image."""
    base = {"nr": nr, "r0": r0, "nu": 0.05, "alpha": 0.07, "g_beta": 0.0, "T0": 0.5, "rho0": 1.0,
            "omega3": 1.0, "omega_hi": 1.0}
    free = W._side(flow=W.FLOW_FREE, swirl=W.SC_NEUMANN, heat=W.SC_NEUMANN)
    half = dict(base, nz=nz, sides=[dict(bottom), free, dict(inner), dict(outer)])
    top = dict(bottom, u_wx=-bottom["u_wx"])  # the mirror image of the bottom wall
    full = dict(base, nz=2 * nz, sides=[dict(bottom), top, dict(inner), dict(outer)])
    return half, full


@pytest.mark.parametrize("geometry", ["cylinder", "annulus"])
def test_free_surface_is_the_mirror_half_of_a_doubled_lattice(geometry):
    nr, nz = 13, 9
    bottom = W._side(heat=W.SC_DIRICHLET, T_w=0.8, omega=0.003, u_wx=0.0, u_wy=0.01)
    if geometry == "cylinder":
        r0, inner = 0.0, W._axis()
    else:
        r0, inner = 4.0, W._side(heat=W.SC_DIRICHLET, T_w=1.0, omega=0.004, u_wy=0.003)
    # lateral walls turn and are porous (both even under the mirror); an axial
    # wall velocity would be odd and break the mirror symmetry of the doubled lattice
    outer = W._side(heat=W.SC_NEUMANN, omega=-0.002, u_wy=-0.002)
    half, full = _mirror_pair(nr, nz, r0, inner, outer, bottom)
    d = _random_dist(half, seed=5)
    dfull = np.concatenate([d, d[MIRX][:, ::-1, :]], axis=1)
    a, b = oracle.Oracle(half), oracle.Oracle(full)
    a.set_dist(d)
    b.set_dist(dfull)
    for _ in range(3):
        a.step(2)
        b.step(2)
        got, want = a.get_dist(), b.get_dist()[:, :nz, :]
        assert np.max(np.abs(got - want)) < 1e-13
        # and the upper half stays the mirror image
        up = b.get_dist()[:, nz:, :]
        assert np.max(np.abs(up - want[MIRX][:, ::-1, :])) < 1e-13
    assert np.max(np.abs(got - d)) > 1e-3  # the state did change


def test_rigid_rotation_persists_under_a_free_surface():
    """Bottom and side wall turning at Omega, a free-surface top: u_theta =
    Omega r and no meridian flow (to the O(Ma^2) of the scheme)."""
    R, u = 12, 1e-3
    c = W.rotating_cylinder(R=R, nz=2 * R, u_wall=u)
    p = dict(c.params)
    p["sides"] = [dict(sd) for sd in p["sides"]]
    p["sides"][1] = W._side(flow=W.FLOW_FREE, swirl=W.SC_NEUMANN, heat=W.SC_NEUMANN)
    o = oracle.Oracle(p)
    o.init_fields(c.fields)
    o.step(30 * R * R)
    fl = o.fields()
    r = W.radii(R, 0.0)
    exact = np.broadcast_to(p["omega_wall"] * r, fl[3].shape)
    assert float(np.linalg.norm(fl[3] - exact) / np.linalg.norm(exact)) < 1e-6
    assert np.max(np.abs(fl[1:3])) < 1e-7


def test_split_top_with_equal_segments_is_the_plain_top():
    c = W.swirling_cylinder(nr=17, nz=11, Re=200.0, Ra=1e4, amp=1e-2, seed=2)
    plain = c.params
    split = dict(plain, top_split=6, top_outer=dict(plain["sides"][1]))
    ramp = dict(split, top_outer=dict(plain["sides"][1], heat=W.SC_RAMP))  # ramp from T_w to the same T_w
    outs = []
    for p in (plain, split, ramp):
        o = oracle.Oracle(p)
        o.init_fields(c.fields)
        o.step(25)
        outs.append(o.get_dist())
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0] - outs[2])) < 1e-15
    # another outer segment changes the result
    other = dict(split, top_outer=dict(plain["sides"][1], omega=0.0))
    o = oracle.Oracle(other)
    o.init_fields(c.fields)
    o.step(25)
    assert np.max(np.abs(o.get_dist() - outs[0])) > 1e-9


def test_ramp_holds_the_linear_conduction_profile():
    """Planar box (no geometric sources) at rest: top split after column 0,
    the inner segment adiabatic, the outer one on the ramp from T_in at the
    split radius to T_out at r0 + nr; lateral walls at the same linear
    profile, adiabatic bottom.  T = T_in + (y - r_s) (T_out - T_in) / (R_o -
    r_s) solves the problem exactly and the scheme keeps it exactly."""
    nr, nz, r0, T_in, T_out = 16, 10, 5.0, 0.2, 0.9
    rs, ro = r0 + 1, r0 + nr
    lin = lambda y: T_in + (y - rs) * (T_out - T_in) / (ro - rs)
    p = {"nr": nr, "nz": nz, "r0": r0, "nu": 0.1, "alpha": 0.08, "g_beta": 0.0, "T0": 0.5, "rho0": 1.0,
         "planar": 1, "omega3": 1.0, "omega_hi": 1.0, "top_split": 1,
         "sides": [W._side(heat=W.SC_NEUMANN, swirl=W.SC_NEUMANN),
                   W._side(heat=W.SC_NEUMANN, swirl=W.SC_NEUMANN, T_w=T_in),
                   W._side(heat=W.SC_DIRICHLET, swirl=W.SC_NEUMANN, T_w=lin(r0)),
                   W._side(heat=W.SC_DIRICHLET, swirl=W.SC_NEUMANN, T_w=lin(ro))],
         "top_outer": W._side(flow=W.FLOW_FREE, heat=W.SC_RAMP, swirl=W.SC_NEUMANN, T_w=T_out)}
    y = W.radii(nr, r0)
    exact = np.broadcast_to(lin(y), (nz, nr))
    fields = W.rest_fields(nz, nr, 0.5)
    o = oracle.Oracle(p)
    o.init_fields(fields)
    o.step(6000)
    T = o.fields()[4]
    assert np.max(np.abs(T - exact)) < 1e-9
    # the ramp read at the node radius: taking it at the face radius y + 1/2
    # would leave an offset of (T_out - T_in) / (2 (R_o - r_s)) = 0.023 on the top row
    assert np.max(np.abs(T[-1] - exact[-1])) < 1e-9


def test_split_column_belongs_to_the_outer_segment():
    """From rest at T0, with the inner top segment at T0 and the outer one at
    T0 + 1, one step changes the stored temperature distributions of exactly
    the top-row nodes of columns j >= top_split (the wall value enters only
    the node next to the wall, and the collision is local)."""
    nr, nz, split, T0 = 12, 6, 5, 0.5
    p = {"nr": nr, "nz": nz, "r0": 3.0, "nu": 0.05, "alpha": 0.07, "g_beta": 0.0, "T0": T0, "rho0": 1.0,
         "omega3": 1.0, "omega_hi": 1.0, "top_split": split,
         "sides": [W._side(), W._side(heat=W.SC_DIRICHLET, T_w=T0), W._side(), W._side()],
         "top_outer": W._side(flow=W.FLOW_FREE, swirl=W.SC_NEUMANN, heat=W.SC_DIRICHLET, T_w=T0 + 1.0)}
    o = oracle.Oracle(p)
    o.init_fields(W.rest_fields(nz, nr, T0))
    before = o.get_dist()
    o.step(1)
    # the stored (post-collision) temperature distributions h of this step
    changed = np.max(np.abs(o.get_dist()[14:] - before[14:]), axis=0) > 1e-12
    want = np.zeros((nz, nr), bool)
    want[nz - 1, split:] = True
    assert np.array_equal(changed, want)
