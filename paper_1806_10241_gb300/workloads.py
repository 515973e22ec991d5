"""Seeded synthetic workloads: lattice parameters and initial fields.

This module holds the problem statements only -- geometry, boundary types,
the map from the paper's dimensionless groups to lattice units, and seeded
initial fields.  It contains none of the lattice Boltzmann arithmetic; both
the CUDA library and the CPU oracle receive exactly the numbers built here.

Dimensionless groups follow the paper: Ra = g beta dT L^3 / (alpha nu),
Pr = nu / alpha (Sec. 3.2), Re = Omega R^2 / nu for the rotating lid
(Sec. 3.4), Re = u_o R_i / nu for Taylor-Couette (Sec. 3.1).  Lattice units:
dx = dt = 1, walls half a cell outside the first and last nodes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# side indices and boundary codes shared by the C ABI (include/lb.h)
BOTTOM, TOP, INNER, OUTER = 0, 1, 2, 3
FLOW_WALL, FLOW_AXIS, FLOW_PERIODIC, FLOW_FREE = 0, 1, 2, 3
SC_DIRICHLET, SC_NEUMANN, SC_AXIS, SC_PERIODIC, SC_RAMP = 0, 1, 2, 3, 4

CS = 1.0 / math.sqrt(3.0)  # lattice speed of sound


def _side(flow=FLOW_WALL, swirl=SC_DIRICHLET, heat=SC_NEUMANN, u_wx=0.0, u_wy=0.0, omega=0.0,
          T_w=0.0):
    return {"flow": flow, "swirl": swirl, "heat": heat, "u_wx": u_wx, "u_wy": u_wy,
            "omega": omega, "T_w": T_w}


def _axis():
    return _side(FLOW_AXIS, SC_AXIS, SC_AXIS)


def _periodic():
    return _side(FLOW_PERIODIC, SC_PERIODIC, SC_PERIODIC)


# ---- seeded perturbation: SplitMix64 (Steele, Lea & Flood 2014) -----------

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 started at `seed` (counter-based form)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n doubles uniform in [-1, 1): the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


# ---- initial fields --------------------------------------------------------

def rest_fields(nz: int, nr: int, T: np.ndarray | float, rho0: float = 1.0,
                u_theta: np.ndarray | float = 0.0) -> np.ndarray:
    """[5, nz, nr] fields rho, u_x, u_y, u_theta, T for a fluid at rest."""
    f = np.zeros((5, nz, nr), np.float64)
    f[0] = rho0
    f[3] = u_theta
    f[4] = T
    return f


def perturbed_T(nz: int, nr: int, base: np.ndarray | float, amp: float, seed: int) -> np.ndarray:
    """base + amp * U(-1, 1), drawn row-major (z then r) from SplitMix64(seed)."""
    noise = uniform_pm1(seed, nz * nr).reshape(nz, nr)
    return np.broadcast_to(np.asarray(base, np.float64), (nz, nr)) + amp * noise


@dataclass
class Case:
    """One lattice: parameter dict (library / oracle) + initial fields."""
    name: str
    params: dict
    fields: np.ndarray

    @property
    def nr(self) -> int:
        return int(self.params["nr"])

    @property
    def nz(self) -> int:
        return int(self.params["nz"])


def radii(nr: int, r0: float) -> np.ndarray:
    """Node radii y_j = r0 + j + 1/2 (half-way walls)."""
    return r0 + np.arange(nr, dtype=np.float64) + 0.5


# ---- the paper's problems ---------------------------------------------------

def annulus_convection(nr: int = 41, nz: int = 41, ratio: float = 2.0, Ra: float = 1e3,
                       Pr: float = 0.7, mach: float = 0.1, swirl_inner: float = 0.0,
                       amp: float = 1e-6, seed: int = 0, T_hot: float = 1.0,
                       T_cold: float = 0.0) -> Case:
    """Natural convection between coaxial vertical cylinders (Sec. 3.2).

    Gap L = nr = R_o - R_i, R_o / R_i = ratio, height H = nz.  Hot inner wall,
    cold outer wall, adiabatic ends, no-slip everywhere.  The buoyancy velocity
    sqrt(g beta dT L) is set to `mach` * c_s.  An optional inner-wall swirl
    speed u_theta(R_i) = swirl_inner (the mixed-convection variant, Sec. 3.5).
    T starts linear in r plus a seeded uniform perturbation of amplitude amp.
    """
    L = float(nr)
    r0 = L / (ratio - 1.0)
    dT = T_hot - T_cold
    U = mach * CS
    g_beta = U * U / (dT * L)
    nu = U * L * math.sqrt(Pr / Ra)
    alpha = nu / Pr
    omega_i = swirl_inner / r0
    sides = [_side(heat=SC_NEUMANN), _side(heat=SC_NEUMANN),
             _side(heat=SC_DIRICHLET, T_w=T_hot, omega=omega_i),
             _side(heat=SC_DIRICHLET, T_w=T_cold)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": nu, "alpha": alpha, "g_beta": g_beta,
              "T0": 0.5 * (T_hot + T_cold), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0,
              "sides": sides}
    y = radii(nr, r0)
    base = T_hot - (y - r0) / L * dT
    T = perturbed_T(nz, nr, base[None, :], amp, seed)
    return Case("annulus_convection", params, rest_fields(nz, nr, T))


def swirling_cylinder(nr: int = 1024, nz: int = 2048, Re: float = 1000.0, Ra: float = 1e5,
                      Pr: float = 0.7, u_lid: float = 0.05, amp: float = 1e-6,
                      seed: int = 0, T_hot: float = 1.0, T_cold: float = 0.0) -> Case:
    """Closed vertical cylinder with a rotating, cooled lid and heated bottom.

    The lid-driven swirling cylinder of Sec. 3.4 (Re = Omega R^2 / nu, lid
    speed u_lid at r = R) with the Rayleigh-Benard heating of Sec. 3.3 added:
    bottom T_hot, lid T_cold, adiabatic side wall, axis of symmetry at r = 0.
    Ra is based on the height H = nz.  Fluid at rest, T = T0 plus a seeded
    perturbation of amplitude amp.
    """
    R, H = float(nr), float(nz)
    omega = u_lid / R
    nu = u_lid * R / Re
    alpha = nu / Pr
    dT = T_hot - T_cold
    g_beta = Ra * nu * alpha / (dT * H ** 3)
    T0 = 0.5 * (T_hot + T_cold)
    sides = [_side(heat=SC_DIRICHLET, T_w=T_hot),
             _side(heat=SC_DIRICHLET, T_w=T_cold, omega=omega),
             _axis(),
             _side(heat=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": 0.0, "nu": nu, "alpha": alpha, "g_beta": g_beta,
              "T0": T0, "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides}
    T = perturbed_T(nz, nr, T0, amp, seed)
    return Case("swirling_cylinder", params, rest_fields(nz, nr, T))


def rayleigh_benard_cylinder(nr: int = 100, nz: int = 100, Ra: float = 5e3, Pr: float = 0.7,
                             tau: float = 0.85, T_init: float = 0.0, amp: float = 0.0, seed: int = 0,
                             T_hot: float = 1.0, T_cold: float = 0.0) -> Case:
    """Rayleigh-Benard convection in a vertical cylinder (Sec. 3.3, Table 2).

    Radius R = nr, height H = nz (aspect ratio H/R = nz / nr), axis of
    symmetry at r = 0, heated bottom T_hot, cooled top T_cold, adiabatic
    side wall, no-slip walls.  The shear relaxation time tau fixes
    nu = (tau - 1/2) / 3; Ra = g beta dT H^3 / (nu alpha).  The fluid starts
    at rest at T = T_init (T_cold gives the up-flow pattern of Fig. 5).
    """
    H = float(nz)
    nu = (tau - 0.5) / 3.0
    alpha = nu / Pr
    dT = T_hot - T_cold
    g_beta = Ra * nu * alpha / (dT * H ** 3)
    sides = [_side(heat=SC_DIRICHLET, T_w=T_hot), _side(heat=SC_DIRICHLET, T_w=T_cold),
             _axis(), _side(heat=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": 0.0, "nu": nu, "alpha": alpha, "g_beta": g_beta,
              "T0": 0.5 * (T_hot + T_cold), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides}
    T = perturbed_T(nz, nr, T_init, amp, seed)
    return Case("rayleigh_benard_cylinder", params, rest_fields(nz, nr, T))


def czochralski(nr: int = 100, nz: int = 100, beta: float = 0.4, Re_x: float = 100.0, Re_c: float = -25.0,
                Pr: float = 0.05, Gr: float = 0.0, u_ref: float = 0.05, amp: float = 0.0, seed: int = 0,
                T_hot: float = 1.0, T_cold: float = 0.0) -> Case:
    """Melt flow in a rotating crucible under a rotating crystal (Sec. 3.6,
    Wheeler's problem).

    Crucible radius R_c = nr, height H = nz (alpha = H / R_c), crystal
    radius R_x = beta R_c = top_split columns.  Re_c = R_c^2 Omega_c / nu,
    Re_x = R_x^2 Omega_x / nu (opposite signs: counter-rotation); the larger
    of the two wall speeds is u_ref, which fixes nu.  Boundaries as Sec. 3.6
    prints them: axis at r = 0; crucible side wall turning with Omega_c at
    T_hot; adiabatic bottom turning with Omega_c; the crystal (r < R_x at
    the top) turning with Omega_x at T_cold; beyond it a free surface (no
    normal velocity, no shear, d u_theta / dz = 0) whose temperature rises
    linearly in r from T_cold at R_x to T_hot at R_c.  Buoyancy from the
    Grashof number Gr = g beta dT R_c^3 / nu^2 (0: forced convection only).
    """
    R, H = float(nr), float(nz)
    split = int(round(beta * nr))
    if not 0 < split < nr:
        raise ValueError("the crystal must cover part of the top (0 < beta nr < nr)")
    Rx = float(split)
    # wall speeds Omega R: crucible Re_c nu / R, crystal Re_x nu / R_x
    nu = u_ref / max(abs(Re_c) / R, abs(Re_x) / Rx)
    om_c, om_x = Re_c * nu / (R * R), Re_x * nu / (Rx * Rx)
    alpha = nu / Pr
    dT = T_hot - T_cold
    g_beta = Gr * nu * nu / (dT * R ** 3)
    sides = [_side(heat=SC_NEUMANN, omega=om_c), _side(heat=SC_DIRICHLET, T_w=T_cold, omega=om_x), _axis(),
             _side(heat=SC_DIRICHLET, T_w=T_hot, omega=om_c)]
    outer = _side(flow=FLOW_FREE, swirl=SC_NEUMANN, heat=SC_RAMP, T_w=T_hot)
    params = {"nr": nr, "nz": nz, "r0": 0.0, "nu": nu, "alpha": alpha, "g_beta": g_beta,
              "T0": 0.5 * (T_hot + T_cold), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides,
              "top_split": split, "top_outer": outer}
    T = perturbed_T(nz, nr, 0.5 * (T_hot + T_cold), amp, seed)
    return Case("czochralski", params, rest_fields(nz, nr, T))


def buoyancy_velocity(params: dict) -> float:
    """sqrt(g beta H dT) of a heated cylinder or annulus (dT from the
    Dirichlet walls), the velocity scale of Table 2."""
    tw = [s["T_w"] for s in params["sides"] if s["heat"] == SC_DIRICHLET]
    return math.sqrt(params["g_beta"] * params["nz"] * (max(tw) - min(tw)))


def mixed_convection_annulus(D: int = 40, eta: float = 10.0, ratio: float = 2.0, Re: float = 100.0,
                             sigma: float = 0.0, Pr: float = 0.7, u_inner: float = 0.05,
                             amp: float = 1e-4, seed: int = 0, T_hot: float = 1.0,
                             T_cold: float = 0.0) -> Case:
    """Mixed convection in a slender annulus with a rotating inner cylinder
    (Sec. 3.5, Table 3).

    Gap D = R_o - R_i = nr, height H = eta D = nz, R_o / R_i = ratio, inner
    wall speed u_inner = Omega_i R_i, Re = Omega_i R_i D / nu,
    Gr = g beta dT D^3 / nu^2 = sigma Re^2.  Hot inner wall, cold outer wall,
    adiabatic ends, fixed outer cylinder and ends.  T starts at the
    conduction profile plus a seeded perturbation that seeds the Taylor cells.
    """
    nr, nz = int(D), int(round(eta * D))
    L = float(nr)
    r0 = L / (ratio - 1.0)
    nu = u_inner * L / Re
    alpha = nu / Pr
    dT = T_hot - T_cold
    g_beta = sigma * Re * Re * nu * nu / (dT * L ** 3)
    sides = [_side(heat=SC_NEUMANN), _side(heat=SC_NEUMANN),
             _side(heat=SC_DIRICHLET, T_w=T_hot, omega=u_inner / r0),
             _side(heat=SC_DIRICHLET, T_w=T_cold)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": nu, "alpha": alpha, "g_beta": g_beta,
              "T0": 0.5 * (T_hot + T_cold), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides}
    y = radii(nr, r0)
    R_o = r0 + L
    base = T_cold + dT * np.log(y / R_o) / math.log(r0 / R_o)
    T = perturbed_T(nz, nr, base[None, :], amp, seed)
    return Case("mixed_convection_annulus", params, rest_fields(nz, nr, T))


def taylor_couette(R_o: int = 50, beta: float = 0.5, kappa: float = 0.1, tau: float = 0.6,
                   Re: float = 5.0, nz: int = 3) -> Case:
    """Circular Couette flow between rotating cylinders (Sec. 3.1).

    Walls at r = R_i = beta R_o and r = R_o, periodic axial direction of nz
    nodes, Omega_o = kappa Omega_i, nu = (tau - 1/2)/3, and u_o = Omega_i R_i
    chosen so that Re = u_o R_i / nu.
    """
    R_i = beta * R_o
    nr = int(round(R_o - R_i))
    nu = (tau - 0.5) / 3.0
    u_o = Re * nu / R_i
    omega_i = u_o / R_i
    omega_o = kappa * omega_i
    sides = [_periodic(), _periodic(),
             _side(omega=omega_i, heat=SC_NEUMANN), _side(omega=omega_o, heat=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": float(R_i), "nu": nu, "alpha": nu, "g_beta": 0.0,
              "T0": 0.0, "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides,
              "omega_i": omega_i, "omega_o": omega_o}
    return Case("taylor_couette", params, rest_fields(nz, nr, 0.0))


def hagen_poiseuille(R: int = 16, G: float = 1e-6, tau: float = 0.8, nz: int = 3) -> Case:
    """Pipe flow driven by a constant axial body force G, axis at r = 0."""
    nu = (tau - 0.5) / 3.0
    sides = [_periodic(), _periodic(), _axis(), _side(heat=SC_NEUMANN)]
    params = {"nr": R, "nz": nz, "r0": 0.0, "nu": nu, "alpha": nu, "g_beta": 0.0, "T0": 0.0,
              "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "body_fx": G, "sides": sides}
    return Case("hagen_poiseuille", params, rest_fields(nz, R, 0.0))


def porous_annulus(nr: int = 16, ratio: float = 2.0, Q: float = 0.02, nu: float = 0.1,
                   alpha: float = 0.1, u_theta_in: float = 1e-3, T_in: float = 1.0,
                   T_out: float = 0.0, G: float = 0.0, nz: int = 3) -> Case:
    """Radial throughflow between porous, rotating, isothermal cylinders.

    R_i = nr / (ratio - 1), R_o = R_i + nr, periodic axial direction.  The
    walls inject / remove fluid with radial velocity Q / R so that u_r = Q / r;
    the inner wall turns with u_theta(R_i) = u_theta_in; optional axial body
    force G.  Steady closed forms (incompressible limit) follow from Eq. 1:
    u_theta = A r^(1 + Q/nu) + B / r, T = C r^(Q/alpha) + D and
    u_z = -G r^2 / (2 (2 nu - Q)) + E r^(Q/nu) + F.
    """
    r0 = nr / (ratio - 1.0)
    R_o = r0 + nr
    sides = [_periodic(), _periodic(),
             _side(heat=SC_DIRICHLET, T_w=T_in, u_wy=Q / r0, omega=u_theta_in / r0),
             _side(heat=SC_DIRICHLET, T_w=T_out, u_wy=Q / R_o)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": nu, "alpha": alpha, "g_beta": 0.0,
              "T0": 0.5 * (T_in + T_out), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0,
              "body_fx": G, "sides": sides}
    return Case("porous_annulus", params, rest_fields(nz, nr, 0.5 * (T_in + T_out)))


def rotating_cylinder(R: int = 16, nz: int = 32, u_wall: float = 1e-3, tau: float = 0.8) -> Case:
    """Closed cylinder turning as a rigid body: the bottom, the lid and the
    side wall rotate at Omega = u_wall / R, axis of symmetry at r = 0, no
    heating.  Steady solution of Eq. 1: u_theta = Omega r, no meridian flow,
    and a radial pressure gradient c^2 d rho / d r = rho Omega^2 r balancing
    the centrifugal term psi^2 / (rho r) of Eq. 4c."""
    nu = (tau - 0.5) / 3.0
    om = u_wall / R
    sides = [_side(heat=SC_NEUMANN, omega=om), _side(heat=SC_NEUMANN, omega=om), _axis(),
             _side(heat=SC_NEUMANN, omega=om)]
    params = {"nr": R, "nz": nz, "r0": 0.0, "nu": nu, "alpha": nu, "g_beta": 0.0, "T0": 0.0,
              "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides, "omega_wall": om}
    return Case("rotating_cylinder", params, rest_fields(nz, R, 0.0))


def axial_couette(nr: int = 16, ratio: float = 2.0, U: float = 1e-3, tau: float = 0.8, nz: int = 3) -> Case:
    """Annulus whose inner cylinder slides along the axis at speed U, outer
    cylinder at rest, periodic along z.  Steady solution of Eq. 1b:
    u_z = U ln(r / R_o) / ln(R_i / R_o), no radial or azimuthal flow."""
    r0 = nr / (ratio - 1.0)
    nu = (tau - 0.5) / 3.0
    sides = [_periodic(), _periodic(), _side(heat=SC_NEUMANN, u_wx=U), _side(heat=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": nu, "alpha": nu, "g_beta": 0.0, "T0": 0.0,
              "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides, "U": U}
    return Case("axial_couette", params, rest_fields(nz, nr, 0.0))


def couette_zero_flux_outer(nr: int = 16, ratio: float = 2.0, u_inner: float = 1e-3, tau: float = 0.8,
                            nz: int = 3) -> Case:
    """Annulus with a rotating inner cylinder (u_theta(R_i) = u_inner) and a
    zero-flux condition on psi at the outer wall, periodic along z.  Steady
    solution: u_theta = A r + B / r with d u_theta / d r = A - B / R_o^2 = 0
    at R_o, i.e. A = u_inner R_i / (R_i^2 + R_o^2), B = A R_o^2."""
    r0 = nr / (ratio - 1.0)
    nu = (tau - 0.5) / 3.0
    sides = [_periodic(), _periodic(), _side(heat=SC_NEUMANN, omega=u_inner / r0),
             _side(heat=SC_NEUMANN, swirl=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": nu, "alpha": nu, "g_beta": 0.0, "T0": 0.0,
              "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides, "u_inner": u_inner}
    return Case("couette_zero_flux_outer", params, rest_fields(nz, nr, 0.0))


def annular_conduction(nr: int = 16, ratio: float = 2.0, alpha: float = 0.1, nz: int = 3,
                       T_in: float = 1.0, T_out: float = 0.0) -> Case:
    """Steady conduction between coaxial cylinders (no flow, periodic in z)."""
    r0 = nr / (ratio - 1.0)
    sides = [_periodic(), _periodic(), _side(heat=SC_DIRICHLET, T_w=T_in),
             _side(heat=SC_DIRICHLET, T_w=T_out)]
    params = {"nr": nr, "nz": nz, "r0": r0, "nu": 0.1, "alpha": alpha, "g_beta": 0.0,
              "T0": 0.5 * (T_in + T_out), "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0,
              "sides": sides}
    return Case("annular_conduction", params, rest_fields(nz, nr, 0.5 * (T_in + T_out)))


def cylinder_conduction(nr: int = 8, nz: int = 16, alpha: float = 0.1) -> Case:
    """Conduction in a closed cylinder: hot bottom, cold top, adiabatic side."""
    sides = [_side(heat=SC_DIRICHLET, T_w=1.0), _side(heat=SC_DIRICHLET, T_w=0.0), _axis(),
             _side(heat=SC_NEUMANN)]
    params = {"nr": nr, "nz": nz, "r0": 0.0, "nu": 0.1, "alpha": alpha, "g_beta": 0.0,
              "T0": 0.5, "rho0": 1.0, "omega3": 1.0, "omega_hi": 1.0, "sides": sides}
    return Case("cylinder_conduction", params, rest_fields(nz, nr, 0.5))


# ---- the benchmark configurations -------------------------------------------

def config_annulus_41() -> Case:
    """Annulus convection, R_o/R_i = 2, H = L, 41 x 41, Ra = 1e3, Pr = 0.7, FP64."""
    return annulus_convection(nr=41, nz=41, ratio=2.0, Ra=1e3, Pr=0.7, amp=1e-6, seed=0)


def config_cylinder(nr: int = 1024, nz: int = 2048, seed: int = 0) -> Case:
    """Swirling heated cylinder, H/R = 2, lid 0.05, Re = 1000, Ra = 1e5, Pr = 0.7."""
    return swirling_cylinder(nr=nr, nz=nz, Re=1000.0, Ra=1e5, Pr=0.7, u_lid=0.05, amp=1e-6,
                             seed=seed)


def batched_instances(count: int = 256, lo: int = 32, hi: int = 512) -> list[Case]:
    """Uneven annulus-convection instances, one per seed 0..count-1.

    Per instance: nr, nz uniform on {lo..hi}, R_o/R_i uniform on [1.5, 3],
    Ra log-uniform on [1e3, 1e5], Pr = 0.7, inner-wall swirl speed uniform on
    [0, 0.05].
    """
    out = []
    for seed in range(count):
        rng = np.random.default_rng(seed)
        nr = int(rng.integers(lo, hi + 1))
        nz = int(rng.integers(lo, hi + 1))
        ratio = float(rng.uniform(1.5, 3.0))
        Ra = float(10.0 ** rng.uniform(3.0, 5.0))
        swirl = float(rng.uniform(0.0, 0.05))
        c = annulus_convection(nr=nr, nz=nz, ratio=ratio, Ra=Ra, Pr=0.7, swirl_inner=swirl,
                               amp=1e-6, seed=seed)
        c.name = f"annulus_{seed}"
        out.append(c)
    return out


@dataclass
class Request:
    rid: int
    arrival: float   # seconds after the start of the stream
    case: Case


def serving_requests(count: int = 2000, rate: float = 50.0, seed: int = 0,
                     nr_lo: int = 64, nr_hi: int = 1024) -> list[Request]:
    """Poisson stream of solve requests: 60 % annulus convection, 40 % cylinder.

    nr uniform on {nr_lo..nr_hi}, nz = nr * U{1, 2}, Ra log-uniform on
    [1e3, 1e5].  Arrival gaps are exponential with mean 1 / rate.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate))
        nr = int(rng.integers(nr_lo, nr_hi + 1))
        nz = nr * int(rng.integers(1, 3))
        Ra = float(10.0 ** rng.uniform(3.0, 5.0))
        if rng.uniform() < 0.6:
            case = annulus_convection(nr=nr, nz=nz, ratio=2.0, Ra=Ra, Pr=0.7, amp=1e-6,
                                      seed=seed * 100003 + rid)
        else:
            case = swirling_cylinder(nr=nr, nz=nz, Re=1000.0, Ra=Ra, Pr=0.7, u_lid=0.05,
                                     amp=1e-6, seed=seed * 100003 + rid)
        case.name = f"req{rid}_{case.name}"
        out.append(Request(rid, t, case))
    return out
