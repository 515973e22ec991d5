/*
 * FP64 CPU oracle of the axisymmetric thermal cascaded LB method
 * (Hajabdollahi, Premnath & Welch, arXiv 1806.10241).
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/, the smoke check and the CPU
 * baseline of bench.py.  It shares nothing with the CUDA library.
 * See orc.h for the algorithm outline and the readings of the paper.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattices --------------------------------------------------------- */
/* D2Q9 particle velocities, Eq. 10a-10b */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* D2Q5 particle velocities, Eq. 28a-28b */
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};

/* speed of sound squared in lattice units (Sec. 2.2, after Eq. 17) and the
 * free D2Q5 parameters c_{s psi}^2 = c_{s phi}^2 = 1/3 (Sec. 2.3, 2.4) */
static const double CS2 = 1.0 / 3.0;

/* derived by search over the velocity sets, not tabulated */
static int OPP9[9], MIRY9[9], MIRX9[9], OPP5[5];
static double W9[9], W5[5];
static int tables_ready = 0;

static void build_tables(void)
{
    if (tables_ready) return;
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            if (EX9[b] == -EX9[a] && EY9[b] == -EY9[a]) OPP9[a] = b;
            if (EX9[b] == EX9[a] && EY9[b] == -EY9[a]) MIRY9[a] = b;
            if (EX9[b] == -EX9[a] && EY9[b] == EY9[a]) MIRX9[a] = b;
        }
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            if (EX5[b] == -EX5[a] && EY5[b] == -EY5[a]) OPP5[a] = b;
    /* rest-state weights = equilibria at unit density and zero velocity */
    orc_eq_d2q9(1.0, 0.0, 0.0, W9);
    orc_eq_d2q5(1.0, 0.0, 0.0, W5);
    tables_ready = 1;
}

/* ---- per-node building blocks ----------------------------------------- */

/* Discrete D2Q9 equilibrium whose raw moments up to kappa'_xxyy are those of
 * the Maxwellian (central moments rho, 0, 0, c^2 rho, c^2 rho, 0, 0, 0,
 * c^4 rho: the attractors of the cascaded collision, Sec. 2.2).  For the
 * D2Q9 set these raw moments factor into per-axis factors: sum_a P(a,u) a^m
 * = 1, u, c^2 + u^2 for m = 0, 1, 2. */
static double axis_factor(int e, double u)
{
    if (e == 0) return 1.0 - CS2 - u * u;
    return 0.5 * (CS2 + u * u + e * u);
}

void orc_eq_d2q9(double rho, double ux, double uy, double feq[9])
{
    for (int a = 0; a < 9; ++a)
        feq[a] = rho * axis_factor(EX9[a], ux) * axis_factor(EY9[a], uy);
}

/* D2Q5 equilibrium of a scalar s advected by u: raw moments s, s u_x, s u_y,
 * s (c^2 + u_x^2), s (c^2 + u_y^2) (Maxwellian central moments with the
 * density replaced by the scalar, Sec. 2.3). */
void orc_eq_d2q5(double s, double ux, double uy, double geq[5])
{
    geq[0] = s * (1.0 - 2.0 * CS2 - ux * ux - uy * uy);
    geq[1] = 0.5 * s * (CS2 + ux * ux + ux);
    geq[3] = 0.5 * s * (CS2 + ux * ux - ux);
    geq[2] = 0.5 * s * (CS2 + uy * uy + uy);
    geq[4] = 0.5 * s * (CS2 + uy * uy - uy);
}

/* Changes of the non-conserved moments under the cascaded collision, Eq. 17,
 * with the raw moments Eq. 15 of the (streamed) distribution f and the
 * density / velocity (rho, ux, uy) handed in by the caller.  om[3..8] are
 * omega_3..omega_8.  ph[0..2] are set to zero (Eq. 16 conserves them; the
 * source steps set them separately, Eq. 26). */
void orc_collide_d2q9(const double f[9], double rho, double ux, double uy,
                      const double om[9], double ph[9])
{
    double kxx = 0, kyy = 0, kxy = 0, kxxy = 0, kxyy = 0, kxxyy = 0;
    for (int a = 0; a < 9; ++a) {
        const double ex = EX9[a], ey = EY9[a];
        kxx += f[a] * ex * ex;
        kyy += f[a] * ey * ey;
        kxy += f[a] * ex * ey;
        kxxy += f[a] * ex * ex * ey;
        kxyy += f[a] * ex * ey * ey;
        kxxyy += f[a] * ex * ex * ey * ey;
    }
    const double ux2 = ux * ux, uy2 = uy * uy;
    const double p3 = om[3] / 12.0 * (2.0 * CS2 * rho + rho * (ux2 + uy2) - (kxx + kyy));
    const double p4 = om[4] / 4.0 * (rho * (ux2 - uy2) - (kxx - kyy));
    const double p5 = om[5] / 4.0 * (rho * ux * uy - kxy);
    const double p6 = om[6] / 4.0 * (2.0 * rho * ux2 * uy + kxxy - 2.0 * ux * kxy - uy * kxx)
                      - 0.5 * uy * (3.0 * p3 + p4) - 2.0 * ux * p5;
    const double p7 = om[7] / 4.0 * (2.0 * rho * ux * uy2 + kxyy - 2.0 * uy * kxy - ux * kyy)
                      - 0.5 * ux * (3.0 * p3 - p4) - 2.0 * uy * p5;
    const double p8 = om[8] / 4.0 * (CS2 * CS2 * rho + 3.0 * rho * ux2 * uy2
                                     - (kxxyy - 2.0 * ux * kxyy - 2.0 * uy * kxxy
                                        + ux2 * kyy + uy2 * kxx + 4.0 * ux * uy * kxy))
                      - 2.0 * p3 - 0.5 * uy2 * (3.0 * p3 + p4) - 0.5 * ux2 * (3.0 * p3 - p4)
                      - 4.0 * ux * uy * p5 - 2.0 * uy * p6 - 2.0 * ux * p7;
    ph[0] = ph[1] = ph[2] = 0.0;
    ph[3] = p3; ph[4] = p4; ph[5] = p5; ph[6] = p6; ph[7] = p7; ph[8] = p8;
}

/* Post-collision distribution f^p = f + K p-hat, Eq. 16a expanded as Eq. 27 */
void orc_post_d2q9(const double f[9], const double p[9], double fp[9])
{
    fp[0] = f[0] + (p[0] - 4.0 * (p[3] - p[8]));
    fp[1] = f[1] + (p[0] + p[1] - p[3] + p[4] + 2.0 * (p[7] - p[8]));
    fp[2] = f[2] + (p[0] + p[2] - p[3] - p[4] + 2.0 * (p[6] - p[8]));
    fp[3] = f[3] + (p[0] - p[1] - p[3] + p[4] - 2.0 * (p[7] + p[8]));
    fp[4] = f[4] + (p[0] - p[2] - p[3] - p[4] - 2.0 * (p[6] + p[8]));
    fp[5] = f[5] + (p[0] + p[1] + p[2] + 2.0 * p[3] + p[5] - p[6] - p[7] + p[8]);
    fp[6] = f[6] + (p[0] - p[1] + p[2] + 2.0 * p[3] - p[5] - p[6] + p[7] + p[8]);
    fp[7] = f[7] + (p[0] - p[1] - p[2] + 2.0 * p[3] + p[5] + p[6] + p[7] + p[8]);
    fp[8] = f[8] + (p[0] + p[1] - p[2] + 2.0 * p[3] - p[5] + p[6] - p[7] + p[8]);
}

/* Changes of the non-conserved D2Q5 moments, Eq. 34 (psi) and Eq. 49 (phi).
 * s is the scalar after the pre-collision source half step, (ux, uy) the
 * flow velocity.  om[1..4] = omega_1..omega_4.  sign_literal selects the
 * printed "+" on the u^2 s terms; the default (0) uses "-", the sign that
 * makes the D2Q5 equilibrium a fixed point. */
void orc_collide_d2q5(const double g[5], double s, double ux, double uy,
                      const double om[5], int sign_literal, double qh[5])
{
    double kx = 0, ky = 0, kxx = 0, kyy = 0;
    for (int a = 0; a < 5; ++a) {
        const double ex = EX5[a], ey = EY5[a];
        kx += g[a] * ex;
        ky += g[a] * ey;
        kxx += g[a] * ex * ex;
        kyy += g[a] * ey * ey;
    }
    const double sg = sign_literal ? 1.0 : -1.0;
    const double q1 = om[1] / 2.0 * (s * ux - kx);
    const double q2 = om[2] / 2.0 * (s * uy - ky);
    const double q3 = om[3] / 4.0 * (2.0 * CS2 * s - (kxx + kyy) + 2.0 * (ux * kx + uy * ky)
                                     + sg * (ux * ux + uy * uy) * s)
                      + ux * q1 + uy * q2;
    const double q4 = om[4] / 4.0 * (-(kxx - kyy) + 2.0 * (ux * kx - uy * ky)
                                     + sg * (ux * ux - uy * uy) * s)
                      + ux * q1 - uy * q2;
    qh[0] = 0.0; qh[1] = q1; qh[2] = q2; qh[3] = q3; qh[4] = q4;
}

/* Post-collision D2Q5 distribution g^p = g + L q-hat, Eq. 42 (and Eq. 52) */
void orc_post_d2q5(const double g[5], const double q[5], double gp[5])
{
    gp[0] = g[0] + (q[0] - 4.0 * q[3]);
    gp[1] = g[1] + (q[0] + q[1] + q[3] + q[4]);
    gp[2] = g[2] + (q[0] + q[2] + q[3] - q[4]);
    gp[3] = g[3] + (q[0] - q[1] + q[3] + q[4]);
    gp[4] = g[4] + (q[0] - q[2] + q[3] - q[4]);
}

/* ---- state ------------------------------------------------------------ */

/* The state of a lattice between steps is its post-collision
 * distributions.  G holds, during a step, the macroscopic fields of that
 * stored state (pass 0); Gn receives the pre-collision fields (pass 2). */
struct orc_state {
    orc_params p;
    size_t n;                 /* nodes                                   */
    double *f, *g, *h;        /* stored post-collision distributions     */
    double *G;                /* [4][n] u_x, u_y, u_theta, T of the stored state */
    double *Gn;               /* [5][n] pre-collision rho, u_x, u_y, u_theta, T */
    double *fs, *gs, *hs;     /* streamed distributions (pass 1)         */
    double *rho, *ux, *uy, *psi, *phi; /* output moments (pass 1)        */
    int64_t step;
};

#define NODE(s, i, j) ((size_t)(i) * (size_t)(s)->p.nr + (size_t)(j))

static int valid_params(const orc_params *p)
{
    if (p->nr < 2 || p->nz < 2) return 0;
    if (!(p->r0 >= 0.0)) return 0;
    if (!(p->nu > 0.0) || !(p->alpha > 0.0) || !(p->rho0 > 0.0)) return 0;
    /* periodicity only along x, on both x sides and for all three fields */
    int per0 = p->side[0].flow == ORC_FLOW_PERIODIC, per1 = p->side[1].flow == ORC_FLOW_PERIODIC;
    if (per0 != per1) return 0;
    for (int s = 0; s < 2; ++s) {
        int per = p->side[s].flow == ORC_FLOW_PERIODIC;
        if ((p->side[s].swirl == ORC_SC_PERIODIC) != per) return 0;
        if ((p->side[s].heat == ORC_SC_PERIODIC) != per) return 0;
        if (p->side[s].flow == ORC_FLOW_AXIS || p->side[s].swirl == ORC_SC_AXIS ||
            p->side[s].heat == ORC_SC_AXIS) return 0;
        if (p->side[s].swirl == ORC_SC_RAMP || p->side[s].heat == ORC_SC_RAMP) return 0;
    }
    if (p->top_split < 0 || p->top_split >= p->nr) return 0;
    if (p->top_split > 0) {
        const orc_side *t = &p->top_outer;
        if (p->side[1].flow == ORC_FLOW_PERIODIC) return 0;
        if (t->flow != ORC_FLOW_WALL && t->flow != ORC_FLOW_FREE) return 0;
        if (t->swirl != ORC_SC_DIRICHLET && t->swirl != ORC_SC_NEUMANN) return 0;
        if (t->heat != ORC_SC_DIRICHLET && t->heat != ORC_SC_NEUMANN && t->heat != ORC_SC_RAMP) return 0;
    }
    for (int s = 2; s < 4; ++s) {
        if (p->side[s].flow == ORC_FLOW_PERIODIC || p->side[s].swirl == ORC_SC_PERIODIC ||
            p->side[s].heat == ORC_SC_PERIODIC) return 0;
        if (p->side[s].flow == ORC_FLOW_FREE || p->side[s].swirl == ORC_SC_RAMP ||
            p->side[s].heat == ORC_SC_RAMP) return 0;
        int ax = p->side[s].flow == ORC_FLOW_AXIS;
        if ((p->side[s].swirl == ORC_SC_AXIS) != ax || (p->side[s].heat == ORC_SC_AXIS) != ax) return 0;
        if (ax && (s != 2 || p->r0 != 0.0)) return 0;
    }
    if (p->r0 == 0.0 && !p->planar && p->side[2].flow != ORC_FLOW_AXIS) return 0;
    return 1;
}

orc_state *orc_create(const orc_params *p)
{
    build_tables();
    if (!valid_params(p)) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    s->n = (size_t)p->nr * (size_t)p->nz;
    s->f = (double *)calloc(s->n * 9, sizeof(double));
    s->g = (double *)calloc(s->n * 5, sizeof(double));
    s->h = (double *)calloc(s->n * 5, sizeof(double));
    s->G = (double *)calloc(s->n * 4, sizeof(double));
    s->Gn = (double *)calloc(s->n * 5, sizeof(double));
    s->fs = (double *)calloc(s->n * 9, sizeof(double));
    s->gs = (double *)calloc(s->n * 5, sizeof(double));
    s->hs = (double *)calloc(s->n * 5, sizeof(double));
    s->rho = (double *)calloc(s->n, sizeof(double));
    s->ux = (double *)calloc(s->n, sizeof(double));
    s->uy = (double *)calloc(s->n, sizeof(double));
    s->psi = (double *)calloc(s->n, sizeof(double));
    s->phi = (double *)calloc(s->n, sizeof(double));
    if (!s->f || !s->g || !s->h || !s->G || !s->Gn || !s->fs || !s->gs || !s->hs || !s->rho || !s->ux ||
        !s->uy || !s->psi || !s->phi) {
        orc_destroy(s);
        return NULL;
    }
    /* rest state: rho0, u = 0, u_theta = 0, T = T0 */
    for (size_t k = 0; k < s->n; ++k) {
        orc_eq_d2q9(p->rho0, 0.0, 0.0, s->f + 9 * k);
        orc_eq_d2q5(0.0, 0.0, 0.0, s->g + 5 * k);
        orc_eq_d2q5(p->T0, 0.0, 0.0, s->h + 5 * k);
    }
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->f); free(s->g); free(s->h); free(s->G); free(s->Gn);
    free(s->fs); free(s->gs); free(s->hs);
    free(s->rho); free(s->ux); free(s->uy); free(s->psi); free(s->phi);
    free(s);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int64_t orc_get_step(const orc_state *s) { return s->step; }

int orc_init_fields(orc_state *s, const double *fields)
{
    const size_t n = s->n;
    for (size_t k = 0; k < n; ++k) {
        const double rho = fields[k], ux = fields[n + k], uy = fields[2 * n + k];
        const double ut = fields[3 * n + k], T = fields[4 * n + k];
        orc_eq_d2q9(rho, ux, uy, s->f + 9 * k);
        orc_eq_d2q5(rho * ut, ux, uy, s->g + 5 * k);
        orc_eq_d2q5(T, ux, uy, s->h + 5 * k);
    }
    s->step = 0;
    return 0;
}

int orc_set_dist(orc_state *s, const double *d)
{
    const size_t n = s->n;
    for (size_t k = 0; k < n; ++k) {
        for (int a = 0; a < 9; ++a) s->f[9 * k + a] = d[(size_t)a * n + k];
        for (int a = 0; a < 5; ++a) s->g[5 * k + a] = d[(size_t)(9 + a) * n + k];
        for (int a = 0; a < 5; ++a) s->h[5 * k + a] = d[(size_t)(14 + a) * n + k];
    }
    return 0;
}

int orc_get_dist(const orc_state *s, double *d)
{
    const size_t n = s->n;
    for (size_t k = 0; k < n; ++k) {
        for (int a = 0; a < 9; ++a) d[(size_t)a * n + k] = s->f[9 * k + a];
        for (int a = 0; a < 5; ++a) d[(size_t)(9 + a) * n + k] = s->g[5 * k + a];
        for (int a = 0; a < 5; ++a) d[(size_t)(14 + a) * n + k] = s->h[5 * k + a];
    }
    return 0;
}

/* ---- pass 0: macroscopic fields of the stored state ------------------- */

/* u_x, u_y, u_theta = psi / rho and T of the stored post-collision
 * distributions: the fields of the previous time level, whose central
 * differences enter the sources of this step. */
static void pass0(orc_state *s)
{
    const size_t n = s->n;
#pragma omp parallel for schedule(static)
    for (long kk = 0; kk < (long)n; ++kk) {
        const size_t k = (size_t)kk;
        double rho = 0, jx = 0, jy = 0, psi = 0, phi = 0;
        for (int a = 0; a < 9; ++a) {
            rho += s->f[9 * k + a];
            jx += s->f[9 * k + a] * EX9[a];
            jy += s->f[9 * k + a] * EY9[a];
        }
        for (int a = 0; a < 5; ++a) {
            psi += s->g[5 * k + a];
            phi += s->h[5 * k + a];
        }
        s->G[k] = jx / rho;
        s->G[n + k] = jy / rho;
        s->G[2 * n + k] = psi / rho;
        s->G[3 * n + k] = phi;
    }
}

/* ---- pass 1: streaming with boundary rules ---------------------------- */

/* u_theta prescribed by a rotating wall: omega * radius, where the radius is
 * that of the node's column on an end wall (lid, Sec. 3.4) and the cylinder
 * radius on a lateral wall (Sec. 3.1, 3.5).  psi_w = rho0 u_theta. */
/* The specification of an end wall at column j: the top's outer segment
 * when the top is split (Sec. 3.6: the crystal inside a free surface), else
 * the side itself. */
static const orc_side *end_side(const orc_params *p, int side, int j)
{
    if (side == 1 && p->top_split > 0 && j >= p->top_split) return &p->top_outer;
    return &p->side[side];
}

/* Wall temperature of an end wall at column j: T_w, or on the top's outer
 * segment with the ramp of Sec. 3.6 the value linear in r from the inner
 * segment's T_w at the split radius r0 + top_split to the outer segment's
 * T_w at r0 + nr, taken at the column's radius. */
static double end_T(const orc_params *p, int side, int j)
{
    const orc_side *sd = end_side(p, side, j);
    if (sd->heat != ORC_SC_RAMP) return sd->T_w;
    const double rs = p->r0 + p->top_split, ro = p->r0 + p->nr, y = p->r0 + j + 0.5;
    return p->side[1].T_w + (y - rs) / (ro - rs) * (sd->T_w - p->side[1].T_w);
}

static double wall_psi(const orc_params *p, int side, int j)
{
    double radius;
    if (side <= 1) radius = p->r0 + j + 0.5;
    else if (side == 2) radius = p->r0;
    else radius = p->r0 + p->nr;
    const double omega = side <= 1 ? end_side(p, side, j)->omega : p->side[side].omega;
    return p->rho0 * omega * radius;
}

/* f_a(x) = f^p_a(x - e_a), Eq. 16b.  A source outside the fluid is replaced
 * by the half-way bounce-back of the population that left x towards the
 * wall, with the moving-wall momentum term 2 w_a rho0 (e_a . u_w) / c^2
 * (no-slip: u_w = 0; a normal component makes a porous wall), or by the
 * mirror image across the axis (the population
 * with e_y reversed, taken at the mirrored source).  A node whose source
 * crosses both an end wall and the axis uses the end wall. */
/* A population entering node (i, j) through a free-surface end wall (Sec.
 * 3.6: no normal velocity, no shear): the specular image of the population
 * that left node (i, j - e_ay) towards the wall, with e_x reversed.  When
 * that node lies beyond a lateral side (a corner), the image is taken
 * across that side too: across the axis the mirror image of the node itself
 * (both components reversed), at a wall its bounce-back with the wall's
 * momentum term. */
static double free_surface_f(const orc_state *s, int i, int j, int a)
{
    const orc_params *p = &s->p;
    const int sj = j - EY9[a];
    if (sj >= 0 && sj < p->nr) return s->f[9 * NODE(s, i, sj) + MIRX9[a]];
    const int lat = sj < 0 ? 2 : 3;
    const double own = s->f[9 * NODE(s, i, j) + OPP9[a]];
    if (p->side[lat].flow == ORC_FLOW_AXIS) return own;
    const double eu = EX9[a] * p->side[lat].u_wx + EY9[a] * p->side[lat].u_wy;
    return own + 2.0 * W9[a] * p->rho0 * eu / CS2;
}

static double pull_f(const orc_state *s, int i, int j, int a)
{
    const orc_params *p = &s->p;
    int si = i - EX9[a], sj = j - EY9[a];
    if (si < 0 || si >= p->nz) {
        const int side = si < 0 ? 0 : 1;
        if (p->side[side].flow == ORC_FLOW_PERIODIC) {
            si = (si + p->nz) % p->nz;
        } else {
            const orc_side *sd = end_side(p, side, j);
            if (sd->flow == ORC_FLOW_FREE) return free_surface_f(s, i, j, a);
            const double eu = EX9[a] * sd->u_wx + EY9[a] * sd->u_wy;
            return s->f[9 * NODE(s, i, j) + OPP9[a]] + 2.0 * W9[a] * p->rho0 * eu / CS2;
        }
    }
    if (sj < 0 || sj >= p->nr) {
        const int side = sj < 0 ? 2 : 3;
        if (p->side[side].flow == ORC_FLOW_AXIS) return s->f[9 * NODE(s, si, j) + MIRY9[a]];
        const double eu = EX9[a] * p->side[side].u_wx + EY9[a] * p->side[side].u_wy;
        return s->f[9 * NODE(s, i, j) + OPP9[a]] + 2.0 * W9[a] * p->rho0 * eu / CS2;
    }
    return s->f[9 * NODE(s, si, sj) + a];
}

/* Scalar pull for g (field 0, psi) and h (field 1, phi), Eq. 33b / 46b.
 * Dirichlet: anti-bounce-back -x^p_abar + 2 w_a s_w; Neumann: bounce-back;
 * axis: mirror image, odd for psi (u_theta = 0 on the axis), even for T. */
static double pull_s(const orc_state *s, int field, int i, int j, int a)
{
    const orc_params *p = &s->p;
    const double *arr = field == 0 ? s->g : s->h;
    int si = i - EX5[a], sj = j - EY5[a];
    int side = -1;
    if (si < 0 || si >= p->nz) {
        side = si < 0 ? 0 : 1;
        const int bc = field == 0 ? p->side[side].swirl : p->side[side].heat;
        if (bc == ORC_SC_PERIODIC) {
            si = (si + p->nz) % p->nz;
            side = -1;
        }
    } else if (sj < 0 || sj >= p->nr) {
        side = sj < 0 ? 2 : 3;
    }
    if (side < 0) return arr[5 * NODE(s, si, sj) + a];
    const orc_side *sd = side <= 1 ? end_side(p, side, j) : &p->side[side];
    const int bc = field == 0 ? sd->swirl : sd->heat;
    const double own = arr[5 * NODE(s, i, j) + OPP5[a]];
    if (bc == ORC_SC_DIRICHLET || bc == ORC_SC_RAMP) {
        const double val = field == 0 ? wall_psi(p, side, j) : (side <= 1 ? end_T(p, side, j) : sd->T_w);
        return -own + 2.0 * W5[a] * val;
    }
    if (bc == ORC_SC_AXIS) return field == 0 ? -own : own;
    return own; /* Neumann */
}

static void pass1(orc_state *s)
{
    const orc_params *p = &s->p;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < p->nz; ++i) {
        for (int j = 0; j < p->nr; ++j) {
            const size_t k = NODE(s, i, j);
            double *fs = s->fs + 9 * k, *gs = s->gs + 5 * k, *hs = s->hs + 5 * k;
            for (int a = 0; a < 9; ++a) fs[a] = pull_f(s, i, j, a);
            for (int a = 0; a < 5; ++a) gs[a] = pull_s(s, 0, i, j, a);
            for (int a = 0; a < 5; ++a) hs[a] = pull_s(s, 1, i, j, a);
            /* output moments, Eq. 18, 35, 47 */
            double rho = 0, jx = 0, jy = 0, psi = 0, phi = 0;
            for (int a = 0; a < 9; ++a) {
                rho += fs[a];
                jx += fs[a] * EX9[a];
                jy += fs[a] * EY9[a];
            }
            for (int a = 0; a < 5; ++a) {
                psi += gs[a];
                phi += hs[a];
            }
            s->rho[k] = rho;
            s->ux[k] = jx / rho;
            s->uy[k] = jy / rho;
            s->psi[k] = psi;
            s->phi[k] = phi;
        }
    }
}

/* ---- pass 2: gradients, sources, collisions --------------------------- */

/* Neighbour values for the central differences of the gradient fields
 * (the macroscopic fields of the stored, previous-step state).  Across a half-way wall
 * the ghost value is the linear extrapolation through the wall value
 * (2 q_w - q_1); across a zero-flux wall it is q_1; across the axis u_x, T
 * are even and u_y, u_theta are odd; a periodic side wraps. */
typedef struct { double ux, uy, w, phi; } nb_t;

static nb_t node_vals(const orc_state *s, int i, int j)
{
    const size_t k = NODE(s, i, j), n = s->n;
    nb_t v = {s->G[k], s->G[n + k], s->G[2 * n + k], s->G[3 * n + k]};
    return v;
}

static nb_t ghost_y(const orc_state *s, int i, int j, int side)
{
    const orc_params *p = &s->p;
    const orc_side *sd = &p->side[side];
    nb_t in = node_vals(s, i, j), g;
    if (sd->flow == ORC_FLOW_AXIS) {
        g.ux = in.ux;
        g.uy = -in.uy;
    } else {
        g.ux = 2.0 * sd->u_wx - in.ux;
        g.uy = 2.0 * sd->u_wy - in.uy;
    }
    if (sd->swirl == ORC_SC_AXIS) g.w = -in.w;
    else if (sd->swirl == ORC_SC_DIRICHLET) g.w = 2.0 * wall_psi(p, side, j) / p->rho0 - in.w;
    else g.w = in.w;
    if (sd->heat == ORC_SC_DIRICHLET) g.phi = 2.0 * sd->T_w - in.phi;
    else g.phi = in.phi;
    return g;
}

/* u_y at row i+di (di = +-1) for the axial derivative of u_y */
static double uy_x_neighbour(const orc_state *s, int i, int j, int di)
{
    const orc_params *p = &s->p;
    const double *Uy = s->G + s->n;
    int ii = i + di;
    if (ii >= 0 && ii < p->nz) return Uy[NODE(s, ii, j)];
    const int side = ii < 0 ? 0 : 1;
    if (p->side[side].flow == ORC_FLOW_PERIODIC) return Uy[NODE(s, (ii + p->nz) % p->nz, j)];
    const orc_side *sd = end_side(p, side, j);
    if (sd->flow == ORC_FLOW_FREE) return Uy[NODE(s, i, j)]; /* no shear: u_y even across the surface */
    return 2.0 * sd->u_wy - Uy[NODE(s, i, j)];
}

static void pass2(orc_state *s, int write)
{
    const orc_params *p = &s->p;
    double om9[9], om5s[5], om5t[5];
    const double om_nu = 1.0 / (3.0 * p->nu + 0.5);    /* nu = c^2 (1/omega - 1/2) */
    const double om_al = 1.0 / (3.0 * p->alpha + 0.5);
    om9[0] = om9[1] = om9[2] = 0.0;
    om9[3] = p->omega3;
    om9[4] = om9[5] = om_nu;
    om9[6] = om9[7] = om9[8] = p->omega_hi;
    om5s[0] = 0.0; om5s[1] = om5s[2] = om_nu; om5s[3] = om5s[4] = p->omega_hi;
    om5t[0] = 0.0; om5t[1] = om5t[2] = om_al; om5t[3] = om5t[4] = p->omega_hi;

#pragma omp parallel for schedule(static)
    for (int i = 0; i < p->nz; ++i) {
        for (int j = 0; j < p->nr; ++j) {
            const size_t k = NODE(s, i, j);
            const double y = p->r0 + j + 0.5;
            const double rho_o = s->rho[k], ux_o = s->ux[k], uy_o = s->uy[k];
            const double psi_o = s->psi[k], phi_o = s->phi[k];

            /* central differences of the previous time level's fields */
            const nb_t up = j + 1 < p->nr ? node_vals(s, i, j + 1) : ghost_y(s, i, j, 3);
            const nb_t dn = j - 1 >= 0 ? node_vals(s, i, j - 1) : ghost_y(s, i, j, 2);
            const double dyux = 0.5 * (up.ux - dn.ux);
            const double dyuy = 0.5 * (up.uy - dn.uy);
            const double dyw = 0.5 * (up.w - dn.w);
            const double dyphi = 0.5 * (up.phi - dn.phi);
            const double dxuy = 0.5 * (uy_x_neighbour(s, i, j, +1) - uy_x_neighbour(s, i, j, -1));

            /* sources (Eq. 4a-4c, 5, 7, 9) and pre-collision half steps (Eq. 21a-21c,
             * 38, 48; dt = 1).  The sources are taken at the pre-collision state
             * (rho, j, psi, phi) itself -- the state the collision uses -- which
             * makes the two half steps of the symmetric split an implicit
             * midpoint rule.  That local implicit relation is solved by two
             * sweeps: the first evaluates the sources at the output state, the
             * second at the state the first one predicts; the mass source is
             * always taken from the newest momentum, M^A = -j_y / y.  With
             * explicit_sources = 1 a single sweep at the output state is used
             * (the literal reading, which has no steady state under a force). */
            const double out[5] = {rho_o, rho_o * ux_o, rho_o * uy_o, psi_o, phi_o};
            double st[5] = {out[0], out[1], out[2], out[3], out[4]};
            double MA = 0, Fx = 0, Fy = 0, Spsi = 0, Sphi = 0;
            const int sweeps = p->explicit_sources ? 1 : 2;
            for (int sw = 0; sw < sweeps; ++sw) {
                const double r = st[0], ux = st[1] / r, uy = st[2] / r, ps = st[3], ph = st[4];
                double MAs = 0, FAx = 0, FAy = 0;
                Spsi = 0;
                Sphi = 0;
                if (!p->planar) {
                    const double mu = r * p->nu;
                    MAs = -r * uy / y;
                    FAx = -r * ux * uy / y + mu * (dxuy + dyux) / y;
                    FAy = ps * ps / (r * y) - r * uy * uy / y + 2.0 * mu * dyuy / y
                          - 2.0 * mu * uy / (y * y);
                    Spsi = -2.0 * uy * ps / y + mu / y * dyw - p->nu * ps / (y * y);
                    Sphi = -uy * ph / y + p->alpha / y * dyphi;
                }
                /* total force, Eq. 5, with the Boussinesq buoyancy along +x */
                Fx = FAx + p->rho0 * p->g_beta * (ph - p->T0) + p->body_fx;
                Fy = FAy;
                st[1] = out[1] + 0.5 * Fx;
                st[2] = out[2] + 0.5 * Fy;
                st[3] = out[3] + 0.5 * Spsi;
                st[4] = out[4] + 0.5 * Sphi;
                MA = (p->planar || p->explicit_sources) ? MAs : -st[2] / y;
                st[0] = out[0] + 0.5 * MA;
            }
            const double rho = st[0], ux = st[1] / rho, uy = st[2] / rho;
            const double psi = st[3], phi = st[4];
            if (!write) {
                s->Gn[k] = rho;
                s->Gn[s->n + k] = ux;
                s->Gn[2 * s->n + k] = uy;
                s->Gn[3 * s->n + k] = psi / rho;
                s->Gn[4 * s->n + k] = phi;
                continue;
            }

            /* cascaded collisions, Eq. 17, 34, 49; source moments Eq. 26, 41, 51 */
            double ph[9], qh[5], rh[5];
            orc_collide_d2q9(s->fs + 9 * k, rho, ux, uy, om9, ph);
            ph[0] = MA / 9.0;
            ph[1] = Fx / 6.0;
            ph[2] = Fy / 6.0;
            orc_collide_d2q5(s->gs + 5 * k, psi, ux, uy, om5s, p->sign_literal, qh);
            qh[0] = Spsi / 5.0;
            orc_collide_d2q5(s->hs + 5 * k, phi, ux, uy, om5t, p->sign_literal, rh);
            rh[0] = Sphi / 5.0;

            /* back-transforms, Eq. 27, 42, 52 */
            orc_post_d2q9(s->fs + 9 * k, ph, s->f + 9 * k);
            orc_post_d2q5(s->gs + 5 * k, qh, s->g + 5 * k);
            orc_post_d2q5(s->hs + 5 * k, rh, s->h + 5 * k);
        }
    }
}

int orc_step(orc_state *s, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        pass0(s);
        pass1(s);
        pass2(s, 1);
        s->step += 1;
    }
    return 0;
}

/* Macroscopic fields of the current state: the pre-collision state
 * (rho, u, u_theta = psi / rho, T after the source half steps) that the
 * next step's collision would use.  Runs passes 0-2 without writing. */
static void precollision_fields(const orc_state *cs)
{
    orc_state *s = (orc_state *)cs; /* touches scratch arrays only */
    pass0(s);
    pass1(s);
    pass2(s, 0);
}

int orc_fields(const orc_state *s, double *fields)
{
    precollision_fields(s);
    memcpy(fields, s->Gn, 5 * s->n * sizeof(double));
    return 0;
}

/* ---- diagnostics ------------------------------------------------------ */

/* Stream function of the meridian flow (Sec. 3.6): dPsi/dy = -y u_x,
 * dPsi/dx = y u_y, Psi = 0 on the inner boundary (axis or inner wall, at
 * y = r0).  Integrated along y with the midpoint rule over whole cells, so
 * psi[i][j] is Psi on the cell face y = r0 + j + 1 of row i:
 * psi[i][j] = -sum_{j' <= j} y_j' u_x(i, j').  Fields of the pre-collision
 * state; psi may be NULL; *psi_max = max |Psi|. */
int orc_stream_function(const orc_state *s, double *psi, double *psi_max)
{
    const orc_params *p = &s->p;
    precollision_fields(s);
    const double *ux = s->Gn + 1 * s->n;
    double m = 0.0;
    for (int i = 0; i < p->nz; ++i) {
        double acc = 0.0;
        for (int j = 0; j < p->nr; ++j) {
            const double y = p->r0 + j + 0.5;
            acc -= y * ux[(size_t)i * p->nr + j];
            if (psi) psi[(size_t)i * p->nr + j] = acc;
            if (fabs(acc) > m) m = fabs(acc);
        }
    }
    *psi_max = m;
    return 0;
}


/* Nusselt numbers (Sec. 3.2): Nu = -R_w / (H dT) int dT/dy dx on a lateral
 * wall of radius R_w.  On an end wall the heat flux is averaged over the
 * wall area: Nu = -(H / dT) (2 / (R_o^2 - R_i^2)) int dT/dx r dr.  The wall
 * gradient is the one-sided second-order difference through the wall value
 * and the first two nodes (wall half a cell away): (-8 T_w + 9 T_1 - T_2)/3
 * along the inward axis; integrals are midpoint sums. */
int orc_diag_compute(const orc_state *s, orc_diag *out)
{
    const orc_params *p = &s->p;
    precollision_fields(s);
    const double *Tf = s->Gn + 4 * s->n;
    memset(out, 0, sizeof(*out));
    const int nr = p->nr, nz = p->nz;
    const double H = nz, Ri = p->r0, Ro = p->r0 + nr;
    double tmin = 0, tmax = 0;
    int ndir = 0;
    for (int sd = 0; sd < 5; ++sd) {
        const orc_side *q = sd < 4 ? &p->side[sd] : &p->top_outer;
        if (sd == 4 && p->top_split == 0) continue;
        if (q->heat == ORC_SC_DIRICHLET || q->heat == ORC_SC_RAMP) {
            const double t = q->T_w;
            if (ndir == 0 || t < tmin) tmin = t;
            if (ndir == 0 || t > tmax) tmax = t;
            ++ndir;
        }
    }
    const double dT = (ndir >= 2 && tmax > tmin) ? tmax - tmin : 1.0;
#define TT(i, j) Tf[NODE(s, i, j)]
    if (p->side[2].heat == ORC_SC_DIRICHLET) {
        const double Tw = p->side[2].T_w;
        double sum = 0;
        for (int i = 0; i < nz; ++i) sum += (-8.0 * Tw + 9.0 * TT(i, 0) - TT(i, 1)) / 3.0;
        out->nu_side[2] = -Ri / (H * dT) * sum;
    }
    if (p->side[3].heat == ORC_SC_DIRICHLET) {
        const double Tw = p->side[3].T_w;
        double sum = 0;
        for (int i = 0; i < nz; ++i) sum += (8.0 * Tw - 9.0 * TT(i, nr - 1) + TT(i, nr - 2)) / 3.0;
        out->nu_side[3] = -Ro / (H * dT) * sum;
    }
    /* mean equivalent conductivity of a lateral wall of an annulus (Sec. 3.5):
     * k_eq = ln(R_o / R_i) / (H dT) * integral over z of (-r dT/dr) at the
     * wall, the integral a midpoint sum over the rows, dT/dr the same
     * one-sided wall derivative as above */
    if (Ri > 0.0) {
        const double lg = log(Ro / Ri);
        if (p->side[2].heat == ORC_SC_DIRICHLET) {
            const double Tw = p->side[2].T_w;
            double integral = 0;
            for (int i = 0; i < nz; ++i) integral += -Ri * (-8.0 * Tw + 9.0 * TT(i, 0) - TT(i, 1)) / 3.0;
            out->k_eq_i = lg / (H * dT) * integral;
        }
        if (p->side[3].heat == ORC_SC_DIRICHLET) {
            const double Tw = p->side[3].T_w;
            double integral = 0;
            for (int i = 0; i < nz; ++i) integral += -Ro * (8.0 * Tw - 9.0 * TT(i, nr - 1) + TT(i, nr - 2)) / 3.0;
            out->k_eq_o = lg / (H * dT) * integral;
        }
    }
    const double area = 0.5 * (Ro * Ro - Ri * Ri);
    if (p->side[0].heat == ORC_SC_DIRICHLET) {
        const double Tw = p->side[0].T_w;
        double sum = 0;
        for (int j = 0; j < nr; ++j)
            sum += (p->r0 + j + 0.5) * (-8.0 * Tw + 9.0 * TT(0, j) - TT(1, j)) / 3.0;
        out->nu_side[0] = -(H / dT) * sum / area;
    }
    /* top: the columns whose segment holds a wall temperature (Dirichlet or
     * the ramp), each with its own wall value */
    {
        double sum = 0;
        int any = 0;
        for (int j = 0; j < nr; ++j) {
            const int ht = end_side(p, 1, j)->heat;
            if (ht != ORC_SC_DIRICHLET && ht != ORC_SC_RAMP) continue;
            const double Tw = end_T(p, 1, j);
            sum += (p->r0 + j + 0.5) * (8.0 * Tw - 9.0 * TT(nz - 1, j) + TT(nz - 2, j)) / 3.0;
            any = 1;
        }
        if (any) out->nu_side[1] = -(H / dT) * sum / area;
    }
#undef TT
    int a = -1, b = -1;
    if (p->side[2].heat == ORC_SC_DIRICHLET && p->side[3].heat == ORC_SC_DIRICHLET) {
        a = 2; b = 3;
    } else if (p->side[0].heat == ORC_SC_DIRICHLET && p->side[1].heat == ORC_SC_DIRICHLET) {
        a = 0; b = 1;
    } else {
        for (int sd = 0; sd < 4; ++sd)
            if (p->side[sd].heat == ORC_SC_DIRICHLET) {
                if (a < 0) a = sd;
                else if (b < 0) b = sd;
            }
    }
    if (a >= 0) out->nu_i = out->nu_side[a];
    if (b >= 0) out->nu_o = out->nu_side[b];
    out->nu_avg = (a >= 0 && b >= 0) ? 0.5 * (out->nu_i + out->nu_o) : out->nu_i;

    /* mass = sum of all f (conserved by streaming; changed only by M^A),
     * mass_r = its radius-weighted sum, T_sum and max |u| from the fields */
    double mass = 0, mass_r = 0, tsum = 0, umax = 0;
    for (int i = 0; i < nz; ++i)
        for (int j = 0; j < nr; ++j) {
            const size_t k = NODE(s, i, j);
            const double y = p->r0 + j + 0.5;
            double m = 0;
            for (int a = 0; a < 9; ++a) m += s->f[9 * k + a];
            mass += m;
            mass_r += m * y;
            tsum += Tf[k];
            const double ux = s->Gn[s->n + k], uy = s->Gn[2 * s->n + k];
            const double um = sqrt(ux * ux + uy * uy);
            if (um > umax) umax = um;
        }
    out->mass = mass;
    out->mass_r = mass_r;
    out->T_sum = tsum;
    out->u_max = umax;
    out->step = s->step;
    return 0;
}
