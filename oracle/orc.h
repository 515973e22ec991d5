/*
 * FP64 CPU oracle for the axisymmetric thermal cascaded central-moment lattice
 * Boltzmann method of Hajabdollahi, Premnath & Welch (arXiv 1806.10241).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * It is a literal, slow, unfused transcription of the paper's algorithm:
 *   pass 0: macroscopic fields of the stored (post-collision) state;
 *   pass 1: pull streaming with boundary rules, output moments (Eq. 16b, 18,
 *           33b, 35, 46b, 47);
 *   pass 2: central-difference gradients of the pass-0 fields,
 *           geometric sources (Eq. 4, 5, 7, 9), pre-collision half step
 *           (Eq. 21, 38, 48), cascaded collisions (Eq. 17, 34, 49), source
 *           moments (Eq. 26, 41, 51), back-transforms (Eq. 27, 42, 52).
 * Distributions are stored as absolute FP64 values, array-of-structures
 * per node (f[9], g[5], h[5]), node index = z * nr + r.
 *
 * Readings of the paper where it is silent or garbled:
 *   - Eq. 34 and 49 print "+(ux^2+uy^2)psi" and "+(ux^2-uy^2)psi"; with that
 *     sign the D2Q5 equilibrium is not a fixed point.  The default uses the
 *     sign obtained by relaxing the central moments (minus); sign_literal=1
 *     reproduces the printed sign.  The q3 bracket's "2 c^2" is read as
 *     "2 c^2 psi" like Eq. 49.
 *   - Sources are evaluated at the pre-collision state of Eq. 21/38/48 (the
 *     state the collision uses), solved by two local sweeps; mu = rho nu.
 *   - Gradients: second-order central differences of the macroscopic
 *     fields of the stored (previous time level) distributions, with ghost
 *     values at half-way walls and the axis (same-step fields make the
 *     staggered momentum mode grow in annuli).
 *   - Walls sit half a cell outside the first node: y_j = r0 + j + 1/2,
 *     x_i = i + 1/2.
 *
 * Parity pins: see tests/test_oracle_*.py (closed forms, invariants, brute
 * force moment matrices).  Absolute Nusselt numbers of the coupled cases are
 * pinned only loosely by Table 1 of the paper.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* side index: 0 = bottom (x = 0), 1 = top (x = nz), 2 = inner (y = r0),
 * 3 = outer (y = r0 + nr) */
/* ORC_FLOW_FREE: a free surface on an end wall (Sec. 3.6): zero normal
 * velocity and zero shear, by specular reflection of f in the wall normal.
 * ORC_SC_RAMP: a Dirichlet temperature linear in r on the outer segment of
 * the top (Sec. 3.6): from the inner segment's T_w at the split radius to
 * the outer segment's T_w at r0 + nr. */
enum { ORC_FLOW_WALL = 0, ORC_FLOW_AXIS = 1, ORC_FLOW_PERIODIC = 2, ORC_FLOW_FREE = 3 };
enum { ORC_SC_DIRICHLET = 0, ORC_SC_NEUMANN = 1, ORC_SC_AXIS = 2, ORC_SC_PERIODIC = 3, ORC_SC_RAMP = 4 };

typedef struct {
    int32_t flow;    /* ORC_FLOW_*                                            */
    int32_t swirl;   /* ORC_SC_* for psi = rho u_theta                        */
    int32_t heat;    /* ORC_SC_* for phi = T                                  */
    int32_t pad;
    double u_wx;     /* wall velocity, axial component                        */
    double u_wy;     /* wall velocity, radial component (porous wall if != 0) */
    double omega;    /* wall angular velocity: u_theta = omega * radius       */
    double T_w;      /* wall temperature (Dirichlet)                          */
} orc_side;

typedef struct {
    int32_t nr, nz;
    double r0;          /* radius of the inner wall; 0 with an axis        */
    double nu;          /* kinematic viscosity (also D_psi, Eq. 6)         */
    double alpha;       /* thermal diffusivity D_phi                       */
    double omega3;      /* bulk relaxation rate                            */
    double omega_hi;    /* omega_6..8 and omega_3,4 of the D2Q5 schemes     */
    double g_beta;      /* buoyancy: F_x^b = rho0 g_beta (T - T0)          */
    double T0;          /* reference temperature                           */
    double body_fx;     /* constant axial body force                       */
    double rho0;        /* reference density                               */
    int32_t planar;     /* 1: drop all geometric (1/y) sources             */
    int32_t sign_literal; /* 1: Eq. 34/49 with the printed "+" sign        */
    int32_t explicit_sources; /* 1: sources at the output state only      */
    int32_t pad;
    orc_side side[4];
    /* the top may consist of two segments (Sec. 3.6, a crystal inside a free
     * surface): columns j >= top_split follow top_outer; 0 = one segment */
    int32_t top_split;
    int32_t pad2;
    orc_side top_outer;
} orc_params;

typedef struct {
    double nu_side[4]; /* Nusselt number on each Dirichlet-T side, else 0 */
    double nu_i, nu_o, nu_avg;
    double mass, mass_r, T_sum, u_max;
    int64_t step;
    double k_eq_i, k_eq_o; /* equivalent conductivity of the lateral walls of
                              an annulus (Sec. 3.5), else 0                 */
} orc_diag;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_params *p);
void orc_destroy(orc_state *s);
void orc_set_threads(int n);
int orc_get_threads(void);

/* initialise every node to the equilibria of the given fields
 * fields: [5][nz][nr] = rho, u_x (axial), u_y (radial), u_theta, T */
int orc_init_fields(orc_state *s, const double *fields);
/* canonical state exchange: [19][nz][nr], f0..f8, g0..g4, h0..h4 */
int orc_set_dist(orc_state *s, const double *d);
int orc_get_dist(const orc_state *s, double *d);
int orc_step(orc_state *s, int nsteps);
/* fields of the current state: the pre-collision state the next step's
 * collision uses, [5][nz][nr] rho, u_x, u_y, u_theta, T */
int orc_fields(const orc_state *s, double *fields);
int orc_diag_compute(const orc_state *s, orc_diag *out);
/* stream function on the cell faces y = r0 + j + 1, [nz][nr] (may be NULL),
 * and max |Psi| */
int orc_stream_function(const orc_state *s, double *psi, double *psi_max);
int64_t orc_get_step(const orc_state *s);

/* per-node building blocks (exported for the brute-force pins) */
void orc_eq_d2q9(double rho, double ux, double uy, double feq[9]);
void orc_eq_d2q5(double s, double ux, double uy, double geq[5]);
void orc_collide_d2q9(const double f[9], double rho, double ux, double uy,
                      const double om[9], double ph[9]);
void orc_post_d2q9(const double f[9], const double ph[9], double fp[9]);
void orc_collide_d2q5(const double g[5], double s, double ux, double uy,
                      const double om[5], int sign_literal, double qh[5]);
void orc_post_d2q5(const double g[5], const double qh[5], double gp[5]);

#ifdef __cplusplus
}
#endif
#endif
