/*
 * lb.h -- C ABI of the GB300 axisymmetric thermal cascaded lattice Boltzmann
 * library (liblbaxi.so).
 *
 * The library advances the three distribution functions of the axisymmetric
 * cascaded central-moment LB method of Hajabdollahi, Premnath & Welch
 * (arXiv 1806.10241) on the meridian (r, z) plane: D2Q9 f for density and
 * axial / radial momentum (Sec. 2.2), D2Q5 g for psi = rho u_theta (Sec. 2.3)
 * and D2Q5 h for the temperature (Sec. 2.4).  Every time step is one fused
 * CUDA kernel: pull streaming with the wall / axis / periodic rules
 * (Eq. 16b, 33b, 46b; Sec. 3), the geometric and body-force sources
 * (Eq. 4a-4c, 5, 7, 9), the pre-collision half steps (Eq. 21, 38, 48), the
 * cascaded collisions (Eq. 17, 34, 49), the source moments (Eq. 26, 41, 51)
 * and the back-transforms (Eq. 27, 42, 52).
 *
 * Coordinates follow Eq. 2: x = z (axial, rows, index i in [0, nz)),
 * y = r (radial, columns, index j in [0, nr)).  Walls sit half a cell outside
 * the first and last nodes: node (i, j) is at x = i + 1/2, y = r_inner + j +
 * 1/2.  Lattice units: dx = dt = 1, c_s^2 = 1/3.
 *
 * Memory ownership: the caller allocates one device buffer of
 * lb_required_bytes() bytes (256-byte aligned) and one CUDA stream and hands
 * both to lb_create(); the library never allocates device memory and never
 * frees the caller's buffer.  All kernels and copies run on that stream.
 *
 * Errors: every call returns an lb_status and never aborts, traps or exits;
 * lb_last_error() gives a one-line description of the last failure of a
 * context.  A context is not thread safe; distinct contexts on distinct
 * streams are independent.
 *
 * Arrays exchanged with the host are row-major [plane][nz][nr] doubles.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LB_EXPORT __attribute__((visibility("default")))
#else
#define LB_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,      /* invalid argument or parameter combination      */
    LB_ERR_NOMEM = 2,    /* the caller's buffer is too small                */
    LB_ERR_CUDA = 3,     /* a CUDA runtime call failed                      */
    LB_ERR_DIVERGED = 4, /* non-finite or out-of-range state (diagnostics)  */
    LB_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out              */
    LB_ERR_STATE = 6     /* call out of order (e.g. step before params)     */
} lb_status;

/* Storage type of the distributions.  LB_FP64 computes in FP64; the other
 * three compute in FP32.  LB_BF16 / LB_FP16 store deviations from the rest
 * state (w_a rho0 for f, w_a T0 for h) in 16 bits. */
typedef enum { LB_FP64 = 0, LB_FP32 = 1, LB_BF16 = 2, LB_FP16 = 3 } lb_storage;

/* Lattice shape.  nr, nz >= 2.  r_inner = 0 puts the axis of symmetry on
 * the inner side (a cylinder); r_inner > 0 makes an annulus. */
typedef struct {
    int32_t nr;        /* radial nodes (columns)                           */
    int32_t nz;        /* axial nodes (rows)                               */
    double r_inner;    /* radius of the inner wall (0: axis)               */
    int32_t storage;   /* lb_storage                                       */
    int32_t reserved;  /* must be 0                                        */
} lb_grid_desc;

/* Boundary sides */
enum { LB_SIDE_BOTTOM = 0, LB_SIDE_TOP = 1, LB_SIDE_INNER = 2, LB_SIDE_OUTER = 3 };

/* Flow (f) boundary types.
 * LB_FLOW_WALL: half-way bounce-back (Sec. 3.2) with the moving-wall
 *   momentum term 2 w_a rho0 (e_a . u_w) / c_s^2 for a wall velocity
 *   u_w = (u_wx, u_wy); u_w = 0 is the no-slip wall, a tangential u_w a
 *   sliding wall, a normal u_w a porous wall.
 * LB_FLOW_AXIS: the symmetry line r = 0, mirror rule for the particle
 *   distributions (Sec. 3.3); only on the inner side with r_inner = 0.
 * LB_FLOW_PERIODIC: periodic along z (Sec. 3.1); bottom and top together.
 * LB_FLOW_FREE: a free surface on an end wall (Sec. 3.6: u_z = 0,
 *   d u_r / dz = 0): specular reflection of the particle distributions in
 *   the wall normal, and an even u_r across it for the central differences.
 *   Where the reflected source lies beyond a lateral side (a corner), the
 *   side's own rule applies to the node itself: across the axis the mirror
 *   image, at a wall the bounce-back with that wall's momentum term. */
enum { LB_FLOW_WALL = 0, LB_FLOW_AXIS = 1, LB_FLOW_PERIODIC = 2, LB_FLOW_FREE = 3 };

/* Scalar (g: psi, h: T) boundary types.
 * LB_SC_DIRICHLET: anti-bounce-back to a wall value (Sec. 3.1, 3.2): for g
 *   psi_w = rho0 * omega * radius (a rotating wall: the column's radius on an
 *   end wall, the wall radius on a lateral wall), for h the value T_w.
 * LB_SC_NEUMANN: zero flux (bounce-back), e.g. an adiabatic wall.
 * LB_SC_AXIS: symmetry line (psi odd, T even).  LB_SC_PERIODIC: along z.
 * LB_SC_RAMP: for h on the outer segment of a split top only (Sec. 3.6, the
 *   melt surface beyond the crystal): Dirichlet to a wall temperature
 *   linear in r, from the inner segment's T_w at the split radius
 *   r_inner + top_split to the outer segment's T_w at r_inner + nr, taken at
 *   each column's radius. */
enum { LB_SC_DIRICHLET = 0, LB_SC_NEUMANN = 1, LB_SC_AXIS = 2, LB_SC_PERIODIC = 3, LB_SC_RAMP = 4 };

typedef struct {
    int32_t flow;    /* LB_FLOW_*                                          */
    int32_t swirl;   /* LB_SC_* for g                                      */
    int32_t heat;    /* LB_SC_* for h                                      */
    int32_t pad;
    double u_wx;     /* wall velocity, axial component                     */
    double u_wy;     /* wall velocity, radial component                    */
    double omega;    /* wall angular velocity (g Dirichlet)                */
    double T_w;      /* wall temperature (h Dirichlet)                     */
} lb_side;

/* Physical parameters in lattice units.
 *   omega_4 = omega_5 = 1 / (3 nu + 1/2) (shear, Sec. 2.2); omega_3 the bulk
 *   rate; omega_6..8 = omega_hi; D2Q5: omega_1,2 = 1 / (3 nu + 1/2) for g and
 *   1 / (3 alpha + 1/2) for h, omega_3,4 = omega_hi (Sec. 2.3, 2.4).
 *   Body force F_x^b = rho0 g_beta (T - T0) + body_fx (buoyancy, Sec. 3.2).
 *   planar = 1 switches off every geometric (1/r) source: plain 2-D flow.
 *   explicit_sources = 1 evaluates the sources once at the post-streaming
 *   state (the literal reading; see the readings of the paper).  The default
 *   evaluates them at the pre-collision state by two local sweeps.
 *   sign_literal = 1 uses the sign printed in Eq. 34 / 49.
 *   top_split > 0 splits the top into two segments (Sec. 3.6: the crystal
 *   and the free melt surface around it): columns j < top_split follow
 *   side[LB_SIDE_TOP], columns j >= top_split follow top_outer (flow WALL or
 *   FREE; swirl DIRICHLET or NEUMANN; heat DIRICHLET, NEUMANN or RAMP).
 *   0 <= top_split < nr; 0 = one segment (top_outer unused). */
typedef struct {
    double nu, alpha, omega3, omega_hi, g_beta, T0, body_fx, rho0;
    int32_t planar;
    int32_t sign_literal;
    int32_t explicit_sources;
    int32_t pad;
    lb_side side[4];
    int32_t top_split;
    int32_t pad2;
    lb_side top_outer;
} lb_params;

/* Diagnostics (Sec. 3.2): Nusselt number on each Dirichlet-T side
 * (lateral wall of radius R_w: -R_w / (H dT) sum dT/dr; end wall:
 * -(H / dT) (2 / (R_o^2 - R_i^2)) sum dT/dz r), the mean of the two
 * opposite heated sides, total mass (sum of f), radius-weighted mass, sum
 * of T and max |u| in the meridian plane, and the mean equivalent
 * conductivity of the inner and outer wall of an annulus (Sec. 3.5):
 * k_eq = ln(R_o / R_i) / (H dT) sum over z of (-R_w dT/dr) at the wall,
 * 1 for pure conduction (0 on a side that is not a Dirichlet-T lateral wall
 * of an annulus) -- all accumulated in FP64 from the pre-collision fields of
 * the current state.  Wall derivatives are one-sided and second order
 * through the wall value, (-8 T_w + 9 T_1 - T_2) / 3 along the inward
 * normal; sums over the wall are midpoint sums.  On a split top the sum
 * covers the columns whose segment holds a wall temperature (DIRICHLET or
 * RAMP), each with its own wall value. */
typedef struct {
    double nu_side[4];
    double nu_i, nu_o, nu_avg;
    double mass, mass_r, T_sum, u_max;
    int64_t step;
    int32_t status;  /* LB_OK or LB_ERR_DIVERGED                          */
    int32_t pad;
    double k_eq_i, k_eq_o;
} lb_diag;

/* Bytes of device memory a lattice of this shape needs (2 distribution
 * buffers + reduction scratch + a table of the column radii y and 1/y,
 * Eq. 2 with half-way walls, computed in FP64 and rounded once).  Returns
 * LB_ERR_ARG for an invalid desc. */
LB_EXPORT lb_status lb_required_bytes(const lb_grid_desc *desc, size_t *bytes);

/* Create a context on the caller's device buffer (>= lb_required_bytes,
 * 256-byte aligned) and CUDA stream (cudaStream_t as void*, NULL = legacy
 * default stream).  The lattice is unusable until lb_set_params(). */
LB_EXPORT lb_status lb_create(const lb_grid_desc *desc, void *dev_buf, size_t bytes, void *cuda_stream,
                    lb_ctx **out);

/* Set the parameters and reset the state to rest: rho0, u = 0, u_theta = 0,
 * T = T0, step = 0; writes the radius table.  Synchronises the stream. */
LB_EXPORT lb_status lb_set_params(lb_ctx *ctx, const lb_params *params);

/* Initialise every node to the equilibria of host fields [5][nz][nr]:
 * rho, u_x, u_y, u_theta, T.  step = 0.  Synchronous. */
LB_EXPORT lb_status lb_init_fields(lb_ctx *ctx, const double *host_fields);

/* Advance nsteps >= 0 time steps, asynchronously on the context's stream. */
LB_EXPORT lb_status lb_step(lb_ctx *ctx, int32_t nsteps);

/* Pre-collision fields of the current state (the rho, u, u_theta, T the
 * next collision uses) into host [5][nz][nr] doubles.  Synchronous. */
LB_EXPORT lb_status lb_get_fields(lb_ctx *ctx, double *host_fields);

/* Diagnostics of the current state.  Synchronous; status LB_ERR_DIVERGED
 * when a field is not finite or rho leaves [0.5, 1.5], LB_ERR_TIMEOUT when a
 * bounded wait of a step kernel ran out (the state is then not valid). */
LB_EXPORT lb_status lb_diagnostics(lb_ctx *ctx, lb_diag *out);

/* Self-test of the failure path of the bounded device waits (no counterpart
 * in the paper): a kernel polls, `polls` times (1..2^22), an mbarrier that
 * nothing arrives at -- the same bounded wait the TMA row rings use -- and
 * sets the context's status word to LB_ERR_TIMEOUT, which the next
 * lb_diagnostics reports; lb_set_params clears it.  No fault, trap or hang:
 * the context stays usable.  Synchronises the stream. */
LB_EXPORT lb_status lb_selftest_timeout(lb_ctx *ctx, int32_t polls);

/* Stream function of the meridian flow (Sec. 3.6: dPsi/dy = -y u_x,
 * dPsi/dx = y u_y), Psi = 0 on the inner boundary (axis or inner wall),
 * integrated along y with the midpoint rule from the pre-collision fields:
 * host_psi[nz][nr] (may be NULL) holds Psi on the cell faces y = r0 + j + 1,
 * *psi_max = max |Psi| (FP64).  Synchronises the stream; uses the idle
 * distribution buffer as scratch. */
LB_EXPORT lb_status lb_stream_function(lb_ctx *ctx, double *host_psi, double *psi_max);

/* Distributions as absolute values, host [19][nz][nr] doubles: f0..f8,
 * g0..g4, h0..h4 (velocity order of Eq. 10 and Eq. 28).  Synchronous.
 * The rest-state offset is added (get) and subtracted (set) in FP64, so a
 * get followed by a set can move a stored deviation by up to half an FP64
 * unit of the rest value (about 3e-17): in FP64 storage any deviation, in
 * FP32 storage only those below about 1e-9 (by one FP32 unit).
 * lb_get_state / lb_set_state restore a state bitwise. */
LB_EXPORT lb_status lb_get_distributions(lb_ctx *ctx, double *host19);
LB_EXPORT lb_status lb_set_distributions(lb_ctx *ctx, const double *host19);

/* Checkpoint: raw state bytes (lb_state_bytes) plus the step counter. */
LB_EXPORT lb_status lb_state_bytes(const lb_ctx *ctx, size_t *bytes);
LB_EXPORT lb_status lb_get_state(lb_ctx *ctx, void *host, size_t bytes);
LB_EXPORT lb_status lb_set_state(lb_ctx *ctx, const void *host, size_t bytes);

/* Steps taken since the last reset. */
LB_EXPORT lb_status lb_get_step(const lb_ctx *ctx, int64_t *step);

/* Tune the launch: rows per z-segment of a warp (0 = automatic), warps per
 * block (0 = automatic, at most 8) and how the FP32 / 16-bit step fetches
 * its rows (0 = automatic, 1 = plain loads, 2 = TMA bulk tensor copies into
 * a shared-memory ring, 3 = the same ring holding rows i - 1, i, i + 1 of
 * the step, read in place).  Results do not depend on the launch shape.
 * LB_ERR_ARG for values out of range. */
LB_EXPORT lb_status lb_set_launch(lb_ctx *ctx, int32_t seg_rows, int32_t warps_per_block, int32_t row_fetch);

/* The launch the next lb_step uses, with the automatic choices resolved:
 * rows per z-segment, warps per block and row fetch (1, 2 or 3 as for
 * lb_set_launch; FP64 storage always 1).  NULL outputs are skipped. */
LB_EXPORT lb_status lb_get_launch(const lb_ctx *ctx, int32_t *seg_rows, int32_t *warps_per_block,
                                  int32_t *row_fetch);

/* Diagnostics of a state held in the caller's device memory, with no context
 * and no scratch memory from the caller; the paper has no counterpart.
 *
 * For callers that cannot allocate device memory -- e.g. a runtime that hands
 * out one fixed device arena at start-up and forbids allocation afterwards,
 * or a tool inspecting checkpoints that another component staged in device
 * memory -- and therefore cannot create a context (lb_create needs a buffer
 * of lb_required_bytes, which includes reduction scratch) or lend scratch.
 * dev_state points at one distribution buffer in the library's layout (the
 * bytes of an lb_get_state blob after its 16-byte header, 256-byte aligned);
 * desc and params describe it and pass the checks of lb_create and
 * lb_set_params; step is copied to out->step.  The reductions use the
 * default launch of the lattice: the result is bitwise that of
 * lb_diagnostics on the same state under the default launch, and equal to
 * reduction round-off under another launch (lb_set_launch, autotuning).
 *
 * Scratch: a 1 MiB array (2^17 doubles) in the library's static device
 * memory, which every GPU that loads the library holds until the process
 * exits.  A lattice needs 16 + 12 x (blocks <= 2048) + 4 (nr + nz) doubles;
 * larger lattices (nr + nz above about 26600) are rejected with LB_ERR_ARG.
 * No call allocates or frees memory.  Every call looks up the array's device
 * address in the current context (cudaGetSymbolAddress); the first call on a
 * device may load the library's device code there, so make it before any
 * stream capture.  Every call reuses the same array and clears the part it
 * uses; calls that overlap on the GPU (other streams, other threads) race on
 * it.  Synchronous on cuda_stream. */
LB_EXPORT lb_status lb_diagnostics_static(const lb_grid_desc *desc, const lb_params *params,
                                          const void *dev_state, int64_t step, void *cuda_stream,
                                          lb_diag *out);

/* ---- batches: many lattices advanced together --------------------------------
 * A batch advances a set of FP32 or 16-bit lattices (any shapes, any
 * parameters) with one kernel launch per step over all their 64-column x
 * z-segment tiles (work items numbered by a prefix sum over the lattices),
 * replayed from a CUDA graph of graph_steps launches when the stream is not
 * the legacy default stream.  Each lattice's
 * update is the one lb_step performs (same arithmetic, same rounding bits).
 * While a batch exists its lattices are stepped through it only; their step
 * counters and current buffers follow the batch, so lb_diagnostics and the
 * other per-lattice calls keep working.  The caller owns the device buffer
 * (lb_batch_required_bytes, 256-byte aligned) holding the descriptors. */
typedef struct lb_batch lb_batch;
LB_EXPORT lb_status lb_batch_required_bytes(int32_t n, size_t *bytes);
LB_EXPORT lb_status lb_batch_create(lb_ctx *const *ctxs, int32_t n, void *dev_buf, size_t bytes, void *cuda_stream,
                                    lb_batch **out);
/* rows per z-segment (0 = keep), warps per block (0 = keep), launches per
 * CUDA graph (0 or 1 = no graph), row fetch (0 = keep, 1 = plain loads on a
 * persistent grid, 3 = TMA ring read in place, one warp per work item; the
 * default is 3; 4 = the same with a ring of three row stages instead of
 * four, FP32 storage only: 12 instead of 10 resident warps per SM, for
 * batches whose step is one wave of work items; 5 = one persistent
 * cooperative launch for all the steps of an lb_batch_step call, every work
 * item resident (lb_batch_get_occupancy: items <= resident warps, else
 * lb_batch_step returns LB_ERR_ARG), an item starting a step once the items
 * around it (windows and z-segments +-1) have finished the previous one --
 * no launch boundary between steps; each wait on a neighbour's progress is
 * bounded (about a second) and a timeout sets the lattice's status to
 * LB_ERR_TIMEOUT).  LB_ERR_ARG for values out of range. */
LB_EXPORT lb_status lb_batch_set_launch(lb_batch *b, int32_t seg_rows, int32_t warps_per_block,
                                        int32_t graph_steps, int32_t row_fetch);
/* Rows per z-segment of each lattice (seg_rows[n], in the order of
 * lb_batch_create; 0 = the batch's common value from lb_batch_set_launch;
 * NULL resets every lattice to it), so that the work items of uneven
 * lattices can be sized per lattice -- e.g. about the same number of rows
 * in every item, and items that fill whole waves of the resident warps.
 * Results do not depend on the segments.  LB_ERR_ARG for a value outside
 * 0..nz. */
LB_EXPORT lb_status lb_batch_set_segments(lb_batch *b, const int32_t *seg_rows);
/* Warps of the batched step that can be resident on the device at once
 * under the current launch, and the number of work items (64-column window x
 * z-segment) of one step.  NULL outputs are skipped. */
LB_EXPORT lb_status lb_batch_get_occupancy(const lb_batch *b, int32_t *resident_warps, int32_t *items);
LB_EXPORT lb_status lb_batch_step(lb_batch *b, int32_t nsteps);
/* lb_diagnostics of every lattice of the batch (out[n], in the order of
 * lb_batch_create), bitwise equal to lb_diagnostics of each lattice: three
 * launches on the batch stream for all lattices (each lattice's reduction
 * grid and order as lb_diagnostics uses them), one copy back; synchronises
 * the batch stream. */
LB_EXPORT lb_status lb_batch_diagnostics(lb_batch *b, lb_diag *out);
LB_EXPORT lb_status lb_batch_destroy(lb_batch *b);

/* Release the context (not the caller's buffer or stream). */
LB_EXPORT lb_status lb_destroy(lb_ctx *ctx);

/* One-line description of the last error on ctx (or of the last failed
 * lb_create / lb_required_bytes when ctx is NULL).  Never NULL. */
LB_EXPORT const char *lb_last_error(const lb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LB_H */
