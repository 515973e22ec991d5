// Internal interface between the C ABI (lb_capi.cu) and the kernels
// (lb_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/lb.h"

namespace lbk {

enum Mode { MODE_STEP = 0, MODE_FIELDS = 1, MODE_DIAG = 2, MODE_DIAG_STRIP = 3 };
enum Storage { ST_FP64 = 0, ST_FP32 = 1, ST_BF16 = 2, ST_FP16 = 3 };

constexpr int NQ = 19;        // 9 (f) + 5 (g) + 5 (h) planes
// FP16 storage holds the deviations times 2^10 (away from the subnormal
// range); kFp16InvScaleBits is 2^-10 as an FP16 bit pattern
constexpr double kFp16Scale = 1024.0;
constexpr unsigned short kFp16InvScaleBits = 0x1400;
constexpr int NSUM = 12;      // diagnostic partial sums per block
constexpr int MAX_DIAG_BLOCKS = 4096;

// Everything a kernel needs about one lattice, in double precision; the
// launchers convert to the compute type.
struct HostParams {
    int nr, nz, pitch;
    long long plane;          // elements per plane = nz * pitch
    int storage;
    double r0;
    double nu, alpha, omega3, omega_hi, g_beta, T0, body_fx, rho0;
    int planar, sign_literal, explicit_sources;
    // sides 0..3 as lb_side; entry 4 the outer segment of a split top
    int flow[5], swirl[5], heat[5];
    double uwx[5], uwy[5], omega[5], Tw[5];
    int top_split;            // columns >= top_split of the top follow entry 4 (0: one segment)
    double scale;             // storage scale of the deviations (16-bit)
    const float *ytab;        // device table: y[pitch] then 1/y[pitch] (FP64, rounded once)
};

struct Launch {
    int seg_rows;             // rows per z-segment
    int warps_per_block;
    int use_tma;              // FP32 / 16-bit rows: 0 plain loads, 1 TMA ring, 2 TMA ring read in place
};

// Elements per row of a plane: nr rounded up to 32 (4- and 8-byte storage)
// or 64 (2-byte storage) elements.
int pitch_for(int nr, int storage);
// The lattice part of h (shape, pitch, storage, storage scale) from a grid
// descriptor, after the checks lb_required_bytes and lb_create make.  On
// failure h is untouched and err (n bytes) holds a one-line message.
lb_status host_from_desc(const lb_grid_desc *d, HostParams *h, char *err, size_t n);
// The physical part of h from lb_params, after the checks lb_set_params
// makes (relaxation rates, boundary codes and their pairing, the axis only on
// the inner side of a cylinder, finite wall values); needs the lattice part
// (r0).  On failure h is untouched and err holds a one-line message.
lb_status host_set_params(const lb_params *p, HostParams *h, char *err, size_t n);

// lb_diag from the NSUM sums of the diagnostics (result[] of launch_diag),
// the device status word (LB_OK, else reported as the status) and the step.
void diag_from_sums(const HostParams &h, const double *res, int kstatus, int64_t step, lb_diag *out);

// One time step src -> dst; `step` seeds the stochastic rounding of 16-bit
// storage.
cudaError_t launch_step(const HostParams &p, const Launch &l, const void *src, void *dst,
                        unsigned long long step, const void *tmap, int *status, cudaStream_t s);
// Tensor map (CUtensorMap, 128 bytes) of a distribution buffer for the TMA
// row fetches of the FP32 / 16-bit step.
cudaError_t make_tensor_map(const HostParams &p, void *buf, void *map_out);
// Pre-collision fields of rows [row0, row1) into out[5][row1-row0][nr] (double).
cudaError_t launch_fields(const HostParams &p, const Launch &l, const void *src, double *out,
                          int row0, int row1, cudaStream_t s);
// Bounded-wait self-test: a warp polls an mbarrier nothing arrives at,
// `polls` times, and sets *status to LB_ERR_TIMEOUT.
cudaError_t launch_wait_selftest(int *status, int polls, cudaStream_t s);
// Stream function of nrows rows from their axial velocity ux[nrows][nr]
// (pre-collision fields): psi[nrows][nr] on the cell faces y = r0 + j + 1
// (psi may be null) and rowmax[nrows] = max |Psi| per row.
cudaError_t launch_psi(const double *ux, double *psi, double *rowmax, int nrows, int nr, double r0, cudaStream_t s);
// Diagnostics of the stored state src: block partial sums (partial), the
// pre-collision T field (tfield, nz * nr doubles of scratch) and the final
// values in result[NSUM]: 0 sum(rho - rho0), 1 sum((rho - rho0) y), 2 sum T,
// 3 max |u|, 4..7 Nusselt number per side, 8 divergence flag, 9 / 10 the
// equivalent conductivity k_eq of the inner / outer wall of an annulus.
cudaError_t launch_diag(const HostParams &p, const Launch &l, const void *src, double *partial,
                        double *tfield, double *result, cudaStream_t s);
// Equilibria of host-format fields [5][rows][nr] (double) into rows [row0,row1) of dst.
cudaError_t launch_init_fields(const HostParams &p, const double *fields, void *dst, int row0,
                               int row1, cudaStream_t s);
// Absolute distributions [19][rows][nr] (double) <-> storage, rows [row0,row1).
cudaError_t launch_export(const HostParams &p, const void *src, double *out, int row0, int row1,
                          cudaStream_t s);
cudaError_t launch_import(const HostParams &p, const double *in, void *dst, int row0, int row1,
                          cudaStream_t s);

size_t storage_bytes(int storage);

// Batched step (FP32 / 16-bit storage): device descriptors built on the host
size_t batch_desc_bytes();
size_t batch_ctl_bytes();
int batch_items(const HostParams &h, int seg_rows);
// One lattice's descriptor: parameters, both buffers and their TMA tensor
// maps, the step count and current buffer when the batch was made, and the
// lattice's device status word (bounded-wait timeouts).
cudaError_t batch_fill_desc(const HostParams &h, void *buf0, void *buf1, unsigned long long step0, int parity0,
                            int seg_rows, int *status, void *out);
int batch_grid(int storage, int wpb);
// Warps of the batched step (row_fetch 1 or 3, wpb warps per block) that can
// be resident on the device at once.
cudaError_t batch_resident_warps(int storage, int row_fetch, int wpb, int *out);
// Kernel attributes of the batched step; called before any stream capture.
cudaError_t batch_prepare(int storage);
// row_fetch: 1 plain loads (persistent grid of `blocks`), 3 TMA ring read in
// place (one warp per work item).  The launch takes batch step t0, plus the
// device counter in ctl when from_counter is set (launches inside a graph).
cudaError_t launch_batch(int storage, int row_fetch, const void *desc, const int *prefix, int n, int total,
                         void *ctl, int wpb, int blocks, unsigned long long t0, int from_counter,
                         cudaStream_t s);
// nsteps batch steps t0 .. t0 + nsteps - 1 in one cooperative launch (every
// work item resident; items wait only for their neighbours' progress in
// done[total], cleared here first).
cudaError_t launch_batch_persist(int storage, const void *desc, const int *prefix, int n, int total, int wpb,
                                 unsigned long long t0, int nsteps, int *done, cudaStream_t s);
// The device counter of a batch: set to value, or advanced by it (add != 0).
cudaError_t launch_batch_counter(void *ctl, unsigned long long value, int add, cudaStream_t s);
// Batched diagnostics: one descriptor per lattice (its partial-sum buffer and
// the grid of its own diagnostics under launch l; returns the number of
// blocks, -1 above MAX_DIAG_BLOCKS), block prefix sums over the lattices, and
// the three launches that write each lattice's sums and status word into
// out + m * slot_doubles after t batch steps.
size_t batch_diag_bytes();
int batch_fill_diag(const HostParams &h, const Launch &l, double *partial, void *out);
cudaError_t launch_batch_diag(int storage, const void *desc, const void *bdiag, const int *bprefix, int n, int total,
                              unsigned long long t, double *out, int slot_doubles, cudaStream_t s);
// Message for lb_last_error(NULL) on this thread.
void set_global_error(const char *msg);
Launch default_launch(const HostParams &p);

}  // namespace lbk
