// Host side of the C ABI declared in include/lb.h.
//
// Device memory layout inside the caller's buffer (256-byte aligned parts):
//   [A: 19 planes][B: 19 planes][partial sums][result, status][radius table]
// The radius table holds y = r_inner + j + 1/2 and 1/y per column (pitch
// entries each), computed in FP64 and rounded once to FP32.
// A and B alternate as source and destination of the time steps; the one
// that is not current doubles as staging space for host exchanges and for
// the temperature field of the diagnostics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"

using lbk::HostParams;
using lbk::Launch;

struct lb_ctx {
    HostParams hp;
    bool params_set;
    char *buf;
    size_t bytes;
    size_t dist_bytes;   // one distribution buffer, rounded to 256
    char *dist[2];
    double *partial;
    double *result;
    cudaStream_t stream;
    int cur;
    int64_t step;
    Launch launch;
    bool launch_auto;
    alignas(64) unsigned char tmap[2][128];  // TMA tensor maps of dist[0], dist[1]
    bool tmap_ready;
    int *status;  // device status word (bounded-wait timeouts of the step kernel)
    char err[256];
};

static thread_local char g_err[256] = "";

void lbk::set_global_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

lb_status fail(lb_ctx *ctx, lb_status st, const char *fmt, ...)
{
    char *dst = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

lb_status cuda_fail(lb_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, LB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

lb_status say(char *err, size_t n, lb_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
    return st;
}

lb_status check_desc(const lb_grid_desc *d, size_t *plane, size_t *dist_bytes)
{
    HostParams h;
    std::memset(&h, 0, sizeof(h));
    const lb_status st = lbk::host_from_desc(d, &h, g_err, sizeof(g_err));
    if (st != LB_OK) return st;
    *plane = (size_t)h.plane;
    *dist_bytes = align256(lbk::NQ * (size_t)h.plane * lbk::storage_bytes(d->storage));
    return LB_OK;
}

size_t scratch_bytes() { return align256((size_t)lbk::MAX_DIAG_BLOCKS * lbk::NSUM * sizeof(double)) + 256; }

size_t table_bytes(int pitch) { return align256(2 * (size_t)pitch * sizeof(float)); }

}  // namespace

int lbk::pitch_for(int nr, int storage)
{
    const int m = lbk::storage_bytes(storage) == 2 ? 64 : 32;
    return (nr + m - 1) / m * m;
}

lb_status lbk::host_from_desc(const lb_grid_desc *d, HostParams *h, char *err, size_t n)
{
    if (!d) return say(err, n, LB_ERR_ARG, "desc is NULL");
    if (d->nr < 2 || d->nz < 2) return say(err, n, LB_ERR_ARG, "nr and nz must be >= 2 (got %d, %d)", d->nr, d->nz);
    if (d->nr > (1 << 20) || d->nz > (1 << 24)) return say(err, n, LB_ERR_ARG, "lattice too large");
    if (!(d->r_inner >= 0.0) || !std::isfinite(d->r_inner)) return say(err, n, LB_ERR_ARG, "r_inner must be >= 0");
    if (d->storage < LB_FP64 || d->storage > LB_FP16)
        return say(err, n, LB_ERR_ARG, "unknown storage %d", d->storage);
    if (d->reserved != 0) return say(err, n, LB_ERR_ARG, "reserved must be 0");
    h->nr = d->nr;
    h->nz = d->nz;
    h->pitch = pitch_for(d->nr, d->storage);
    h->plane = (long long)h->nz * h->pitch;
    h->storage = d->storage;
    h->r0 = d->r_inner;
    h->scale = d->storage == LB_FP16 ? lbk::kFp16Scale : 1.0;
    return LB_OK;
}

lb_status lbk::host_set_params(const lb_params *p, HostParams *h, char *err, size_t n)
{
    if (!p) return say(err, n, LB_ERR_ARG, "params is NULL");
    if (!(p->nu > 0.0) || !(p->alpha > 0.0) || !(p->rho0 > 0.0))
        return say(err, n, LB_ERR_ARG, "nu, alpha and rho0 must be > 0");
    if (!(p->omega3 > 0.0 && p->omega3 < 2.0) || !(p->omega_hi > 0.0 && p->omega_hi < 2.0))
        return say(err, n, LB_ERR_ARG, "omega3 and omega_hi must lie in (0, 2)");
    const double vals[] = {p->g_beta, p->T0, p->body_fx};
    for (double v : vals)
        if (!std::isfinite(v)) return say(err, n, LB_ERR_ARG, "non-finite g_beta, T0 or body_fx");
    const int per0 = p->side[0].flow == LB_FLOW_PERIODIC, per1 = p->side[1].flow == LB_FLOW_PERIODIC;
    if (per0 != per1) return say(err, n, LB_ERR_ARG, "periodicity needs both end sides");
    for (int s = 0; s < 4; ++s) {
        const lb_side &sd = p->side[s];
        if (sd.flow < 0 || sd.flow > 3 || sd.swirl < 0 || sd.swirl > 4 || sd.heat < 0 || sd.heat > 4)
            return say(err, n, LB_ERR_ARG, "side %d: unknown boundary code", s);
        const bool per = sd.flow == LB_FLOW_PERIODIC;
        const bool ax = sd.flow == LB_FLOW_AXIS;
        if ((sd.swirl == LB_SC_PERIODIC) != per || (sd.heat == LB_SC_PERIODIC) != per)
            return say(err, n, LB_ERR_ARG, "side %d: periodic must apply to f, g and h together", s);
        if ((sd.swirl == LB_SC_AXIS) != ax || (sd.heat == LB_SC_AXIS) != ax)
            return say(err, n, LB_ERR_ARG, "side %d: the axis must apply to f, g and h together", s);
        if (per && s >= 2) return say(err, n, LB_ERR_ARG, "periodicity only along z");
        if (ax && (s != 2 || h->r0 != 0.0))
            return say(err, n, LB_ERR_ARG, "the axis is only the inner side of a cylinder");
        const double wv[4] = {sd.u_wx, sd.u_wy, sd.omega, sd.T_w};
        for (double v : wv)
            if (!std::isfinite(v)) return say(err, n, LB_ERR_ARG, "side %d: non-finite wall value", s);
    }
    if (h->r0 == 0.0 && !p->planar && p->side[2].flow != LB_FLOW_AXIS)
        return say(err, n, LB_ERR_ARG, "r_inner = 0 needs the axis on the inner side");
    for (int s = 0; s < 4; ++s) {
        const lb_side &sd = p->side[s];
        if (sd.flow == LB_FLOW_FREE && s >= 2) return say(err, n, LB_ERR_ARG, "a free surface only on an end wall");
        if (sd.heat == LB_SC_RAMP || sd.swirl == LB_SC_RAMP)
            return say(err, n, LB_ERR_ARG, "the temperature ramp only on the outer segment of a split top");
    }
    if (p->top_split < 0 || p->top_split >= h->nr) return say(err, n, LB_ERR_ARG, "top_split must lie in 0..nr-1");
    if (p->top_split > 0) {
        const lb_side &t = p->top_outer;
        if (p->side[1].flow == LB_FLOW_PERIODIC) return say(err, n, LB_ERR_ARG, "a periodic top cannot be split");
        if (!(t.flow == LB_FLOW_WALL || t.flow == LB_FLOW_FREE) ||
            !(t.swirl == LB_SC_DIRICHLET || t.swirl == LB_SC_NEUMANN) ||
            !(t.heat == LB_SC_DIRICHLET || t.heat == LB_SC_NEUMANN || t.heat == LB_SC_RAMP))
            return say(err, n, LB_ERR_ARG, "top_outer: flow WALL or FREE, swirl DIRICHLET or NEUMANN, "
                                           "heat DIRICHLET, NEUMANN or RAMP");
        const double tv[4] = {t.u_wx, t.u_wy, t.omega, t.T_w};
        for (double v : tv)
            if (!std::isfinite(v)) return say(err, n, LB_ERR_ARG, "top_outer: non-finite wall value");
    }
    h->nu = p->nu;
    h->alpha = p->alpha;
    h->omega3 = p->omega3;
    h->omega_hi = p->omega_hi;
    h->g_beta = p->g_beta;
    h->T0 = p->T0;
    h->body_fx = p->body_fx;
    h->rho0 = p->rho0;
    h->planar = p->planar;
    h->sign_literal = p->sign_literal;
    h->explicit_sources = p->explicit_sources;
    for (int s = 0; s < 5; ++s) {
        // entry 4: the top's outer segment, or a copy of the top when it is not split
        const lb_side &sd = s < 4 ? p->side[s] : (p->top_split > 0 ? p->top_outer : p->side[1]);
        h->flow[s] = sd.flow;
        h->swirl[s] = sd.swirl;
        h->heat[s] = sd.heat;
        h->uwx[s] = sd.u_wx;
        h->uwy[s] = sd.u_wy;
        h->omega[s] = sd.omega;
        h->Tw[s] = sd.T_w;
    }
    h->top_split = p->top_split;
    return LB_OK;
}

void lbk::diag_from_sums(const HostParams &h, const double *res, int kstatus, int64_t step, lb_diag *out)
{
    std::memset(out, 0, sizeof(*out));
    const double N = (double)h.nr * h.nz;
    const double sum_y = (double)h.nz * (h.nr * h.r0 + 0.5 * (double)h.nr * h.nr);
    out->mass = h.rho0 * N + res[0];
    out->mass_r = h.rho0 * sum_y + res[1];
    out->T_sum = res[2];
    out->u_max = res[3];
    for (int s = 0; s < 4; ++s) out->nu_side[s] = res[4 + s];
    int a = -1, b = -1;
    if (h.heat[2] == LB_SC_DIRICHLET && h.heat[3] == LB_SC_DIRICHLET) {
        a = 2;
        b = 3;
    } else if (h.heat[0] == LB_SC_DIRICHLET && h.heat[1] == LB_SC_DIRICHLET) {
        a = 0;
        b = 1;
    } else {
        for (int s = 0; s < 4; ++s)
            if (h.heat[s] == LB_SC_DIRICHLET) {
                if (a < 0) a = s;
                else if (b < 0) b = s;
            }
    }
    if (a >= 0) out->nu_i = out->nu_side[a];
    if (b >= 0) out->nu_o = out->nu_side[b];
    out->nu_avg = (a >= 0 && b >= 0) ? 0.5 * (out->nu_i + out->nu_o) : out->nu_i;
    out->k_eq_i = res[9];
    out->k_eq_o = res[10];
    out->step = step;
    const bool bad = res[8] > 0.0 || !std::isfinite(res[0]) || !std::isfinite(res[2]);
    out->status = kstatus ? kstatus : (bad ? LB_ERR_DIVERGED : LB_OK);
}

namespace {

// Rows of `planes` doubles per node that fit in the staging area.
lb_status staging(lb_ctx *ctx, int planes, double **ptr, int *rows)
{
    const size_t per_row = (size_t)planes * ctx->hp.nr * sizeof(double);
    size_t avail = ctx->dist_bytes;
    char *base = ctx->dist[1 - ctx->cur];
    if (avail < per_row) {  // tiny 16-bit lattices: use the reduction scratch
        avail = (size_t)lbk::MAX_DIAG_BLOCKS * lbk::NSUM * sizeof(double);
        base = (char *)ctx->partial;
        if (avail < per_row) return fail(ctx, LB_ERR_NOMEM, "no staging space for one row");
    }
    size_t r = avail / per_row;
    if (r > (size_t)ctx->hp.nz) r = ctx->hp.nz;
    *ptr = (double *)base;
    *rows = (int)r;
    return LB_OK;
}

lb_status need_params(lb_ctx *ctx)
{
    if (!ctx) return fail(nullptr, LB_ERR_ARG, "ctx is NULL");
    if (!ctx->params_set) return fail(ctx, LB_ERR_STATE, "lb_set_params has not been called");
    return LB_OK;
}

Launch diag_launch(const lb_ctx *ctx)
{
    Launch l = ctx->launch;
    if (l.seg_rows < 32) l.seg_rows = 32;  // the diagnostics march: longer segments, fewer partial sums
    const long long nwin = (ctx->hp.nr + 29) / 30;
    const long long bx = (nwin + 3) / 4;
    long long segs = (ctx->hp.nz + l.seg_rows - 1) / l.seg_rows;
    if (bx * segs > lbk::MAX_DIAG_BLOCKS) {
        segs = lbk::MAX_DIAG_BLOCKS / bx;
        if (segs < 1) segs = 1;
        l.seg_rows = (int)((ctx->hp.nz + segs - 1) / segs);
    }
    return l;
}

}  // namespace

extern "C" {

lb_status lb_required_bytes(const lb_grid_desc *desc, size_t *bytes)
{
    size_t plane, dist;
    lb_status st = check_desc(desc, &plane, &dist);
    if (st != LB_OK) return st;
    if (!bytes) return fail(nullptr, LB_ERR_ARG, "bytes is NULL");
    *bytes = 2 * dist + scratch_bytes() + table_bytes(lbk::pitch_for(desc->nr, desc->storage));
    return LB_OK;
}

lb_status lb_create(const lb_grid_desc *desc, void *dev_buf, size_t bytes, void *cuda_stream, lb_ctx **out)
{
    if (!out) return fail(nullptr, LB_ERR_ARG, "out is NULL");
    *out = nullptr;
    size_t plane, dist;
    lb_status st = check_desc(desc, &plane, &dist);
    if (st != LB_OK) return st;
    const size_t need = 2 * dist + scratch_bytes() + table_bytes(lbk::pitch_for(desc->nr, desc->storage));
    if (!dev_buf) return fail(nullptr, LB_ERR_ARG, "dev_buf is NULL");
    if (((uintptr_t)dev_buf & 255) != 0) return fail(nullptr, LB_ERR_ARG, "dev_buf must be 256-byte aligned");
    if (bytes < need) return fail(nullptr, LB_ERR_NOMEM, "buffer holds %zu bytes, %zu needed", bytes, need);
    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return fail(nullptr, LB_ERR_NOMEM, "host allocation failed");
    HostParams &h = c->hp;
    std::memset(&h, 0, sizeof(h));
    lbk::host_from_desc(desc, &h, g_err, sizeof(g_err));  // checked above
    c->buf = (char *)dev_buf;
    c->bytes = bytes;
    c->dist_bytes = dist;
    c->dist[0] = c->buf;
    c->dist[1] = c->buf + dist;
    c->partial = (double *)(c->buf + 2 * dist);
    c->result = (double *)(c->buf + 2 * dist + align256((size_t)lbk::MAX_DIAG_BLOCKS * lbk::NSUM * sizeof(double)));
    c->status = (int *)((char *)c->result + 128);
    h.ytab = (const float *)(c->buf + 2 * dist + scratch_bytes());
    c->tmap_ready = false;
    c->stream = (cudaStream_t)cuda_stream;
    c->cur = 0;
    c->step = 0;
    c->params_set = false;
    c->launch = lbk::default_launch(h);
    c->launch_auto = true;
    c->err[0] = 0;
    *out = c;
    return LB_OK;
}

lb_status lb_set_params(lb_ctx *ctx, const lb_params *p)
{
    if (!ctx || !p) return fail(ctx, LB_ERR_ARG, "NULL argument");
    lb_status st = lbk::host_set_params(p, &ctx->hp, ctx->err, sizeof(ctx->err));
    if (st != LB_OK) return st;
    HostParams &h = ctx->hp;
    // rest state: every stored deviation is zero; clear the status word;
    // radius table (entries past nr - 1 repeat the last radius)
    std::vector<float> tab(2 * (size_t)h.pitch);
    for (int j = 0; j < h.pitch; ++j) {
        const double y = h.r0 + (j < h.nr ? j : h.nr - 1) + 0.5;
        tab[j] = (float)y;
        tab[h.pitch + j] = (float)(1.0 / y);
    }
    cudaError_t e = cudaMemsetAsync(ctx->dist[0], 0, ctx->dist_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h.ytab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // tab is freed on return
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reset");
    ctx->cur = 0;
    ctx->step = 0;
    ctx->params_set = true;
    return LB_OK;
}

lb_status lb_init_fields(lb_ctx *ctx, const double *host_fields)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host_fields) return fail(ctx, LB_ERR_ARG, "host_fields is NULL");
    double *stage;
    int rows;
    if ((st = staging(ctx, 5, &stage, &rows)) != LB_OK) return st;
    const int nr = ctx->hp.nr, nz = ctx->hp.nz;
    const size_t N = (size_t)nr * nz;
    for (int r0 = 0; r0 < nz; r0 += rows) {
        const int r1 = r0 + rows < nz ? r0 + rows : nz;
        const size_t n = (size_t)(r1 - r0) * nr;
        for (int q = 0; q < 5; ++q) {
            cudaError_t e = cudaMemcpyAsync(stage + q * n, host_fields + q * N + (size_t)r0 * nr, n * sizeof(double),
                                            cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "init upload");
        }
        cudaError_t e = lbk::launch_init_fields(ctx->hp, stage, ctx->dist[ctx->cur], r0, r1, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "init kernel");
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init sync");
    ctx->step = 0;
    return LB_OK;
}

lb_status lb_step(lb_ctx *ctx, int32_t nsteps)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (nsteps < 0) return fail(ctx, LB_ERR_ARG, "nsteps < 0");
    if (ctx->hp.storage != LB_FP64 && !ctx->tmap_ready) {
        for (int b = 0; b < 2; ++b) {
            cudaError_t e = lbk::make_tensor_map(ctx->hp, ctx->dist[b], ctx->tmap[b]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor map");
        }
        ctx->tmap_ready = true;
    }
    for (int32_t t = 0; t < nsteps; ++t) {
        const void *map = ctx->tmap_ready ? ctx->tmap[ctx->cur] : nullptr;
        cudaError_t e = lbk::launch_step(ctx->hp, ctx->launch, ctx->dist[ctx->cur], ctx->dist[1 - ctx->cur],
                                         (unsigned long long)ctx->step, map, ctx->status, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
        ctx->cur ^= 1;
        ctx->step += 1;
    }
    return LB_OK;
}

lb_status lb_get_fields(lb_ctx *ctx, double *host_fields)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host_fields) return fail(ctx, LB_ERR_ARG, "host_fields is NULL");
    double *stage;
    int rows;
    if ((st = staging(ctx, 5, &stage, &rows)) != LB_OK) return st;
    const int nr = ctx->hp.nr, nz = ctx->hp.nz;
    const size_t N = (size_t)nr * nz;
    for (int r0 = 0; r0 < nz; r0 += rows) {
        const int r1 = r0 + rows < nz ? r0 + rows : nz;
        const size_t n = (size_t)(r1 - r0) * nr;
        cudaError_t e = lbk::launch_fields(ctx->hp, ctx->launch, ctx->dist[ctx->cur], stage, r0, r1, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fields kernel");
        for (int q = 0; q < 5; ++q) {
            e = cudaMemcpyAsync(host_fields + q * N + (size_t)r0 * nr, stage + q * n, n * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "fields download");
        }
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fields sync");
    }
    return LB_OK;
}

lb_status lb_selftest_timeout(lb_ctx *ctx, int32_t polls)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (polls < 1 || polls > (1 << 22)) return fail(ctx, LB_ERR_ARG, "1 <= polls <= 2^22");
    cudaError_t e = lbk::launch_wait_selftest(ctx->status, polls, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test");
    return LB_OK;
}

lb_status lb_stream_function(lb_ctx *ctx, double *host_psi, double *psi_max)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!psi_max) return fail(ctx, LB_ERR_ARG, "psi_max is NULL");
    double *stage;
    int rows;
    if ((st = staging(ctx, 5, &stage, &rows)) != LB_OK) return st;
    const int nr = ctx->hp.nr, nz = ctx->hp.nz;
    std::vector<double> rowmax((size_t)nz);
    for (int r0 = 0; r0 < nz; r0 += rows) {
        const int r1 = r0 + rows < nz ? r0 + rows : nz;
        const size_t n = (size_t)(r1 - r0) * nr;
        // fields into planes 0..4 of the stage; Psi over plane 0, row maxima over plane 2
        cudaError_t e = lbk::launch_fields(ctx->hp, ctx->launch, ctx->dist[ctx->cur], stage, r0, r1, ctx->stream);
        if (e == cudaSuccess)
            e = lbk::launch_psi(stage + n, stage, stage + 2 * n, r1 - r0, nr, ctx->hp.r0, ctx->stream);
        if (e == cudaSuccess && host_psi)
            e = cudaMemcpyAsync(host_psi + (size_t)r0 * nr, stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(rowmax.data() + r0, stage + 2 * n, (size_t)(r1 - r0) * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream function");
    }
    double m = 0.0;
    for (double v : rowmax) m = v > m ? v : m;
    *psi_max = m;
    return LB_OK;
}

// lb_diag from the NSUM device sums of the diagnostics and the status word
static void fill_diag(const lb_ctx *ctx, const double *res, int kstatus, lb_diag *out)
{
    lbk::diag_from_sums(ctx->hp, res, kstatus, ctx->step, out);
}

lb_status lb_diagnostics(lb_ctx *ctx, lb_diag *out)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!out) return fail(ctx, LB_ERR_ARG, "out is NULL");
    const HostParams &h = ctx->hp;
    double res[lbk::NSUM];
    int kstatus = 0;
    cudaError_t e = lbk::launch_diag(h, diag_launch(ctx), ctx->dist[ctx->cur], ctx->partial,
                                     (double *)ctx->dist[1 - ctx->cur], ctx->result, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "diagnostics kernel");
    e = cudaMemcpyAsync(&kstatus, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, ctx->result, sizeof(res), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "diagnostics download");
    fill_diag(ctx, res, kstatus, out);
    return LB_OK;
}

lb_status lb_get_distributions(lb_ctx *ctx, double *host19)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host19) return fail(ctx, LB_ERR_ARG, "host19 is NULL");
    double *stage;
    int rows;
    if ((st = staging(ctx, lbk::NQ, &stage, &rows)) != LB_OK) return st;
    const int nr = ctx->hp.nr, nz = ctx->hp.nz;
    const size_t N = (size_t)nr * nz;
    for (int r0 = 0; r0 < nz; r0 += rows) {
        const int r1 = r0 + rows < nz ? r0 + rows : nz;
        const size_t n = (size_t)(r1 - r0) * nr;
        cudaError_t e = lbk::launch_export(ctx->hp, ctx->dist[ctx->cur], stage, r0, r1, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "export kernel");
        for (int q = 0; q < lbk::NQ; ++q) {
            e = cudaMemcpyAsync(host19 + q * N + (size_t)r0 * nr, stage + q * n, n * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "export download");
        }
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "export sync");
    }
    return LB_OK;
}

lb_status lb_set_distributions(lb_ctx *ctx, const double *host19)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host19) return fail(ctx, LB_ERR_ARG, "host19 is NULL");
    double *stage;
    int rows;
    if ((st = staging(ctx, lbk::NQ, &stage, &rows)) != LB_OK) return st;
    const int nr = ctx->hp.nr, nz = ctx->hp.nz;
    const size_t N = (size_t)nr * nz;
    for (int r0 = 0; r0 < nz; r0 += rows) {
        const int r1 = r0 + rows < nz ? r0 + rows : nz;
        const size_t n = (size_t)(r1 - r0) * nr;
        for (int q = 0; q < lbk::NQ; ++q) {
            cudaError_t e = cudaMemcpyAsync(stage + q * n, host19 + q * N + (size_t)r0 * nr, n * sizeof(double),
                                            cudaMemcpyHostToDevice, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "import upload");
        }
        cudaError_t e = lbk::launch_import(ctx->hp, stage, ctx->dist[ctx->cur], r0, r1, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "import kernel");
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "import sync");
    }
    return LB_OK;
}

lb_status lb_state_bytes(const lb_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return fail(nullptr, LB_ERR_ARG, "NULL argument");
    *bytes = 16 + ctx->dist_bytes;
    return LB_OK;
}

lb_status lb_get_state(lb_ctx *ctx, void *host, size_t bytes)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host || bytes < 16 + ctx->dist_bytes) return fail(ctx, LB_ERR_ARG, "state buffer too small");
    int64_t hdr[2] = {ctx->step, (int64_t)ctx->hp.storage};
    std::memcpy(host, hdr, 16);
    cudaError_t e = cudaMemcpyAsync((char *)host + 16, ctx->dist[ctx->cur], ctx->dist_bytes, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state download");
    return LB_OK;
}

lb_status lb_set_state(lb_ctx *ctx, const void *host, size_t bytes)
{
    lb_status st = need_params(ctx);
    if (st != LB_OK) return st;
    if (!host || bytes < 16 + ctx->dist_bytes) return fail(ctx, LB_ERR_ARG, "state buffer too small");
    int64_t hdr[2];
    std::memcpy(hdr, host, 16);
    if (hdr[1] != ctx->hp.storage) return fail(ctx, LB_ERR_ARG, "state was saved with another storage type");
    cudaError_t e = cudaMemcpyAsync(ctx->dist[ctx->cur], (const char *)host + 16, ctx->dist_bytes,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "state upload");
    ctx->step = hdr[0];
    return LB_OK;
}

lb_status lb_get_step(const lb_ctx *ctx, int64_t *step)
{
    if (!ctx || !step) return fail(nullptr, LB_ERR_ARG, "NULL argument");
    *step = ctx->step;
    return LB_OK;
}

lb_status lb_set_launch(lb_ctx *ctx, int32_t seg_rows, int32_t warps_per_block, int32_t row_fetch)
{
    if (!ctx) return fail(nullptr, LB_ERR_ARG, "ctx is NULL");
    if (seg_rows < 0 || warps_per_block < 0 || warps_per_block > 8 || row_fetch < 0 || row_fetch > 3)
        return fail(ctx, LB_ERR_ARG, "seg_rows >= 0, 0 <= warps_per_block <= 8, 0 <= row_fetch <= 3");
    if (seg_rows && (ctx->hp.nz + seg_rows - 1) / seg_rows > 65535)
        return fail(ctx, LB_ERR_ARG, "seg_rows too small for nz (more than 65535 segments)");
    Launch d = lbk::default_launch(ctx->hp);
    ctx->launch.seg_rows = seg_rows ? seg_rows : d.seg_rows;
    ctx->launch.warps_per_block = warps_per_block ? warps_per_block : d.warps_per_block;
    ctx->launch.use_tma = row_fetch == 0 ? d.use_tma : (row_fetch >= 2 && ctx->hp.storage != LB_FP64 ? row_fetch - 1 : 0);
    ctx->launch_auto = seg_rows == 0 && warps_per_block == 0 && row_fetch == 0;
    return LB_OK;
}

lb_status lb_get_launch(const lb_ctx *ctx, int32_t *seg_rows, int32_t *warps_per_block, int32_t *row_fetch)
{
    if (!ctx) return fail(nullptr, LB_ERR_ARG, "ctx is NULL");
    if (seg_rows) *seg_rows = ctx->launch.seg_rows;
    if (warps_per_block) *warps_per_block = ctx->launch.warps_per_block;
    if (row_fetch) *row_fetch = ctx->launch.use_tma + 1;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx *ctx)
{
    delete ctx;
    return LB_OK;
}

const char *lb_last_error(const lb_ctx *ctx) { return ctx ? ctx->err : g_err; }

// ---- batches ---------------------------------------------------------------------

struct lb_batch {
    std::vector<lb_ctx *> ctxs;
    std::vector<unsigned long long> step0;
    std::vector<int> parity0;
    int storage;
    char *buf;
    size_t bytes;
    void *d_desc;
    int *d_prefix;
    void *d_ctl;
    char *d_diag;
    std::vector<char> hdiag;
    cudaStream_t stream;
    int seg_rows, wpb, blocks, total, graph_steps, row_fetch;
    std::vector<int> seg_of;             // per lattice rows per z-segment (0: seg_rows)
    unsigned long long counter;
    cudaGraphExec_t gexec;
    bool graph_valid;
    cudaEvent_t ev;                      // orders the batch stream against the lattices' streams
    std::vector<cudaStream_t> streams;   // the lattices' distinct streams other than the batch's
    std::vector<unsigned char> hdesc;
    std::vector<int> hprefix;
    // batched diagnostics: per-lattice descriptors and block prefix sums
    void *d_bdiag;
    int *d_bprefix;
    std::vector<unsigned char> hbdiag;
    std::vector<int> hbprefix;
    bool bdiag_uploaded;
    int *d_flags;  // progress counters of the persistent step (row fetch 5)
};

// Work queued on the lattices' own streams (initialisation, state uploads,
// diagnostics) and the batch's launches stay ordered both ways.
static cudaError_t batch_streams_wait(lb_batch *b, bool batch_waits)
{
    cudaError_t e = cudaSuccess;
    for (cudaStream_t s : b->streams) {
        cudaStream_t from = batch_waits ? s : b->stream, to = batch_waits ? b->stream : s;
        e = cudaEventRecord(b->ev, from);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(to, b->ev, 0);
        if (e != cudaSuccess) break;
    }
    return e;
}

constexpr size_t kDiagSlot = 256;  // per lattice: its NSUM sums and status word, gathered on the device

// Batch buffer: descriptors, item prefix sums, step counter, gathered
// diagnostics, diagnostics descriptors, diagnostics block prefix sums.
// Work items the persistent batched step (row fetch 5) can track: one
// progress counter each.
constexpr int kMaxPersistItems = 16384;

static size_t batch_layout(int32_t n, size_t *desc_off, size_t *prefix_off, size_t *ctl_off, size_t *diag_off,
                           size_t *bdiag_off = nullptr, size_t *bprefix_off = nullptr, size_t *flags_off = nullptr)
{
    const size_t d = align256((size_t)n * lbk::batch_desc_bytes());
    const size_t p = align256((size_t)(n + 1) * sizeof(int));
    const size_t t = align256(lbk::batch_ctl_bytes());
    const size_t g = align256((size_t)n * kDiagSlot);
    const size_t bd = align256((size_t)n * lbk::batch_diag_bytes());
    const size_t bp = align256((size_t)(n + 1) * sizeof(int));
    *desc_off = 0;
    *prefix_off = d;
    *ctl_off = d + p;
    *diag_off = d + p + t;
    if (bdiag_off) *bdiag_off = d + p + t + g;
    if (bprefix_off) *bprefix_off = d + p + t + g + bd;
    if (flags_off) *flags_off = d + p + t + g + bd + bp;
    return d + p + t + g + bd + bp + (size_t)kMaxPersistItems * sizeof(int);
}

static lb_status batch_upload(lb_batch *b)
{
    const int n = (int)b->ctxs.size();
    const size_t db = lbk::batch_desc_bytes();
    b->hdesc.assign((size_t)n * db, 0);
    b->hprefix.assign((size_t)n + 1, 0);
    for (int m = 0; m < n; ++m) {
        lb_ctx *c = b->ctxs[m];
        const int seg = b->seg_of[m] ? b->seg_of[m] : b->seg_rows;
        cudaError_t e = lbk::batch_fill_desc(c->hp, c->dist[0], c->dist[1], b->step0[m], b->parity0[m], seg,
                                             c->status, b->hdesc.data() + (size_t)m * db);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch descriptor (tensor map)");
        const long long items = (long long)b->hprefix[m] + lbk::batch_items(c->hp, seg);
        if (items > (1LL << 30)) return fail(nullptr, LB_ERR_ARG, "too many work items in the batch");
        b->hprefix[m + 1] = (int)items;
    }
    b->total = b->hprefix[n];
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->hdesc.data(), b->hdesc.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_prefix, b->hprefix.data(), b->hprefix.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch upload");
    if (b->graph_valid) {
        cudaGraphExecDestroy(b->gexec);
        b->graph_valid = false;
    }
    return LB_OK;
}

lb_status lb_batch_required_bytes(int32_t n, size_t *bytes)
{
    if (n < 1 || !bytes) return fail(nullptr, LB_ERR_ARG, "n >= 1 and bytes required");
    size_t a, b, c, d;
    *bytes = batch_layout(n, &a, &b, &c, &d);
    return LB_OK;
}

lb_status lb_batch_create(lb_ctx *const *ctxs, int32_t n, void *dev_buf, size_t bytes, void *cuda_stream,
                          lb_batch **out)
{
    if (!out || !ctxs || n < 1 || !dev_buf) return fail(nullptr, LB_ERR_ARG, "NULL argument or n < 1");
    *out = nullptr;
    size_t doff, poff, coff, goff, bdoff, bpoff, foff;
    const size_t need = batch_layout(n, &doff, &poff, &coff, &goff, &bdoff, &bpoff, &foff);
    if (bytes < need) return fail(nullptr, LB_ERR_NOMEM, "batch buffer holds %zu bytes, %zu needed", bytes, need);
    if (((uintptr_t)dev_buf & 255) != 0) return fail(nullptr, LB_ERR_ARG, "dev_buf must be 256-byte aligned");
    const int storage = ctxs[0] ? ctxs[0]->hp.storage : -1;
    if (storage == LB_FP64 || storage < 0) return fail(nullptr, LB_ERR_ARG, "batches take FP32 or 16-bit lattices");
    for (int m = 0; m < n; ++m) {
        if (!ctxs[m] || !ctxs[m]->params_set) return fail(nullptr, LB_ERR_STATE, "lattice %d has no parameters", m);
        if (ctxs[m]->hp.storage != storage) return fail(nullptr, LB_ERR_ARG, "lattices of a batch share the storage");
        for (int q = 0; q < m; ++q)
            if (ctxs[q] == ctxs[m]) return fail(nullptr, LB_ERR_ARG, "lattice %d appears twice", m);
    }
    lb_batch *b = new (std::nothrow) lb_batch();
    if (!b) return fail(nullptr, LB_ERR_NOMEM, "host allocation failed");
    b->ctxs.assign(ctxs, ctxs + n);
    for (int m = 0; m < n; ++m) {
        b->step0.push_back((unsigned long long)ctxs[m]->step);
        b->parity0.push_back(ctxs[m]->cur);
    }
    b->storage = storage;
    b->buf = (char *)dev_buf;
    b->bytes = bytes;
    b->d_desc = b->buf + doff;
    b->d_prefix = (int *)(b->buf + poff);
    b->d_ctl = b->buf + coff;
    b->d_diag = b->buf + goff;
    b->hdiag.assign((size_t)n * kDiagSlot, 0);
    b->d_bdiag = b->buf + bdoff;
    b->d_bprefix = (int *)(b->buf + bpoff);
    b->d_flags = (int *)(b->buf + foff);
    b->bdiag_uploaded = false;
    b->stream = (cudaStream_t)cuda_stream;
    b->seg_rows = 4;
    b->seg_of.assign((size_t)n, 0);
    b->wpb = 1;
    b->graph_steps = 8;
    b->row_fetch = 3;
    b->counter = 0;
    b->graph_valid = false;
    b->blocks = lbk::batch_grid(storage, b->wpb);
    b->ev = nullptr;
    for (int m = 0; m < n; ++m) {
        cudaStream_t s = ctxs[m]->stream;
        bool seen = s == b->stream;
        for (cudaStream_t t : b->streams) seen = seen || t == s;
        if (!seen) b->streams.push_back(s);
    }
    cudaError_t e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = lbk::batch_prepare(storage);
    if (e == cudaSuccess) e = batch_streams_wait(b, true);  // the lattices' pending work precedes the batch
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, lbk::batch_ctl_bytes(), b->stream);
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        return cuda_fail(nullptr, e, "batch reset");
    }
    lb_status st = batch_upload(b);
    if (st != LB_OK) {
        lb_batch_destroy(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_set_launch(lb_batch *b, int32_t seg_rows, int32_t warps_per_block, int32_t graph_steps,
                              int32_t row_fetch)
{
    if (!b || seg_rows < 0 || warps_per_block < 0 || warps_per_block > 8 || graph_steps < 0 ||
        !(row_fetch == 0 || row_fetch == 1 || row_fetch == 3 || row_fetch == 4 || row_fetch == 5))
        return fail(nullptr, LB_ERR_ARG,
                    "seg_rows >= 0, 0 <= warps_per_block <= 8, graph_steps >= 0, row_fetch 0, 1, 3, 4 or 5");
    if (row_fetch == 4 && b->storage != LB_FP32)
        return fail(nullptr, LB_ERR_ARG, "row_fetch 4 (three ring stages) is for FP32 storage");
    if (row_fetch) b->row_fetch = row_fetch;
    if (seg_rows) b->seg_rows = seg_rows;
    if (warps_per_block) {
        b->wpb = warps_per_block;
        b->blocks = lbk::batch_grid(b->storage, b->wpb);
    }
    b->graph_steps = graph_steps;
    return batch_upload(b);
}

lb_status lb_batch_set_segments(lb_batch *b, const int32_t *seg_rows)
{
    if (!b) return fail(nullptr, LB_ERR_ARG, "batch is NULL");
    const int n = (int)b->ctxs.size();
    if (seg_rows)
        for (int m = 0; m < n; ++m)
            if (seg_rows[m] < 0 || seg_rows[m] > b->ctxs[m]->hp.nz)
                return fail(nullptr, LB_ERR_ARG, "lattice %d: rows per z-segment must lie in 0..nz", m);
    for (int m = 0; m < n; ++m) b->seg_of[m] = seg_rows ? seg_rows[m] : 0;
    return batch_upload(b);
}

lb_status lb_batch_get_occupancy(const lb_batch *b, int32_t *resident_warps, int32_t *items)
{
    if (!b) return fail(nullptr, LB_ERR_ARG, "batch is NULL");
    if (resident_warps) {
        int r = 0;
        cudaError_t e = lbk::batch_resident_warps(b->storage, b->row_fetch, b->wpb, &r);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "occupancy");
        *resident_warps = r;
    }
    if (items) *items = b->total;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int32_t nsteps)
{
    if (!b || nsteps < 0) return fail(nullptr, LB_ERR_ARG, "batch is NULL or nsteps < 0");
    {
        cudaError_t e = batch_streams_wait(b, true);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch stream order");
    }
    if (b->row_fetch == 5 && nsteps > 0) {  // one persistent launch for all the steps
        int resident = 0;
        cudaError_t e = lbk::batch_resident_warps(b->storage, 5, b->wpb, &resident);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "occupancy");
        if (b->total > resident || b->total > kMaxPersistItems)
            return fail(nullptr, LB_ERR_ARG,
                        "row fetch 5 needs every work item resident: %d items, %d resident warps (at most %d items)",
                        b->total, resident, kMaxPersistItems);
        e = lbk::launch_batch_persist(b->storage, b->d_desc, b->d_prefix, (int)b->ctxs.size(), b->total, b->wpb,
                                      b->counter, nsteps, b->d_flags, b->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "persistent batch launch");
        b->counter += (unsigned long long)nsteps;
        for (size_t m = 0; m < b->ctxs.size(); ++m) {
            lb_ctx *c = b->ctxs[m];
            c->step = (int64_t)(b->step0[m] + b->counter);
            c->cur = (int)((b->parity0[m] + b->counter) & 1ULL);
        }
        e = batch_streams_wait(b, false);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch stream order");
        return LB_OK;
    }
    int32_t left = nsteps;
    unsigned long long t = b->counter;  // batch step of the next launch
    const bool use_graph = b->graph_steps > 1 && b->stream != nullptr && left >= b->graph_steps;
    if (use_graph && !b->graph_valid) {
        // launches j = 0 .. K - 1 take steps counter + j; the last node adds K
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        for (int j = 0; e == cudaSuccess && j < b->graph_steps; ++j)
            e = lbk::launch_batch(b->storage, b->row_fetch, b->d_desc, b->d_prefix, (int)b->ctxs.size(), b->total,
                                  b->d_ctl, b->wpb, b->blocks, (unsigned long long)j, 1, b->stream);
        if (e == cudaSuccess)
            e = lbk::launch_batch_counter(b->d_ctl, (unsigned long long)b->graph_steps, 1, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
        }
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch graph");
        b->graph_valid = true;
    }
    if (use_graph) {
        cudaError_t e = lbk::launch_batch_counter(b->d_ctl, t, 0, b->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch counter");
        for (; left >= b->graph_steps; left -= b->graph_steps, t += (unsigned long long)b->graph_steps) {
            e = cudaGraphLaunch(b->gexec, b->stream);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch graph launch");
        }
    }
    for (; left > 0; --left, ++t) {
        cudaError_t e = lbk::launch_batch(b->storage, b->row_fetch, b->d_desc, b->d_prefix, (int)b->ctxs.size(), b->total,
                                          b->d_ctl, b->wpb, b->blocks, t, 0, b->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch launch");
    }
    b->counter += (unsigned long long)nsteps;
    for (size_t m = 0; m < b->ctxs.size(); ++m) {
        lb_ctx *c = b->ctxs[m];
        c->step = (int64_t)(b->step0[m] + b->counter);
        c->cur = (int)((b->parity0[m] + b->counter) & 1ULL);
    }
    cudaError_t e = batch_streams_wait(b, false);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch stream order");
    return LB_OK;
}

lb_status lb_batch_diagnostics(lb_batch *b, lb_diag *out)
{
    if (!b || !out) return fail(nullptr, LB_ERR_ARG, "batch or out is NULL");
    cudaError_t e = batch_streams_wait(b, true);
    // each lattice's diagnostics grid as lb_diagnostics would launch it (its
    // launch settings may have changed since the last call)
    const int n = (int)b->ctxs.size();
    const size_t gb = lbk::batch_diag_bytes();
    std::vector<unsigned char> hd((size_t)n * gb);
    std::vector<int> hp((size_t)n + 1, 0);
    for (int m = 0; m < n; ++m) {
        lb_ctx *c = b->ctxs[m];
        const int nb = lbk::batch_fill_diag(c->hp, diag_launch(c), c->partial, hd.data() + (size_t)m * gb);
        if (nb < 1) return fail(nullptr, LB_ERR_ARG, "lattice %d: diagnostics grid too large", m);
        hp[m + 1] = hp[m] + nb;
    }
    if (e == cudaSuccess && (!b->bdiag_uploaded || hd != b->hbdiag || hp != b->hbprefix)) {
        b->hbdiag.swap(hd);
        b->hbprefix.swap(hp);
        e = cudaMemcpyAsync(b->d_bdiag, b->hbdiag.data(), b->hbdiag.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_bprefix, b->hbprefix.data(), b->hbprefix.size() * sizeof(int),
                                cudaMemcpyHostToDevice, b->stream);
        b->bdiag_uploaded = e == cudaSuccess;
    }
    if (e == cudaSuccess)
        e = lbk::launch_batch_diag(b->storage, b->d_desc, b->d_bdiag, b->d_bprefix, n, b->hbprefix[n], b->counter,
                                   (double *)b->d_diag, (int)(kDiagSlot / sizeof(double)), b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->hdiag.data(), b->d_diag, b->hdiag.size(), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = batch_streams_wait(b, false);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch diagnostics");
    for (size_t m = 0; m < b->ctxs.size(); ++m) {
        const char *slot = b->hdiag.data() + m * kDiagSlot;
        int kstatus;
        std::memcpy(&kstatus, slot + 128, sizeof(int));
        fill_diag(b->ctxs[m], reinterpret_cast<const double *>(slot), kstatus, &out[m]);
    }
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch *b)
{
    if (b && b->graph_valid) cudaGraphExecDestroy(b->gexec);
    if (b && b->ev) cudaEventDestroy(b->ev);
    delete b;
    return LB_OK;
}

}  // extern "C"
