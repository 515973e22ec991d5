// Fused time-step kernel of the axisymmetric thermal cascaded LB method
// (arXiv 1806.10241) for sm_103a, plus the field, diagnostic and
// import/export kernels.
//
// Data layout (per lattice, per buffer): 19 planes [q][z][pitch] of the
// storage type: f0..f8, g0..g4, h0..h4 in the velocity order of Eq. 10 and
// Eq. 28.  f and h are stored as deviations from the rest state (w_a rho0,
// w_a T0), g as is, all multiplied by `scale` (1 except for FP16).
//
// Work decomposition: one thread owns one radial column c and marches along
// z over a segment of rows.  Each plane row is loaded once, at the thread's
// own column (aligned, coalesced 128-byte rows per warp).  Pull streaming
// (Eq. 16b, 33b, 46b) shifts in r by warp shuffles and in z by carrying the
// row groups in registers: populations with e_x = +1 come from the previous
// row, e_x = 0 from the current row and e_x = -1 from the next row.  The
// macroscopic fields of the stored (previous time level) state -- the
// moments of the same loaded values -- give the central differences of the
// geometric sources.  A warp covers 32 columns and updates the 30 inner
// ones; lanes 0 and 31 are halo columns.  HBM traffic is therefore 19 loads
// and 19 stores per node update.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace lbk {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int OUT_COLS = 30;  // columns updated per warp
#ifndef LB_MARCH_UNROLL
#define LB_MARCH_UNROLL 2
#endif
constexpr int kMarchUnroll = LB_MARCH_UNROLL;  // rows per unrolled march iteration

// ---- storage conversions ------------------------------------------------

template <typename S, typename C> struct Cvt;
template <> struct Cvt<double, double> {
    static __device__ __forceinline__ double cv(double x) { return x; }
    static __device__ __forceinline__ double ld(const double *p) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Cvt<float, float> {
    static __device__ __forceinline__ float cv(float x) { return x; }
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Cvt<__nv_bfloat16, float> {
    static __device__ __forceinline__ float cv(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <> struct Cvt<__half, float> {
    static __device__ __forceinline__ float cv(__half x) { return __half2float(x); }
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};

// 1/x: the hardware reciprocal for FP32 (|error| <= 2 ulp, far inside the
// FP32 parity tolerances), a correctly rounded division for FP64
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// FP16 storage is scaled (deviations x 1024, away from the subnormal range);
// the other storage types are not, and skip the multiplications.
template <typename S> struct Scaled { static constexpr bool value = std::is_same<S, __half>::value; };

// ---- kernel parameters in the compute type --------------------------------

template <typename C> struct KP {
    int nr, nz, pitch, xper;
    long long plane;
    double r0;
    C om3, om4, omhi, omg, omh;
    C nu, alpha, gbeta, T0, bfx, rho0;
    int planar, sign_lit, explicit_src;
    // sides 0..3; entry 4 the outer segment of a split top (a copy of the top
    // when the top is one segment): columns >= top_split of the top follow it
    int flow[5], swirl[5], heat[5];
    C uwx[5], uwy[5], omega[5], Tw[5];
    int top_split;
    C ramp0, ramp1;       // wall temperature ramp of entry 4: T_w(y) = ramp0 + ramp1 y
    C scale, inv_scale;
    C r0c, roc;           // inner and outer wall radii, rounded once
    // Lateral walls (sides 2 and 3), computed once in the kernel's precision
    // with the operations the per-row rules would do (pair kernels): latf, the
    // moving-wall terms of the populations entering from the wall (f2, f5, f6
    // at the inner side, f4, f7, f8 at the outer); (latgs, latgc) and
    // (laths, lathc), the sign and constant of the scalar rule of g and h,
    // x = s x_own + c; (gha, ghb), the ghost values a q + b of u_x, u_y,
    // u_theta and T for the central differences.
    C latf[2][3], latgs[2], latgc[2], laths[2], lathc[2], gha[2][4], ghb[2][4];
    const float *ytab;    // y[pitch] then 1/y[pitch] (pair kernels)
    // Nusselt and equivalent-conductivity scales per side (diagnostics)
    double nu_scale[4], keq_scale[4];
};

template <typename C> KP<C> make_kp(const HostParams &h)
{
    KP<C> k;
    k.nr = h.nr;
    k.nz = h.nz;
    k.pitch = h.pitch;
    k.plane = h.plane;
    k.xper = h.flow[0] == 2;
    k.r0 = h.r0;
    const double omn = 1.0 / (3.0 * h.nu + 0.5), oma = 1.0 / (3.0 * h.alpha + 0.5);
    k.om3 = (C)h.omega3;
    k.om4 = (C)omn;
    k.omhi = (C)h.omega_hi;
    k.omg = (C)omn;
    k.omh = (C)oma;
    k.nu = (C)h.nu;
    k.alpha = (C)h.alpha;
    k.gbeta = (C)h.g_beta;
    k.T0 = (C)h.T0;
    k.bfx = (C)h.body_fx;
    k.rho0 = (C)h.rho0;
    k.planar = h.planar;
    k.sign_lit = h.sign_literal;
    k.explicit_src = h.explicit_sources;
    for (int s = 0; s < 5; ++s) {
        k.flow[s] = h.flow[s];
        k.swirl[s] = h.swirl[s];
        k.heat[s] = h.heat[s];
        k.uwx[s] = (C)h.uwx[s];
        k.uwy[s] = (C)h.uwy[s];
        k.omega[s] = (C)h.omega[s];
        k.Tw[s] = (C)h.Tw[s];
    }
    k.top_split = h.top_split;
    {  // Sec. 3.6 surface temperature: linear in r from the top's T_w at the
       // split radius to the outer segment's T_w at the outer wall
        const double rs = h.r0 + h.top_split, ro = h.r0 + h.nr;
        const double slope = h.top_split > 0 ? (h.Tw[4] - h.Tw[1]) / (ro - rs) : 0.0;
        k.ramp0 = (C)(h.Tw[1] - slope * rs);
        k.ramp1 = (C)slope;
    }
    k.scale = (C)h.scale;
    k.inv_scale = (C)(1.0 / h.scale);
    k.r0c = (C)h.r0;
    k.roc = (C)(h.r0 + h.nr);
    for (int j = 0; j < 2; ++j) {
        const int sd = 2 + j;
        const C rw = k.rho0, ux = k.uwx[sd], uy = k.uwy[sd], radius = j == 0 ? k.r0c : k.roc;
        const C c9 = (C)(6.0 / 9.0), c36 = (C)(6.0 / 36.0), two = (C)2;
        if (j == 0) {  // Sec. 3.1 moving wall (R11) at the inner side
            k.latf[0][0] = rw * c9 * uy;
            k.latf[0][1] = rw * c36 * (ux + uy);
            k.latf[0][2] = rw * c36 * (-ux + uy);
        } else {
            k.latf[1][0] = rw * c9 * (-uy);
            k.latf[1][1] = rw * c36 * (-ux - uy);
            k.latf[1][2] = rw * c36 * (ux - uy);
        }
        // scalar rules (R12, R13): Dirichlet -x + (2/6) w, odd axis -x, else x
        const C psi_w = k.rho0 * k.omega[sd] * radius, t_w = k.Tw[sd] - k.T0;
        k.latgs[j] = (C)(k.swirl[sd] == 0 || k.swirl[sd] == 2 ? -1 : 1);
        k.latgc[j] = k.swirl[sd] == 0 ? (C)(2.0 / 6.0) * psi_w : (C)0;
        k.laths[j] = (C)(k.heat[sd] == 0 ? -1 : 1);
        k.lathc[j] = k.heat[sd] == 0 ? (C)(2.0 / 6.0) * t_w : (C)0;
        // ghosts (R7): wall 2 q_w - q, zero flux q, axis u_x, T even, u_y, u_theta odd
        const bool axis = k.flow[sd] == 1;
        k.gha[j][0] = (C)(axis ? 1 : -1);
        k.ghb[j][0] = axis ? (C)0 : two * ux;
        k.gha[j][1] = (C)-1;
        k.ghb[j][1] = axis ? (C)0 : two * uy;
        k.gha[j][2] = (C)(k.swirl[sd] == 0 || k.swirl[sd] == 2 ? -1 : 1);
        k.ghb[j][2] = k.swirl[sd] == 0 ? two * k.omega[sd] * radius : (C)0;
        k.gha[j][3] = (C)(k.heat[sd] == 0 ? -1 : 1);
        k.ghb[j][3] = k.heat[sd] == 0 ? two * k.Tw[sd] : (C)0;
    }
    k.ytab = h.ytab;
    // Nusselt normalisation (Sec. 3.2): lateral walls -R_w / (H dT), end
    // walls -(H / dT) * 2 / (R_o^2 - R_i^2); dT from the Dirichlet values.
    double tmin = 0, tmax = 0;
    int nd = 0;
    for (int s = 0; s < 5; ++s)
        if ((h.heat[s] == 0 || h.heat[s] == 4) && (s < 4 || h.top_split > 0)) {
            if (nd == 0 || h.Tw[s] < tmin) tmin = h.Tw[s];
            if (nd == 0 || h.Tw[s] > tmax) tmax = h.Tw[s];
            ++nd;
        }
    const double dT = (nd >= 2 && tmax > tmin) ? tmax - tmin : 1.0;
    const double H = h.nz, Ri = h.r0, Ro = h.r0 + h.nr;
    k.nu_scale[0] = k.nu_scale[1] = -(H / dT) * 2.0 / (Ro * Ro - Ri * Ri);
    k.nu_scale[2] = -Ri / (H * dT);
    k.nu_scale[3] = -Ro / (H * dT);
    // mean equivalent conductivity of a lateral wall of an annulus (Sec. 3.5):
    // ln(R_o / R_i) / (H dT) times the sum over z of -R_w dT/dr
    const double lg = Ri > 0.0 ? std::log(Ro / Ri) : 0.0;
    k.keq_scale[0] = k.keq_scale[1] = 0.0;
    k.keq_scale[2] = -Ri * lg / (H * dT);
    k.keq_scale[3] = -Ro * lg / (H * dT);
    return k;
}

// ---- per-row helpers -------------------------------------------------------

// Plane indices
enum { F0 = 0, G0 = 9, H0 = 14 };

template <typename C> struct PM {  // macroscopic fields of the stored state
    C rd, ux, uy, ut, T;
};

template <typename S, typename C> __device__ __forceinline__ PM<C> moments(const C v[NQ], const KP<C> &k)
{
    // rho = rho0 + sum f_dev, j = sum f_dev e, psi = sum g, T = T0 + sum h_dev
    C rd = v[0] + v[1] + v[2] + v[3] + v[4] + v[5] + v[6] + v[7] + v[8];
    C jx = v[1] - v[3] + v[5] - v[6] - v[7] + v[8];
    C jy = v[2] - v[4] + v[5] + v[6] - v[7] - v[8];
    C ps = v[9] + v[10] + v[11] + v[12] + v[13];
    C td = v[14] + v[15] + v[16] + v[17] + v[18];
    if (Scaled<S>::value) {
        const C is = k.inv_scale;
        rd *= is;
        jx *= is;
        jy *= is;
        ps *= is;
        td *= is;
    }
    const C ir = rcp(k.rho0 + rd);
    PM<C> m;
    m.rd = rd;
    m.ux = jx * ir;
    m.uy = jy * ir;
    m.ut = ps * ir;
    m.T = k.T0 + td;
    return m;
}

template <typename C> __device__ __forceinline__ C shup(C v) { return __shfl_up_sync(FULL, v, 1); }
template <typename C> __device__ __forceinline__ C shdn(C v) { return __shfl_down_sync(FULL, v, 1); }

// Row groups (already shifted in r):
//   XM (from row i-1): f1, f5, f8, g1, h1
//   X0 (from row i)  : f0, f2, f4, g0, g2, g4, h0, h2, h4
//   XP (from row i+1): f3, f6, f7, g3, h3
template <typename C>
__device__ __forceinline__ void groups(const C v[NQ], C xm[5], C x0[9], C xp[5])
{
    xm[0] = v[1];
    xm[1] = shup(v[5]);
    xm[2] = shdn(v[8]);
    xm[3] = v[G0 + 1];
    xm[4] = v[H0 + 1];
    x0[0] = v[0];
    x0[1] = shup(v[2]);
    x0[2] = shdn(v[4]);
    x0[3] = v[G0 + 0];
    x0[4] = shup(v[G0 + 2]);
    x0[5] = shdn(v[G0 + 4]);
    x0[6] = v[H0 + 0];
    x0[7] = shup(v[H0 + 2]);
    x0[8] = shdn(v[H0 + 4]);
    xp[0] = v[3];
    xp[1] = shup(v[6]);
    xp[2] = shdn(v[7]);
    xp[3] = v[G0 + 3];
    xp[4] = v[H0 + 3];
}

template <typename S, typename C>
__device__ __forceinline__ void load_row(const S *__restrict__ src, const KP<C> &k, int row, int col,
                                         C v[NQ])
{
    const S *p = src + (long long)row * k.pitch + col;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = Cvt<S, C>::ld(p + q * k.plane);
}

// raw (unconverted) loads of one row, issued ahead of their use
template <typename S, typename C>
__device__ __forceinline__ void load_raw(const S *__restrict__ src, const KP<C> &k, int row, int col, S r[NQ])
{
    const S *p = src + (long long)row * k.pitch + col;
#pragma unroll
    for (int q = 0; q < NQ; ++q) r[q] = p[q * k.plane];
}

template <typename S, typename C>
__device__ __forceinline__ C own(const S *__restrict__ src, const KP<C> &k, int q, int row, int col)
{
    return Cvt<S, C>::ld(src + q * k.plane + (long long)row * k.pitch + col);
}

// psi on a rotating wall: rho0 * omega * radius (side 4: the top's outer segment)
template <typename C> __device__ __forceinline__ C wall_psi(const KP<C> &k, int side, C y)
{
    const C radius = (side <= 1 || side == 4) ? y : (side == 2 ? k.r0c : k.roc);
    return k.rho0 * k.omega[side] * radius;
}

// the entry of an end wall at column col: the top's outer segment (4) for
// columns >= top_split of a split top, else the side itself
template <typename C> __device__ __forceinline__ int end_seg(const KP<C> &k, int side, int col)
{
    return (side == 1 && k.top_split > 0 && col >= k.top_split) ? 4 : side;
}

// wall temperature of an end-wall entry at the column radius y (the ramp of
// Sec. 3.6 on entry 4 with heat type 4), and the entry's h rule with the ramp
// read as Dirichlet
template <typename C> __device__ __forceinline__ C end_T(const KP<C> &k, int seg, C y)
{
    return k.heat[seg] == 4 ? k.ramp0 + k.ramp1 * y : k.Tw[seg];
}
template <typename C> __device__ __forceinline__ int heat_rule(const KP<C> &k, int seg)
{
    return k.heat[seg] == 4 ? 0 : k.heat[seg];
}
// a side whose wall temperatures enter its Nusselt number (Sec. 3.2): a
// Dirichlet side, or a top any of whose segments holds a wall temperature
template <typename C> __device__ __forceinline__ bool wall_heated(const KP<C> &k, int sd)
{
    if (sd == 1 && k.top_split > 0) return k.heat[1] == 0 || k.heat[4] == 0 || k.heat[4] == 4;
    return k.heat[sd] == 0;
}

// Scalar boundary value for the population entering from a wall (Sec. 3):
// Dirichlet anti-bounce-back -x_own + 2 w s_w (w = 1/6, deviation form for h),
// Neumann / even axis bounce-back x_own, odd axis (psi) -x_own.
template <typename C>
__device__ __forceinline__ C scalar_bc(int bc, C own_v, C wall_dev_scaled, bool odd_axis)
{
    if (bc == 0) return -own_v + (C)(2.0 / 6.0) * wall_dev_scaled;
    if (bc == 2 && odd_axis) return -own_v;
    return own_v;
}

// ---- the node update -------------------------------------------------------

template <typename C> struct NodeOut {
    C f[9], g[5], h[5];
    C rho, ux, uy, ut, T;  // pre-collision fields
};

// Pulled (deviation, unscaled) values in fv/gv/hv; gradient inputs.
template <typename C>
__device__ __forceinline__ void update_node(const KP<C> &k, C y, C iy, C fv[9], C gv[5], C hv[5],
                                            C dxuy, C dyux, C dyuy, C dyut, C dyT, NodeOut<C> &o)
{
    // output moments, Eq. 18, 35, 47 (deviation form: rest parts cancel)
    const C rdo = fv[0] + fv[1] + fv[2] + fv[3] + fv[4] + fv[5] + fv[6] + fv[7] + fv[8];
    const C jxo = fv[1] - fv[3] + fv[5] - fv[6] - fv[7] + fv[8];
    const C jyo = fv[2] - fv[4] + fv[5] + fv[6] - fv[7] - fv[8];
    const C pso = gv[0] + gv[1] + gv[2] + gv[3] + gv[4];
    const C tdo = hv[0] + hv[1] + hv[2] + hv[3] + hv[4];

    // sources (Eq. 4a-4c, 5, 7, 9) at the pre-collision state, two sweeps.
    // Written per unit of the swept state (rd, j, psi, td): with mu = rho nu,
    //   F_x^A = -j_x u_y / y + rho nu (d_x u_y + d_y u_x) / y
    //   F_y^A = psi^2 / (rho y) - j_y u_y / y + rho 2 nu d_y u_y / y - 2 nu j_y / y^2
    //   S_psi = -2 u_y psi / y + rho nu d_y u_theta / y - nu psi / y^2
    //   S_phi = -u_y T / y + alpha d_y T / y
    // so the gradient factors are formed once per node.
    C rd = rdo, jx = jxo, jy = jyo, ps = pso, td = tdo;
    C MA = 0, Fx = 0, Fy = 0, Sps = 0, Sph = 0;
    const bool geo = !k.planar;
    const C Gx = geo ? k.nu * (dxuy + dyux) * iy : (C)0;
    const C Gy = geo ? (C)2 * k.nu * dyuy * iy : (C)0;
    const C Gw = geo ? k.nu * dyut * iy : (C)0;
    const C Gt = geo ? k.alpha * dyT * iy : (C)0;
    const C iy2nu = geo ? k.nu * iy * iy : (C)0;
    const C gy = geo ? iy : (C)0;
    const C Fb = k.rho0 * k.gbeta;
    const int sweeps = k.explicit_src ? 1 : 2;
    for (int sw = 0; sw < sweeps; ++sw) {
        const C r = k.rho0 + rd, ir = rcp(r);
        const C uyy = jy * ir * gy;  // u_y / y
        const C ph = k.T0 + td;
        const C FAx = -jx * uyy + r * Gx;
        const C FAy = (ps * ps - jy * jy) * ir * gy + r * Gy - (C)2 * jy * iy2nu;
        Sps = (C)-2 * uyy * ps + r * Gw - iy2nu * ps;
        Sph = -uyy * ph + Gt;
        Fx = FAx + Fb * td + k.bfx;
        Fy = FAy;
        jx = jxo + (C)0.5 * Fx;
        jy = jyo + (C)0.5 * Fy;
        ps = pso + (C)0.5 * Sps;
        td = tdo + (C)0.5 * Sph;
        // M^A = -j_y / y, from the newest momentum (from the output momentum
        // in the single-evaluation mode)
        MA = -(k.explicit_src ? jyo : jy) * gy;
        rd = rdo + (C)0.5 * MA;
    }
    const C r = k.rho0 + rd, ir = rcp(r);
    const C ux = jx * ir, uy = jy * ir;
    const C phi = k.T0 + td;
    o.rho = r;
    o.ux = ux;
    o.uy = uy;
    o.ut = ps * ir;
    o.T = phi;

    // D2Q9 cascaded collision, Eq. 17 (raw moments of the streamed f; the
    // rest-state parts rho0/3, rho0/9 written out)
    const C third = (C)(1.0 / 3.0);
    const C Dxx = fv[1] + fv[3] + fv[5] + fv[6] + fv[7] + fv[8];
    const C Dyy = fv[2] + fv[4] + fv[5] + fv[6] + fv[7] + fv[8];
    const C Dxy = fv[5] - fv[6] + fv[7] - fv[8];
    const C Dxxy = fv[5] + fv[6] - fv[7] - fv[8];
    const C Dxyy = fv[5] - fv[6] - fv[7] + fv[8];
    const C Dxxyy = fv[5] + fv[6] + fv[7] + fv[8];
    const C Kxx = k.rho0 * third + Dxx, Kyy = k.rho0 * third + Dyy;
    const C ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const C p3 = k.om3 * (C)(1.0 / 12.0) * ((C)(2.0 / 3.0) * rd + r * (ux2 + uy2) - (Dxx + Dyy));
    const C p4 = k.om4 * (C)0.25 * (r * (ux2 - uy2) - (Dxx - Dyy));
    const C p5 = k.om4 * (C)0.25 * (r * uxy - Dxy);
    const C q34p = (C)3 * p3 + p4, q34m = (C)3 * p3 - p4;
    const C p6 = k.omhi * (C)0.25 * ((C)2 * r * ux2 * uy + Dxxy - (C)2 * ux * Dxy - uy * Kxx)
                 - (C)0.5 * uy * q34p - (C)2 * ux * p5;
    const C p7 = k.omhi * (C)0.25 * ((C)2 * r * ux * uy2 + Dxyy - (C)2 * uy * Dxy - ux * Kyy)
                 - (C)0.5 * ux * q34m - (C)2 * uy * p5;
    const C p8 = k.omhi * (C)0.25 *
                     (rd * (C)(1.0 / 9.0) + (C)3 * r * ux2 * uy2 -
                      (Dxxyy - (C)2 * ux * Dxyy - (C)2 * uy * Dxxy + ux2 * Kyy + uy2 * Kxx + (C)4 * uxy * Dxy)) -
                 (C)2 * p3 - (C)0.5 * uy2 * q34p - (C)0.5 * ux2 * q34m - (C)4 * uxy * p5 - (C)2 * uy * p6 -
                 (C)2 * ux * p7;
    // source moments, Eq. 26
    const C p0 = MA * (C)(1.0 / 9.0), p1 = Fx * (C)(1.0 / 6.0), p2 = Fy * (C)(1.0 / 6.0);
    // back-transform, Eq. 27
    o.f[0] = fv[0] + (p0 - (C)4 * (p3 - p8));
    o.f[1] = fv[1] + (p0 + p1 - p3 + p4 + (C)2 * (p7 - p8));
    o.f[2] = fv[2] + (p0 + p2 - p3 - p4 + (C)2 * (p6 - p8));
    o.f[3] = fv[3] + (p0 - p1 - p3 + p4 - (C)2 * (p7 + p8));
    o.f[4] = fv[4] + (p0 - p2 - p3 - p4 - (C)2 * (p6 + p8));
    o.f[5] = fv[5] + (p0 + p1 + p2 + (C)2 * p3 + p5 - p6 - p7 + p8);
    o.f[6] = fv[6] + (p0 - p1 + p2 + (C)2 * p3 - p5 - p6 + p7 + p8);
    o.f[7] = fv[7] + (p0 - p1 - p2 + (C)2 * p3 + p5 + p6 + p7 + p8);
    o.f[8] = fv[8] + (p0 + p1 - p2 + (C)2 * p3 - p5 + p6 - p7 + p8);

    // D2Q5 cascaded collisions, Eq. 34 (psi) and Eq. 49 (T), with the sign
    // that makes the equilibrium a fixed point unless sign_lit is set
    const C sg = k.sign_lit ? (C)1 : (C)-1;
    const C uu = ux2 + uy2, ud = ux2 - uy2;
    {
        const C kx = gv[1] - gv[3], ky = gv[2] - gv[4];
        const C kxx = gv[1] + gv[3], kyy = gv[2] + gv[4];
        const C q1 = k.omg * (C)0.5 * (ps * ux - kx);
        const C q2 = k.omg * (C)0.5 * (ps * uy - ky);
        const C q3 = k.omhi * (C)0.25 * ((C)(2.0 / 3.0) * ps - (kxx + kyy) + (C)2 * (ux * kx + uy * ky) + sg * uu * ps)
                     + ux * q1 + uy * q2;
        const C q4 = k.omhi * (C)0.25 * (-(kxx - kyy) + (C)2 * (ux * kx - uy * ky) + sg * ud * ps) + ux * q1 - uy * q2;
        const C q0 = Sps * (C)0.2;  // Eq. 41
        // Eq. 42
        o.g[0] = gv[0] + (q0 - (C)4 * q3);
        o.g[1] = gv[1] + (q0 + q1 + q3 + q4);
        o.g[2] = gv[2] + (q0 + q2 + q3 - q4);
        o.g[3] = gv[3] + (q0 - q1 + q3 + q4);
        o.g[4] = gv[4] + (q0 - q2 + q3 - q4);
    }
    {
        const C kx = hv[1] - hv[3], ky = hv[2] - hv[4];
        const C Hxx = hv[1] + hv[3], Hyy = hv[2] + hv[4];
        const C r1 = k.omh * (C)0.5 * (phi * ux - kx);
        const C r2 = k.omh * (C)0.5 * (phi * uy - ky);
        const C r3 = k.omhi * (C)0.25 * ((C)(2.0 / 3.0) * td - (Hxx + Hyy) + (C)2 * (ux * kx + uy * ky) + sg * uu * phi)
                     + ux * r1 + uy * r2;
        const C r4 = k.omhi * (C)0.25 * (-(Hxx - Hyy) + (C)2 * (ux * kx - uy * ky) + sg * ud * phi) + ux * r1 - uy * r2;
        const C r0 = Sph * (C)0.2;  // Eq. 51
        // Eq. 52
        o.h[0] = hv[0] + (r0 - (C)4 * r3);
        o.h[1] = hv[1] + (r0 + r1 + r3 + r4);
        o.h[2] = hv[2] + (r0 + r2 + r3 - r4);
        o.h[3] = hv[3] + (r0 - r1 + r3 + r4);
        o.h[4] = hv[4] + (r0 - r2 + r3 - r4);
    }
}

// ---- diagnostics accumulator ------------------------------------------------

struct DiagAcc {
    double mass_dev, mass_r_dev, tsum, umax, bad;
};

// ---- the march ---------------------------------------------------------------

template <typename S, typename C, int MODE>
__device__ __forceinline__ void march(const KP<C> &k, const S *__restrict__ src, S *__restrict__ dst,
                                      double *__restrict__ fout, int fout_row0, int fout_rows, int c,
                                      int row_s, int row_e, DiagAcc *acc)
{
    const int lane = threadIdx.x & 31;
    const int nr = k.nr, nz = k.nz;
    const int cl = c < 0 ? 0 : (c >= nr ? nr - 1 : c);
    const bool out_lane = lane >= 1 && lane <= OUT_COLS && c < nr;
    const bool at_c0 = c == 0, at_cN = c == nr - 1;
    const bool edge_warp = __any_sync(FULL, at_c0 || at_cN);
    // radius of the column, its inverse computed in FP64 and rounded once
    const double yd = k.r0 + cl + 0.5;
    const C y = (C)yd, iy = (C)(1.0 / yd);
    const C is = k.inv_scale, sc = k.scale;

    C v[NQ];
    C xm_prev[5], xm_cur[5], x0_cur[9];
    PM<C> pm_cur;
    C uy_prev = 0;
    bool has_m;

    // prologue: rows s-1 and s
    if (row_s > 0 || k.xper) {
        const int rm = row_s > 0 ? row_s - 1 : nz - 1;
        load_row<S, C>(src, k, rm, cl, v);
        C x0t[9], xpt[5];
        groups<C>(v, xm_prev, x0t, xpt);
        uy_prev = moments<S, C>(v, k).uy;
        has_m = true;
    } else {
        has_m = false;
#pragma unroll
        for (int q = 0; q < 5; ++q) xm_prev[q] = 0;
    }
    // software pipeline: the raw values of row i+1 are loaded during the
    // iteration for row i-1, so a row's DRAM latency overlaps the previous
    // row's arithmetic
    S nb[NQ];
    if ((row_s + 1 < nz) || k.xper) load_raw<S, C>(src, k, row_s + 1 < nz ? row_s + 1 : 0, cl, nb);
    {
        load_row<S, C>(src, k, row_s, cl, v);
        C xpt[5];
        groups<C>(v, xm_cur, x0_cur, xpt);
        pm_cur = moments<S, C>(v, k);
    }

#pragma unroll kMarchUnroll
    for (int i = row_s; i < row_e; ++i) {
        const bool has_p = (i + 1 < nz) || k.xper;
        C xp_n[5], x0_n[9], xm_n[5];
        PM<C> pm_n;
        if (has_p) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] = Cvt<S, C>::cv(nb[q]);
        }
        if (i + 1 < row_e && ((i + 2 < nz) || k.xper))
            load_raw<S, C>(src, k, i + 2 < nz ? i + 2 : i + 2 - nz, cl, nb);
        if (has_p) {
            groups<C>(v, xm_n, x0_n, xp_n);
            pm_n = moments<S, C>(v, k);
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) xp_n[q] = xm_n[q] = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) x0_n[q] = 0;
            pm_n = pm_cur;
        }

        // pulled values (scaled storage units)
        C fv[9], gv[5], hv[5];
        fv[1] = xm_prev[0]; fv[5] = xm_prev[1]; fv[8] = xm_prev[2]; gv[1] = xm_prev[3]; hv[1] = xm_prev[4];
        fv[0] = x0_cur[0]; fv[2] = x0_cur[1]; fv[4] = x0_cur[2];
        gv[0] = x0_cur[3]; gv[2] = x0_cur[4]; gv[4] = x0_cur[5];
        hv[0] = x0_cur[6]; hv[2] = x0_cur[7]; hv[4] = x0_cur[8];
        fv[3] = xp_n[0]; fv[6] = xp_n[1]; fv[7] = xp_n[2]; gv[3] = xp_n[3]; hv[3] = xp_n[4];

        // lateral boundaries (Sec. 3): the population entering from r < r0 or
        // r > r0 + nr is rebuilt from the node's own stored values
        if (edge_warp) {
            if (at_c0) {
                const int sd = 2;
                const C rw = k.rho0 * sc;
                if (k.flow[sd] == 1) {  // axis: mirror images
                    fv[2] = own<S, C>(src, k, 4, i, 0);
                    if (has_m) fv[5] = own<S, C>(src, k, 8, i > 0 ? i - 1 : nz - 1, 0);
                    if (has_p) fv[6] = own<S, C>(src, k, 7, i + 1 < nz ? i + 1 : 0, 0);
                } else {  // wall: bounce-back + moving-wall term 6 w rho0 (e.u_w)
                    const C ux_w = k.uwx[sd], uy_w = k.uwy[sd];
                    fv[2] = own<S, C>(src, k, 4, i, 0) + rw * (C)(6.0 / 9.0) * uy_w;
                    fv[5] = own<S, C>(src, k, 7, i, 0) + rw * (C)(6.0 / 36.0) * (ux_w + uy_w);
                    fv[6] = own<S, C>(src, k, 8, i, 0) + rw * (C)(6.0 / 36.0) * (-ux_w + uy_w);
                }
                gv[2] = scalar_bc<C>(k.swirl[sd], own<S, C>(src, k, G0 + 4, i, 0), wall_psi<C>(k, sd, y) * sc, true);
                hv[2] = scalar_bc<C>(k.heat[sd], own<S, C>(src, k, H0 + 4, i, 0), (k.Tw[sd] - k.T0) * sc, false);
            }
            if (at_cN) {
                const int sd = 3;
                const C rw = k.rho0 * sc;
                const C ux_w = k.uwx[sd], uy_w = k.uwy[sd];
                fv[4] = own<S, C>(src, k, 2, i, nr - 1) + rw * (C)(6.0 / 9.0) * (-uy_w);
                fv[7] = own<S, C>(src, k, 5, i, nr - 1) + rw * (C)(6.0 / 36.0) * (-ux_w - uy_w);
                fv[8] = own<S, C>(src, k, 6, i, nr - 1) + rw * (C)(6.0 / 36.0) * (ux_w - uy_w);
                gv[4] = scalar_bc<C>(k.swirl[sd], own<S, C>(src, k, G0 + 2, i, nr - 1), wall_psi<C>(k, sd, y) * sc, true);
                hv[4] = scalar_bc<C>(k.heat[sd], own<S, C>(src, k, H0 + 2, i, nr - 1), (k.Tw[sd] - k.T0) * sc, false);
            }
        }
        // end walls (rows 0 and nz-1 unless periodic); they win in corners.  A
        // free surface (Sec. 3.6) reflects f specularly: the population that
        // left the neighbour column towards the wall, e_x reversed; at a corner
        // column the lateral side's rule for the node itself
        if (!has_m) {
            const int sd = end_seg(k, 0, cl);
            const C rw = k.rho0 * sc, ux_w = k.uwx[sd], uy_w = k.uwy[sd];
            if (k.flow[sd] == 3) {
                fv[1] = own<S, C>(src, k, 3, i, cl);
                fv[5] = at_c0 ? own<S, C>(src, k, 7, i, 0) +
                                    (k.flow[2] == 1 ? (C)0 : rw * (C)(6.0 / 36.0) * (k.uwx[2] + k.uwy[2]))
                              : own<S, C>(src, k, 6, i, cl > 0 ? cl - 1 : 0);
                fv[8] = at_cN ? own<S, C>(src, k, 6, i, cl) + rw * (C)(6.0 / 36.0) * (k.uwx[3] - k.uwy[3])
                              : own<S, C>(src, k, 7, i, cl + 1 < nr ? cl + 1 : cl);
            } else {
                fv[1] = own<S, C>(src, k, 3, i, cl) + rw * (C)(6.0 / 9.0) * ux_w;
                fv[5] = own<S, C>(src, k, 7, i, cl) + rw * (C)(6.0 / 36.0) * (ux_w + uy_w);
                fv[8] = own<S, C>(src, k, 6, i, cl) + rw * (C)(6.0 / 36.0) * (ux_w - uy_w);
            }
            gv[1] = scalar_bc<C>(k.swirl[sd], own<S, C>(src, k, G0 + 3, i, cl), wall_psi<C>(k, sd, y) * sc, true);
            hv[1] = scalar_bc<C>(heat_rule(k, sd), own<S, C>(src, k, H0 + 3, i, cl), (end_T(k, sd, y) - k.T0) * sc,
                                 false);
        }
        if (!has_p) {
            const int sd = end_seg(k, 1, cl);
            const C rw = k.rho0 * sc, ux_w = k.uwx[sd], uy_w = k.uwy[sd];
            if (k.flow[sd] == 3) {
                fv[3] = own<S, C>(src, k, 1, i, cl);
                fv[6] = at_c0 ? own<S, C>(src, k, 8, i, 0) +
                                    (k.flow[2] == 1 ? (C)0 : rw * (C)(6.0 / 36.0) * (-k.uwx[2] + k.uwy[2]))
                              : own<S, C>(src, k, 5, i, cl > 0 ? cl - 1 : 0);
                fv[7] = at_cN ? own<S, C>(src, k, 5, i, cl) + rw * (C)(6.0 / 36.0) * (-k.uwx[3] - k.uwy[3])
                              : own<S, C>(src, k, 8, i, cl + 1 < nr ? cl + 1 : cl);
            } else {
                fv[3] = own<S, C>(src, k, 1, i, cl) + rw * (C)(6.0 / 9.0) * (-ux_w);
                fv[6] = own<S, C>(src, k, 8, i, cl) + rw * (C)(6.0 / 36.0) * (-ux_w + uy_w);
                fv[7] = own<S, C>(src, k, 5, i, cl) + rw * (C)(6.0 / 36.0) * (-ux_w - uy_w);
            }
            gv[3] = scalar_bc<C>(k.swirl[sd], own<S, C>(src, k, G0 + 1, i, cl), wall_psi<C>(k, sd, y) * sc, true);
            hv[3] = scalar_bc<C>(heat_rule(k, sd), own<S, C>(src, k, H0 + 1, i, cl), (end_T(k, sd, y) - k.T0) * sc,
                                 false);
        }
        if (Scaled<S>::value) {
#pragma unroll
            for (int q = 0; q < 9; ++q) fv[q] *= is;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                gv[q] *= is;
                hv[q] *= is;
            }
        }

        // central differences of the stored-state fields, with ghosts
        // (a free surface: no shear, u_y even across it)
        const int sb = end_seg(k, 0, cl), st = end_seg(k, 1, cl);
        const C uy_xm = has_m ? uy_prev : (k.flow[sb] == 3 ? pm_cur.uy : (C)2 * k.uwy[sb] - pm_cur.uy);
        const C uy_xp = has_p ? pm_n.uy : (k.flow[st] == 3 ? pm_cur.uy : (C)2 * k.uwy[st] - pm_cur.uy);
        C ux_l = shup(pm_cur.ux), uy_l = shup(pm_cur.uy), ut_l = shup(pm_cur.ut), T_l = shup(pm_cur.T);
        C ux_r = shdn(pm_cur.ux), uy_r = shdn(pm_cur.uy), ut_r = shdn(pm_cur.ut), T_r = shdn(pm_cur.T);
        if (edge_warp) {
            if (at_c0) {
                const int sd = 2;
                if (k.flow[sd] == 1) {
                    ux_l = pm_cur.ux;
                    uy_l = -pm_cur.uy;
                } else {
                    ux_l = (C)2 * k.uwx[sd] - pm_cur.ux;
                    uy_l = (C)2 * k.uwy[sd] - pm_cur.uy;
                }
                const int sw = k.swirl[sd], ht = k.heat[sd];
                ut_l = sw == 2 ? -pm_cur.ut : (sw == 0 ? (C)2 * k.omega[sd] * (C)k.r0 - pm_cur.ut : pm_cur.ut);
                T_l = ht == 0 ? (C)2 * k.Tw[sd] - pm_cur.T : pm_cur.T;
            }
            if (at_cN) {
                const int sd = 3;
                ux_r = (C)2 * k.uwx[sd] - pm_cur.ux;
                uy_r = (C)2 * k.uwy[sd] - pm_cur.uy;
                const int sw = k.swirl[sd], ht = k.heat[sd];
                ut_r = sw == 0 ? (C)2 * k.omega[sd] * (C)(k.r0 + k.nr) - pm_cur.ut : pm_cur.ut;
                T_r = ht == 0 ? (C)2 * k.Tw[sd] - pm_cur.T : pm_cur.T;
            }
        }
        const C dxuy = (C)0.5 * (uy_xp - uy_xm);
        const C dyux = (C)0.5 * (ux_r - ux_l);
        const C dyuy = (C)0.5 * (uy_r - uy_l);
        const C dyut = (C)0.5 * (ut_r - ut_l);
        const C dyT = (C)0.5 * (T_r - T_l);

        NodeOut<C> o;
        update_node<C>(k, y, iy, fv, gv, hv, dxuy, dyux, dyuy, dyut, dyT, o);

        if (MODE == MODE_STEP) {
            if (out_lane) {
                S *p = dst + (long long)i * k.pitch + c;
                const C m = Scaled<S>::value ? sc : (C)1;
#pragma unroll
                for (int q = 0; q < 9; ++q) Cvt<S, C>::st(p + q * k.plane, Scaled<S>::value ? o.f[q] * m : o.f[q]);
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    Cvt<S, C>::st(p + (G0 + q) * k.plane, Scaled<S>::value ? o.g[q] * m : o.g[q]);
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    Cvt<S, C>::st(p + (H0 + q) * k.plane, Scaled<S>::value ? o.h[q] * m : o.h[q]);
            }
        } else if (MODE == MODE_FIELDS) {
            if (out_lane) {
                const long long n = (long long)fout_rows * nr;  // plane stride of the output chunk
                double *p = fout + (long long)(i - fout_row0) * nr + c;
                p[0] = (double)o.rho;
                p[n] = (double)o.ux;
                p[2 * n] = (double)o.uy;
                p[3 * n] = (double)o.ut;
                p[4 * n] = (double)o.T;
            }
        } else {  // MODE_DIAG
            if (out_lane) {
                const double rdp = (double)pm_cur.rd;
                acc->mass_dev += rdp;
                acc->mass_r_dev += rdp * yd;
                acc->tsum += (double)o.T;
                const double um = sqrt((double)o.ux * (double)o.ux + (double)o.uy * (double)o.uy);
                acc->umax = fmax(acc->umax, um);
                const bool finite = isfinite((double)o.rho) && isfinite((double)o.ux) &&
                                    isfinite((double)o.uy) && isfinite((double)o.ut) &&
                                    isfinite((double)o.T);
                if (!finite || o.rho < (C)0.5 || o.rho > (C)1.5) acc->bad = 1.0;
                if (MODE == MODE_DIAG) {
                    fout[(long long)i * nr + c] = (double)o.T;  // for the wall fluxes
                } else {
                    // wall-adjacent temperatures only: rows 0, 1, nz-2, nz-1
                    // (4 x nr values), then columns 0, 1, nr-2, nr-1 (4 x nz)
                    const double T = (double)o.T;
                    if (i == 0) fout[c] = T;
                    if (i == 1) fout[nr + c] = T;
                    if (i == nz - 2) fout[2 * nr + c] = T;
                    if (i == nz - 1) fout[3 * nr + c] = T;
                    double *cs = fout + 4LL * nr;
                    if (c == 0) cs[i] = T;
                    if (c == 1) cs[nz + i] = T;
                    if (c == nr - 2) cs[2LL * nz + i] = T;
                    if (c == nr - 1) cs[3LL * nz + i] = T;
                }
            }
        }

        // rotate the row window
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            xm_prev[q] = xm_cur[q];
            xm_cur[q] = xm_n[q];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) x0_cur[q] = x0_n[q];
        uy_prev = pm_cur.uy;
        pm_cur = pm_n;
        has_m = true;
    }
}

#include "lb_pair.cuh"

// Programmatic dependent launch (sm_90+): the kernels of consecutive steps
// are launched with programmatic stream serialisation, so a step's blocks
// may start while the previous step's last blocks run.  Each block first
// allows the next launch to begin, then waits until every earlier grid of
// the stream has completed and its writes are visible, before it reads or
// writes any distribution.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void grid_dependency_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_trigger_and_wait()
{
    grid_dependency_trigger();
    grid_dependency_wait();
}

template <typename S, typename C>
__device__ __forceinline__ void step_body(const KP<C> &k, const S *__restrict__ src, S *__restrict__ dst,
                                          int seg_rows, int nwin)
{
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= nwin) return;  // whole warps only
    const int c = warp * OUT_COLS - 1 + (threadIdx.x & 31);
    const int s = blockIdx.y * seg_rows;
    const int e = min(k.nz, s + seg_rows);
    grid_dependency_trigger_and_wait();
    march<S, C, MODE_STEP>(k, src, dst, nullptr, 0, 0, c, s, e, nullptr);
}

// FP64 step (the GPU FP64 reference path): the scalar march, 30 columns per warp
template <typename S, typename C>
__global__ void __maxnreg__(255) k_step64(KP<C> k, const S *__restrict__ src, S *__restrict__ dst,
                                          int seg_rows, int nwin)
{
    step_body<S, C>(k, src, dst, seg_rows, nwin);
}

// Block of a step grid in traversal order: every other step (rev = 1) the
// blocks take the lattice from its last row segment back to its first.  A step
// then starts on the rows the previous step wrote last, which are still in
// the L2 (129 MB against the 319 MB of the 1024 x 2048 FP32 lattice); the
// results do not depend on the order.
__device__ __forceinline__ void step_block(int rev, int &bx, int &by)
{
    const unsigned nb = gridDim.x * gridDim.y, b0 = blockIdx.y * gridDim.x + blockIdx.x;
    const unsigned b = rev ? nb - 1u - b0 : b0;
    bx = (int)(b % gridDim.x);
    by = (int)(b / gridDim.x);
}

// FP32-compute step on column pairs (lb_pair.cuh): 64 aligned columns per warp
#ifndef LB_STEP2_MAXREG
#define LB_STEP2_MAXREG 232
#endif
template <typename S>
__global__ void __maxnreg__(LB_STEP2_MAXREG) k_step2(KP<float> k, const S *__restrict__ src, S *__restrict__ dst,
                                                     int seg_rows, int nwin2, uint32_t salt, int rev)
{
    int bx, by;
    step_block(rev, bx, by);
    const int warp = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= nwin2) return;
    const int lane = threadIdx.x & 31;
    const int s = by * seg_rows;
    const int e = min(k.nz, s + seg_rows);
    const int A = warp * 64 + 2 * lane;
    const int Amax = (k.nr - 1) & ~1;
    int hcol = lane == 0 ? warp * 64 - 1 : warp * 64 + 64;
    hcol = hcol < 0 ? 0 : (hcol >= k.nr ? k.nr - 1 : hcol);
    RowDirect<S> rs{src, &k, A <= Amax ? A : Amax, hcol, (s > 0 || k.xper) ? s - 1 : s, k.nz, 0,
                    lane == 0 || lane == 31};
    grid_dependency_trigger_and_wait();
    march2<S>(k, src, dst, warp * 64, s, e, salt, rs);
}

// The same step with the rows of each warp fetched by TMA into a ring of
// shared-memory stages (one bulk tensor copy per row), so that a warp has
// up to kTmaStages rows in flight without holding them in registers.
template <typename S>
__global__ void __maxnreg__(LB_STEP2_MAXREG)
    k_step2_tma(KP<float> k, const __grid_constant__ CUtensorMap map, const S *__restrict__ src,
                S *__restrict__ dst, int seg_rows, int nwin2, uint32_t salt, int *status, int rev)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int wib = threadIdx.x >> 5;
    int bx, by;
    step_block(rev, bx, by);
    const int warp = bx * (blockDim.x >> 5) + wib;
    if (warp >= nwin2) return;
    const int lane = threadIdx.x & 31;
    const int s = by * seg_rows;
    const int e = min(k.nz, s + seg_rows);
    const bool has_m = s > 0 || k.xper, has_last = e < k.nz || k.xper;
    const int nrows = (e - s) + (has_m ? 1 : 0) + (has_last ? 1 : 0);
    const int per_warp = kTmaStages * TmaGeom<S>::stage_bytes + 128;  // keeps every ring 128-byte aligned
    unsigned char *ring = smem + per_warp * wib;
    RowTma<S> rs;
    rs.map = &map;
    rs.k = &k;
    rs.ring = ring;
    rs.ring_s = smem_u32(ring);
    rs.bar_s = smem_u32(ring + kTmaStages * TmaGeom<S>::stage_bytes);
    rs.first = has_m ? s - 1 : s;
    rs.nrows = nrows;
    rs.nz = k.nz;
    rs.taken = 0;
    rs.lane = lane;
    rs.x0 = warp * 64 - TmaGeom<S>::off;
    rs.status = status;
    grid_dependency_trigger_and_wait();
    rs.start();
    march2<S>(k, src, dst, warp * 64, s, e, salt, rs);
}

// The step with the rows resident in the TMA ring (march3): no row carried
// in registers.  kRingStages<S> stages of one row each per warp: rows i-1,
// i, i+1 of the step and one more in flight.
#ifndef LB_STEP3_MAXREG
#define LB_STEP3_MAXREG 168
#endif
template <typename S> constexpr int kRingStages = 4;
// march3 forms, as measured on GB300 (all give the same bits): the
// single-lattice FP32 step takes the separate interior form of the row update
// (+5 %; in 16-bit storage it cost 2-3 %) and every kernel reads the wall and
// axis values from the ring (the batched FP32 step on serving-size lattices,
// where nearly every warp holds a wall or the axis: +10 % over global loads).
template <typename S> constexpr bool kStepSplit = sizeof(S) == 4;

template <typename S>
__host__ __device__ size_t ring_smem_bytes(int wpb)
{
    return (size_t)wpb * (kRingStages<S> * TmaGeom<S>::stage_bytes + 128);
}

template <typename S>
__global__ void __maxnreg__(LB_STEP3_MAXREG)
    k_step3_tma(KP<float> k, const __grid_constant__ CUtensorMap map, const S *__restrict__ src,
                S *__restrict__ dst, int seg_rows, int nwin2, uint32_t salt, int *status, int rev)
{
    constexpr int R = kRingStages<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int wib = threadIdx.x >> 5;
    int bx, by;
    step_block(rev, bx, by);
    const int warp = bx * (blockDim.x >> 5) + wib;
    if (warp >= nwin2) return;
    const int s = by * seg_rows;
    const int e = min(k.nz, s + seg_rows);
    const bool has_m = s > 0 || k.xper, has_last = e < k.nz || k.xper;
    const int per_warp = R * TmaGeom<S>::stage_bytes + 128;  // keeps every ring 128-byte aligned
    unsigned char *ring = smem + per_warp * wib;
    RowRing<S, R> rs;
    rs.map = &map;
    rs.ring = ring;
    rs.ring_s = smem_u32(ring);
    rs.bar_s = smem_u32(ring + R * TmaGeom<S>::stage_bytes);
    rs.bar_stride = 8;
    rs.first = has_m ? s - 1 : s;
    rs.nrows = (e - s) + (has_m ? 1 : 0) + (has_last ? 1 : 0);
    rs.nz = k.nz;
    rs.x0 = warp * 64 - TmaGeom<S>::off;
    rs.lane = threadIdx.x & 31;
    rs.status = status;
    // programmatic dependent launch: let the next step's blocks become
    // resident now, and touch no distribution before the previous step is done
    grid_dependency_trigger_and_wait();
    rs.start();
    march3<S, R, kStepSplit<S>, true>(k, src, dst, warp * 64, s, e, salt, rs);
}

// Stream function of the meridian flow (Sec. 3.6): dPsi/dy = -y u_x with
// Psi = 0 on the inner boundary y = r0, midpoint sums over whole cells, so
// psi[i][j] is Psi on the face y = r0 + j + 1 of row i.  One warp per row:
// an FP64 warp scan per 32 columns plus the carry; rowmax[i] = max |Psi|.
__global__ void __launch_bounds__(128) k_psi(const double *__restrict__ ux, double *__restrict__ psi,
                                             double *__restrict__ rowmax, int nrows, int nr, double r0)
{
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nrows) return;
    const int lane = threadIdx.x & 31;
    double carry = 0.0, m = 0.0;
    for (int j0 = 0; j0 < nr; j0 += 32) {
        const int j = j0 + lane;
        double v = j < nr ? -(r0 + j + 0.5) * ux[(long long)row * nr + j] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double w = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += w;
        }
        v += carry;
        if (j < nr) {
            if (psi) psi[(long long)row * nr + j] = v;
            m = fmax(m, fabs(v));
        }
        carry = __shfl_sync(FULL, v, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(FULL, m, o));
    if (lane == 0) rowmax[row] = m;
}

constexpr int kFieldRows = 32;  // rows per z-segment of the field export

template <typename S, typename C>
__global__ void __launch_bounds__(256) k_fields(KP<C> k, const S *__restrict__ src, double *__restrict__ out,
                                                int row0, int row1, int nwin)
{
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= nwin) return;
    const int c = warp * OUT_COLS - 1 + (threadIdx.x & 31);
    const int s = row0 + blockIdx.y * kFieldRows, e = min(row1, s + kFieldRows);
    march<S, C, MODE_FIELDS>(k, src, nullptr, out, row0, row1 - row0, c, s, e, nullptr);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
    return v;
}

// One warp per 30-column window, whole height (the end-wall fluxes need rows
// 0, 1 and nz-2, nz-1 in the same march).  Block partial sums in a fixed
// order, then a single-block final reduction: deterministic.
// Block (bx, by) of a diagnostics grid gx blocks wide; 128 threads.
template <typename S, typename C>
__device__ __forceinline__ void diag_block(const KP<C> &k, const S *__restrict__ src, double *__restrict__ partial,
                                           double *__restrict__ tfield, int seg_rows, int nwin, int bx, int by,
                                           int gx)
{
    __shared__ double sh[4][NSUM];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = bx * (blockDim.x >> 5) + wib;
    DiagAcc a = {0, 0, 0, 0, 0};
    if (warp < nwin) {
        const int c = warp * OUT_COLS - 1 + lane;
        const int s = by * seg_rows, e = min(k.nz, s + seg_rows);
        march<S, C, MODE_DIAG>(k, src, nullptr, tfield, 0, 0, c, s, e, &a);
    }
    double vals[NSUM] = {a.mass_dev, a.mass_r_dev, a.tsum, a.umax, 0, 0, 0, 0, a.bad, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < NSUM; ++q) vals[q] = (q == 3 || q == 8) ? warp_max(vals[q]) : warp_sum(vals[q]);
    if (lane == 0)
        for (int q = 0; q < NSUM; ++q) sh[wib][q] = vals[q];
    __syncthreads();
    if (threadIdx.x < NSUM) {
        const int q = threadIdx.x;
        double r = sh[0][q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = (q == 3 || q == 8) ? fmax(r, sh[w][q]) : r + sh[w][q];
        partial[(by * gx + bx) * NSUM + q] = r;
    }
}

template <typename S, typename C>
__global__ void __launch_bounds__(128) k_diag(KP<C> k, const S *__restrict__ src, double *__restrict__ partial,
                                              double *__restrict__ tfield, int seg_rows, int nwin)
{
    diag_block<S, C>(k, src, partial, tfield, seg_rows, nwin, blockIdx.x, blockIdx.y, gridDim.x);
}

// Wall heat-flux sums (Sec. 3.2) from the pre-collision T field: one-sided
// second-order derivative through the wall value, wall half a cell away,
// (-8 T_w + 9 T_1 - T_2) / 3 along the inward direction; end walls weighted
// by the radius.  One block, fixed-order tree reduction (deterministic).
template <typename C>
__device__ __forceinline__ void wall_block(const KP<C> &k, const double *__restrict__ T, double *__restrict__ result)
{
    __shared__ double sh[256];
    const int nr = k.nr, nz = k.nz;
    for (int sd = 0; sd < 4; ++sd) {
        double acc = 0;
        if (wall_heated(k, sd)) {
            const double Tw = (double)k.Tw[sd];
            if (sd == 2)
                for (int i = threadIdx.x; i < nz; i += blockDim.x)
                    acc += (-8.0 * Tw + 9.0 * T[(long long)i * nr] - T[(long long)i * nr + 1]) / 3.0;
            else if (sd == 3)
                for (int i = threadIdx.x; i < nz; i += blockDim.x)
                    acc += (8.0 * Tw - 9.0 * T[(long long)i * nr + nr - 1] + T[(long long)i * nr + nr - 2]) / 3.0;
            else if (sd == 0)
                for (int j = threadIdx.x; j < nr; j += blockDim.x)
                    acc += (k.r0 + j + 0.5) * (-8.0 * Tw + 9.0 * T[j] - T[nr + j]) / 3.0;
            else  // the top: the columns whose segment holds a wall temperature, each with its own value
                for (int j = threadIdx.x; j < nr; j += blockDim.x) {
                    const int sg = end_seg(k, 1, j);
                    if (k.heat[sg] != 0 && k.heat[sg] != 4) continue;
                    const double Tj = (double)end_T(k, sg, (C)(k.r0 + j + 0.5));
                    acc += (k.r0 + j + 0.5) *
                           (8.0 * Tj - 9.0 * T[(long long)(nz - 1) * nr + j] + T[(long long)(nz - 2) * nr + j]) / 3.0;
                }
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            result[4 + sd] = wall_heated(k, sd) ? sh[0] * k.nu_scale[sd] : 0.0;
            if (sd >= 2) result[7 + sd] = k.heat[sd] == 0 ? sh[0] * k.keq_scale[sd] : 0.0;  // 9, 10: k_eq
        }
        __syncthreads();
    }
}

template <typename C>
__global__ void __launch_bounds__(256) k_wall(KP<C> k, const double *__restrict__ T, double *__restrict__ result)
{
    wall_block<C>(k, T, result);
}

// Variant of k_diag whose temperature output is the wall-adjacent strips
// only (4 (nr + nz) doubles), for the scratch-free diagnostics entry point.
template <typename S, typename C>
__global__ void __launch_bounds__(128) k_diag_strip(KP<C> k, const S *__restrict__ src,
                                                    double *__restrict__ partial, double *__restrict__ strips,
                                                    int seg_rows, int nwin)
{
    __shared__ double sh[4][NSUM];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    DiagAcc a = {0, 0, 0, 0, 0};
    if (warp < nwin) {
        const int c = warp * OUT_COLS - 1 + lane;
        const int s = blockIdx.y * seg_rows, e = min(k.nz, s + seg_rows);
        march<S, C, MODE_DIAG_STRIP>(k, src, nullptr, strips, 0, 0, c, s, e, &a);
    }
    double vals[NSUM] = {a.mass_dev, a.mass_r_dev, a.tsum, a.umax, 0, 0, 0, 0, a.bad, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < NSUM; ++q) vals[q] = (q == 3 || q == 8) ? warp_max(vals[q]) : warp_sum(vals[q]);
    if (lane == 0)
        for (int q = 0; q < NSUM; ++q) sh[wib][q] = vals[q];
    __syncthreads();
    if (threadIdx.x < NSUM) {
        const int q = threadIdx.x;
        double r = sh[0][q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = (q == 3 || q == 8) ? fmax(r, sh[w][q]) : r + sh[w][q];
        partial[(blockIdx.y * gridDim.x + blockIdx.x) * NSUM + q] = r;
    }
}

// k_wall on the strips written by k_diag_strip (same summation order).
template <typename C>
__global__ void __launch_bounds__(256) k_wall_strip(KP<C> k, const double *__restrict__ strips,
                                                    double *__restrict__ result)
{
    __shared__ double sh[256];
    const int nr = k.nr, nz = k.nz;
    const double *r0 = strips, *r1 = strips + nr, *r2 = strips + 2 * nr, *r3 = strips + 3 * nr;
    const double *c0 = strips + 4 * nr, *c1 = c0 + nz, *c2 = c0 + 2 * nz, *c3 = c0 + 3 * nz;
    for (int sd = 0; sd < 4; ++sd) {
        double acc = 0;
        if (wall_heated(k, sd)) {
            const double Tw = (double)k.Tw[sd];
            if (sd == 2)
                for (int i = threadIdx.x; i < nz; i += blockDim.x) acc += (-8.0 * Tw + 9.0 * c0[i] - c1[i]) / 3.0;
            else if (sd == 3)
                for (int i = threadIdx.x; i < nz; i += blockDim.x) acc += (8.0 * Tw - 9.0 * c3[i] + c2[i]) / 3.0;
            else if (sd == 0)
                for (int j = threadIdx.x; j < nr; j += blockDim.x)
                    acc += (k.r0 + j + 0.5) * (-8.0 * Tw + 9.0 * r0[j] - r1[j]) / 3.0;
            else
                for (int j = threadIdx.x; j < nr; j += blockDim.x) {
                    const int sg = end_seg(k, 1, j);
                    if (k.heat[sg] != 0 && k.heat[sg] != 4) continue;
                    const double Tj = (double)end_T(k, sg, (C)(k.r0 + j + 0.5));
                    acc += (k.r0 + j + 0.5) * (8.0 * Tj - 9.0 * r3[j] + r2[j]) / 3.0;
                }
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            result[4 + sd] = wall_heated(k, sd) ? sh[0] * k.nu_scale[sd] : 0.0;
            if (sd >= 2) result[7 + sd] = k.heat[sd] == 0 ? sh[0] * k.keq_scale[sd] : 0.0;  // 9, 10: k_eq
        }
        __syncthreads();
    }
}

// One block of 256 threads: per sum, strided partial sums in a fixed order,
// then a fixed tree (deterministic for a given number of blocks).
__device__ __forceinline__ void diag_final_block(const double *__restrict__ partial, int nblocks,
                                                 double *__restrict__ result)
{
    __shared__ double sh[256];
    for (int q = 0; q < NSUM; ++q) {
        if ((q >= 4 && q < 8) || q == 9 || q == 10) continue;  // 4..7, 9, 10: wall sums (k_wall)
        const bool mx = q == 3 || q == 8;
        double r = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double v = partial[b * NSUM + q];
            r = mx ? fmax(r, v) : r + v;
        }
        sh[threadIdx.x] = r;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] = mx ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                                            : sh[threadIdx.x] + sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) result[q] = sh[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_diag_final(const double *__restrict__ partial, int nblocks,
                                                    double *__restrict__ result)
{
    diag_final_block(partial, nblocks, result);
}

// ---- initialisation and exchange ---------------------------------------------

// D2Q9 equilibrium with Maxwellian raw moments, factorised per axis
__device__ __forceinline__ double axis_factor(int e, double u)
{
    const double c2 = 1.0 / 3.0;
    return e == 0 ? 1.0 - c2 - u * u : 0.5 * (c2 + u * u + e * u);
}

__constant__ int c_ex9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_ey9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ double c_w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
__constant__ double c_w5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};

__device__ __forceinline__ void eq_d2q5(double s, double ux, double uy, double o[5])
{
    const double c2 = 1.0 / 3.0;
    o[0] = s * (1.0 - 2.0 * c2 - ux * ux - uy * uy);
    o[1] = 0.5 * s * (c2 + ux * ux + ux);
    o[3] = 0.5 * s * (c2 + ux * ux - ux);
    o[2] = 0.5 * s * (c2 + uy * uy + uy);
    o[4] = 0.5 * s * (c2 + uy * uy - uy);
}

template <typename S>
__global__ void k_init_fields(HostParams h, const double *__restrict__ fields, S *__restrict__ dst, int row0,
                              int row1)
{
    const long long nrow = row1 - row0;
    const long long n = nrow * h.nr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = row0 + (int)(t / h.nr), j = (int)(t % h.nr);
        const double rho = fields[t], ux = fields[n + t], uy = fields[2 * n + t];
        const double ut = fields[3 * n + t], T = fields[4 * n + t];
        S *p = dst + (long long)i * h.pitch + j;
        for (int a = 0; a < 9; ++a) {
            const double fe = rho * axis_factor(c_ex9[a], ux) * axis_factor(c_ey9[a], uy);
            Cvt<S, typename std::conditional<std::is_same<S, double>::value, double, float>::type>::st(
                p + a * h.plane, (fe - c_w9[a] * h.rho0) * h.scale);
        }
        double ge[5], he[5];
        eq_d2q5(rho * ut, ux, uy, ge);
        eq_d2q5(T, ux, uy, he);
        for (int a = 0; a < 5; ++a) {
            Cvt<S, typename std::conditional<std::is_same<S, double>::value, double, float>::type>::st(
                p + (G0 + a) * h.plane, ge[a] * h.scale);
            Cvt<S, typename std::conditional<std::is_same<S, double>::value, double, float>::type>::st(
                p + (H0 + a) * h.plane, (he[a] - c_w5[a] * h.T0) * h.scale);
        }
    }
}

template <typename S>
__global__ void k_export(HostParams h, const S *__restrict__ src, double *__restrict__ out, int row0, int row1)
{
    using C = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
    const long long n = (long long)(row1 - row0) * h.nr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = row0 + (int)(t / h.nr), j = (int)(t % h.nr);
        const S *p = src + (long long)i * h.pitch + j;
        for (int q = 0; q < NQ; ++q) {
            double rest = q < 9 ? c_w9[q] * h.rho0 : (q < 14 ? 0.0 : c_w5[q - 14] * h.T0);
            out[q * n + t] = (double)Cvt<S, C>::ld(p + q * h.plane) / h.scale + rest;
        }
    }
}

template <typename S>
__global__ void k_import(HostParams h, const double *__restrict__ in, S *__restrict__ dst, int row0, int row1)
{
    using C = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
    const long long n = (long long)(row1 - row0) * h.nr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = row0 + (int)(t / h.nr), j = (int)(t % h.nr);
        S *p = dst + (long long)i * h.pitch + j;
        for (int q = 0; q < NQ; ++q) {
            double rest = q < 9 ? c_w9[q] * h.rho0 : (q < 14 ? 0.0 : c_w5[q - 14] * h.T0);
            Cvt<S, C>::st(p + q * h.plane, (C)((in[q * n + t] - rest) * h.scale));
        }
    }
}

int nwindows(int nr) { return (nr + OUT_COLS - 1) / OUT_COLS; }

// ---- batched step: many lattices, one launch per step ----------------------------

// SplitMix64 finaliser of a step counter (the same function as step_salt on
// the host: a lattice draws the same rounding bits alone and in a batch)
__host__ __device__ __forceinline__ uint32_t salt_of(unsigned long long step)
{
    unsigned long long z = step + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return (uint32_t)(z ^ (z >> 31));
}

struct alignas(128) BatchDesc {
    unsigned char map[2][128];  // CUtensorMap of buf[0], buf[1] (64-byte aligned in the device array)
    KP<float> k;
    void *buf[2];
    int *status;               // the lattice's device status word
    unsigned long long step0;  // the lattice's step count when the batch was made
    int parity0;               // its current buffer then
    int nwin2, seg_rows, pad;
};

// The batch's step counter in device memory: the step at the start of the
// running CUDA graph replay.  A graph holds K launches that take steps
// counter + 0 .. counter + K - 1 and then a one-thread launch that adds K, so
// every replay is the same; launches outside a graph get their step as a
// parameter.
struct BatchCtl {
    unsigned long long counter;
    unsigned long long pad;
};

__global__ void k_batch_counter(BatchCtl *ctl, unsigned long long value, int add)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) ctl->counter = add ? ctl->counter + value : value;
}

// Instance of a work item: the last m < n with prefix[m] <= item (prefix is
// non-decreasing, prefix[0] = 0 <= item < prefix[n]).  Each round tests 32
// evenly spaced candidates of the remaining span with one load per lane and
// a ballot: one round for n <= 32, two for n <= 1024.
__device__ __forceinline__ int batch_instance(const int *__restrict__ prefix, int n, int item, int lane)
{
    int lo = 0, span = n;
    while (span > 1) {
        const int step = (span + 31) >> 5;
        const int m = lo + lane * step;
        const bool le = m < lo + span && prefix[m] <= item;
        const unsigned mask = __ballot_sync(FULL, le);  // bit 0 set: prefix[lo] <= item
        const int nlo = lo + (31 - __clz(mask)) * step;
        span = min(step, lo + span - nlo);
        lo = nlo;
    }
    return lo;
}

// Work items (instance, 64-column window, z-segment) are numbered by a prefix
// sum over the instances and dealt to the warps of a persistent grid.  The
// step is t0, plus the device counter when from_counter is set (inside a
// graph), so that every replay of a graph is the same.  Dynamic shared
// memory: one KP per warp.
template <typename S>
__global__ void __maxnreg__(LB_STEP2_MAXREG) k_batch(const BatchDesc *__restrict__ d, const int *__restrict__ prefix,
                                                     int n, int total, const BatchCtl *ctl, unsigned long long t0,
                                                     int from_counter)
{
    extern __shared__ __align__(128) unsigned char smem[];
    KP<float> *skp = reinterpret_cast<KP<float> *>(smem);
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const unsigned long long t = t0 + (from_counter ? *(volatile const unsigned long long *)&ctl->counter : 0ULL);
    for (int item = blockIdx.x * wpb + wib; item < total; item += gridDim.x * wpb) {
        const int lo = batch_instance(prefix, n, item, lane);
        const BatchDesc *bd = d + lo;
        __syncwarp();
        {
            const uint32_t *s = reinterpret_cast<const uint32_t *>(&bd->k);
            uint32_t *o = reinterpret_cast<uint32_t *>(&skp[wib]);
            for (int w = lane; w < (int)(sizeof(KP<float>) / 4); w += 32) o[w] = s[w];
        }
        __syncwarp();
        const KP<float> &k = skp[wib];
        const int local = item - prefix[lo];
        const int nw2 = bd->nwin2;
        const int w = local % nw2, sg = local / nw2;
        const int cur = (bd->parity0 + (int)(t & 1ULL)) & 1;
        const S *src = (const S *)bd->buf[cur];
        S *dst = (S *)bd->buf[cur ^ 1];
        const int seg = bd->seg_rows;
        const int s = sg * seg, e = min(k.nz, s + seg);
        const int A = w * 64 + 2 * lane, Amax = (k.nr - 1) & ~1;
        int hcol = lane == 0 ? w * 64 - 1 : w * 64 + 64;
        hcol = hcol < 0 ? 0 : (hcol >= k.nr ? k.nr - 1 : hcol);
        RowDirect<S> rs{src, &k, A <= Amax ? A : Amax, hcol, (s > 0 || k.xper) ? s - 1 : s, k.nz, 0,
                        lane == 0 || lane == 31};
        march2<S>(k, src, dst, w * 64, s, e, salt_of(bd->step0 + t), rs);
    }
}

// The batched step with the rows read in place from the TMA ring (march3):
// one warp per work item, tensor maps from the lattice's descriptor; the
// step as in k_batch.  Dynamic shared memory: the warps' rings (each a
// multiple of 128 bytes), then one KP per warp.  Each stage's mbarrier sits in
// the padding after the stage's box, which the copies never write, so that
// ten FP32 warps still fit on an SM (22,272 bytes per warp).
// R ring stages per warp: 4 by default (one more row in flight); 3 in the
// FP32 variant that fits 12 instead of 10 warps on an SM (16.9 instead of
// 22.3 KB of shared memory per warp), for batches too small to fill the GPU,
// whose step time is the latency of one wave of work items.
template <typename S, int R>
__host__ __device__ constexpr size_t batch3_ring_bytes()
{
    static_assert(TmaGeom<S>::stage_bytes - TmaGeom<S>::box_bytes >= 8 && TmaGeom<S>::box_bytes % 8 == 0,
                  "room for the stage's mbarrier after its box");
    return (size_t)R * TmaGeom<S>::stage_bytes;
}
template <typename S, int R = kRingStages<S>>
__host__ __device__ size_t batch3_smem_bytes(int wpb)
{
    return (size_t)wpb * (batch3_ring_bytes<S, R>() + sizeof(KP<float>));
}

template <typename S, int R>
__global__ void __maxnreg__(LB_STEP3_MAXREG) k_batch3(const BatchDesc *__restrict__ d, const int *__restrict__ prefix,
                                                      int n, int total, const BatchCtl *ctl, unsigned long long t0,
                                                      int from_counter, int rev)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    unsigned char *ring = smem + batch3_ring_bytes<S, R>() * wib;
    KP<float> *skp = reinterpret_cast<KP<float> *>(smem + batch3_ring_bytes<S, R>() * wpb);
    // Programmatic dependent launch: the next step's blocks may become
    // resident now.  The instance lookup and the parameter copy read only
    // what no launch of the batch writes (the prefix sums, the descriptors),
    // so they overlap the previous launch's last blocks; the step counter and
    // the rows are read after the wait below.
    grid_dependency_trigger();
    const int item0 = blockIdx.x * wpb + wib;
    const int item = rev ? total - 1 - item0 : item0;  // every other step from the last item back
    if (item0 < total) {
        const int lo = batch_instance(prefix, n, item, lane);
        const BatchDesc *bd = d + lo;
        {
            const uint32_t *s = reinterpret_cast<const uint32_t *>(&bd->k);
            uint32_t *o = reinterpret_cast<uint32_t *>(&skp[wib]);
            for (int w = lane; w < (int)(sizeof(KP<float>) / 4); w += 32) o[w] = s[w];
        }
        __syncwarp();
        const KP<float> &k = skp[wib];
        const int local = item - prefix[lo];
        const int nw2 = bd->nwin2;
        const int w = local % nw2, sg = local / nw2;
        const int seg = bd->seg_rows;
        const int s = sg * seg, e = min(k.nz, s + seg);
        const bool has_m = s > 0 || k.xper, has_last = e < k.nz || k.xper;
        if (lane < 2)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                             (unsigned long long)bd->map[lane])
                         : "memory");
        grid_dependency_wait();  // the previous launch is complete and its writes are visible
        const unsigned long long t =
            t0 + (from_counter ? *(volatile const unsigned long long *)&ctl->counter : 0ULL);
        const int cur = (bd->parity0 + (int)(t & 1ULL)) & 1;
        const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(bd->map[cur]);
        RowRing<S, R> rs;
        rs.map = map;
        rs.ring = ring;
        rs.ring_s = smem_u32(ring);
        rs.bar_s = smem_u32(ring + TmaGeom<S>::box_bytes);
        rs.bar_stride = TmaGeom<S>::stage_bytes;
        rs.first = has_m ? s - 1 : s;
        rs.nrows = (e - s) + (has_m ? 1 : 0) + (has_last ? 1 : 0);
        rs.nz = k.nz;
        rs.x0 = w * 64 - TmaGeom<S>::off;
        rs.lane = lane;
        rs.status = bd->status;
        rs.start();
        march3<S, R, false, true>(k, (const S *)bd->buf[cur], (S *)bd->buf[cur ^ 1], w * 64, s, e,
                                               salt_of(bd->step0 + t), rs);
    }
}

// The batched step as one persistent launch for nsteps steps, for batches
// whose work items all fit on the device at once (a cooperative launch, one
// warp per item).  Instead of a launch boundary after each step, an item
// starts step j once the up-to-eight items around it (windows and z-segments
// +-1 in its lattice; segments wrap on a periodic lattice) have completed
// step j - 1: their halo rows and columns are then written (read after write)
// and no longer read from the buffer that step j overwrites (write after
// read).  done[item] counts the steps an item has completed in this launch,
// stored with release semantics after its writes; lanes 0..7 poll one
// neighbour each with acquire loads, at most kFlagWaitLimit times with a
// short sleep between polls (about a second), after which the lattice's
// status word gets LB_ERR_TIMEOUT and the warp leaves.
constexpr int kFlagWaitLimit = 1 << 20;

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename S, int R>
__global__ void __maxnreg__(LB_STEP3_MAXREG) k_batch3p(const BatchDesc *__restrict__ d, const int *__restrict__ prefix,
                                                       int n, int total, unsigned long long t0, int nsteps, int *done)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    unsigned char *ring = smem + batch3_ring_bytes<S, R>() * wib;
    KP<float> *skp = reinterpret_cast<KP<float> *>(smem + batch3_ring_bytes<S, R>() * wpb);
    const int item = blockIdx.x * wpb + wib;
    if (item >= total) return;
    const int lo = batch_instance(prefix, n, item, lane);
    const BatchDesc *bd = d + lo;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&bd->k);
        uint32_t *o = reinterpret_cast<uint32_t *>(&skp[wib]);
        for (int q = lane; q < (int)(sizeof(KP<float>) / 4); q += 32) o[q] = src[q];
    }
    __syncwarp();
    const KP<float> &k = skp[wib];
    const int local = item - prefix[lo];
    const int nw2 = bd->nwin2;
    const int w = local % nw2, sg = local / nw2;
    const int seg = bd->seg_rows, nseg = (k.nz + seg - 1) / seg;
    const int s = sg * seg, e = min(k.nz, s + seg);
    const bool has_m = s > 0 || k.xper, has_last = e < k.nz || k.xper;
    // the neighbour item this lane watches (lanes 0..7), -1 for none
    int nb = -1;
    if (lane < 8) {
        const int c = lane < 4 ? lane : lane + 1;  // the 3 x 3 block without its centre
        const int dw = c % 3 - 1, dg = c / 3 - 1;
        const int w2 = w + dw;
        int g2 = sg + dg;
        if (k.xper) g2 = (g2 + nseg) % nseg;
        if (w2 >= 0 && w2 < nw2 && g2 >= 0 && g2 < nseg && g2 * nw2 + w2 != local) nb = prefix[lo] + g2 * nw2 + w2;
    }
    if (lane < 2)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((unsigned long long)bd->map[lane])
                     : "memory");
    RowRing<S, R> rs;
    rs.ring = ring;
    rs.ring_s = smem_u32(ring);
    rs.bar_s = smem_u32(ring + TmaGeom<S>::box_bytes);
    rs.bar_stride = TmaGeom<S>::stage_bytes;
    rs.first = has_m ? s - 1 : s;
    rs.nrows = (e - s) + (has_m ? 1 : 0) + (has_last ? 1 : 0);
    rs.nz = k.nz;
    rs.x0 = w * 64 - TmaGeom<S>::off;
    rs.lane = lane;
    rs.status = bd->status;
    for (int j = 0; j < nsteps; ++j) {
        if (j > 0) {
            bool ok = true;
            if (nb >= 0) {
                int it = 0;
                while (ld_acquire_gpu(done + nb) < j) {
                    if (++it > kFlagWaitLimit) {
                        ok = false;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            if (!__all_sync(FULL, ok)) {
                if (lane == 0) atomicExch(bd->status, (int)LB_ERR_TIMEOUT);
                return;
            }
            // the neighbours' writes, acquired by the watching lanes, before this
            // warp's bulk-tensor reads; the ring stages read by the last step
            // before the copies that refill them
            __threadfence();
            asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        const unsigned long long t = t0 + (unsigned long long)j;
        const int cur = (bd->parity0 + (int)(t & 1ULL)) & 1;
        rs.map = reinterpret_cast<const CUtensorMap *>(bd->map[cur]);
        if (j == 0) rs.start();  // the barriers, once
        else rs.prime();
        march3<S, R, false, true>(k, (const S *)bd->buf[cur], (S *)bd->buf[cur ^ 1], w * 64, s, e,
                                  salt_of(bd->step0 + t), rs);
        if (*(volatile const int *)bd->status != 0) return;  // a ring wait ran out
        rs.advance();
        // publish: this item's writes, then its progress
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_gpu(done + item, j + 1);
    }
}

// Diagnostics of every lattice of a batch in three launches instead of three
// per lattice: the blocks of all the lattices' diagnostics grids in one grid,
// then one final-reduction block and one wall-flux block per lattice.  Each
// lattice keeps the grid and summation order of its own diagnostics, so the
// results are bitwise those of lb_diagnostics.
struct BatchDiag {
    double *partial;         // the lattice's block partial sums
    int gx, gy, seg, nwin;   // its diagnostics grid (diag_t)
};

template <typename S>
__global__ void __launch_bounds__(128) k_batch_diag(const BatchDesc *__restrict__ d,
                                                    const BatchDiag *__restrict__ dd, const int *__restrict__ prefix,
                                                    int n, unsigned long long t)
{
    // the lattice of this block: the last m with prefix[m] <= blockIdx.x
    const int blk = blockIdx.x;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= blk) lo = mid;
        else hi = mid;
    }
    const BatchDesc &bd = d[lo];
    const BatchDiag &g = dd[lo];
    const int local = blk - prefix[lo];
    const int cur = (bd.parity0 + (int)(t & 1ULL)) & 1;  // the lattice's current buffer after t batch steps
    diag_block<S, float>(bd.k, (const S *)bd.buf[cur], g.partial, (double *)bd.buf[cur ^ 1], g.seg, g.nwin,
                         local % g.gx, local / g.gx, g.gx);
}

// out: one slot of slot_doubles per lattice, its NSUM sums and, 128 bytes in,
// the lattice's status word
__global__ void __launch_bounds__(256) k_batch_diag_final(const BatchDesc *__restrict__ d,
                                                          const BatchDiag *__restrict__ dd, double *__restrict__ out,
                                                          int slot_doubles)
{
    const int m = blockIdx.x;
    double *res = out + (size_t)m * slot_doubles;
    diag_final_block(dd[m].partial, dd[m].gx * dd[m].gy, res);
    if (threadIdx.x == 0) *reinterpret_cast<int *>(res + 16) = *d[m].status;
}

__global__ void __launch_bounds__(256) k_batch_wall(const BatchDesc *__restrict__ d, double *__restrict__ out,
                                                    int slot_doubles, unsigned long long t)
{
    const int m = blockIdx.x;
    const BatchDesc &bd = d[m];
    const int cur = (bd.parity0 + (int)(t & 1ULL)) & 1;
    wall_block<float>(bd.k, (const double *)bd.buf[cur ^ 1], out + (size_t)m * slot_doubles);
}

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// arrives at, for `polls` polls of the same bounded wait the TMA rings use;
// the timeout must reach the status word as it does for a row that never
// arrives.  Nothing is in flight when the kernel ends.
__global__ void k_wait_selftest(int *status, int polls)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(b, 0u, polls);
    if (!__all_sync(FULL, ok) && threadIdx.x == 0) atomicExch(status, (int)LB_ERR_TIMEOUT);
}

int nwindows2(int nr) { return (nr + 63) / 64; }

// random bits of the stochastic rounding differ from step to step
uint32_t step_salt(unsigned long long step) { return salt_of(step); }

template <typename S>
size_t tma_smem_bytes(int wpb)
{
    return (size_t)wpb * (kTmaStages * TmaGeom<S>::stage_bytes + 128);
}

// The dynamic shared-memory limit of a kernel is a per-device attribute:
// set it once on every device that launches the kernel (devices 0..63;
// beyond that it is set at every launch).
template <typename K>
cudaError_t smem_limit_once(K kernel, int bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ULL << dev : 0ULL;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Launch configuration with programmatic stream serialisation (see
// grid_dependency_trigger_and_wait)
void pdl_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, dim3 grid, dim3 block, size_t smem,
                cudaStream_t s)
{
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

template <typename S, typename C>
cudaError_t step_t(const HostParams &h, const Launch &l, const void *src, void *dst, unsigned long long step,
                   const void *tmap, int *status, cudaStream_t s)
{
    const KP<C> k = make_kp<C>(h);
    const int wpb = l.warps_per_block;
    const int seg = l.seg_rows;
    if constexpr (std::is_same<C, double>::value) {
        const int nwin = nwindows(h.nr);
        dim3 grid((nwin + wpb - 1) / wpb, (h.nz + seg - 1) / seg);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute pdl[1];
        pdl_config(cfg, pdl, grid, dim3(32 * wpb), 0, s);
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_step64<S, C>, k, (const S *)src, (S *)dst, seg, nwin);
        if (e != cudaSuccess) return e;
    } else {
        const int nwin2 = nwindows2(h.nr);
        dim3 grid((nwin2 + wpb - 1) / wpb, (h.nz + seg - 1) / seg);
        if (tmap && l.use_tma == 2) {
            const size_t sm = ring_smem_bytes<S>(wpb);
            static std::atomic<unsigned long long> attr_set{0};
            cudaError_t e = smem_limit_once(k_step3_tma<S>, (int)ring_smem_bytes<S>(8), attr_set);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute pdl[1];
            pdl_config(cfg, pdl, grid, dim3(32 * wpb), sm, s);
            e = cudaLaunchKernelEx(&cfg, k_step3_tma<S>, k, *(const CUtensorMap *)tmap, (const S *)src, (S *)dst,
                                   seg, nwin2, step_salt(step), status, (int)(step & 1ULL));
            if (e != cudaSuccess) return e;
        } else if (tmap && l.use_tma) {
            const size_t sm = tma_smem_bytes<S>(wpb);
            static std::atomic<unsigned long long> attr_set{0};
            cudaError_t e = smem_limit_once(k_step2_tma<S>, (int)tma_smem_bytes<S>(8), attr_set);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute pdl[1];
            pdl_config(cfg, pdl, grid, dim3(32 * wpb), sm, s);
            e = cudaLaunchKernelEx(&cfg, k_step2_tma<S>, k, *(const CUtensorMap *)tmap, (const S *)src, (S *)dst,
                                   seg, nwin2, step_salt(step), status, (int)(step & 1ULL));
            if (e != cudaSuccess) return e;
        } else {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute pdl[1];
            pdl_config(cfg, pdl, grid, dim3(32 * wpb), 0, s);
            cudaError_t e = cudaLaunchKernelEx(&cfg, k_step2<S>, k, (const S *)src, (S *)dst, seg, nwin2,
                                               step_salt(step), (int)(step & 1ULL));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t fields_t(const HostParams &h, const Launch &l, const void *src, double *out, int row0, int row1,
                     cudaStream_t s)
{
    const KP<C> k = make_kp<C>(h);
    const int nwin = nwindows(h.nr);
    const int wpb = l.warps_per_block;
    dim3 grid((nwin + wpb - 1) / wpb, (row1 - row0 + kFieldRows - 1) / kFieldRows);
    k_fields<S, C><<<grid, 32 * wpb, 0, s>>>(k, (const S *)src, out, row0, row1, nwin);
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t diag_t(const HostParams &h, const Launch &l, const void *src, double *partial, double *tfield,
                   double *result, cudaStream_t s)
{
    const KP<C> k = make_kp<C>(h);
    const int nwin = nwindows(h.nr);
    const int wpb = 4;
    const int seg = l.seg_rows;
    dim3 grid((nwin + wpb - 1) / wpb, (h.nz + seg - 1) / seg);
    const int nb = grid.x * grid.y;
    if (nb > MAX_DIAG_BLOCKS) return cudaErrorInvalidValue;
    k_diag<S, C><<<grid, 32 * wpb, 0, s>>>(k, (const S *)src, partial, tfield, seg, nwin);
    k_diag_final<<<1, 256, 0, s>>>(partial, nb, result);
    k_wall<C><<<1, 256, 0, s>>>(k, tfield, result);
    return cudaGetLastError();
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

size_t storage_bytes(int storage)
{
    switch (storage) {
        case ST_FP64: return 8;
        case ST_FP32: return 4;
        default: return 2;
    }
}

// SMs of the current device (152 on GB300; also the answer without a device)
static int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0) {
        cudaGetLastError();  // clear the error of a query without a device
        return 152;
    }
    return sms;
}

Launch default_launch(const HostParams &p)
{
    Launch l;
    l.warps_per_block = p.storage == ST_FP64 ? 4 : 1;
    l.use_tma = p.storage != ST_FP64 ? 2 : 0;
    // FP64: 32-row segments; pair kernels: 4-row segments in FP32, 6 in
    // 16-bit storage (measured on the 1024 x 2048 lattice; short segments
    // balance the last wave, and their halo rows are re-read from L2); fewer
    // rows when the lattice would otherwise leave SMs idle
    const int nwin = p.storage == ST_FP64 ? nwindows(p.nr) : nwindows2(p.nr);
    int seg = p.storage == ST_FP64 ? 32 : (p.storage == ST_FP32 ? 4 : 6);
    const long long warps = (long long)nwin * ((p.nz + seg - 1) / seg);
    const long long want = 16LL * sm_count();  // about two waves of resident warps
    if (warps < want) {
        const long long segs = (want + nwin - 1) / nwin;
        seg = (int)((p.nz + segs - 1) / segs);
        if (seg < 4) seg = 4;
    }
    if ((p.nz + seg - 1) / seg > 65535) seg = (p.nz + 65534) / 65535;  // grid.y limit
    l.seg_rows = seg;
    return l;
}

#define DISPATCH(p, CALL)                                                   \
    switch ((p).storage) {                                                  \
        case ST_FP64: { using S = double; using C = double; return CALL; }   \
        case ST_FP32: { using S = float; using C = float; return CALL; }     \
        case ST_BF16: { using S = __nv_bfloat16; using C = float; return CALL; } \
        case ST_FP16: { using S = __half; using C = float; return CALL; }    \
        default: return cudaErrorInvalidValue;                              \
    }

cudaError_t launch_step(const HostParams &p, const Launch &l, const void *src, void *dst, unsigned long long step,
                        const void *tmap, int *status, cudaStream_t s)
{
    DISPATCH(p, (step_t<S, C>(p, l, src, dst, step, tmap, status, s)));
}

// Tensor map of one distribution buffer for the TMA row fetches: a 3-D view
// [19 planes][nz rows][pitch columns], box of TmaGeom::cols x 1 x 19.
cudaError_t make_tensor_map(const HostParams &p, void *buf, void *map_out)
{
    if (p.storage == ST_FP64) return cudaErrorInvalidValue;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int es = (int)storage_bytes(p.storage);
    const CUtensorMapDataType dt = p.storage == ST_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : p.storage == ST_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)p.pitch, (cuuint64_t)p.nz, (cuuint64_t)NQ};
    const cuuint64_t strides[2] = {(cuuint64_t)p.pitch * es, (cuuint64_t)p.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)(64 + 2 * (16 / es)), 1u, (cuuint32_t)NQ};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode((CUtensorMap *)map_out, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_wait_selftest(int *status, int polls, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(status, polls);
    return cudaGetLastError();
}

cudaError_t launch_psi(const double *ux, double *psi, double *rowmax, int nrows, int nr, double r0, cudaStream_t s)
{
    if (nrows < 1) return cudaSuccess;
    k_psi<<<(nrows + 3) / 4, 128, 0, s>>>(ux, psi, rowmax, nrows, nr, r0);
    return cudaGetLastError();
}

cudaError_t launch_fields(const HostParams &p, const Launch &l, const void *src, double *out, int row0, int row1,
                          cudaStream_t s)
{
    DISPATCH(p, (fields_t<S, C>(p, l, src, out, row0, row1, s)));
}

cudaError_t launch_diag(const HostParams &p, const Launch &l, const void *src, double *partial, double *tfield,
                        double *result, cudaStream_t s)
{
    DISPATCH(p, (diag_t<S, C>(p, l, src, partial, tfield, result, s)));
}

#define DISPATCH_S(p, CALL)                                         \
    switch ((p).storage) {                                          \
        case ST_FP64: { using S = double; CALL; break; }            \
        case ST_FP32: { using S = float; CALL; break; }             \
        case ST_BF16: { using S = __nv_bfloat16; CALL; break; }     \
        case ST_FP16: { using S = __half; CALL; break; }            \
        default: return cudaErrorInvalidValue;                      \
    }

cudaError_t launch_init_fields(const HostParams &p, const double *fields, void *dst, int row0, int row1,
                               cudaStream_t s)
{
    const int nb = blocks_for((long long)(row1 - row0) * p.nr);
    DISPATCH_S(p, (k_init_fields<S><<<nb, 256, 0, s>>>(p, fields, (S *)dst, row0, row1)));
    return cudaGetLastError();
}

cudaError_t launch_export(const HostParams &p, const void *src, double *out, int row0, int row1, cudaStream_t s)
{
    const int nb = blocks_for((long long)(row1 - row0) * p.nr);
    DISPATCH_S(p, (k_export<S><<<nb, 256, 0, s>>>(p, (const S *)src, out, row0, row1)));
    return cudaGetLastError();
}

cudaError_t launch_import(const HostParams &p, const double *in, void *dst, int row0, int row1, cudaStream_t s)
{
    const int nb = blocks_for((long long)(row1 - row0) * p.nr);
    DISPATCH_S(p, (k_import<S><<<nb, 256, 0, s>>>(p, in, (S *)dst, row0, row1)));
    return cudaGetLastError();
}

}  // namespace lbk

namespace lbk {

size_t batch_desc_bytes() { return sizeof(BatchDesc); }
size_t batch_ctl_bytes() { return sizeof(BatchCtl); }

int batch_items(const HostParams &h, int seg_rows)
{
    return nwindows2(h.nr) * ((h.nz + seg_rows - 1) / seg_rows);
}

cudaError_t batch_fill_desc(const HostParams &h, void *buf0, void *buf1, unsigned long long step0, int parity0,
                            int seg_rows, int *status, void *out)
{
    BatchDesc d;
    std::memset(&d, 0, sizeof(d));
    cudaError_t e = make_tensor_map(h, buf0, d.map[0]);
    if (e == cudaSuccess) e = make_tensor_map(h, buf1, d.map[1]);
    if (e != cudaSuccess) return e;
    d.k = make_kp<float>(h);
    d.buf[0] = buf0;
    d.buf[1] = buf1;
    d.status = status;
    d.step0 = step0;
    d.parity0 = parity0;
    d.nwin2 = nwindows2(h.nr);
    d.seg_rows = seg_rows;
    std::memcpy(out, &d, sizeof(d));
    return cudaSuccess;
}

cudaError_t batch_prepare(int storage)
{
    switch (storage) {
        case ST_FP32: {
            cudaError_t e = cudaFuncSetAttribute(k_batch3<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)batch3_smem_bytes<float, 4>(8));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_batch3p<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch3_smem_bytes<float, 3>(8));
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(k_batch3<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)batch3_smem_bytes<float, 3>(8));
        }
        case ST_FP16: {
            cudaError_t e = cudaFuncSetAttribute(k_batch3p<__half, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)batch3_smem_bytes<__half>(8));
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(k_batch3<__half, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)batch3_smem_bytes<__half>(8));
        }
        case ST_BF16: {
            cudaError_t e = cudaFuncSetAttribute(k_batch3p<__nv_bfloat16, 4>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)batch3_smem_bytes<__nv_bfloat16>(8));
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(k_batch3<__nv_bfloat16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)batch3_smem_bytes<__nv_bfloat16>(8));
        }
        default: return cudaErrorInvalidValue;
    }
}

int batch_grid(int storage, int wpb)
{
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = (size_t)wpb * sizeof(KP<float>);
    switch (storage) {
        case ST_FP32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<float>, 32 * wpb, sm); break;
        case ST_FP16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<__half>, 32 * wpb, sm); break;
        case ST_BF16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<__nv_bfloat16>, 32 * wpb, sm); break;
        default: per = 1;
    }
    return sms * (per > 0 ? per : 1);
}

cudaError_t batch_resident_warps(int storage, int row_fetch, int wpb, int *out)
{
    if (row_fetch == 1) {
        *out = batch_grid(storage, wpb) * wpb;
        return cudaSuccess;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = batch_prepare(storage);
    if (e != cudaSuccess) return e;
    if (row_fetch == 5) {
        switch (storage) {
            case ST_FP32:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3p<float, 3>, 32 * wpb,
                                                                  batch3_smem_bytes<float, 3>(wpb));
                break;
            case ST_FP16:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3p<__half, 4>, 32 * wpb,
                                                                  batch3_smem_bytes<__half>(wpb));
                break;
            case ST_BF16:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3p<__nv_bfloat16, 4>, 32 * wpb,
                                                                  batch3_smem_bytes<__nv_bfloat16>(wpb));
                break;
            default: return cudaErrorInvalidValue;
        }
        *out = sms * per * wpb;
        return e;
    }
    switch (storage) {
        case ST_FP32:
            if (row_fetch == 4)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3<float, 3>, 32 * wpb,
                                                                  batch3_smem_bytes<float, 3>(wpb));
            else
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3<float, 4>, 32 * wpb,
                                                                  batch3_smem_bytes<float, 4>(wpb));
            break;
        case ST_FP16:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3<__half, 4>, 32 * wpb,
                                                              batch3_smem_bytes<__half>(wpb));
            break;
        case ST_BF16:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3<__nv_bfloat16, 4>, 32 * wpb,
                                                              batch3_smem_bytes<__nv_bfloat16>(wpb));
            break;
        default: return cudaErrorInvalidValue;
    }
    *out = sms * per * wpb;
    return e;
}

cudaError_t launch_batch_persist(int storage, const void *desc, const int *prefix, int n, int total, int wpb,
                                 unsigned long long t0, int nsteps, int *done, cudaStream_t s)
{
    if (total < 1 || nsteps < 1) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(done, 0, (size_t)total * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const BatchDesc *dd = (const BatchDesc *)desc;
    void *args[] = {(void *)&dd, (void *)&prefix, (void *)&n, (void *)&total, (void *)&t0, (void *)&nsteps,
                    (void *)&done};
    const dim3 grid((total + wpb - 1) / wpb), block(32 * wpb);
    switch (storage) {
        case ST_FP32:
            return cudaLaunchCooperativeKernel((const void *)k_batch3p<float, 3>, grid, block, args,
                                               batch3_smem_bytes<float, 3>(wpb), s);
        case ST_FP16:
            return cudaLaunchCooperativeKernel((const void *)k_batch3p<__half, 4>, grid, block, args,
                                               batch3_smem_bytes<__half>(wpb), s);
        case ST_BF16:
            return cudaLaunchCooperativeKernel((const void *)k_batch3p<__nv_bfloat16, 4>, grid, block, args,
                                               batch3_smem_bytes<__nv_bfloat16>(wpb), s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_counter(void *ctl, unsigned long long value, int add, cudaStream_t s)
{
    k_batch_counter<<<1, 32, 0, s>>>((BatchCtl *)ctl, value, add);
    return cudaGetLastError();
}

cudaError_t launch_batch(int storage, int row_fetch, const void *desc, const int *prefix, int n, int total,
                         void *ctl, int wpb, int blocks, unsigned long long t0, int from_counter, cudaStream_t s)
{
    const int need = (total + wpb - 1) / wpb;
    if (need < 1) return cudaSuccess;
    const BatchDesc *dd = (const BatchDesc *)desc;
    const BatchCtl *cc = (const BatchCtl *)ctl;
    // the item order alternates with the step (inside a graph with the launch
    // index, t0 = j there): a step starts on the items the previous one wrote last
    const int rev = (int)(t0 & 1ULL);
    if (row_fetch == 3 || row_fetch == 4) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute pdl[1];
        switch (storage) {
            case ST_FP32:
                if (row_fetch == 4) {
                    pdl_config(cfg, pdl, dim3(need), dim3(32 * wpb), batch3_smem_bytes<float, 3>(wpb), s);
                    return cudaLaunchKernelEx(&cfg, k_batch3<float, 3>, dd, prefix, n, total, cc, t0, from_counter, rev);
                }
                pdl_config(cfg, pdl, dim3(need), dim3(32 * wpb), batch3_smem_bytes<float, 4>(wpb), s);
                return cudaLaunchKernelEx(&cfg, k_batch3<float, 4>, dd, prefix, n, total, cc, t0, from_counter, rev);
            case ST_FP16:
                pdl_config(cfg, pdl, dim3(need), dim3(32 * wpb), batch3_smem_bytes<__half>(wpb), s);
                return cudaLaunchKernelEx(&cfg, k_batch3<__half, 4>, dd, prefix, n, total, cc, t0, from_counter, rev);
            case ST_BF16:
                pdl_config(cfg, pdl, dim3(need), dim3(32 * wpb), batch3_smem_bytes<__nv_bfloat16>(wpb), s);
                return cudaLaunchKernelEx(&cfg, k_batch3<__nv_bfloat16, 4>, dd, prefix, n, total, cc, t0,
                                          from_counter, rev);
            default: return cudaErrorInvalidValue;
        }
    }
    const int grid = blocks < need ? blocks : need;
    const size_t sm = (size_t)wpb * sizeof(KP<float>);
    switch (storage) {
        case ST_FP32: k_batch<float><<<grid, 32 * wpb, sm, s>>>(dd, prefix, n, total, cc, t0, from_counter); break;
        case ST_FP16: k_batch<__half><<<grid, 32 * wpb, sm, s>>>(dd, prefix, n, total, cc, t0, from_counter); break;
        case ST_BF16:
            k_batch<__nv_bfloat16><<<grid, 32 * wpb, sm, s>>>(dd, prefix, n, total, cc, t0, from_counter);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t batch_diag_bytes() { return sizeof(BatchDiag); }

int batch_fill_diag(const HostParams &h, const Launch &l, double *partial, void *out)
{
    BatchDiag g;
    g.partial = partial;
    g.nwin = nwindows(h.nr);
    g.seg = l.seg_rows;
    g.gx = (g.nwin + 3) / 4;
    g.gy = (h.nz + g.seg - 1) / g.seg;
    std::memcpy(out, &g, sizeof g);
    const int nb = g.gx * g.gy;
    return nb <= MAX_DIAG_BLOCKS ? nb : -1;
}

cudaError_t launch_batch_diag(int storage, const void *desc, const void *bdiag, const int *bprefix, int n, int total,
                              unsigned long long t, double *out, int slot_doubles, cudaStream_t s)
{
    const BatchDesc *d = (const BatchDesc *)desc;
    const BatchDiag *dd = (const BatchDiag *)bdiag;
    switch (storage) {
        case ST_FP32: k_batch_diag<float><<<total, 128, 0, s>>>(d, dd, bprefix, n, t); break;
        case ST_FP16: k_batch_diag<__half><<<total, 128, 0, s>>>(d, dd, bprefix, n, t); break;
        case ST_BF16: k_batch_diag<__nv_bfloat16><<<total, 128, 0, s>>>(d, dd, bprefix, n, t); break;
        default: return cudaErrorInvalidValue;
    }
    k_batch_diag_final<<<n, 256, 0, s>>>(d, dd, out, slot_doubles);
    k_batch_wall<<<n, 256, 0, s>>>(d, out, slot_doubles, t);
    return cudaGetLastError();
}

}  // namespace lbk

// ---- diagnostics without scratch memory from the caller ------------------------
//
// lb_diagnostics_static() evaluates the diagnostics of a state the caller
// holds in device memory, with no context and no scratch from the caller:
// its block partial sums and wall temperature strips live in the file-scope
// array below (1 MiB, allocated by the CUDA runtime when the module loads on
// a device and held by every device that loads the library until the process
// exits).  Host code must not pass the array's name to a kernel -- in host
// code it is only a stand-in for the symbol -- so every call looks up the
// device address of the array in the current device's context with
// cudaGetSymbolAddress.  The address is not cached: after cudaDeviceReset, or
// under another context on the same device, the module is loaded again at
// another address.

static __device__ __align__(256) double g_diag_scratch[1 << 17];

namespace lbk {
namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 17;
constexpr int kScratchMaxBlocks = 2048;

cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (e != cudaSuccess) return e;
    *out = (double *)p;
    return cudaSuccess;
}

template <typename S, typename C>
cudaError_t diag_static_t(const HostParams &h, const Launch &l, const void *src, double *scratch, int nb,
                          cudaStream_t s)
{
    const KP<C> k = make_kp<C>(h);
    const int nwin = nwindows(h.nr);
    dim3 grid((nwin + 3) / 4, (h.nz + l.seg_rows - 1) / l.seg_rows);
    double *result = scratch, *partial = scratch + 16, *strips = scratch + 16 + (size_t)nb * NSUM;
    k_diag_strip<S, C><<<grid, 128, 0, s>>>(k, (const S *)src, partial, strips, l.seg_rows, nwin);
    k_diag_final<<<1, 256, 0, s>>>(partial, nb, result);
    k_wall_strip<C><<<1, 256, 0, s>>>(k, strips, result);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbk

extern "C" lb_status lb_diagnostics_static(const lb_grid_desc *desc, const lb_params *p, const void *dev_state,
                                           int64_t step, void *cuda_stream, lb_diag *out)
{
    using namespace lbk;
    if (!desc || !p || !dev_state || !out) {
        set_global_error("lb_diagnostics_static: NULL argument");
        return LB_ERR_ARG;
    }
    HostParams h;
    std::memset(&h, 0, sizeof(h));
    char why[200];
    if (host_from_desc(desc, &h, why, sizeof(why)) != LB_OK || host_set_params(p, &h, why, sizeof(why)) != LB_OK) {
        char msg[256];
        snprintf(msg, sizeof(msg), "lb_diagnostics_static: %s", why);
        set_global_error(msg);
        return LB_ERR_ARG;
    }
    if (((uintptr_t)dev_state & 255) != 0) {
        set_global_error("lb_diagnostics_static: dev_state must be 256-byte aligned");
        return LB_ERR_ARG;
    }
    // launch shape within the static scratch: at most kScratchMaxBlocks blocks
    Launch l = default_launch(h);
    if (l.seg_rows < 32) l.seg_rows = 32;  // as lb_diagnostics
    const long long bx = (nwindows(h.nr) + 3) / 4;
    long long segs = (h.nz + l.seg_rows - 1) / l.seg_rows;
    if (bx * segs > kScratchMaxBlocks) {
        segs = kScratchMaxBlocks / bx;
        if (segs < 1) segs = 1;
        l.seg_rows = (int)((h.nz + segs - 1) / segs);
        segs = (h.nz + l.seg_rows - 1) / l.seg_rows;
    }
    const long long nb = bx * segs;
    const size_t need = 16 + (size_t)nb * NSUM + 4 * ((size_t)h.nr + (size_t)h.nz);
    if (nb > kScratchMaxBlocks || need > kScratchDoubles) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "lb_diagnostics_static: a %d x %d lattice needs %zu scratch doubles, the static array holds %zu "
                 "(nr + nz must stay below about 26600)",
                 h.nr, h.nz, need, kScratchDoubles);
        set_global_error(msg);
        return LB_ERR_ARG;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, need * sizeof(double), st);
    if (e == cudaSuccess) {
        switch (h.storage) {
            case ST_FP64: e = diag_static_t<double, double>(h, l, dev_state, scratch, (int)nb, st); break;
            case ST_FP32: e = diag_static_t<float, float>(h, l, dev_state, scratch, (int)nb, st); break;
            case ST_BF16: e = diag_static_t<__nv_bfloat16, float>(h, l, dev_state, scratch, (int)nb, st); break;
            default: e = diag_static_t<__half, float>(h, l, dev_state, scratch, (int)nb, st); break;
        }
    }
    double res[NSUM];
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, scratch, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "lb_diagnostics_static: %s", cudaGetErrorString(e));
        set_global_error(msg);
        return LB_ERR_CUDA;
    }
    diag_from_sums(h, res, 0, step, out);
    return LB_OK;
}
