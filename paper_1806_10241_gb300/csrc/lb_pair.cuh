// Two radial columns per lane (included by lb_kernels.cu inside its
// anonymous namespace; FP32 arithmetic, FP32 / FP16 / BF16 storage).
//
// A warp owns 64 adjacent, 64-aligned columns: lane l holds columns
// c0 + 2l ("x" of every pair) and c0 + 2l + 1 ("y").  Rows are read and
// written as float2 / half2 pairs, so each warp touches whole 128-byte lines
// of every plane.  Two marches share the row update (row_tail):
//   * march2 takes whole rows from a row source (plain loads, or a TMA ring
//     copied into registers), carries the row groups in registers and does
//     the radial streaming shift with one shuffle per plane, the halo
//     columns c0 - 1 and c0 + 64 coming from lanes 0 and 31;
//   * march3 reads the pulled values in place from a TMA ring holding rows
//     i - 1, i and i + 1 (the radial shift is a column offset in the stage).
// The node arithmetic runs on pairs with the packed FP32x2 instructions
// (FADD2 / FMUL2 / FFMA2) of sm_100+.
//
// The arithmetic is the scalar update_node() reorganised into shared
// subexpressions and fused multiply-adds; both follow the same equations of
// the paper and are compared against the FP64 oracle.

struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 mk2(float a, float b)
{
    F2 r;
    r.v = make_float2(a, b);
    return r;
}
__device__ __forceinline__ F2 sp(float s) { return mk2(s, s); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
// a * b + c
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
// a - b, exactly (one rounding of b * (-1) + a)
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return fma2(b, sp(-1.0f), a); }
__device__ __forceinline__ F2 rcp2(F2 a) { return mk2(__fdividef(1.0f, a.v.x), __fdividef(1.0f, a.v.y)); }
__device__ __forceinline__ F2 sel2(bool px, bool py, F2 a, F2 b)  // per component: p ? a : b
{
    return mk2(px ? a.v.x : b.v.x, py ? a.v.y : b.v.y);
}

// ---- pair loads / stores ------------------------------------------------------

// Counter-based random words for stochastic rounding: the PCG hash of
// Jarzynski & Olano (2020) seeds a xorshift32 sequence (Marsaglia 2003).
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v)
{
    const uint32_t s = v * 747796405u + 2891336453u;
    const uint32_t w = ((s >> ((s >> 28u) + 4u)) ^ s) * 277803737u;
    return (w >> 22u) ^ w;
}
__device__ __forceinline__ uint32_t xorshift32(uint32_t x)
{
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
}

template <typename S> struct PairIO;
template <> struct PairIO<float> {
    static constexpr bool rounds = false;
    static __device__ __forceinline__ F2 ld(const float *p)
    {
        F2 r;
        r.v = *reinterpret_cast<const float2 *>(p);
        return r;
    }
    static __device__ __forceinline__ void st(float *p, F2 v, uint32_t) { *reinterpret_cast<float2 *>(p) = v.v; }
};
// 16-bit storage: stochastic rounding (cvt.rs, sm_100+), so that the
// rounding errors of successive steps do not accumulate a bias
template <> struct PairIO<__half> {
    static constexpr bool rounds = true;
    static __device__ __forceinline__ F2 ld(const __half *p)
    {
        F2 r;
        r.v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        return r;
    }
    static __device__ __forceinline__ void st(__half *p, F2 v, uint32_t rbits)
    {
        uint32_t d;
        // d = {hi: v.y, lo: v.x}: x stays at the lower address
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(rbits));
        *reinterpret_cast<uint32_t *>(p) = d;
    }
};
template <> struct PairIO<__nv_bfloat16> {
    static constexpr bool rounds = true;
    static __device__ __forceinline__ F2 ld(const __nv_bfloat16 *p)
    {
        F2 r;
        r.v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        return r;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, F2 v, uint32_t rbits)
    {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(rbits));
        *reinterpret_cast<uint32_t *>(p) = d;
    }
};

// Stored values to FP32, times the inverse storage scale.  For FP16 one
// mixed-precision FMA per value (fma.rn.f32.f16, sm_100+) converts and
// scales at once: h * 2^-10 + (-0) is exact, so the result is bitwise that
// of a conversion followed by a multiplication.
template <typename S> struct LoadScaled {
    static __device__ __forceinline__ F2 pair(const S *p, float is)
    {
        const F2 v = PairIO<S>::ld(p);
        return Scaled<S>::value ? v * sp(is) : v;
    }
    static __device__ __forceinline__ float one(const S *p, float is)
    {
        const float v = Cvt<S, float>::ld(p);
        return Scaled<S>::value ? v * is : v;
    }
};
template <> struct LoadScaled<__half> {
    static_assert(kFp16Scale == 1024.0 && kFp16InvScaleBits == 0x1400, "FP16 scale is 2^10");
    static __device__ __forceinline__ F2 pair(const __half *p, float)
    {
        const uint32_t raw = *reinterpret_cast<const uint32_t *>(p);
        float x, y;
        asm("{\n\t.reg .f16 lo, hi, s;\n\tmov.b32 {lo, hi}, %2;\n\tmov.b16 s, %3;\n\t"
            "fma.rn.f32.f16 %0, lo, s, %4;\n\tfma.rn.f32.f16 %1, hi, s, %4;\n\t}"
            : "=f"(x), "=f"(y)
            : "r"(raw), "h"(kFp16InvScaleBits), "f"(-0.0f));
        return mk2(x, y);
    }
    static __device__ __forceinline__ float one(const __half *p, float)
    {
        const unsigned short raw = *reinterpret_cast<const unsigned short *>(p);
        float x;
        asm("{\n\t.reg .f16 s;\n\tmov.b16 s, %2;\n\tfma.rn.f32.f16 %0, %1, s, %3;\n\t}"
            : "=f"(x)
            : "h"(raw), "h"(kFp16InvScaleBits), "f"(-0.0f));
        return x;
    }
};

// ---- the node update on pairs ------------------------------------------------

struct NodeOut2 {
    F2 f[9], g[5], h[5];
};

// The post-collision values come out multiplied by osc, a power of two (the
// FP16 storage scale, else 1): osc is folded into the constants of the
// post-collision moments and into the fused multiply-add that adds them to
// the streamed values.  Scaling by a power of two commutes with every
// rounding, so the results are exactly osc times the unscaled ones.
__device__ __forceinline__ void update_node2(const KP<float> &k, F2 iy, const F2 fv[9], const F2 gv[5],
                                             const F2 hv[5], F2 dxuy, F2 dyux, F2 dyuy, F2 dyut, F2 dyT,
                                             float osc, NodeOut2 &o)
{
    const F2 OS = sp(osc);
    // output moments, Eq. 18, 35, 47 (deviation form)
    const F2 a57 = fv[5] - fv[7], a86 = fv[8] - fv[6];
    const F2 s57 = fv[5] + fv[7], s68 = fv[6] + fv[8];
    const F2 s13 = fv[1] + fv[3], s24 = fv[2] + fv[4];
    const F2 s5678 = s57 + s68;
    const F2 rdo = (fv[0] + s13) + (s24 + s5678);
    const F2 jxo = (fv[1] - fv[3]) + (a57 + a86);
    const F2 jyo = (fv[2] - fv[4]) + (a57 - a86);
    const F2 pso = (gv[0] + gv[1]) + (gv[2] + gv[3]) + gv[4];
    const F2 tdo = (hv[0] + hv[1]) + (hv[2] + hv[3]) + hv[4];

    // sources at the pre-collision state, two sweeps (see update_node)
    const bool geo = !k.planar;
    const F2 gy = geo ? iy : sp(0.0f);
    const F2 ngy = gy * sp(-1.0f);
    const F2 nuiy = gy * sp(k.nu);
    const F2 Gx = (dxuy + dyux) * nuiy;
    const F2 Gy = dyuy * (nuiy + nuiy);
    const F2 Gw = dyut * nuiy;
    const F2 Gt = dyT * (gy * sp(k.alpha));
    const F2 iy2nu = nuiy * gy;
    const F2 m2iy2nu = iy2nu * sp(-2.0f);
    const F2 Fbx = sp(k.bfx);
    const F2 Fb = sp(k.rho0 * k.gbeta), rho0 = sp(k.rho0), T0 = sp(k.T0), half = sp(0.5f);
    F2 rd = rdo, jx = jxo, jy = jyo, ps = pso, td = tdo;
    F2 MA = sp(0.0f), Fx = sp(0.0f), Fy = sp(0.0f), Sps = sp(0.0f), Sph = sp(0.0f);
    const int sweeps = k.explicit_src ? 1 : 2;
    for (int sw = 0; sw < sweeps; ++sw) {
        const F2 r = rho0 + rd, ir = rcp2(r);
        const F2 uyyn = (jy * ir) * ngy;  // -u_y / y
        const F2 igy = ir * gy;
        const F2 FAx = fma2(jx, uyyn, r * Gx);
        const F2 FAy = fma2(jy, m2iy2nu, fma2(r, Gy, ((ps - jy) * (ps + jy)) * igy));
        Sps = fma2(ps, fma2(uyyn, sp(2.0f), iy2nu * sp(-1.0f)), r * Gw);
        Sph = fma2(uyyn, T0 + td, Gt);
        Fx = fma2(Fb, td, FAx + Fbx);
        Fy = FAy;
        jx = fma2(Fx, half, jxo);
        jy = fma2(Fy, half, jyo);
        ps = fma2(Sps, half, pso);
        td = fma2(Sph, half, tdo);
        MA = (k.explicit_src ? jyo : jy) * ngy;
        rd = fma2(MA, half, rdo);
    }
    const F2 r = rho0 + rd, ir = rcp2(r);
    const F2 ux = jx * ir, uy = jy * ir;
    const F2 phi = T0 + td;

    // D2Q9 cascaded collision, Eq. 17
    const F2 Dxx = s13 + s5678, Dyy = s24 + s5678;
    const F2 Dxy = s57 - s68, Dxxy = a57 - a86, Dxyy = a57 + a86, Dxxyy = s5678;
    const F2 k3 = sp(k.rho0 * (1.0f / 3.0f));
    const F2 Kxx = k3 + Dxx, Kyy = k3 + Dyy;
    const F2 ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const F2 uu = ux2 + uy2, ud = ux2 - uy2;
    const F2 p3 = (fma2(rd, sp(2.0f / 3.0f), r * uu) - (Dxx + Dyy)) * sp(k.om3 * (1.0f / 12.0f) * osc);
    const F2 c4 = sp(k.om4 * 0.25f * osc);
    const F2 p4 = ((r * ud) - (Dxx - Dyy)) * c4;
    const F2 p5 = ((r * uxy) - Dxy) * c4;
    const F2 q34p = fma2(p3, sp(3.0f), p4), q34m = fma2(p3, sp(3.0f), p4 * sp(-1.0f));
    const F2 ch = sp(k.omhi * 0.25f * osc);
    const F2 m2p5 = p5 * sp(-2.0f);
    const F2 m2Dxy = Dxy * sp(-2.0f);
    const F2 r2 = r + r;
    // p6: (2 r ux^2 uy + Dxxy - 2 ux Dxy - uy Kxx) omhi/4 - uy (3 p3 + p4)/2 - 2 ux p5
    F2 Z = fma2(r2 * ux2, uy, Dxxy);
    Z = fma2(ux, m2Dxy, Z);
    Z = fma2(uy, Kxx * sp(-1.0f), Z);
    const F2 p6 = fma2(Z, ch, fma2(uy, q34p * sp(-0.5f), ux * m2p5));
    F2 Y = fma2(r2 * ux, uy2, Dxyy);
    Y = fma2(uy, m2Dxy, Y);
    Y = fma2(ux, Kyy * sp(-1.0f), Y);
    const F2 p7 = fma2(Y, ch, fma2(ux, q34m * sp(-0.5f), uy * m2p5));
    // p8
    F2 B = fma2(ux2, Kyy, Dxxyy);
    B = fma2(uy2, Kxx, B);
    B = fma2(uxy, Dxy * sp(4.0f), B);
    B = fma2(ux, Dxyy * sp(-2.0f), B);
    B = fma2(uy, Dxxy * sp(-2.0f), B);
    const F2 W = fma2(rd, sp(1.0f / 9.0f), (r * sp(3.0f)) * (ux2 * uy2)) - B;
    F2 p8 = W * ch;
    p8 = fma2(p3, sp(-2.0f), p8);
    p8 = fma2(uy2, q34p * sp(-0.5f), p8);
    p8 = fma2(ux2, q34m * sp(-0.5f), p8);
    p8 = fma2(uxy, p5 * sp(-4.0f), p8);
    p8 = fma2(uy, p6 * sp(-2.0f), p8);
    p8 = fma2(ux, p7 * sp(-2.0f), p8);
    // source moments, Eq. 26
    const F2 p0 = MA * sp((1.0f / 9.0f) * osc), p1 = Fx * sp((1.0f / 6.0f) * osc), p2 = Fy * sp((1.0f / 6.0f) * osc);
    // back-transform, Eq. 27, grouped
    {
        const F2 A0 = p0 - p3;
        const F2 E = A0 + p4, Fm = A0 - p4;
        const F2 t78m = p7 - p8, t78p = p7 + p8, t68m = p6 - p8, t68p = p6 + p8;
        o.f[0] = fma2(p3 - p8, sp(-4.0f), fma2(fv[0], OS, p0));
        o.f[1] = fma2(fv[1], OS, E) + fma2(t78m, sp(2.0f), p1);
        o.f[3] = fma2(fv[3], OS, E) - fma2(t78p, sp(2.0f), p1);
        o.f[2] = fma2(fv[2], OS, Fm) + fma2(t68m, sp(2.0f), p2);
        o.f[4] = fma2(fv[4], OS, Fm) - fma2(t68p, sp(2.0f), p2);
        const F2 B0 = fma2(p3, sp(2.0f), p0 + p8);
        const F2 u12 = p1 + p2, v12 = p1 - p2, s67 = p6 + p7, d67 = p6 - p7;
        const F2 C5 = B0 + p5, C6 = B0 - p5;
        const F2 us = u12 - s67, vd = v12 + d67;
        o.f[5] = fma2(fv[5], OS, C5) + us;
        o.f[7] = fma2(fv[7], OS, C5) - us;
        o.f[6] = fma2(fv[6], OS, C6) - vd;
        o.f[8] = fma2(fv[8], OS, C6) + vd;
    }

    // D2Q5 cascaded collisions, Eq. 34 / 49 (sign reading of the paper: -)
    const F2 coefu = fma2(sp(k.sign_lit ? 1.0f : -1.0f), uu, sp(2.0f / 3.0f));
    const F2 coefd = sp(k.sign_lit ? 1.0f : -1.0f) * ud;
    {
        const F2 kxn = gv[3] - gv[1], kyn = gv[4] - gv[2];  // -kappa'_x, -kappa'_y
        const F2 kxx = gv[1] + gv[3], kyy = gv[2] + gv[4];
        const F2 cg = sp(k.omg * 0.5f * osc);
        const F2 q1 = fma2(ps, ux, kxn) * cg;
        const F2 q2 = fma2(ps, uy, kyn) * cg;
        const F2 m = fma2(ux, kxn, uy * kyn);  // -(ux kx + uy ky)
        const F2 mm = fma2(ux, kxn, uy * (gv[2] - gv[4]));  // -(ux kx - uy ky)
        const F2 X3 = fma2(ps, coefu, fma2(m, sp(-2.0f), (kxx + kyy) * sp(-1.0f)));
        const F2 X4 = fma2(ps, coefd, fma2(mm, sp(-2.0f), (kxx - kyy) * sp(-1.0f)));
        const F2 q3 = fma2(X3, ch, fma2(ux, q1, uy * q2));
        const F2 q4 = fma2(X4, ch, fma2(ux, q1, uy * q2 * sp(-1.0f)));
        const F2 q0 = Sps * sp(0.2f * osc);
        const F2 Q = q0 + q3, Qp = Q + q4, Qm = Q - q4;
        o.g[0] = fma2(q3, sp(-4.0f), fma2(gv[0], OS, q0));
        o.g[1] = fma2(gv[1], OS, Qp) + q1;
        o.g[3] = fma2(gv[3], OS, Qp) - q1;
        o.g[2] = fma2(gv[2], OS, Qm) + q2;
        o.g[4] = fma2(gv[4], OS, Qm) - q2;
    }
    {
        const F2 kxn = hv[3] - hv[1], kyn = hv[4] - hv[2];
        const F2 Hxx = hv[1] + hv[3], Hyy = hv[2] + hv[4];
        const F2 ct = sp(k.omh * 0.5f * osc);
        const F2 r1 = fma2(phi, ux, kxn) * ct;
        const F2 r2t = fma2(phi, uy, kyn) * ct;
        const F2 m = fma2(ux, kxn, uy * kyn);
        const F2 mm = fma2(ux, kxn, uy * (hv[2] - hv[4]));
        // 2 c^2 phi - (kxx + kyy) with the rest parts written out: 2/3 td - (Hxx + Hyy)
        const F2 X3 = fma2(sp(2.0f / 3.0f), td, fma2(phi, coefu - sp(2.0f / 3.0f), fma2(m, sp(-2.0f),
                                                                                    (Hxx + Hyy) * sp(-1.0f))));
        const F2 X4 = fma2(phi, coefd, fma2(mm, sp(-2.0f), (Hxx - Hyy) * sp(-1.0f)));
        const F2 r3 = fma2(X3, ch, fma2(ux, r1, uy * r2t));
        const F2 r4 = fma2(X4, ch, fma2(ux, r1, uy * r2t * sp(-1.0f)));
        const F2 r0 = Sph * sp(0.2f * osc);
        const F2 Q = r0 + r3, Qp = Q + r4, Qm = Q - r4;
        o.h[0] = fma2(r3, sp(-4.0f), fma2(hv[0], OS, r0));
        o.h[1] = fma2(hv[1], OS, Qp) + r1;
        o.h[3] = fma2(hv[3], OS, Qp) - r1;
        o.h[2] = fma2(hv[2], OS, Qm) + r2t;
        o.h[4] = fma2(hv[4], OS, Qm) - r2t;
    }
}

// ---- the march on pairs ---------------------------------------------------------

struct PM2 {
    F2 rd, ux, uy, ut, T;
};

__device__ __forceinline__ PM2 moments2(const F2 v[NQ], const KP<float> &k)
{
    PM2 m;
    const F2 s13 = v[1] + v[3], s24 = v[2] + v[4], s5678 = (v[5] + v[7]) + (v[6] + v[8]);
    m.rd = (v[0] + s13) + (s24 + s5678);
    const F2 a57 = v[5] - v[7], a86 = v[8] - v[6];
    const F2 jx = (v[1] - v[3]) + (a57 + a86);
    const F2 jy = (v[2] - v[4]) + (a57 - a86);
    const F2 ps = (v[9] + v[10]) + (v[11] + v[12]) + v[13];
    const F2 td = (v[14] + v[15]) + (v[16] + v[17]) + v[18];
    const F2 ir = rcp2(sp(k.rho0) + m.rd);
    m.ux = jx * ir;
    m.uy = jy * ir;
    m.ut = ps * ir;
    m.T = sp(k.T0) + td;
    return m;
}

// values at column c - 1 (for e_y = +1) and c + 1 (for e_y = -1) of a pair;
// lanes 0 / 31 take the halo column's value
__device__ __forceinline__ F2 from_left(F2 v, float halo, int lane)
{
    float l = __shfl_up_sync(FULL, v.v.y, 1);
    if (lane == 0) l = halo;
    return mk2(l, v.v.x);
}
__device__ __forceinline__ F2 from_right(F2 v, float halo, int lane)
{
    float r = __shfl_down_sync(FULL, v.v.x, 1);
    if (lane == 31) r = halo;
    return mk2(v.v.y, r);
}

template <typename S>
__device__ __forceinline__ void load_pair_row(const S *__restrict__ src, const KP<float> &k, int row, int Ac, int hcol,
                                              bool hlane, F2 v[NQ], float hv[NQ])
{
    const S *p = src + (long long)row * k.pitch;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v[q] = PairIO<S>::ld(p + q * k.plane + Ac);
        hv[q] = hlane ? Cvt<S, float>::ld(p + q * k.plane + hcol) : 0.0f;
    }
    if (Scaled<S>::value) {
        const float is = k.inv_scale;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            v[q] = v[q] * sp(is);
            hv[q] *= is;
        }
    }
}

// Row groups of pairs, shifted in r (see groups())
__device__ __forceinline__ void groups2(const F2 v[NQ], const float hv[NQ], int lane, F2 xm[5], F2 x0[9], F2 xp[5])
{
    xm[0] = v[1];
    xm[1] = from_left(v[5], hv[5], lane);
    xm[2] = from_right(v[8], hv[8], lane);
    xm[3] = v[G0 + 1];
    xm[4] = v[H0 + 1];
    x0[0] = v[0];
    x0[1] = from_left(v[2], hv[2], lane);
    x0[2] = from_right(v[4], hv[4], lane);
    x0[3] = v[G0 + 0];
    x0[4] = from_left(v[G0 + 2], hv[G0 + 2], lane);
    x0[5] = from_right(v[G0 + 4], hv[G0 + 4], lane);
    x0[6] = v[H0 + 0];
    x0[7] = from_left(v[H0 + 2], hv[H0 + 2], lane);
    x0[8] = from_right(v[H0 + 4], hv[H0 + 4], lane);
    xp[0] = v[3];
    xp[1] = from_left(v[6], hv[6], lane);
    xp[2] = from_right(v[7], hv[7], lane);
    xp[3] = v[G0 + 3];
    xp[4] = v[H0 + 3];
}

template <typename S>
__device__ __forceinline__ F2 own2(const S *__restrict__ src, const KP<float> &k, int q, int row, int Ac)
{
    F2 v = PairIO<S>::ld(src + q * k.plane + (long long)row * k.pitch + Ac);
    if (Scaled<S>::value) v = v * sp(k.inv_scale);
    return v;
}

// ---- row sources ------------------------------------------------------------------
//
// march2 consumes the rows of its segment strictly in order (row s-1 when it
// exists, s, s+1, ..., and the look-ahead row e when it exists, indices taken
// modulo nz).  A row source delivers them as pairs plus the lane's halo value.

// Plain global loads.
template <typename S> struct RowDirect {
    const S *src;
    const KP<float> *k;
    int Ac, hcol, first, nz, taken;
    bool hlane;
    __device__ __forceinline__ bool get(F2 v[NQ], float hv[NQ])
    {
        int row = first + taken++;
        row = row >= nz ? row - nz : (row < 0 ? row + nz : row);
        load_pair_row<S>(src, *k, row, Ac, hcol, hlane, v, hv);
        return true;
    }
    __device__ __forceinline__ void finish() {}
};

// TMA ring (sm_90+ bulk tensor copies): one 3-D box per row -- TmaGeom::cols
// columns starting TmaGeom::off columns left of the warp's window, one row,
// all 19 planes -- into a stage of shared memory, completion signalled on an
// mbarrier.  Lane 0 issues the copies; every wait is bounded and a timeout
// sets the device status word instead of spinning for ever.
template <typename S> struct TmaGeom {
    static constexpr int es = (int)sizeof(S);
    static constexpr int off = 16 / es;               // x start stays 16-byte aligned
    static constexpr int cols = 64 + 2 * off;          // 72 (FP32) or 80 (16-bit) columns
    static constexpr int box_bytes = NQ * cols * es;
    static constexpr int stage_bytes = (box_bytes + 127) / 128 * 128;
};
constexpr int kTmaStages = 3;
// Bounded mbarrier polls of a row wait: a poll of a phase that does not
// complete returns after about 4 us on GB300 (measured by
// lb_selftest_timeout), so 2^18 polls give up after about a second; a row in
// flight normally completes within a few polls.
constexpr int kTmaWaitLimit = 1 << 18;

// Poll the mbarrier at shared address bar for the phase of the given parity
// at most `limit` times; false when it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit)
{
    uint32_t ok = 0;
    for (int it = 0; it < limit && !ok; ++it)
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename S> struct RowTma {
    const CUtensorMap *map;
    const KP<float> *k;
    const unsigned char *ring;  // this warp's stages
    uint32_t ring_s, bar_s;     // shared addresses of the stages and of the barriers
    int first, nrows, nz, taken, lane, x0;
    int *status;

    __device__ __forceinline__ void issue(int f)
    {
        int row = first + f;
        row = row >= nz ? row - nz : (row < 0 ? row + nz : row);
        const int st = f % kTmaStages;
        const uint32_t bar = bar_s + 8u * st, dst = ring_s + (uint32_t)(TmaGeom<S>::stage_bytes * st);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)TmaGeom<S>::box_bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst),
            "l"((unsigned long long)map), "r"(x0), "r"(row), "r"(0), "r"(bar)
            : "memory");
    }

    __device__ __forceinline__ void start()
    {
        if (lane == 0) {
            for (int s = 0; s < kTmaStages; ++s)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + 8u * s) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int f = 0; f < kTmaStages && f < nrows; ++f) issue(f);
        }
        __syncwarp();
    }

    __device__ __forceinline__ bool wait_stage(int t)
    {
        return mbar_wait_bounded(bar_s + 8u * (t % kTmaStages), (uint32_t)((t / kTmaStages) & 1), kTmaWaitLimit);
    }

    __device__ __forceinline__ bool get(F2 v[NQ], float hv[NQ])
    {
        const int t = taken++;
        if (!__all_sync(FULL, wait_stage(t))) {
            if (lane == 0) atomicExch(status, (int)LB_ERR_TIMEOUT);
            return false;
        }
        const S *b = reinterpret_cast<const S *>(ring + TmaGeom<S>::stage_bytes * (t % kTmaStages));
        constexpr int C = TmaGeom<S>::cols, O = TmaGeom<S>::off;
        const int hc = lane == 0 ? O - 1 : O + 64;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            v[q] = PairIO<S>::ld(b + q * C + O + 2 * lane);
            hv[q] = Cvt<S, float>::ld(b + q * C + hc);
        }
        if (Scaled<S>::value) {
            const float is = k->inv_scale;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                v[q] = v[q] * sp(is);
                hv[q] *= is;
            }
        }
        __syncwarp();  // every lane has read the stage
        if (lane == 0 && t + kTmaStages < nrows) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + kTmaStages);
        }
        return true;
    }

    // after an error: give the copies still in flight a bounded wait
    __device__ __forceinline__ void finish()
    {
        for (int t = taken; t < nrows && t < taken + kTmaStages; ++t) (void)wait_stage(t);
    }
};

// Per-lane constants of a pair march.
struct Lane2 {
    int lane, A, Ac;
    bool outA, atA0, atAN, atBN, edge_warp;
    F2 y2, iy;
};

__device__ __forceinline__ Lane2 lane2(const KP<float> &k, int c0)
{
    Lane2 L;
    L.lane = threadIdx.x & 31;
    L.A = c0 + 2 * L.lane;
    const int B = L.A + 1, nr = k.nr;
    const int Amax = (nr - 1) & ~1;
    L.Ac = L.A <= Amax ? L.A : Amax;  // even pair start inside the padded row
    L.outA = L.A < nr;
    L.atA0 = L.A == 0;
    L.atAN = L.A == nr - 1;
    L.atBN = B == nr - 1;
    L.edge_warp = __any_sync(FULL, L.atA0 || L.atAN || L.atBN);
    // y and 1/y of the pair from the table (FP64 on the host, rounded once;
    // entries past nr - 1 repeat the last radius)
    const float2 yv = *reinterpret_cast<const float2 *>(k.ytab + L.Ac);
    const float2 iyv = *reinterpret_cast<const float2 *>(k.ytab + k.pitch + L.Ac);
    L.y2 = mk2(yv.x, yv.y);
    L.iy = mk2(iyv.x, iyv.y);
    return L;
}

__device__ __forceinline__ void halo_fields(const KP<float> &k, const float h[NQ], float &ux, float &uy, float &ut,
                                            float &T)
{
    const float rd = h[0] + h[1] + h[2] + h[3] + h[4] + h[5] + h[6] + h[7] + h[8];
    const float ir = __fdividef(1.0f, k.rho0 + rd);
    ux = (h[1] - h[3] + h[5] - h[6] - h[7] + h[8]) * ir;
    uy = (h[2] - h[4] + h[5] + h[6] - h[7] - h[8]) * ir;
    ut = (h[9] + h[10] + h[11] + h[12] + h[13]) * ir;
    T = k.T0 + (h[14] + h[15] + h[16] + h[17] + h[18]);
}

// Own post-collision values that the wall and axis rules need (own(q): the
// lane's pair on row i; own0(q): column 0 on row i; m8 / p7: f8 on row i - 1
// and f7 on row i + 1 at column 0, for the axis mirror).  OwnGlobal reads them
// from the source buffer; OwnStage from the TMA ring, where they already are,
// so that a warp at a wall or the axis waits on no global load.
// shl(q) / shr(q): the pair's values of plane q one column to the left
// (A - 1, A) and to the right (A + 1, A + 2) on row i (free-surface end walls;
// columns outside the lattice are clamped, their values replaced by the
// corner rules).
template <typename S> struct OwnGlobal {
    const S *src;
    const KP<float> *k;
    int i, Ac;
    __device__ __forceinline__ F2 own(int q) const { return own2<S>(src, *k, q, i, Ac); }
    __device__ __forceinline__ float own0(int q) const { return own2<S>(src, *k, q, i, 0).v.x; }
    __device__ __forceinline__ float m8() const { return own2<S>(src, *k, 8, i > 0 ? i - 1 : k->nz - 1, 0).v.x; }
    __device__ __forceinline__ float p7() const { return own2<S>(src, *k, 7, i + 1 < k->nz ? i + 1 : 0, 0).v.x; }
    __device__ __forceinline__ float at(int q, int col) const
    {
        col = col < 0 ? 0 : (col >= k->nr ? k->nr - 1 : col);
        return LoadScaled<S>::one(src + q * k->plane + (long long)i * k->pitch + col, k->inv_scale);
    }
    __device__ __forceinline__ F2 shl(int q) const { return mk2(at(q, Ac - 1), at(q, Ac)); }
    __device__ __forceinline__ F2 shr(int q) const { return mk2(at(q, Ac + 1), at(q, Ac + 2)); }
};
template <typename S> struct OwnStage {
    const S *b;  // stage of row i
    int cA;      // column of the lane's pair in the stage
    float is, m8v, p7v;
    // FP32: the loads are volatile so that they stay inside the wall lanes'
    // branches.  Plain loads were hoisted ahead of the branches, which kept
    // every own value live in registers: the batched step then needed more
    // than its 168 and spilled (measured 2.5-4 % slower than reading the
    // values from global memory; 10 % faster with these loads).
    __device__ __forceinline__ F2 own(int q) const
    {
        if constexpr (sizeof(S) == 4) {
            float x, y;
            const uint32_t a = smem_u32(b + q * TmaGeom<S>::cols + cA);
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a) : "memory");
            return mk2(x, y);
        } else {
            return LoadScaled<S>::pair(b + q * TmaGeom<S>::cols + cA, is);
        }
    }
    __device__ __forceinline__ float own0(int q) const
    {
        if constexpr (sizeof(S) == 4) {
            float x;
            const uint32_t a = smem_u32(b + q * TmaGeom<S>::cols + cA);
            asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x) : "r"(a) : "memory");
            return x;
        } else {
            return LoadScaled<S>::one(b + q * TmaGeom<S>::cols + cA, is);
        }
    }
    __device__ __forceinline__ float m8() const { return m8v; }
    __device__ __forceinline__ float p7() const { return p7v; }
    __device__ __forceinline__ F2 shl(int q) const
    {
        const S *p = b + q * TmaGeom<S>::cols + cA;
        return mk2(LoadScaled<S>::one(p - 1, is), LoadScaled<S>::one(p, is));
    }
    __device__ __forceinline__ F2 shr(int q) const
    {
        const S *p = b + q * TmaGeom<S>::cols + cA;
        return mk2(LoadScaled<S>::one(p + 1, is), LoadScaled<S>::one(p + 2, is));
    }
};

// The rest of a row update once the pulled values of the pair are in fv, gv,
// hv5: wall and axis rules (the own post-collision values they need are read
// from src), central differences of the stored-state fields with ghosts, the
// node update and the stores.  kBc = false is the interior form, for a warp
// with no wall or axis column on a row with both neighbour rows: the rules are
// left out at compile time instead of being branched or predicated around.
template <typename S, bool kBc, typename Own>
__device__ __forceinline__ void row_tail(const KP<float> &k, const Own &own, S *__restrict__ dst,
                                         const Lane2 &L, int i, bool has_m_, bool has_p_, uint32_t salt, F2 fv[9],
                                         F2 gv[5], F2 hv5[5], const PM2 &pm_cur, const PM2 &pm_n, F2 uy_prev,
                                         float pmh_ux, float pmh_uy, float pmh_ut, float pmh_T)
{
    const int lane = L.lane, A = L.A, Ac = L.Ac, nz = k.nz;
    const bool has_m = kBc ? has_m_ : true, has_p = kBc ? has_p_ : true;
    const bool outA = L.outA, atA0 = L.atA0, atAN = L.atAN, atBN = L.atBN, edge_warp = kBc && L.edge_warp;
    const F2 y2 = L.y2, iy = L.iy;
    const float sc = k.scale;
    // lateral boundaries: column 0 is always the x of a pair, column
    // nr - 1 the x or the y
    // (the wall terms and rule coefficients come precomputed in k.latf,
    // k.latgs / latgc, k.laths / lathc: one add or one FMA per value)
    if (edge_warp) {
        if (atA0) {
            if (k.flow[2] == 1) {  // axis: mirror images
                fv[2].v.x = own.own0(4);
                if (has_m) fv[5].v.x = own.m8();
                if (has_p) fv[6].v.x = own.p7();
            } else {
                fv[2].v.x = own.own0(4) + k.latf[0][0];
                fv[5].v.x = own.own0(7) + k.latf[0][1];
                fv[6].v.x = own.own0(8) + k.latf[0][2];
            }
            gv[2].v.x = __fmaf_rn(k.latgs[0], own.own0(G0 + 4), k.latgc[0]);
            hv5[2].v.x = __fmaf_rn(k.laths[0], own.own0(H0 + 4), k.lathc[0]);
        }
        if (atAN || atBN) {
            const F2 o2 = own.own(2), o5 = own.own(5), o6 = own.own(6);
            const F2 og = own.own(G0 + 2), oh = own.own(H0 + 2);
            if (atAN) {
                fv[4].v.x = o2.v.x + k.latf[1][0];
                fv[7].v.x = o5.v.x + k.latf[1][1];
                fv[8].v.x = o6.v.x + k.latf[1][2];
                gv[4].v.x = __fmaf_rn(k.latgs[1], og.v.x, k.latgc[1]);
                hv5[4].v.x = __fmaf_rn(k.laths[1], oh.v.x, k.lathc[1]);
            }
            if (atBN) {
                fv[4].v.y = o2.v.y + k.latf[1][0];
                fv[7].v.y = o5.v.y + k.latf[1][1];
                fv[8].v.y = o6.v.y + k.latf[1][2];
                gv[4].v.y = __fmaf_rn(k.latgs[1], og.v.y, k.latgc[1]);
                hv5[4].v.y = __fmaf_rn(k.laths[1], oh.v.y, k.lathc[1]);
            }
        }
    }
    // end walls; they win in corners.  Each node of the pair takes the rules
    // of its own segment (a split top, Sec. 3.6); a free surface reflects f
    // specularly (the population that left the neighbour column towards the
    // wall, e_x reversed) and at a corner column takes the lateral side's rule
    // for the node itself.
    if (!has_m) {
        const int sx = end_seg(k, 0, A), sy = end_seg(k, 0, A + 1);
        if (k.flow[sx] == 3 || k.flow[sy] == 3) {
            const F2 o3 = own.own(3), l6 = own.shl(6), r7 = own.shr(7);
            float c5 = 0.0f, c8x = 0.0f, c8y = 0.0f;
            if (atA0) c5 = own.own0(7) + (k.flow[2] == 1 ? 0.0f : k.rho0 * (6.0f / 36.0f) * (k.uwx[2] + k.uwy[2]));
            if (atAN || atBN) {
                const F2 o6 = own.own(6);
                const float t8 = k.rho0 * (6.0f / 36.0f) * (k.uwx[3] - k.uwy[3]);
                c8x = o6.v.x + t8;
                c8y = o6.v.y + t8;
            }
            const F2 f5 = mk2(atA0 ? c5 : l6.v.x, l6.v.y);
            const F2 f8 = mk2(atAN ? c8x : r7.v.x, atBN ? c8y : r7.v.y);
            const F2 w1 = own.own(3), w5 = own.own(7), w8 = own.own(6);
            fv[1] = mk2(k.flow[sx] == 3 ? o3.v.x : w1.v.x + k.rho0 * (6.0f / 9.0f) * k.uwx[sx],
                        k.flow[sy] == 3 ? o3.v.y : w1.v.y + k.rho0 * (6.0f / 9.0f) * k.uwx[sy]);
            fv[5] = mk2(k.flow[sx] == 3 ? f5.v.x : w5.v.x + k.rho0 * (6.0f / 36.0f) * (k.uwx[sx] + k.uwy[sx]),
                        k.flow[sy] == 3 ? f5.v.y : w5.v.y + k.rho0 * (6.0f / 36.0f) * (k.uwx[sy] + k.uwy[sy]));
            fv[8] = mk2(k.flow[sx] == 3 ? f8.v.x : w8.v.x + k.rho0 * (6.0f / 36.0f) * (k.uwx[sx] - k.uwy[sx]),
                        k.flow[sy] == 3 ? f8.v.y : w8.v.y + k.rho0 * (6.0f / 36.0f) * (k.uwx[sy] - k.uwy[sy]));
        } else {
            const int sd = 0;
            const float ux_w = k.uwx[sd], uy_w = k.uwy[sd];
            fv[1] = own.own(3) + sp(k.rho0 * (6.0f / 9.0f) * ux_w);
            fv[5] = own.own(7) + sp(k.rho0 * (6.0f / 36.0f) * (ux_w + uy_w));
            fv[8] = own.own(6) + sp(k.rho0 * (6.0f / 36.0f) * (ux_w - uy_w));
        }
        const F2 og = own.own(G0 + 3), oh = own.own(H0 + 3);
        gv[1] = mk2(scalar_bc<float>(k.swirl[sx], og.v.x, wall_psi<float>(k, sx, y2.v.x), true),
                    scalar_bc<float>(k.swirl[sy], og.v.y, wall_psi<float>(k, sy, y2.v.y), true));
        hv5[1] = mk2(scalar_bc<float>(heat_rule(k, sx), oh.v.x, end_T(k, sx, y2.v.x) - k.T0, false),
                     scalar_bc<float>(heat_rule(k, sy), oh.v.y, end_T(k, sy, y2.v.y) - k.T0, false));
    }
    if (!has_p) {
        const int sx = end_seg(k, 1, A), sy = end_seg(k, 1, A + 1);
        if (k.flow[sx] == 3 || k.flow[sy] == 3) {
            const F2 o1 = own.own(1), l5 = own.shl(5), r8 = own.shr(8);
            float c6 = 0.0f, c7x = 0.0f, c7y = 0.0f;
            if (atA0) c6 = own.own0(8) + (k.flow[2] == 1 ? 0.0f : k.rho0 * (6.0f / 36.0f) * (-k.uwx[2] + k.uwy[2]));
            if (atAN || atBN) {
                const F2 o5 = own.own(5);
                const float t7 = k.rho0 * (6.0f / 36.0f) * (-k.uwx[3] - k.uwy[3]);
                c7x = o5.v.x + t7;
                c7y = o5.v.y + t7;
            }
            const F2 f6 = mk2(atA0 ? c6 : l5.v.x, l5.v.y);
            const F2 f7 = mk2(atAN ? c7x : r8.v.x, atBN ? c7y : r8.v.y);
            const F2 w3 = own.own(1), w6 = own.own(8), w7 = own.own(5);
            fv[3] = mk2(k.flow[sx] == 3 ? o1.v.x : w3.v.x + k.rho0 * (6.0f / 9.0f) * (-k.uwx[sx]),
                        k.flow[sy] == 3 ? o1.v.y : w3.v.y + k.rho0 * (6.0f / 9.0f) * (-k.uwx[sy]));
            fv[6] = mk2(k.flow[sx] == 3 ? f6.v.x : w6.v.x + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sx] + k.uwy[sx]),
                        k.flow[sy] == 3 ? f6.v.y : w6.v.y + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sy] + k.uwy[sy]));
            fv[7] = mk2(k.flow[sx] == 3 ? f7.v.x : w7.v.x + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sx] - k.uwy[sx]),
                        k.flow[sy] == 3 ? f7.v.y : w7.v.y + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sy] - k.uwy[sy]));
        } else if (sx != sy || sx == 4) {  // a split top without a free surface: per-node wall velocities
            const F2 w3 = own.own(1), w6 = own.own(8), w7 = own.own(5);
            fv[3] = mk2(w3.v.x + k.rho0 * (6.0f / 9.0f) * (-k.uwx[sx]), w3.v.y + k.rho0 * (6.0f / 9.0f) * (-k.uwx[sy]));
            fv[6] = mk2(w6.v.x + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sx] + k.uwy[sx]),
                        w6.v.y + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sy] + k.uwy[sy]));
            fv[7] = mk2(w7.v.x + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sx] - k.uwy[sx]),
                        w7.v.y + k.rho0 * (6.0f / 36.0f) * (-k.uwx[sy] - k.uwy[sy]));
        } else {
            const int sd = 1;
            const float ux_w = k.uwx[sd], uy_w = k.uwy[sd];
            fv[3] = own.own(1) + sp(k.rho0 * (6.0f / 9.0f) * (-ux_w));
            fv[6] = own.own(8) + sp(k.rho0 * (6.0f / 36.0f) * (-ux_w + uy_w));
            fv[7] = own.own(5) + sp(k.rho0 * (6.0f / 36.0f) * (-ux_w - uy_w));
        }
        const F2 og = own.own(G0 + 1), oh = own.own(H0 + 1);
        gv[3] = mk2(scalar_bc<float>(k.swirl[sx], og.v.x, wall_psi<float>(k, sx, y2.v.x), true),
                    scalar_bc<float>(k.swirl[sy], og.v.y, wall_psi<float>(k, sy, y2.v.y), true));
        hv5[3] = mk2(scalar_bc<float>(heat_rule(k, sx), oh.v.x, end_T(k, sx, y2.v.x) - k.T0, false),
                     scalar_bc<float>(heat_rule(k, sy), oh.v.y, end_T(k, sy, y2.v.y) - k.T0, false));
    }

    // central differences of the stored-state fields, with ghosts (a free
    // surface: no shear, u_y even across it)
    F2 uy_xm = uy_prev, uy_xp = pm_n.uy;
    if (!has_m) {
        const int sx = end_seg(k, 0, A), sy = end_seg(k, 0, A + 1);
        uy_xm = mk2(k.flow[sx] == 3 ? pm_cur.uy.v.x : 2.0f * k.uwy[sx] - pm_cur.uy.v.x,
                    k.flow[sy] == 3 ? pm_cur.uy.v.y : 2.0f * k.uwy[sy] - pm_cur.uy.v.y);
    }
    if (!has_p) {
        const int sx = end_seg(k, 1, A), sy = end_seg(k, 1, A + 1);
        uy_xp = mk2(k.flow[sx] == 3 ? pm_cur.uy.v.x : 2.0f * k.uwy[sx] - pm_cur.uy.v.x,
                    k.flow[sy] == 3 ? pm_cur.uy.v.y : 2.0f * k.uwy[sy] - pm_cur.uy.v.y);
    }
    float lux = __shfl_up_sync(FULL, pm_cur.ux.v.y, 1), luy = __shfl_up_sync(FULL, pm_cur.uy.v.y, 1);
    float lut = __shfl_up_sync(FULL, pm_cur.ut.v.y, 1), lT = __shfl_up_sync(FULL, pm_cur.T.v.y, 1);
    float rux = __shfl_down_sync(FULL, pm_cur.ux.v.x, 1), ruy = __shfl_down_sync(FULL, pm_cur.uy.v.x, 1);
    float rut = __shfl_down_sync(FULL, pm_cur.ut.v.x, 1), rT = __shfl_down_sync(FULL, pm_cur.T.v.x, 1);
    if (lane == 0) {
        lux = pmh_ux;
        luy = pmh_uy;
        lut = pmh_ut;
        lT = pmh_T;
    }
    if (lane == 31) {
        rux = pmh_ux;
        ruy = pmh_uy;
        rut = pmh_ut;
        rT = pmh_T;
    }
    F2 Lux = mk2(lux, pm_cur.ux.v.x), Luy = mk2(luy, pm_cur.uy.v.x);
    F2 Lut = mk2(lut, pm_cur.ut.v.x), LT = mk2(lT, pm_cur.T.v.x);
    F2 Rux = mk2(pm_cur.ux.v.y, rux), Ruy = mk2(pm_cur.uy.v.y, ruy);
    F2 Rut = mk2(pm_cur.ut.v.y, rut), RT = mk2(pm_cur.T.v.y, rT);
    // ghosts at the lateral walls, a q + b (k.gha, k.ghb)
    if (edge_warp) {
        if (atA0) {
            Lux.v.x = __fmaf_rn(k.gha[0][0], pm_cur.ux.v.x, k.ghb[0][0]);
            Luy.v.x = __fmaf_rn(k.gha[0][1], pm_cur.uy.v.x, k.ghb[0][1]);
            Lut.v.x = __fmaf_rn(k.gha[0][2], pm_cur.ut.v.x, k.ghb[0][2]);
            LT.v.x = __fmaf_rn(k.gha[0][3], pm_cur.T.v.x, k.ghb[0][3]);
        }
        if (atAN) {
            Rux.v.x = __fmaf_rn(k.gha[1][0], pm_cur.ux.v.x, k.ghb[1][0]);
            Ruy.v.x = __fmaf_rn(k.gha[1][1], pm_cur.uy.v.x, k.ghb[1][1]);
            Rut.v.x = __fmaf_rn(k.gha[1][2], pm_cur.ut.v.x, k.ghb[1][2]);
            RT.v.x = __fmaf_rn(k.gha[1][3], pm_cur.T.v.x, k.ghb[1][3]);
        }
        if (atBN) {
            Rux.v.y = __fmaf_rn(k.gha[1][0], pm_cur.ux.v.y, k.ghb[1][0]);
            Ruy.v.y = __fmaf_rn(k.gha[1][1], pm_cur.uy.v.y, k.ghb[1][1]);
            Rut.v.y = __fmaf_rn(k.gha[1][2], pm_cur.ut.v.y, k.ghb[1][2]);
            RT.v.y = __fmaf_rn(k.gha[1][3], pm_cur.T.v.y, k.ghb[1][3]);
        }
    }
    const F2 hf = sp(0.5f);
    const F2 dxuy = (uy_xp - uy_xm) * hf;
    const F2 dyux = (Rux - Lux) * hf;
    const F2 dyuy = (Ruy - Luy) * hf;
    const F2 dyut = (Rut - Lut) * hf;
    const F2 dyT = (RT - LT) * hf;

    // FP16 storage: the update returns the values already times the scale
    NodeOut2 o;
    update_node2(k, iy, fv, gv, hv5, dxuy, dyux, dyuy, dyut, dyT, Scaled<S>::value ? sc : 1.0f, o);

    if (outA) {
        S *p = dst + (long long)i * k.pitch + A;
        uint32_t w = 0;
        if (PairIO<S>::rounds) w = pcg_hash(((uint32_t)i * (uint32_t)k.pitch + (uint32_t)A) ^ salt) | 1u;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (PairIO<S>::rounds) w = xorshift32(w);
            PairIO<S>::st(p + q * k.plane, o.f[q], w);
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (PairIO<S>::rounds) w = xorshift32(w);
            PairIO<S>::st(p + (G0 + q) * k.plane, o.g[q], w);
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (PairIO<S>::rounds) w = xorshift32(w);
            PairIO<S>::st(p + (H0 + q) * k.plane, o.h[q], w);
        }
    }

}

template <typename S, typename RS>
__device__ __forceinline__ void march2(const KP<float> &k, const S *__restrict__ src, S *__restrict__ dst, int c0,
                                       int row_s, int row_e, uint32_t salt, RS &rs)
{
    const Lane2 L = lane2(k, c0);
    const int lane = L.lane, nz = k.nz;

    F2 v[NQ];
    float hv[NQ];
    F2 xm_prev[5], xm_cur[5], x0_cur[9];
    PM2 pm_cur;
    float pmh_ux, pmh_uy, pmh_ut, pmh_T;  // halo column fields (lanes 0 / 31)
    F2 uy_prev = sp(0.0f);
    bool has_m;

    if (row_s > 0 || k.xper) {
        if (!rs.get(v, hv)) return rs.finish();
        F2 x0t[9], xpt[5];
        groups2(v, hv, lane, xm_prev, x0t, xpt);
        uy_prev = moments2(v, k).uy;
        has_m = true;
    } else {
        has_m = false;
#pragma unroll
        for (int q = 0; q < 5; ++q) xm_prev[q] = sp(0.0f);
    }
    {
        if (!rs.get(v, hv)) return rs.finish();
        F2 xpt[5];
        groups2(v, hv, lane, xm_cur, x0_cur, xpt);
        pm_cur = moments2(v, k);
        halo_fields(k, hv, pmh_ux, pmh_uy, pmh_ut, pmh_T);
    }

    for (int i = row_s; i < row_e; ++i) {
        const bool has_p = (i + 1 < nz) || k.xper;
        F2 xp_n[5], x0_n[9], xm_n[5];
        PM2 pm_n;
        float nh_ux = 0, nh_uy = 0, nh_ut = 0, nh_T = 0;
        if (has_p) {
            if (!rs.get(v, hv)) return rs.finish();
            groups2(v, hv, lane, xm_n, x0_n, xp_n);
            pm_n = moments2(v, k);
            halo_fields(k, hv, nh_ux, nh_uy, nh_ut, nh_T);
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) xp_n[q] = xm_n[q] = sp(0.0f);
#pragma unroll
            for (int q = 0; q < 9; ++q) x0_n[q] = sp(0.0f);
            pm_n = pm_cur;
        }

        // pulled values of the pair
        F2 fv[9], gv[5], hv5[5];
        fv[1] = xm_prev[0]; fv[5] = xm_prev[1]; fv[8] = xm_prev[2]; gv[1] = xm_prev[3]; hv5[1] = xm_prev[4];
        fv[0] = x0_cur[0]; fv[2] = x0_cur[1]; fv[4] = x0_cur[2];
        gv[0] = x0_cur[3]; gv[2] = x0_cur[4]; gv[4] = x0_cur[5];
        hv5[0] = x0_cur[6]; hv5[2] = x0_cur[7]; hv5[4] = x0_cur[8];
        fv[3] = xp_n[0]; fv[6] = xp_n[1]; fv[7] = xp_n[2]; gv[3] = xp_n[3]; hv5[3] = xp_n[4];

        row_tail<S, true>(k, OwnGlobal<S>{src, &k, i, L.Ac}, dst, L, i, has_m, has_p, salt, fv, gv, hv5, pm_cur, pm_n, uy_prev, pmh_ux, pmh_uy,
                    pmh_ut, pmh_T);

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
        pmh_ux = nh_ux;
        pmh_uy = nh_uy;
        pmh_ut = nh_ut;
        pmh_T = nh_T;
        has_m = true;
    }
}

// ---- the march with the rows resident in shared memory ------------------------
//
// The same row update with no row carried in registers: the TMA ring keeps
// the rows i - 1, i and i + 1 of the step in shared memory and the pulled
// values are read straight from them, the radial shift being a column offset
// (the stage holds the two halo columns).  Row i - 1 is released once its
// e_x = +1 group is read, so that the copy of row i + 2 is in flight during
// the step.  R stages (R >= 3) per warp; with R = 4 one more row is in flight.

template <typename S, int R> struct RowRing {
    static_assert(R >= 3, "rows i - 1, i and i + 1 must fit");
    const CUtensorMap *map;
    const unsigned char *ring;  // this warp's stages
    uint32_t ring_s, bar_s;     // shared addresses of the stages and of barrier 0
    uint32_t bar_stride;        // bytes between consecutive barriers
    int first, nrows, nz, x0, lane, waited, issued;
    int *status;
    // Sequence number of row 0 of the current march: a warp that marches
    // several times through one ring (one time step after another) keeps its
    // barriers, initialised once, and continues their phases instead of
    // initialising them again (which a valid mbarrier does not allow).
    int base = 0;

    __device__ __forceinline__ void issue(int t)
    {
        int row = first + t;
        row = row >= nz ? row - nz : (row < 0 ? row + nz : row);
        const int st = (base + t) % R;
        const uint32_t bar = bar_s + bar_stride * st, dst = ring_s + (uint32_t)(TmaGeom<S>::stage_bytes * st);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)TmaGeom<S>::box_bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst),
            "l"((unsigned long long)map), "r"(x0), "r"(row), "r"(0), "r"(bar)
            : "memory");
    }

    __device__ __forceinline__ void start()
    {
        if (lane == 0) {
            for (int s = 0; s < R; ++s)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s + bar_stride * s) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        prime();
    }

    // the first copies of a march (barriers already initialised)
    __device__ __forceinline__ void prime()
    {
        waited = 0;
        issued = nrows < R ? nrows : R;
        if (lane == 0)
            for (int t = 0; t < issued; ++t) issue(t);
        __syncwarp();
    }

    // the next march through the same ring continues the sequence
    __device__ __forceinline__ void advance() { base += nrows; }

    __device__ __forceinline__ bool wait_one(int t)
    {
        const int q = base + t;
        return mbar_wait_bounded(bar_s + bar_stride * (q % R), (uint32_t)((q / R) & 1), kTmaWaitLimit);
    }

    // rows up to sequence index t have landed (false after a timeout, with
    // the status word set)
    __device__ __forceinline__ bool wait_upto(int t)
    {
        bool ok = true;
        while (waited <= t) {
            if (!wait_one(waited)) {
                ok = false;
                break;
            }
            ++waited;
        }
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicExch(status, (int)LB_ERR_TIMEOUT);
            return false;
        }
        return true;
    }

    __device__ __forceinline__ const S *stage(int t) const
    {
        return reinterpret_cast<const S *>(ring + TmaGeom<S>::stage_bytes * ((base + t) % R));
    }

    // every lane is done with row t: its stage takes row t + R
    __device__ __forceinline__ void release(int t)
    {
        __syncwarp();
        if (t + R < nrows) {
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(t + R);
            }
            issued = t + R + 1;
        }
    }

    // after an error: give the copies still in flight a bounded wait
    __device__ __forceinline__ void finish()
    {
        for (int t = waited; t < issued; ++t) (void)wait_one(t);
    }
};

// stage reads: the pair (A, B), the pair shifted one column left (A - 1, A)
// or right (B, B + 1), and one column (the halo lanes)
template <typename S> struct StageRd {
    const S *b;
    int cA;  // column of A inside the stage
    float is;
    __device__ __forceinline__ F2 pair(int q) const
    {
        return LoadScaled<S>::pair(b + q * TmaGeom<S>::cols + cA, is);
    }
    __device__ __forceinline__ F2 left(int q) const
    {
        const S *p = b + q * TmaGeom<S>::cols + cA;
        return mk2(LoadScaled<S>::one(p - 1, is), LoadScaled<S>::one(p, is));
    }
    __device__ __forceinline__ F2 right(int q) const
    {
        const S *p = b + q * TmaGeom<S>::cols + cA;
        return mk2(LoadScaled<S>::one(p + 1, is), LoadScaled<S>::one(p + 2, is));
    }
    __device__ __forceinline__ float col(int q, int c) const
    {
        return LoadScaled<S>::one(b + q * TmaGeom<S>::cols + c, is);
    }
};

// kSplit: interior rows of warps without wall or axis columns take the
// interior form of row_tail.  kOwnStage: the wall and axis rules read the own
// values from the ring (else from src).
template <typename S, int R, bool kSplit, bool kOwnStage>
__device__ __forceinline__ void march3(const KP<float> &k, const S *__restrict__ src, S *__restrict__ dst, int c0,
                                       int row_s, int row_e, uint32_t salt, RowRing<S, R> &rs)
{
    const Lane2 L = lane2(k, c0);
    const int lane = L.lane, nz = k.nz;
    constexpr int O = TmaGeom<S>::off;
    const int hc = lane == 0 ? O - 1 : O + 64;  // halo column of lanes 0 / 31
    const int first = (row_s > 0 || k.xper) ? row_s - 1 : row_s;
    StageRd<S> rd{nullptr, O + 2 * lane, k.inv_scale};

    // stored-state fields of row row_s (and u_y of row row_s - 1)
    PM2 pm_cur;
    float pmh_ux, pmh_uy, pmh_ut, pmh_T;
    F2 uy_prev = sp(0.0f);
    {
        if (!rs.wait_upto(row_s - first)) return rs.finish();
        F2 v[NQ];
        float hv[NQ];
        if (row_s > first) {
            rd.b = rs.stage(0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] = rd.pair(q);
            uy_prev = moments2(v, k).uy;
        }
        rd.b = rs.stage(row_s - first);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            v[q] = rd.pair(q);
            hv[q] = rd.col(q, hc);
        }
        pm_cur = moments2(v, k);
        halo_fields(k, hv, pmh_ux, pmh_uy, pmh_ut, pmh_T);
    }

    for (int i = row_s; i < row_e; ++i) {
        const bool has_m = i > 0 || k.xper;
        const bool has_p = (i + 1 < nz) || k.xper;
        const int t = i - first;
        if (has_p && !rs.wait_upto(t + 1)) return rs.finish();

        F2 fv[9], gv[5], hv5[5];
        OwnStage<S> own{rs.stage(t), O + 2 * lane, k.inv_scale, 0.0f, 0.0f};
        // e_x = +1 group from row i - 1, then that row's stage is free
        if (has_m) {
            rd.b = rs.stage(t - 1);
            fv[1] = rd.pair(1);
            fv[5] = rd.left(5);
            fv[8] = rd.right(8);
            gv[1] = rd.pair(G0 + 1);
            hv5[1] = rd.pair(H0 + 1);
            if (kOwnStage && L.edge_warp) own.m8v = rd.pair(8).v.x;  // f8 of row i - 1, the lane's column
            rs.release(t - 1);
        } else {
            fv[1] = fv[5] = fv[8] = gv[1] = hv5[1] = sp(0.0f);
        }
        // e_x = 0 group from row i
        rd.b = rs.stage(t);
        fv[0] = rd.pair(0);
        fv[2] = rd.left(2);
        fv[4] = rd.right(4);
        gv[0] = rd.pair(G0 + 0);
        gv[2] = rd.left(G0 + 2);
        gv[4] = rd.right(G0 + 4);
        hv5[0] = rd.pair(H0 + 0);
        hv5[2] = rd.left(H0 + 2);
        hv5[4] = rd.right(H0 + 4);
        // e_x = -1 group and the stored-state fields of row i + 1
        PM2 pm_n;
        float nh_ux = 0, nh_uy = 0, nh_ut = 0, nh_T = 0;
        if (has_p) {
            rd.b = rs.stage(t + 1);
            F2 v[NQ];
            float hv[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                v[q] = rd.pair(q);
                hv[q] = rd.col(q, hc);
            }
            pm_n = moments2(v, k);
            halo_fields(k, hv, nh_ux, nh_uy, nh_ut, nh_T);
            fv[3] = v[3];
            fv[6] = rd.left(6);
            fv[7] = rd.right(7);
            gv[3] = v[G0 + 3];
            hv5[3] = v[H0 + 3];
            own.p7v = v[7].v.x;  // f7 of row i + 1 at the lane's column (axis mirror)
        } else {
            fv[3] = fv[6] = fv[7] = gv[3] = hv5[3] = sp(0.0f);
            pm_n = pm_cur;
        }

        if (kSplit && has_m && has_p && !L.edge_warp)
            row_tail<S, false>(k, own, dst, L, i, has_m, has_p, salt, fv, gv, hv5, pm_cur, pm_n, uy_prev, pmh_ux,
                               pmh_uy, pmh_ut, pmh_T);
        else if (kOwnStage)
            row_tail<S, true>(k, own, dst, L, i, has_m, has_p, salt, fv, gv, hv5, pm_cur, pm_n, uy_prev, pmh_ux,
                              pmh_uy, pmh_ut, pmh_T);
        else
            row_tail<S, true>(k, OwnGlobal<S>{src, &k, i, L.Ac}, dst, L, i, has_m, has_p, salt, fv, gv, hv5, pm_cur,
                              pm_n, uy_prev, pmh_ux, pmh_uy, pmh_ut, pmh_T);

        uy_prev = pm_cur.uy;
        pm_cur = pm_n;
        pmh_ux = nh_ux;
        pmh_uy = nh_uy;
        pmh_ut = nh_ut;
        pmh_T = nh_T;
    }
}
