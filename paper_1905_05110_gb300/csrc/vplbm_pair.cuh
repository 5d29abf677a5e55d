// Packed FP32x2 arithmetic for two nodes at once (Blackwell FFMA2 / FADD2 /
// FMUL2) and the VP-MRT update of two fluid nodes away from the body.
// Internal to the library.
#pragma once

#include "vplbm_node.cuh"

namespace vplbm {
namespace {

struct V2 {
    float2 v;
};
__device__ __forceinline__ V2 mk(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return {__fadd2_rn(a.v, b.v)}; }
// a - b as one fused op: b * (-1) is exact, so the single rounding equals a - b
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

__device__ __forceinline__ float2 ld2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 ld2(const __half *p) { return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p))); }
__device__ __forceinline__ void st2(float *p, V2 x) { *reinterpret_cast<float2 *>(p) = x.v; }
__device__ __forceinline__ void st2(__half *p, V2 x) { *reinterpret_cast<__half2 *>(p) = __float22half2_rn(x.v); }

// VP-MRT update of two fluid nodes away from the body (chi = 0): Eqs. (19),
// (22) with chi = 0, (14)-(17) in the closed forms of vplbm_node.cuh.
template <int P>
__device__ __forceinline__ void pair_update(const StepParams &p, const V2 f[NQ], typename Prec<P>::S *fout, long long b)
{
    const PairConsts &k = p.pc;
    const V2 d13 = f[1] - f[3], d24 = f[2] - f[4];
    const V2 b13 = f[1] + f[3], b24 = f[2] + f[4];
    const V2 d56 = f[5] - f[6], d87 = f[8] - f[7];
    const V2 a56 = f[5] + f[6], a78 = f[7] + f[8];
    const V2 sx = d56 + d87, ty = a56 - a78;
    const V2 sa = b13 + b24, sd = a56 + a78;
    const V2 rs = (f[0] + sa) + sd;
    const V2 rho = rs + mk(p.rho0f);
    const V2 jx = d13 + sx, qx = fma2(mk(-2.f), d13, sx);
    const V2 jy = d24 + ty, qy = fma2(mk(-2.f), d24, ty);
    const V2 e = fma2(mk(-4.f), f[0], fma2(mk(2.f), sd, mk(0.f) - sa));
    const V2 ep = fma2(mk(4.f), f[0], fma2(mk(-2.f), sa, sd));
    const V2 pxx = b13 - b24;
    const V2 pxy = (f[5] + f[7]) - (f[6] + f[8]);

    const V2 inv = {make_float2(__frcp_rn(rho.v.x), __frcp_rn(rho.v.y))};
    const V2 ux = fma2(jx, inv, mk(k.hgx));
    const V2 uy = fma2(jy, inv, mk(k.hgy));
    const V2 Gx = rho * mk(p.gxf), Gy = rho * mk(p.gyf);

    const V2 ux2 = ux * ux, uy2 = uy * uy;
    const V2 u2r = rho * (ux2 + uy2);
    const V2 uG = fma2(ux, Gx, uy * Gy);
    const V2 e_s = fma2(mk(k.om1), e, fma2(mk(p.sf[1]), fma2(mk(3.f), u2r, mk(-2.f) * rs), mk(k.h1x6) * uG));
    const V2 ep_s = fma2(mk(k.om2), ep, fma2(mk(p.sf[2]), fma2(mk(-3.f), u2r, rs), mk(k.mh2x6) * uG));
    const V2 jx_s = jx + Gx, jy_s = jy + Gy;
    const V2 qx_s = fma2(mk(k.om4), qx, fma2(mk(-p.sf[4]), rho * ux, mk(k.mh4) * Gx));
    const V2 qy_s = fma2(mk(k.om6), qy, fma2(mk(-p.sf[6]), rho * uy, mk(k.mh6) * Gy));
    const V2 pxx_s = fma2(mk(k.om7), pxx, fma2(mk(p.sf[7]), rho * (ux2 - uy2), mk(k.h7x2) * (ux * Gx - uy * Gy)));
    const V2 pxy_s = fma2(mk(k.om8), pxy, fma2(mk(p.sf[8]), rho * (ux * uy), mk(k.h8) * fma2(ux, Gy, uy * Gx)));

    // back to populations, M^-1 = M^T diag(1/|row|^2)
    const V2 r9 = rs * mk(1.f / 9.f);
    const V2 A = fma2(mk(-1.f / 36.f), e_s, fma2(mk(-1.f / 18.f), ep_s, r9));
    const V2 B = fma2(mk(1.f / 18.f), e_s, fma2(mk(1.f / 36.f), ep_s, r9));
    const V2 X1 = (jx_s - qx_s) * mk(1.f / 6.f);
    const V2 Y1 = (jy_s - qy_s) * mk(1.f / 6.f);
    const V2 X2 = fma2(jx_s, mk(1.f / 6.f), qx_s * mk(1.f / 12.f));
    const V2 Y2 = fma2(jy_s, mk(1.f / 6.f), qy_s * mk(1.f / 12.f));
    const V2 Pq = pxx_s * mk(0.25f), Rq = pxy_s * mk(0.25f);
    const V2 AP = A + Pq, AM = A - Pq, BP = B + Rq, BM = B - Rq;
    const V2 XY = X2 + Y2, XmY = X2 - Y2;
    const long long ps = p.ps;
    st2(fout + b, fma2(mk(-1.f / 9.f), e_s, fma2(mk(1.f / 9.f), ep_s, r9)));
    st2(fout + ps + b, AP + X1);
    st2(fout + 2 * ps + b, AM + Y1);
    st2(fout + 3 * ps + b, AP - X1);
    st2(fout + 4 * ps + b, AM - Y1);
    st2(fout + 5 * ps + b, BP + XY);
    st2(fout + 6 * ps + b, BM - XmY);
    st2(fout + 7 * ps + b, BP - XY);
    st2(fout + 8 * ps + b, BM + XmY);

    const float r0 = rho.v.x, r1 = rho.v.y;
    if (!(r0 > 0.f) || !(r0 < 1e30f) || !(r1 > 0.f) || !(r1 < 1e30f)) *p.err = ERR_NONFINITE;
}

}  // namespace
}  // namespace vplbm
