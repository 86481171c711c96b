// Double-float ("float-float") arithmetic on the float32 pipes: a value is the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2 after
// normalisation, carrying ~48 significant bits.  Products use the exact
// two-product of an FMA (Dekker), sums the error-free two-sum (Knuth).  This
// GPU's float64 rate is a small fraction of its float32 rate, so
// float64-accurate streaming arithmetic (the Gram-Schmidt projections of the
// mixed-precision GMRES) runs faster this way than in float64.
//
// A complex double-float is stored as float4 (hi.re, hi.im, lo.re, lo.im):
// the 16 bytes of a double2.
#pragma once
#include <cuda_runtime.h>

namespace vie {

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_norm(float& hi, float& lo) {  // fast two-sum, |hi| >= |lo|
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}

// (ah, al) += (xh + xl) (yh + yl), dropping the xl yl term (~2^-48 relative);
// the accumulator is left unnormalised (al collects the error terms)
__device__ __forceinline__ void df_acc(float& ah, float& al, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    float s, t;
    df_two_sum(ah, p, s, t);
    ah = s;
    al += t + e;
}

__device__ __forceinline__ float4 df_from(double2 v) {
    const float hx = (float)v.x, hy = (float)v.y;
    return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}
__device__ __forceinline__ double2 df_to(float4 v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// acc += conj(v) w (complex, unnormalised accumulators: re (h, l), im (h, l))
__device__ __forceinline__ void df_cmac_conj(float4& acc, float4 v, float4 w) {
    df_acc(acc.x, acc.z, v.x, v.z, w.x, w.z);
    df_acc(acc.x, acc.z, v.y, v.w, w.y, w.w);
    df_acc(acc.y, acc.w, v.x, v.z, w.y, w.w);
    df_acc(acc.y, acc.w, -v.y, -v.w, w.x, w.z);
}
// acc -= v h
__device__ __forceinline__ void df_cmsub(float4& acc, float4 v, float4 h) {
    df_acc(acc.x, acc.z, -v.x, -v.z, h.x, h.z);
    df_acc(acc.x, acc.z, v.y, v.w, h.y, h.w);
    df_acc(acc.y, acc.w, -v.x, -v.z, h.y, h.w);
    df_acc(acc.y, acc.w, -v.y, -v.w, h.x, h.z);
}
__device__ __forceinline__ float4 df_normed(float4 a) {
    df_norm(a.x, a.z);
    df_norm(a.y, a.w);
    return a;
}
// s v for a real double-float s = (sh, sl)
__device__ __forceinline__ float4 df_scale(float4 v, float sh, float sl) {
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    df_acc(r.x, r.z, v.x, v.z, sh, sl);
    df_acc(r.y, r.w, v.y, v.w, sh, sl);
    return df_normed(r);
}

}  // namespace vie
