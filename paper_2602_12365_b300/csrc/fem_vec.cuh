// Lane-vector arithmetic for the element kernels.
//
// V is the type one lane computes with: double (FP64 calls), float (FP32
// calls, one element per lane) or F2 (FP32 calls, two elements per lane in
// the two halves of a packed pair, evaluated with the sm_100+ paired FP32
// instructions __ffma2_rn / __fadd2_rn / __fmul2_rn).  Every routine in
// fem_material.cuh is written once against this interface.
#pragma once
#include <cuda_runtime.h>

namespace fem {

struct F2 {
    float2 v;
};

__device__ __forceinline__ F2 mk2(float a, float b) { return F2{make_float2(a, b)}; }

template <class V>
struct VT;
template <>
struct VT<float> {
    using S = float;
    static constexpr int N = 1;
};
template <>
struct VT<double> {
    using S = double;
    static constexpr int N = 1;
};
template <>
struct VT<F2> {
    using S = float;
    static constexpr int N = 2;
};

template <class V>
__device__ __forceinline__ V splat(typename VT<V>::S s);
template <>
__device__ __forceinline__ float splat<float>(float s) {
    return s;
}
template <>
__device__ __forceinline__ double splat<double>(double s) {
    return s;
}
template <>
__device__ __forceinline__ F2 splat<F2>(float s) {
    return mk2(s, s);
}

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
// a - b as b * (-1) + a: one rounding, identical to the scalar difference
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    return F2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)};
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2{__fmul2_rn(a.v, make_float2(-1.f, -1.f))}; }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) {
    a = a + b;
    return a;
}
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) {
    a = a - b;
    return a;
}

// ---------------------------------------------------------------------------
// reciprocal: the hardware approximation (rcp.approx) refined by one Newton
// step r' = r + r (1 - x r), which leaves about one ulp of error in FP32
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vrcp(float x) {
    const float r = rcp_approx(x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double vrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 vrcp(F2 x) {
    const F2 r = mk2(rcp_approx(x.v.x), rcp_approx(x.v.y));
    const F2 e = F2{__ffma2_rn(make_float2(-x.v.x, -x.v.y), r.v, make_float2(1.f, 1.f))};
    return F2{__ffma2_rn(r.v, e.v, r.v)};
}

// ---------------------------------------------------------------------------
// ln(1 + x) in FP32 from ln z = 2 artanh((z - 1) / (z + 1)) (Abramowitz and
// Stegun 4.1.27): with s = x / (2 + x), ln(1 + x) = 2 (s + s^3/3 + s^5/5 +
// ... + s^13/13).  For |x| <= 3/8, |s| <= 0.231 and the truncation error is
// below 2e-9 relative, so the result keeps about 2 ulp; outside that window
// the library log1pf is used.  FP64 calls use the library log1p.
// ---------------------------------------------------------------------------
constexpr float kLogSeriesMax = 0.375f;

template <class V>
__device__ __forceinline__ V log1p_series(V x, V two, V c3, V c5, V c7, V c9, V c11, V c13) {
    const V s = x * vrcp(two + x);
    const V s2 = s * s;
    V p = vfma(s2, c13, c11);
    p = vfma(s2, p, c9);
    p = vfma(s2, p, c7);
    p = vfma(s2, p, c5);
    p = vfma(s2, p, c3);
    const V t = vfma(s * s2, p, s);
    return t + t;
}

__device__ __forceinline__ float vlog1p(float x) {
    if (fabsf(x) > kLogSeriesMax) return log1pf(x);
    return log1p_series<float>(x, 2.f, 1.f / 3, 1.f / 5, 1.f / 7, 1.f / 9, 1.f / 11, 1.f / 13);
}
__device__ __forceinline__ double vlog1p(double x) { return log1p(x); }
__device__ __forceinline__ F2 vlog1p(F2 x) {
    if (fabsf(x.v.x) > kLogSeriesMax || fabsf(x.v.y) > kLogSeriesMax)
        return mk2(log1pf(x.v.x), log1pf(x.v.y));
    auto k = [](float c) { return mk2(c, c); };
    return log1p_series<F2>(x, k(2.f), k(1.f / 3), k(1.f / 5), k(1.f / 7), k(1.f / 9), k(1.f / 11),
                            k(1.f / 13));
}

// ln(1 + x) for x > -1 without a branch (the pair kernels, whose element
// arithmetic must stay one straight-line block): with 1 + x = 2^e m,
// m in [sqrt(1/2), sqrt(2)) (e from the exponent bits of 1 + x),
// ln(1 + x) = e ln 2 + ln(1 + z), z = m - 1 = x 2^-e + (2^-e - 1) formed by one
// FMA (exact scaling, one rounding), and ln(1 + z) by the artanh series above
// (|z| <= 0.415, |s| <= 0.172: truncation below 1e-12 relative).  For
// 1 + x in [sqrt(1/2), sqrt(2)) the scale is 1 and z = x exactly, so small
// strains keep full relative accuracy.  FP64 calls do not use it.
__device__ __forceinline__ int ln_exponent(float x, float& scale) {
    const int e = (__float_as_int(1.0f + x) - 0x3f3504f3) >> 23;  // floor(log2((1 + x) / sqrt(1/2)))
    scale = __int_as_float((127 - e) << 23);                     // 2^-e
    return e;
}
constexpr float kLn2 = 0.693147180559945309f;
__device__ __forceinline__ float vlog1p_bf(float x) {
    float sc;
    const int e = ln_exponent(x, sc);
    const float z = fmaf(x, sc, sc - 1.0f);
    return fmaf((float)e, kLn2, log1p_series<float>(z, 2.f, 1.f / 3, 1.f / 5, 1.f / 7, 1.f / 9, 1.f / 11, 1.f / 13));
}
__device__ __forceinline__ F2 vlog1p_bf(F2 x) {
    float s0, s1;
    const int e0 = ln_exponent(x.v.x, s0), e1 = ln_exponent(x.v.y, s1);
    const F2 sc = mk2(s0, s1);
    const F2 z = F2{__ffma2_rn(x.v, sc.v, make_float2(s0 - 1.0f, s1 - 1.0f))};
    auto k = [](float c) { return mk2(c, c); };
    const F2 l = log1p_series<F2>(z, k(2.f), k(1.f / 3), k(1.f / 5), k(1.f / 7), k(1.f / 9), k(1.f / 11),
                                  k(1.f / 13));
    return F2{__ffma2_rn(make_float2((float)e0, (float)e1), make_float2(kLn2, kLn2), l.v)};
}

__device__ __forceinline__ float vabs(float x) { return fabsf(x); }
__device__ __forceinline__ double vabs(double x) { return fabs(x); }
__device__ __forceinline__ F2 vabs(F2 x) { return mk2(fabsf(x.v.x), fabsf(x.v.y)); }

// bit c set when component c is > 0
__device__ __forceinline__ int vpos(float x) { return x > 0.f ? 1 : 0; }
__device__ __forceinline__ int vpos(double x) { return x > 0.0 ? 1 : 0; }
__device__ __forceinline__ int vpos(F2 x) { return (x.v.x > 0.f ? 1 : 0) | (x.v.y > 0.f ? 2 : 0); }

// keep components whose bit is set, replace the others by `alt`
__device__ __forceinline__ float vsel(int bits, float x, float alt) { return (bits & 1) ? x : alt; }
__device__ __forceinline__ double vsel(int bits, double x, double alt) { return (bits & 1) ? x : alt; }
__device__ __forceinline__ F2 vsel(int bits, F2 x, float alt) {
    return mk2((bits & 1) ? x.v.x : alt, (bits & 2) ? x.v.y : alt);
}

// component c as double (for FP64 accumulation)
__device__ __forceinline__ double vget(float x, int) { return (double)x; }
__device__ __forceinline__ double vget(double x, int) { return x; }
__device__ __forceinline__ double vget(F2 x, int c) { return (double)(c ? x.v.y : x.v.x); }

__device__ __forceinline__ float vcomp(float x, int) { return x; }
__device__ __forceinline__ double vcomp(double x, int) { return x; }
__device__ __forceinline__ float vcomp(F2 x, int c) { return c ? x.v.y : x.v.x; }

}  // namespace fem
