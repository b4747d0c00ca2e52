// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits, from FP32 operations only
// (Dekker, "A floating-point technique for extending the available precision", 1971;
// Knuth's TwoSum; the exact product by FMA).  On this GPU FP64 runs at 1/64 of the FP32
// rate, so the one quantity of the mixed form that needs more than FP32 -- the
// reprojection residual f s p - u, whose ~500 px terms cancel to ~1 px -- is computed
// this way.  The error-free transformations use the _rn intrinsics so the compiler
// neither contracts nor reassociates them.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace gbba {

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_from(float a) { return {a, 0.0f}; }

// hi + lo of a double, rounded twice.
__device__ __forceinline__ DF df_from_double(double a) {
    const float hi = (float)a;
    return {hi, (float)(a - (double)hi)};
}

__device__ __forceinline__ float df_to_float(DF a) { return __fadd_rn(a.hi, a.lo); }

// s + e = a + b exactly (Knuth's TwoSum, no condition on the operands).
__device__ __forceinline__ DF two_sum_f(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ DF fast_two_sum_f(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum_f(a.hi, b.hi);
    return fast_two_sum_f(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
    const DF s = two_sum_f(a.hi, b);
    return fast_two_sum_f(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }

// a b: the exact product of the high parts (fma gives its error), plus the cross terms.
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum_f(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum_f(p, e);
}

// 1 / b: the FP32 reciprocal x of b.hi, then one Newton step y = x + x (1 - b x) with
// 1 - b x taken in df (b x is within an ulp of 1, so 1 - hi(b x) is exact).
__device__ __forceinline__ DF df_rcp(DF b) {
    const float x = __frcp_rn(b.hi);
    const DF bx = df_mul_f(b, x);
    const float e = __fsub_rn(__fsub_rn(1.0f, bx.hi), bx.lo);
    return fast_two_sum_f(x, __fmul_rn(x, e));
}

// Camera of a df residual: FP32 record plus its low-order record.
struct CamDF {
    DF R[9], t[3], f, k1, k2;
};

__device__ __forceinline__ CamDF load_cam_df(const float* __restrict__ rec, const float* __restrict__ lo) {
    const float4* r4 = reinterpret_cast<const float4*>(rec);
    const float4* l4 = reinterpret_cast<const float4*>(lo);
    float h[16], l[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 a = __ldg(r4 + k), b = __ldg(l4 + k);
        h[4 * k] = a.x; h[4 * k + 1] = a.y; h[4 * k + 2] = a.z; h[4 * k + 3] = a.w;
        l[4 * k] = b.x; l[4 * k + 1] = b.y; l[4 * k + 2] = b.z; l[4 * k + 3] = b.w;
    }
    CamDF c;
#pragma unroll
    for (int i = 0; i < 9; ++i) c.R[i] = {h[CP_R + i], l[CP_R + i]};
#pragma unroll
    for (int i = 0; i < 3; ++i) c.t[i] = {h[CP_T + i], l[CP_T + i]};
    c.f = {h[CP_F], l[CP_F]};
    c.k1 = {h[CP_K1], l[CP_K1]};
    c.k2 = {h[CP_K2], l[CP_K2]};
    return c;
}

// The Snavely residual of Sec. VI-A in df arithmetic: P = R X + t, d = P.z -+ eps
// (d_safe), p = -P.xy / d, s = 1 + k1 |p|^2 + k2 |p|^4, r = f s p - u.  Its error is a
// few units of 2^-48 of the ~500 px terms, so rounded to FP32 it is the exact residual
// to within an ulp of itself.
__device__ __forceinline__ void residual_df(const CamDF& c, const DF (&X)[3], float eps, float u0, float u1,
                                            DF& r0, DF& r1) {
    DF P[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        DF a = df_mul(c.R[3 * i], X[0]);
        a = df_add(a, df_mul(c.R[3 * i + 1], X[1]));
        a = df_add(a, df_mul(c.R[3 * i + 2], X[2]));
        P[i] = df_add(a, c.t[i]);
    }
    const DF d = df_add_f(P[2], P[2].hi >= 0.0f ? eps : -eps);
    const DF iz = df_rcp(d);
    const DF p0 = df_neg(df_mul(P[0], iz)), p1 = df_neg(df_mul(P[1], iz));
    const DF n2 = df_add(df_mul(p0, p0), df_mul(p1, p1));
    const DF s = df_add_f(df_mul(n2, df_add(c.k1, df_mul(c.k2, n2))), 1.0f);
    const DF fs = df_mul(c.f, s);
    r0 = df_add_f(df_mul(fs, p0), -u0);
    r1 = df_add_f(df_mul(fs, p1), -u1);
}

}  // namespace gbba
