// egfem_df64.cuh -- "double-float" numbers: an unevaluated sum hi + lo of two FP32 values,
// giving a 48-bit significand with FP32 exponent range, computed on the FP32 pipe.
//
// The mixed-precision Krylov solver keeps its vectors in this format: GB300 executes FP32
// at about 58 times the FP64 rate, so df64 vector arithmetic costs little while its
// precision keeps BiCGStab's recurrences as stable as in FP64 (plain FP32 vectors make
// BiCGStab diverge on the 2D problems of interest, see egfem_krylov.cuh).
//
// The operations are the classical error-free transformations -- Knuth's TwoSum, Dekker's
// Fast2Sum, and the FMA-based exact product -- composed as in double-double arithmetic
// (Dekker 1971; Hida, Li & Bailey 2001), written here for FP32 pairs.  Explicit _rn
// intrinsics keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace egfem {

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df64 df_from(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - double(hi))};
}

__device__ __forceinline__ df64 df_from(float x) { return {x, 0.f}; }

__device__ __forceinline__ double df_to_double(df64 a) { return double(a.hi) + double(a.lo); }

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    df64 s = df_two_sum(a.hi, b.hi);
    const df64 t = df_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64 df_neg(df64 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64 df_mul(float a, df64 b) {
    const float p = __fmul_rn(a, b.hi);
    float e = __fmaf_rn(a, b.hi, -p);
    e = __fmaf_rn(a, b.lo, e);
    return df_fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ df64 df_fma(float a, df64 b, df64 c) { return df_add(df_mul(a, b), c); }

}  // namespace egfem
