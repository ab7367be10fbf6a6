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

// c + a b for double-float a, b accumulated into c: the exact product of the high words plus the
// cross terms, then TwoSum of the high words with the low words and errors carried (the
// compensated accumulation of the inner products, kept as a pair)
__device__ __forceinline__ df64 df_acc_prod(df64 c, df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df64 s = df_two_sum(c.hi, p);
    return df_fast_two_sum(s.hi, __fadd_rn(__fadd_rn(c.lo, e), s.lo));
}

// c + a for double-float a, c (TwoSum of the high words, low words and error carried)
__device__ __forceinline__ df64 df_acc(df64 c, df64 a) {
    const df64 s = df_two_sum(c.hi, a.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(__fadd_rn(c.lo, a.lo), s.lo));
}

// x 2^-sc as a pair of floats (hi, lo) built from the bit pattern with integer operations (no
// FP64 instruction): hi holds the leading 24 significand bits, lo the next 23 (lo = 0 below 2^-80
// after scaling), so hi + lo equals x 2^-sc to a relative error below 2^-46.  Zero and values
// below 2^-126 after scaling give (0, 0); infinities, NaN and values beyond the float range after
// scaling give a non-finite hi, so a non-finite input still makes the results non-finite.
__device__ __forceinline__ df64 split_dbl(double x, int sc) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi32 = unsigned(b >> 32), lo32 = unsigned(b);
    const unsigned sign = hi32 & 0x80000000u;
    const int eb = int((hi32 >> 20) & 0x7ffu);
    const int e = eb - sc;
    df64 r;
    if (eb == 0x7ff || e > 1150) {
        const bool nan = eb == 0x7ff && ((hi32 & 0xfffffu) | lo32) != 0u;
        r.hi = __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
        r.lo = 0.f;
    } else if (e < 897) {
        r.hi = 0.f;
        r.lo = 0.f;
    } else {
        r.hi = __uint_as_float(sign | (unsigned(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
        const float f = __fsub_rn(__uint_as_float(0x4B000000u | ((lo32 >> 6) & 0x7fffffu)), 8388608.0f);
        r.lo = e >= 943 ? __fmul_rn(f, __uint_as_float(sign | (unsigned(e - 942) << 23))) : 0.f;
    }
    return r;
}

// A float as a double, exactly, from its bit pattern (integer operations; subnormal floats, which
// the accumulations here never produce at a relevant size, give 0)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double(static_cast<long long>(sign));
    const unsigned long long ex = e == 0xffu ? 0x7ffull : static_cast<unsigned long long>(e + 896u);
    return __longlong_as_double(static_cast<long long>(sign | (ex << 52) | (static_cast<unsigned long long>(u & 0x7fffffu) << 29)));
}

// hi + lo rounded to a double: two exact conversions and one FP64 addition
__device__ __forceinline__ double df_to_double_bits(df64 a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace egfem
