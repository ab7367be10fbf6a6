// egfem_krylov.cuh -- BiCGStab (van der Vorst 1992) on the Jacobi-scaled system
// (D J) x = D b, D = diag(J)^{-1}, with the matrix in the slice-interleaved (SELL-32)
// layout of the tensor's local columns.
//
// V is the vector/matrix type: double (FP64 path) or float (mixed path).  Every thread
// owns R = 16 / sizeof(V) consecutive rows (2 in FP64, 4 in FP32) and moves them with
// one 128-bit load or store per array, so a warp keeps 512 B per stream in flight.
// Vectors are padded to whole slices (pad entries stay zero), so no kernel needs a
// bounds check inside a slice.  Dot products are summed per thread in V and across
// threads and blocks in double, in a fixed order (deterministic results).
//
// FP32 operator application uses the difference form
//     (A p)_i = s_i p_i + sum_{c != i} A_ic (p_c - p_i),   s_i = sum_c A_ic,
// with the row sum s_i stored in place of the diagonal.  For the smooth vectors of an
// elliptic problem the plain FP32 sum cancels O(|A||p|) terms down to O(h^2 |p|) and
// loses ~5 digits (BiCGStab then diverges); the difference form does not cancel.
//
// Every kernel of an iteration reads the device state first and returns at once when
// the solve has finished, so a captured chunk of iterations can overshoot the last one
// at the cost of empty launches only.  Cross-block reductions use the "last block
// finishes" pattern (one atomic ticket per block, no waiting), so no kernel spins.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "egfem_df64.cuh"
#include "egfem_internal.h"

namespace egfem {

constexpr int KRY_BLOCK = 256;

enum KDone : int32_t { K_RUNNING = 0, K_CONVERGED = 1, K_MAXIT = 2, K_BREAKDOWN = 3, K_NONFINITE = 4, K_STAGNATED = 5 };

struct KState {
    double rho, alpha, omega, beta;
    double rr;          // ||r||^2 of the current iterate
    double rr0;         // ||r_0||^2
    double tol2;        // stop when rr <= tol2
    double best_rr;     // smallest rr so far (stagnation guard)
    double stall_rr;    // the stagnation guard acts only once best_rr <= stall_rr
    double scratch[2];
    int32_t iter, maxit, done, last_improve;
    int32_t stall;      // iterations without a 10% improvement before K_STAGNATED (0: off)
    uint32_t ticket;
};

// Per vector type V: the 128-bit word moved per load (type), the index word (idx), the
// rows per thread (R), the operator value type (mat) and whether the operator is applied in
// the difference form (diff).  df64 vectors use an FP32 operator in difference form.
template <typename V> struct VecT;
template <> struct VecT<double> {
    using type = double2; using idx = int2; using mat = double; static constexpr int R = 2; static constexpr bool diff = false;
};
template <> struct VecT<float> {
    using type = float4; using idx = int4; using mat = float; static constexpr int R = 4; static constexpr bool diff = true;
};
template <> struct VecT<df64> {
    using type = float4; using idx = int2; using mat = float; static constexpr int R = 2; static constexpr bool diff = true;
};

// conversions and arithmetic that read the same for double, float and df64
template <typename V> __device__ __forceinline__ V cvt(double x);
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return float(x); }
template <> __device__ __forceinline__ df64 cvt<df64>(double x) { return df_from(x); }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return double(x); }
__device__ __forceinline__ double to_d(df64 x) { return df_to_double(x); }
__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return df_sub(a, b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 operator*(float a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { a = df_add(a, b); return a; }
__device__ __forceinline__ double ldg1(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldg1(const float *p) { return __ldg(p); }
__device__ __forceinline__ df64 ldg1(const df64 *p) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    return {t.x, t.y};
}

template <typename V>
struct Pack {
    V v[VecT<V>::R];
};

template <typename V>
__device__ __forceinline__ Pack<V> ldv(const V *p) {
    Pack<V> o;
    const typename VecT<V>::type t = *reinterpret_cast<const typename VecT<V>::type *>(p);
    if constexpr (std::is_same<V, df64>::value) { o.v[0] = {t.x, t.y}; o.v[1] = {t.z, t.w}; }
    else if constexpr (VecT<V>::R == 2) { o.v[0] = t.x; o.v[1] = t.y; }
    else { o.v[0] = t.x; o.v[1] = t.y; o.v[2] = t.z; o.v[3] = t.w; }
    return o;
}

template <typename V>
__device__ __forceinline__ void stv(V *p, const Pack<V> &o) {
    typename VecT<V>::type t;
    if constexpr (std::is_same<V, df64>::value) { t.x = o.v[0].hi; t.y = o.v[0].lo; t.z = o.v[1].hi; t.w = o.v[1].lo; }
    else if constexpr (VecT<V>::R == 2) { t.x = o.v[0]; t.y = o.v[1]; }
    else { t.x = o.v[0]; t.y = o.v[1]; t.z = o.v[2]; t.w = o.v[3]; }
    *reinterpret_cast<typename VecT<V>::type *>(p) = t;
}

template <typename M, int R>
// operator values and column indices are read-only during a solve: non-coherent loads, which
// the compiler may also schedule ahead of the solve's vector stores
__device__ __forceinline__ void ldm(const M *p, M (&o)[R]) {
    if constexpr (sizeof(M) * R == 16) {
        if constexpr (R == 2) { const double2 t = __ldg(reinterpret_cast<const double2 *>(p)); o[0] = t.x; o[1] = t.y; }
        else { const float4 t = __ldg(reinterpret_cast<const float4 *>(p)); o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w; }
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));   // two FP32 values (df64 rows)
        o[0] = t.x; o[1] = t.y;
    }
}

template <typename V>
__device__ __forceinline__ void ldi(const int32_t *p, int32_t (&c)[VecT<V>::R]) {
    const typename VecT<V>::idx t = __ldg(reinterpret_cast<const typename VecT<V>::idx *>(p));
    if constexpr (VecT<V>::R == 2) { c[0] = t.x; c[1] = t.y; }
    else { c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w; }
}

template <typename V>
struct KVecs {
    int64_t n_pad;      // rows rounded up to whole slices
    const SliceMeta *meta;
    const int32_t *col_idx;
    const int32_t *slice_off;   // column offsets of uniform slices
    const typename VecT<V>::mat *A;
    V *x, *r, *rh, *p, *v, *s, *t;
    const V *b;
    KState *st;
    double *part;       // [2 * gridDim.x]
};

// Per-thread dot-product accumulators.  FP64: plain FMA.  FP32: compensated dot product
// (Ogita, Rump & Oishi 2005, "Dot2"): each product is split exactly by an FMA and summed
// with Knuth's TwoSum, so the result is as accurate as if computed in twice the working
// precision.  BiCGStab's inner products cancel strongly once r is nearly orthogonal to
// the shadow residual; rounded FP32 products there give wrong alpha/beta and divergence.
// Explicit _rn intrinsics keep the compiler from contracting the error-free transforms.
template <typename V> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<df64> {
    float hi = 0.f, lo = 0.f;
    // a.hi b.hi exactly (FMA split) plus the cross terms a.hi b.lo + a.lo b.hi
    __device__ __forceinline__ void add(df64 a, df64 b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        const float t = __fadd_rn(hi, p);
        const float z = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
        lo = __fadd_rn(lo, __fadd_rn(err, e));
        hi = t;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};
template <> struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(hi, p);
        const float z = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
        lo = __fadd_rn(lo, __fadd_rn(err, e));
        hi = t;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-reduce NV values, store the block partials, and return true in the last block to
// finish, after which tot[0..NV) hold the grid totals (summed in block order).
template <int NV>
__device__ bool grid_reduce(double (&val)[NV], double *part, uint32_t *ticket, double (&tot)[NV]) {
    __shared__ double sh[NV][KRY_BLOCK / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = warp_sum(val[k]);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (int q = 0; q < KRY_BLOCK / 32; ++q) x += sh[k][q];
            part[k * gridDim.x + blockIdx.x] = x;
        }
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = 0.0;
        for (int q = threadIdx.x; q < int(gridDim.x); q += KRY_BLOCK) x += __ldcg(&part[k * gridDim.x + q]);
        x = warp_sum(x);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = 0.0;
        for (int q = 0; q < KRY_BLOCK / 32; ++q) x += sh[k][q];
        tot[k] = x;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// column indices of local column c for the R rows starting at r0: from the slice's
// offsets when the slice is uniform (no index traffic), else from col_idx
template <typename V>
__device__ __forceinline__ void row_cols(const KVecs<V> &K, const SliceMeta &M, int64_t r0, int64_t q, int c,
                                         int32_t (&col)[VecT<V>::R]) {
    if (M.off_base >= 0) {
        const int32_t o = __ldg(K.slice_off + M.off_base + c);
#pragma unroll
        for (int j = 0; j < VecT<V>::R; ++j) col[j] = int32_t(r0 + j) + o;
    } else {
        ldi<V>(K.col_idx + q, col);
    }
}

// y[r0 .. r0+R) = A xin for the R rows starting at r0 (r0 a multiple of R).
template <typename V>
__device__ __forceinline__ Pack<V> sell_rows(const KVecs<V> &K, int64_t r0, const V *xin) {
    constexpr int R = VecT<V>::R;
    using M_t = typename VecT<V>::mat;
    const SliceMeta M = K.meta[r0 / SLICE];
    const int lane = int(r0 % SLICE);
    Pack<V> y;
    if constexpr (VecT<V>::diff) {
        // difference form: column 0 holds the row sum s_i and the row's own value
        const Pack<V> xi = ldv(xin + r0);
        M_t a0[R];
        ldm(K.A + M.col_base + lane, a0);
#pragma unroll
        for (int j = 0; j < R; ++j) y.v[j] = a0[j] * xi.v[j];
        for (int c = 1; c < M.ncol; ++c) {
            const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
            M_t a[R];
            ldm(K.A + q, a);
            int32_t col[R];
            row_cols(K, M, r0, q, c, col);
#pragma unroll
            for (int j = 0; j < R; ++j) y.v[j] += a[j] * (ldg1(xin + col[j]) - xi.v[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) y.v[j] = cvt<V>(0.0);
        for (int c = 0; c < M.ncol; ++c) {
            const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
            M_t a[R];
            ldm(K.A + q, a);
            int32_t col[R];
            row_cols(K, M, r0, q, c, col);
#pragma unroll
            for (int j = 0; j < R; ++j) y.v[j] += a[j] * ldg1(xin + col[j]);
        }
    }
    return y;
}

__device__ __forceinline__ bool finished(const KState *st) { return *(volatile const int32_t *)&st->done != K_RUNNING; }

#define KRY_LOOP(K) \
    for (int64_t r0 = (int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x) * VecT<V>::R; r0 < (K).n_pad; \
         r0 += int64_t(gridDim.x) * KRY_BLOCK * VecT<V>::R)

// setup: x = 0, r = rh = p = b, v = 0, rho = (r, r)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_setup(KVecs<V> K, double rtol, int32_t maxit, int32_t stall) {
    constexpr int R = VecT<V>::R;
    double acc[1] = {0.0};
    Pack<V> z;
#pragma unroll
    for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
    KRY_LOOP(K) {
        const Pack<V> b = ldv(K.b + r0);
        stv(K.x + r0, z); stv(K.v + r0, z);
        stv(K.r + r0, b); stv(K.rh + r0, b); stv(K.p + r0, b);
#pragma unroll
        for (int j = 0; j < R; ++j) acc[0] += to_d(b.v[j]) * to_d(b.v[j]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        S.rho = tot[0]; S.rr = tot[0]; S.rr0 = tot[0]; S.best_rr = tot[0];
        S.tol2 = rtol * rtol * tot[0];
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0;
        S.iter = 0; S.maxit = maxit; S.last_improve = 0; S.stall = stall;
        S.stall_rr = 4e-6 * tot[0];   // the guard waits for a 500x residual reduction
        S.done = (tot[0] == 0.0) ? K_CONVERGED : (!isfinite(tot[0]) ? K_NONFINITE : K_RUNNING);
    }
}

// v = A p;  alpha = rho / (rh, v)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_v(KVecs<V> K) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    DotAcc<V> a;
    KRY_LOOP(K) {
        const Pack<V> y = sell_rows(K, r0, K.p);
        stv(K.v + r0, y);
        const Pack<V> rh = ldv(K.rh + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) a.add(rh.v[j], y.v[j]);
    }
    double acc[1] = {a.value()}, tot[1];
    if (grid_reduce<1>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (tot[0] == 0.0 || !isfinite(tot[0])) S.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
        else S.alpha = S.rho / tot[0];
    }
}

// s = r - alpha v
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_s(KVecs<V> K) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V alpha = cvt<V>(K.st->alpha);
    KRY_LOOP(K) {
        const Pack<V> r = ldv(K.r + r0), v = ldv(K.v + r0);
        Pack<V> s;
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = r.v[j] - alpha * v.v[j];
        stv(K.s + r0, s);
    }
}

// t = A s;  omega = (t, s) / (t, t)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_t(KVecs<V> K) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    DotAcc<V> ts, tt;
    KRY_LOOP(K) {
        const Pack<V> y = sell_rows(K, r0, K.s);
        stv(K.t + r0, y);
        const Pack<V> s = ldv(K.s + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) { ts.add(y.v[j], s.v[j]); tt.add(y.v[j], y.v[j]); }
    }
    double acc[2] = {ts.value(), tt.value()}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
        else S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
    }
}

// x += alpha p + omega s;  r = s - omega t;  rho' = (rh, r);  beta; convergence test on (r, r)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_x(KVecs<V> K) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V alpha = cvt<V>(K.st->alpha), omega = cvt<V>(K.st->omega);
    DotAcc<V> rho, rr;
    KRY_LOOP(K) {
        const Pack<V> s = ldv(K.s + r0), p = ldv(K.p + r0), t = ldv(K.t + r0), rh = ldv(K.rh + r0);
        Pack<V> x = ldv(K.x + r0), r;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            x.v[j] += alpha * p.v[j] + omega * s.v[j];
            r.v[j] = s.v[j] - omega * t.v[j];
            rho.add(rh.v[j], r.v[j]);
            rr.add(r.v[j], r.v[j]);
        }
        stv(K.x + r0, x);
        stv(K.r + r0, r);
    }
    double acc[2] = {rho.value(), rr.value()}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        S.iter += 1;
        S.rr = tot[1];
        if (tot[1] < 0.81 * S.best_rr) { S.best_rr = tot[1]; S.last_improve = S.iter; }
        // a diverged iteration stops before it overflows; a guarded (FP32) solve gives up
        // once its residual is 1000 times the initial one
        const double blowup = S.stall > 0 ? 1e6 : 1e24;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || tot[1] > blowup * S.rr0) S.done = K_NONFINITE;
        else if (tot[1] <= S.tol2) S.done = K_CONVERGED;
        else if (tot[0] == 0.0 || S.omega == 0.0) S.done = K_BREAKDOWN;
        else if (S.iter >= S.maxit) S.done = K_MAXIT;
        else if (S.stall > 0 && S.best_rr <= S.stall_rr && S.iter - S.last_improve >= S.stall) S.done = K_STAGNATED;
        else {
            S.beta = (tot[0] / S.rho) * (S.alpha / S.omega);
            S.rho = tot[0];
        }
    }
}

// p = r + beta (p - omega v)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_p(KVecs<V> K) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V beta = cvt<V>(K.st->beta), omega = cvt<V>(K.st->omega);
    KRY_LOOP(K) {
        const Pack<V> r = ldv(K.r + r0), v = ldv(K.v + r0);
        Pack<V> p = ldv(K.p + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) p.v[j] = r.v[j] + beta * (p.v[j] - omega * v.v[j]);
        stv(K.p + r0, p);
    }
}


// ---------------------------------------------------------------------------------
// Newton-level helpers
// ---------------------------------------------------------------------------------

// out = sum over free rows of r_i^2 (deterministic), written to *out
__global__ void __launch_bounds__(KRY_BLOCK) norm2_free_kernel(int64_t n, const double *r, const uint8_t *dir,
                                                               double *part, uint32_t *ticket, double *out) {
    double acc[1] = {0.0};
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < n; i += int64_t(gridDim.x) * KRY_BLOCK)
        if (!dir[i]) acc[0] += r[i] * r[i];
    double tot[1];
    if (grid_reduce<1>(acc, part, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

// u -= lambda x (Newton update with step length lambda), x in the Krylov type
template <typename V>
__global__ void newton_update_kernel(int64_t n, double *u, const V *x, double lambda) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) u[i] -= lambda * to_d(x[i]);
}

// CSR values -> Jacobi-scaled SELL operator and scaled right-hand side (egfem_bicgstab).
// FP32 operators keep the scaled row sum in column 0 (difference form, see above).
template <typename V>
__global__ void csr_to_sell_kernel(int64_t n, const SliceMeta *meta, const int32_t *col_slot, const double *vals,
                                   const double *rhs, typename VecT<V>::mat *A, V *b, int32_t *status) {
    using M_t = typename VecT<V>::mat;
    const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const SliceMeta M = meta[row / SLICE];
    const int lane = int(row % SLICE);
    const double diag = vals[col_slot[M.col_base + lane]];
    double dinv = 0.0;
    if (diag != 0.0) dinv = 1.0 / diag;
    else atomicOr(status, 1);
    double rs = 0.0;
    for (int c = 0; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const int32_t s = col_slot[q];
        const double a = s >= 0 ? (c == 0 && dinv != 0.0 ? 1.0 : vals[s] * dinv) : 0.0;   // unit diagonal
        rs += a;
        A[q] = M_t(a);
    }
    if (VecT<V>::diff) A[M.col_base + lane] = M_t(rs);
    b[row] = cvt<V>(rhs[row] * dinv);
}

// Replace column 0 of a scaled SELL operator by its row sum (FP32 difference form).
template <typename V>
__global__ void rowsum_form_kernel(int64_t n, const SliceMeta *meta, V *A) {   // V: the operator value type
    const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const SliceMeta M = meta[row / SLICE];
    const int lane = int(row % SLICE);
    double rs = 0.0;
    for (int c = 0; c < M.ncol; ++c) rs += double(A[M.col_base + int64_t(c) * SLICE + lane]);
    A[M.col_base + lane] = V(rs);
}

// y = J x from CSR values (egfem_spmv)
__global__ void csr_spmv_kernel(int64_t n, const int32_t *rowptr, const int32_t *cols, const double *vals,
                                const double *x, double *y) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) s += vals[q] * x[cols[q]];
    y[i] = s;
}

template <typename S, typename D>
__global__ void cast_kernel(int64_t n, const S *a, D *b) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = cvt<D>(to_d(a[i]));
}

// ---------------------------------------------------------------------------------
// Fused iteration for double-float vectors: three kernels instead of five.
//
// On the FP32 pipe a few extra additions are cheap, so each SpMV recomputes the vector
// it multiplies at the gathered columns from the vectors it came from, instead of
// reading a stored copy written by a separate kernel:
//   kry_vp:  p' = r + beta (p - omega v)  (own rows stored);  v' = A p';  alpha = rho / (rh, v')
//   kry_st:  s = r - alpha v';            t = A s;            omega = (t, s) / (t, t)
//   kry_xr:  x += alpha p' + omega s;     r = s - omega t;    rho', beta, convergence
// p and v alternate between two buffers (odd / even iterations), since kry_vp reads the
// old values at neighbouring rows while it writes the new ones.
// ---------------------------------------------------------------------------------

template <typename V, typename F>
__device__ __forceinline__ Pack<V> sell_rows_f(const KVecs<V> &K, int64_t r0, const Pack<V> &xi, F xval) {
    constexpr int R = VecT<V>::R;
    using M_t = typename VecT<V>::mat;
    const SliceMeta M = K.meta[r0 / SLICE];
    const int lane = int(r0 % SLICE);
    Pack<V> y;
    M_t a0[R];
    ldm(K.A + M.col_base + lane, a0);
#pragma unroll
    for (int j = 0; j < R; ++j) y.v[j] = a0[j] * xi.v[j];
    for (int c = 1; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        M_t a[R];
        ldm(K.A + q, a);
        int32_t col[R];
        row_cols(K, M, r0, q, c, col);
#pragma unroll
        for (int j = 0; j < R; ++j) y.v[j] += a[j] * (xval(col[j]) - xi.v[j]);
    }
    return y;
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_vp(KVecs<V> K, V *p_out, V *v_out, const V *p_in, const V *v_in) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V beta = cvt<V>(K.st->beta), omega = cvt<V>(K.st->omega);
    auto pnew = [&](int32_t j) { return ldg1(K.r + j) + beta * (ldg1(p_in + j) - omega * ldg1(v_in + j)); };
    DotAcc<V> a;
    KRY_LOOP(K) {
        const Pack<V> r = ldv(K.r + r0), p = ldv(p_in + r0), v = ldv(v_in + r0);
        Pack<V> pi;
#pragma unroll
        for (int j = 0; j < R; ++j) pi.v[j] = r.v[j] + beta * (p.v[j] - omega * v.v[j]);
        stv(p_out + r0, pi);
        const Pack<V> y = sell_rows_f(K, r0, pi, pnew);
        stv(v_out + r0, y);
        const Pack<V> rh = ldv(K.rh + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) a.add(rh.v[j], y.v[j]);
    }
    double acc[1] = {a.value()}, tot[1];
    if (grid_reduce<1>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (tot[0] == 0.0 || !isfinite(tot[0])) S.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
        else S.alpha = S.rho / tot[0];
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_st(KVecs<V> K, const V *v_cur) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V alpha = cvt<V>(K.st->alpha);
    auto sval = [&](int32_t j) { return ldg1(K.r + j) - alpha * ldg1(v_cur + j); };
    DotAcc<V> ts, tt;
    KRY_LOOP(K) {
        const Pack<V> r = ldv(K.r + r0), v = ldv(v_cur + r0);
        Pack<V> s;
#pragma unroll
        for (int j = 0; j < R; ++j) s.v[j] = r.v[j] - alpha * v.v[j];
        const Pack<V> y = sell_rows_f(K, r0, s, sval);
        stv(K.t + r0, y);
#pragma unroll
        for (int j = 0; j < R; ++j) { ts.add(y.v[j], s.v[j]); tt.add(y.v[j], y.v[j]); }
    }
    double acc[2] = {ts.value(), tt.value()}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
        else S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_xr(KVecs<V> K, const V *p_cur, const V *v_cur) {
    constexpr int R = VecT<V>::R;
    if (finished(K.st)) return;
    const V alpha = cvt<V>(K.st->alpha), omega = cvt<V>(K.st->omega);
    DotAcc<V> rho, rr;
    KRY_LOOP(K) {
        const Pack<V> r0v = ldv(K.r + r0), v = ldv(v_cur + r0), p = ldv(p_cur + r0), t = ldv(K.t + r0),
                      rh = ldv(K.rh + r0);
        Pack<V> x = ldv(K.x + r0), r;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const V s = r0v.v[j] - alpha * v.v[j];
            x.v[j] += alpha * p.v[j] + omega * s;
            r.v[j] = s - omega * t.v[j];
            rho.add(rh.v[j], r.v[j]);
            rr.add(r.v[j], r.v[j]);
        }
        stv(K.x + r0, x);
        stv(K.r + r0, r);
    }
    double acc[2] = {rho.value(), rr.value()}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        S.iter += 1;
        S.rr = tot[1];
        if (tot[1] < 0.81 * S.best_rr) { S.best_rr = tot[1]; S.last_improve = S.iter; }
        const double blowup = S.stall > 0 ? 1e6 : 1e24;
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || tot[1] > blowup * S.rr0) S.done = K_NONFINITE;
        else if (tot[1] <= S.tol2) S.done = K_CONVERGED;
        else if (tot[0] == 0.0 || S.omega == 0.0) S.done = K_BREAKDOWN;
        else if (S.iter >= S.maxit) S.done = K_MAXIT;
        else if (S.stall > 0 && S.best_rr <= S.stall_rr && S.iter - S.last_improve >= S.stall) S.done = K_STAGNATED;
        else {
            S.beta = (tot[0] / S.rho) * (S.alpha / S.omega);
            S.rho = tot[0];
        }
    }
}

#undef KRY_LOOP

}  // namespace egfem
