// egfem_krylov.cuh -- BiCGStab (van der Vorst 1992) on the Jacobi-scaled system
// (D J) x = D b, D = diag(J)^{-1}, with the matrix in the slice-interleaved (SELL-32)
// layout of the tensor's local columns.  V is the vector/matrix type (double for the
// FP64 path, float for the mixed path); dot products are summed per thread in V and
// across threads and blocks in double, in a fixed order (deterministic results).
//
// Every kernel of an iteration reads the device state first and returns at once when
// the solve has finished, so a captured chunk of iterations can overshoot the last one
// at the cost of empty launches only.  Cross-block reductions use the "last block
// finishes" pattern (one atomic ticket per block, no waiting), so no kernel spins.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "egfem_internal.h"

namespace egfem {

constexpr int KRY_BLOCK = 256;

enum KDone : int32_t { K_RUNNING = 0, K_CONVERGED = 1, K_MAXIT = 2, K_BREAKDOWN = 3, K_NONFINITE = 4 };

struct KState {
    double rho, alpha, omega, beta;
    double rr;          // ||r||^2 of the current iterate
    double rr0;         // ||r_0||^2
    double tol2;        // stop when rr <= tol2
    double scratch[4];
    int32_t iter, maxit, done, pad;
    uint32_t ticket;
};

template <typename V>
struct KVecs {
    int64_t n;
    const SliceMeta *meta;
    const int32_t *col_idx;
    const V *A;
    V *x, *r, *rh, *p, *v, *s, *t;
    const V *b;
    KState *st;
    double *part;       // [3 * gridDim.x]
};

template <typename V> struct Acc { using type = V; };

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

// y_row = sum_c A[q] x[col(q)] over the row's local columns (SELL-32 layout).
template <typename V>
__device__ __forceinline__ V sell_row(const KVecs<V> &K, int64_t row, const V *xin) {
    const SliceMeta M = K.meta[row / SLICE];
    const int lane = int(row % SLICE);
    V y = V(0);
    for (int c = 0; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        y += K.A[q] * xin[K.col_idx[q]];
    }
    return y;
}

__device__ __forceinline__ bool finished(const KState *st) { return *(volatile const int32_t *)&st->done != K_RUNNING; }

// setup: x = 0, r = rh = p = b, rho = (r, r)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_setup(KVecs<V> K, double rtol, int32_t maxit) {
    double acc[1] = {0.0};
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK) {
        const V b = K.b[i];
        K.x[i] = V(0); K.r[i] = b; K.rh[i] = b; K.p[i] = b; K.v[i] = V(0);
        acc[0] += double(b) * double(b);
    }
    double tot[1];
    if (grid_reduce<1>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        S.rho = tot[0]; S.rr = tot[0]; S.rr0 = tot[0];
        S.tol2 = rtol * rtol * tot[0];
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0;
        S.iter = 0; S.maxit = maxit;
        S.done = (tot[0] == 0.0) ? K_CONVERGED : (!isfinite(tot[0]) ? K_NONFINITE : K_RUNNING);
    }
}

// v = A p;  alpha = rho / (rh, v)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_v(KVecs<V> K) {
    if (finished(K.st)) return;
    typename Acc<V>::type a = 0;
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK) {
        const V y = sell_row(K, i, K.p);
        K.v[i] = y;
        a += K.rh[i] * y;
    }
    double acc[1] = {double(a)}, tot[1];
    if (grid_reduce<1>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (tot[0] == 0.0 || !isfinite(tot[0])) S.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
        else S.alpha = S.rho / tot[0];
    }
}

// s = r - alpha v
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_s(KVecs<V> K) {
    if (finished(K.st)) return;
    const V alpha = V(K.st->alpha);
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK)
        K.s[i] = K.r[i] - alpha * K.v[i];
}

// t = A s;  omega = (t, s) / (t, t)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_t(KVecs<V> K) {
    if (finished(K.st)) return;
    typename Acc<V>::type ts = 0, tt = 0;
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK) {
        const V y = sell_row(K, i, K.s);
        K.t[i] = y;
        ts += y * K.s[i];
        tt += y * y;
    }
    double acc[2] = {double(ts), double(tt)}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
        else S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
    }
}

// x += alpha p + omega s;  r = s - omega t;  rho' = (rh, r);  beta; convergence test on (r, r)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_x(KVecs<V> K) {
    if (finished(K.st)) return;
    const V alpha = V(K.st->alpha), omega = V(K.st->omega);
    typename Acc<V>::type rho = 0, rr = 0;
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK) {
        const V s = K.s[i];
        K.x[i] += alpha * K.p[i] + omega * s;
        const V r = s - omega * K.t[i];
        K.r[i] = r;
        rho += K.rh[i] * r;
        rr += r * r;
    }
    double acc[2] = {double(rho), double(rr)}, tot[2];
    if (grid_reduce<2>(acc, K.part, &K.st->ticket, tot) && threadIdx.x == 0) {
        KState &S = *K.st;
        S.iter += 1;
        S.rr = tot[1];
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
        else if (tot[1] <= S.tol2) S.done = K_CONVERGED;
        else if (tot[0] == 0.0 || S.omega == 0.0) S.done = K_BREAKDOWN;
        else if (S.iter >= S.maxit) S.done = K_MAXIT;
        else {
            S.beta = (tot[0] / S.rho) * (S.alpha / S.omega);
            S.rho = tot[0];
        }
    }
}

// p = r + beta (p - omega v)
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kry_p(KVecs<V> K) {
    if (finished(K.st)) return;
    const V beta = V(K.st->beta), omega = V(K.st->omega);
    for (int64_t i = int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x; i < K.n; i += int64_t(gridDim.x) * KRY_BLOCK)
        K.p[i] = K.r[i] + beta * (K.p[i] - omega * K.v[i]);
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

// u -= x (Newton update), x in the Krylov type
template <typename V>
__global__ void newton_update_kernel(int64_t n, double *u, const V *x) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) u[i] -= double(x[i]);
}

// CSR values -> Jacobi-scaled SELL operator and scaled right-hand side (egfem_bicgstab)
template <typename V>
__global__ void csr_to_sell_kernel(int64_t n, const SliceMeta *meta, const int32_t *col_slot, const double *vals,
                                   const double *rhs, V *A, V *b, int32_t *status) {
    const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const SliceMeta M = meta[row / SLICE];
    const int lane = int(row % SLICE);
    const double diag = vals[col_slot[M.col_base + lane]];
    double dinv = 0.0;
    if (diag != 0.0) dinv = 1.0 / diag;
    else atomicOr(status, 1);
    for (int c = 0; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const int32_t s = col_slot[q];
        A[q] = V(s >= 0 ? vals[s] * dinv : 0.0);
    }
    b[row] = V(rhs[row] * dinv);
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
    if (i < n) b[i] = D(a[i]);
}

}  // namespace egfem
