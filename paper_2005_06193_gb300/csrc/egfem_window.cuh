// egfem_window.cuh -- BiCGStab (van der Vorst 1992) on one Jacobi-scaled system as one
// persistent cooperative kernel with TWO grid-wide reductions per iteration.
//
// pk_solve1 separates its phases by five grid barriers per iteration: three for the inner
// products and two because each operator application needs its neighbours' rows of the
// vector it multiplies (s after B1, p after D).  Each barrier waits for the slowest block,
// and the block sums that follow are a chain of L2 round trips, so at 1 M rows the FP64
// iteration stalls on barriers about as long as it computes.
//
// Here block b owns one contiguous tile of rows [r_begin, r_end) and the WINDOW [w_lo, w_hi)
// of every column its rows touch (the tile plus the stencil halo; 2D structured meshes in
// lexicographic order: one grid line of the mesh on each side).  Before each operator
// application the block evaluates the vector it multiplies on its whole window into shared
// memory, recomputing the halo rows from vectors that every block finished before the last
// reduction, with the same instructions the owners use, so the halo values are bit-identical
// to the owners' values.  No barrier is then needed before an operator application, and the
// inner products are regrouped so that each iteration has two reductions:
//
//   A_k (after G2 of k-1):  window: r_k = s - w t,  p_k = r_k + b (p_{k-1} - w v_{k-1})
//                           tile:   x_k = x_{k-1} + a p_{k-1} + w s;  v_k = A p_k
//                           sums:   (r_k, r_k), (rh, v_k)                       -> G1
//       after G1: the convergence and failure tests on r_k (pk_solve1's, with the same
//       quantities), then alpha_k = rho_k / (rh, v_k)
//   B_k:                    window: s = r_k - alpha_k v_k
//                           tile:   t = A s
//                           sums:   (t, s), (t, t), (rh, s), (rh, t)            -> G2
//       after G2: omega_k = (t, s) / (t, t), rho_{k+1} = (rh, s) - omega_k (rh, t) (equal to
//       (rh, r_{k+1}) in exact arithmetic; r_{k+1} itself is formed only in A_{k+1}),
//       beta_k = (rho_{k+1} / rho_k) (alpha_k / omega_k)
//
// x_0 = 0, so r_0 = p_0 = b and the shadow residual rh is b itself (not stored).  The
// iteration count and the stopping decisions are those of the five-barrier form: the tests
// on r_k run at G1 of step k, before alpha_k is used, and x_k is complete by then.  p and v
// alternate between two buffers (a block reads p_{k-1} and v_{k-1} at its halo rows while
// their owners write p_k and v_k); r, s and t are read at halo rows only after the reduction
// that follows their writes.
//
// The barrier, its bounded wait and the timeout path are pk_solve1's (pk1_sync): every wait
// ends after PK_WAIT_NS of %globaltimer at the latest, and the host reports the timeout.
//
// pkwb_solve is the same iteration for a batch of independent systems (block-diagonal
// operator, instances of uneven size), as pk_solveb is for pk_solve1: tiles lie inside one
// instance and are dealt to blocks round-robin; a block takes its tiles one after another in
// each phase (one window in shared memory at a time), keeps the state of each owned tile's
// system, and after each barrier adds all partials of that system (pkb_sync's barrier, which
// also counts the blocks that still own a running tile and so ends the loop).
#pragma once

#include "egfem_persist.cuh"

namespace egfem {

constexpr int PKW_BLOCK = 512;    // threads per block of the one-system kernel (2 resident per SM)
constexpr int PKW_MIN_BLOCKS = 2;
constexpr int PKWB_BLOCK = 512;   // threads per block of the batched kernel (2 resident per SM)
constexpr int PKWB_MIN_BLOCKS = 2;
// shared memory of a block's reduction staging, carved from the window buffer (free while a tile's
// partials are formed): the window allocation is at least this large
constexpr size_t PKW_STAGE_BYTES = 4 * PKW_BLOCK * sizeof(double);

struct PkWin {
    int64_t lo, hi;   // window rows [lo, hi), multiples of the thread row count
};

template <typename V>
struct PkwArgs {
    KVecs<V> K;               // x, r, p (p_k, even k), v (even k), s, t, b; K.rh unused (rh = b)
    V *p2, *v2;               // p and v of odd k
    const BTile *tiles;       // pkw_solve: one tile per block; pkwb_solve: tiles grouped by system
    const PkWin *win;         // one window per tile
    int64_t ntiles;
    KState *st;               // [systems] final states
    double *part;             // [4 * G] (pkw_solve) or [4 * ntiles] (pkwb_solve) partials
    const uint8_t *active;    // [systems] or null (all)
    const double *rtol;       // [systems] or null (rtol0)
    double rtol0;
    PGrid *bar;
    int64_t n;                // rows of the (batch) system (K.n_pad - n padding rows follow)
    int32_t maxit, stall;
};

// Column indices of local column c for the R rows at r0, as row_cols, except that a padding row
// (index >= n, all of its operator values zero) names itself: the builder gives padding rows
// column 0, which lies outside any window but the first.
template <typename V>
__device__ __forceinline__ void pkw_cols(const KVecs<V> &K, const SliceMeta &M, int64_t r0, int64_t q, int c, int64_t n,
                                         int32_t (&col)[VecT<V>::R]) {
    row_cols(K, M, r0, q, c, col);
    if (M.off_base < 0) {
#pragma unroll
        for (int j = 0; j < VecT<V>::R; ++j)
            if (r0 + j >= n) col[j] = int32_t(r0 + j);
    }
}

// y = A x for the R rows at r0, with x gathered from the shared-memory window xw (row j at
// xw[j - lo]); xi = x at those rows; n = the system's rows (padding rows follow).  Arithmetic as
// pk_spmv.
template <typename V>
__device__ __forceinline__ Pack<V> pkw_spmv(const KVecs<V> &K, int64_t r0, const V *xw, int64_t lo, int64_t n,
                                            const Pack<V> &xi) {
    constexpr int R = VecT<V>::R;
    constexpr bool DF = std::is_same<V, df64>::value;
    using M_t = typename VecT<V>::mat;
    const SliceMeta M = K.meta[r0 / SLICE];
    const int lane = int(r0 % SLICE);
    double y64[R];
    float hi[R], lo_[R];
    if constexpr (DF) {
        M_t a0[R];
        ldm(K.A + M.col_base + lane, a0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            hi[j] = __fmul_rn(a0[j], xi.v[j].hi);
            lo_[j] = __fmaf_rn(a0[j], xi.v[j].lo, __fmaf_rn(a0[j], xi.v[j].hi, -hi[j]));
        }
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) y64[j] = xi.v[j];
    }
#pragma unroll 4
    for (int c = 1; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        M_t a[R];
        int32_t col[R];
        ldm(K.A + q, a);
        pkw_cols(K, M, r0, q, c, n, col);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const V xc = xw[col[j] - int32_t(lo)];
            if constexpr (DF) df_acc_diff(hi[j], lo_[j], a[j], xc, xi.v[j]);
            else y64[j] = fma(a[j], xc, y64[j]);
        }
    }
    Pack<V> y;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if constexpr (DF) y.v[j] = df_fast_two_sum(hi[j], lo_[j]);
        else y.v[j] = y64[j];
    }
    return y;
}

// Inner products of the solve: double-float accumulators on the FP32 pipe.  FP64 vectors enter
// through split_dbl with the system's scale (a power of two near the root mean square of b, so
// that every product stays in the float range); double-float vectors enter as they are.
template <typename V> struct PkwIn;
template <> struct PkwIn<double> {
    static __device__ __forceinline__ df64 get(double x, int sc) { return split_dbl(x, sc); }
};
template <> struct PkwIn<df64> {
    static __device__ __forceinline__ df64 get(df64 x, int) { return x; }
};

// Block partials of NV (2 or 4) accumulators (DotAcc<df64>, or DotAcc<double> for the first sums
// of an FP64 solve): the per-thread values go to shared memory (`stage`, PKW_STAGE_BYTES of the
// window buffer, which no thread reads any more), warp w adds chunk w / NV of value
// w % NV, and warp k < NV adds the chunk sums of value k and stores it in part[k * stride +
// index] (double-float pairs in the 8-byte slots, or doubles).  One fixed order, on the FP32
// pipe for double-float values.  Ends with the stores issued (the caller's barrier orders them).
template <int BLOCK, typename A, int NV>
__device__ __forceinline__ void pkw_block_partial(const A (&acc)[NV], double *part, int64_t stride, int64_t index,
                                                  void *stage) {
    constexpr bool DF = std::is_same<A, DotAcc<df64>>::value;
    using T = typename std::conditional<DF, df64, double>::type;
    constexpr int NW = BLOCK / 32, CH = NW / NV, PER = BLOCK / CH;
    static_assert(NV == 2 || NV == 4, "two or four sums");
    static_assert(PER % 32 == 0, "whole warps per chunk");
    static_assert(NV * BLOCK * sizeof(T) <= PKW_STAGE_BYTES, "staging fits the window buffer");
    T *s_acc = reinterpret_cast<T *>(stage);
    __shared__ T s_ch[NV][CH];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // the window's readers (and the previous partial's readers of s_ch) are done
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if constexpr (DF) s_acc[k * BLOCK + threadIdx.x] = df_two_sum(acc[k].hi, acc[k].lo);
        else s_acc[k * BLOCK + threadIdx.x] = acc[k].value();
    }
    __syncthreads();
    {
        const int k = w % NV, c = w / NV;
        T x = s_acc[k * BLOCK + c * PER + lane];
#pragma unroll
        for (int q = lane + 32; q < PER; q += 32) {
            if constexpr (DF) x = df_add(x, s_acc[k * BLOCK + c * PER + q]);
            else x = x + s_acc[k * BLOCK + c * PER + q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if constexpr (DF) x = df_add(x, shfl_xor_df(x, o));
            else x = x + __shfl_xor_sync(0xffffffffu, x, o);
        }
        if (lane == 0) s_ch[k][c] = x;
    }
    __syncthreads();
    if (w < NV && lane == 0) {
        T x = s_ch[w][0];
#pragma unroll
        for (int c = 1; c < CH; ++c) {
            if constexpr (DF) x = df_add(x, s_ch[w][c]);
            else x = x + s_ch[w][c];
        }
        if constexpr (DF) reinterpret_cast<float2 *>(part)[int64_t(w) * stride + index] = make_float2(x.hi, x.lo);
        else part[int64_t(w) * stride + index] = x;
    }
}

// One warp: the sum of the n partials part[k * stride + q0 .. q0 + n) in one fixed order (lanes
// over partials, then the warp's tree), in double-float (DF) or FP64; every lane returns it.
template <bool DF>
__device__ __forceinline__ double pkw_warp_sum(const double *part, int64_t k, int64_t stride, int64_t q0, int64_t n) {
    const int lane = threadIdx.x & 31;
    if constexpr (DF) {
        df64 x = {0.f, 0.f};
        for (int64_t q = lane; q < n; q += 32) {
            const float2 t = __ldcg(reinterpret_cast<const float2 *>(part) + k * stride + q0 + q);
            x = df_add(x, df64{t.x, t.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = df_add(x, shfl_xor_df(x, o));
        return df_to_double(x);
    } else {
        double x = 0.0;
        for (int64_t q = lane; q < n; q += 32) x += __ldcg(part + k * stride + q0 + q);
        return warp_sum(x);
    }
}

// x + (a p + w s): two FMAs in FP64, the sloppy double-float sums for double-float vectors
__device__ __forceinline__ double pkw_xupd(double x, double a, double p, double w, double s) { return fma(w, s, fma(a, p, x)); }
__device__ __forceinline__ df64 pkw_xupd(df64 x, df64 a, df64 p, df64 w, df64 s) { return dfs_add(x, dfs_add(a * p, w * s)); }

// ---- the phases of one tile (all threads of the block; BLOCK threads, R rows each per trip)

// A, window: r_k = s - w t and p_k = r_k + b (p_{k-1} - w v_{k-1}) on [lo, hi) into xw (k = 0:
// r = p = b); on the tile [rb, re): x_k (k = 0: 0), r_k and p_k stored, (r_k, r_k) accumulated
// (FP64 at k = 0 of an FP64 solve, else split double-float)
template <typename V, int BLOCK>
__device__ __forceinline__ void pkw_a_window(const KVecs<V> &K, V *xw, int64_t lo, int64_t hi, int64_t rb, int64_t re,
                                             int32_t k, double a_, double w_, double b_, const V *p_old, const V *v_old,
                                             V *p_new, int sc, DotAcc<df64> &acc, DotAcc<double> &acc0) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    constexpr bool F64 = std::is_same<V, double>::value;
    const V al = cvt<V>(a_), om = cvt<V>(w_), be = cvt<V>(b_);
#pragma unroll 1
    for (int64_t j0 = lo + int64_t(threadIdx.x) * R; j0 < hi; j0 += int64_t(BLOCK) * R) {
        Pack<V> rk, pk;
        const bool own = j0 >= rb && j0 < re;
        if (k == 0) {
            rk = ldv(K.b + j0);
            pk = rk;
            if (own) {
                Pack<V> z;
#pragma unroll
                for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
                stv(K.x + j0, z);
            }
        } else {
            const Pack<V> s = ldcv(K.s + j0), tv = ldcv(K.t + j0), po = ldcv(p_old + j0), vo = ldcv(v_old + j0);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                rk.v[j] = Op::sub(s.v[j], om * tv.v[j]);
                pk.v[j] = Op::add(rk.v[j], be * Op::sub(po.v[j], om * vo.v[j]));
            }
            if (own) {
                Pack<V> x = ldcv(K.x + j0);
#pragma unroll
                for (int j = 0; j < R; ++j) x.v[j] = pkw_xupd(x.v[j], al, po.v[j], om, s.v[j]);
                stv(K.x + j0, x);
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) xw[j0 - lo + j] = pk.v[j];
        if (own) {
            stv(K.r + j0, rk);
            stv(p_new + j0, pk);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (F64 && k == 0) acc0.add(to_d(rk.v[j]), to_d(rk.v[j]));
                else { const df64 q = PkwIn<V>::get(rk.v[j], sc); acc.add(q, q); }
            }
        }
    }
}

// A, operator: v_k = A p_k on the tile from the window; (rh, v_k) with rh = b
template <typename V, int BLOCK>
__device__ __forceinline__ void pkw_a_spmv(const KVecs<V> &K, const V *xw, int64_t lo, int64_t rb, int64_t re, int64_t n,
                                           int32_t k, V *v_new, int sc, DotAcc<df64> &acc, DotAcc<double> &acc0) {
    constexpr int R = VecT<V>::R;
    constexpr bool F64 = std::is_same<V, double>::value;
#pragma unroll 1
    for (int64_t r0 = rb + int64_t(threadIdx.x) * R; r0 < re; r0 += int64_t(BLOCK) * R) {
        Pack<V> pi;
#pragma unroll
        for (int j = 0; j < R; ++j) pi.v[j] = xw[r0 - lo + j];
        const Pack<V> y = pkw_spmv(K, r0, xw, lo, n, pi);
        stv(v_new + r0, y);
        const Pack<V> rh = ldv(K.b + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (F64 && k == 0) acc0.add(to_d(rh.v[j]), to_d(y.v[j]));
            else acc.add(PkwIn<V>::get(rh.v[j], sc), PkwIn<V>::get(y.v[j], sc));
        }
    }
}

// B, window: s = r_k - alpha v_k on [lo, hi) into xw, stored on the tile
template <typename V, int BLOCK>
__device__ __forceinline__ void pkw_b_window(const KVecs<V> &K, V *xw, int64_t lo, int64_t hi, int64_t rb, int64_t re,
                                             double a_, const V *v_new) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    const V al = cvt<V>(a_);
#pragma unroll 1
    for (int64_t j0 = lo + int64_t(threadIdx.x) * R; j0 < hi; j0 += int64_t(BLOCK) * R) {
        const Pack<V> r = ldcv(K.r + j0), v = ldcv(v_new + j0);
        Pack<V> s;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            s.v[j] = Op::sub(r.v[j], al * v.v[j]);
            xw[j0 - lo + j] = s.v[j];
        }
        if (j0 >= rb && j0 < re) stv(K.s + j0, s);
    }
}

// B, operator: t = A s on the tile from the window; (t, s), (t, t), (rh, s), (rh, t)
template <typename V, int BLOCK>
__device__ __forceinline__ void pkw_b_spmv(const KVecs<V> &K, const V *xw, int64_t lo, int64_t rb, int64_t re, int64_t n,
                                           int sc, DotAcc<df64> (&acc)[4]) {
    constexpr int R = VecT<V>::R;
#pragma unroll 1
    for (int64_t r0 = rb + int64_t(threadIdx.x) * R; r0 < re; r0 += int64_t(BLOCK) * R) {
        Pack<V> si;
#pragma unroll
        for (int j = 0; j < R; ++j) si.v[j] = xw[r0 - lo + j];
        const Pack<V> y = pkw_spmv(K, r0, xw, lo, n, si);
        stv(K.t + r0, y);
        const Pack<V> rh = ldv(K.b + r0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const df64 qt = PkwIn<V>::get(y.v[j], sc), qs = PkwIn<V>::get(si.v[j], sc), qb = PkwIn<V>::get(rh.v[j], sc);
            acc[0].add(qt, qs);
            acc[1].add(qt, qt);
            acc[2].add(qb, qs);
            acc[3].add(qb, qt);
        }
    }
}

// ---- the scalar updates (one thread per system copy)

// After G1 of step k: at k = 0 the setup of the state from (b, b) (and, for an FP64 solve, the
// scale of the later inner products: 2^sc near ||b||, the same in every block that holds a part of
// the system); then the tests of pk_after_c on r_k (beta was formed at G2 and is used only if
// running) and alpha_k.
__device__ __forceinline__ void pkw_after_g1(KState &S, int32_t k, double rr, double rv, double rho_next, double rt,
                                             int32_t maxit, int32_t stall, bool f64, int &sc) {
    if (k == 0) {
        S.iter = 0; S.last_improve = 0; S.maxit = maxit; S.stall = stall; S.ticket = 0u;
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0; S.scratch[0] = S.scratch[1] = 0.0;
        S.rho = S.rr = S.rr0 = S.best_rr = rr;
        S.tol2 = rt * rt * rr;
        S.stall_rr = 4e-6 * rr;
        S.done = (rr == 0.0) ? K_CONVERGED : (!isfinite(rr) ? K_NONFINITE : (maxit <= 0 ? K_MAXIT : K_RUNNING));
        if (f64 && S.done == K_RUNNING) {
            int ex = 0;
            frexp(sqrt(rr), &ex);
            sc = ex;
        }
    } else {
        const double beta = S.beta;
        pk_after_c(S, rho_next, rr, maxit, stall);
        S.beta = beta;
    }
    if (S.done == K_RUNNING) {
        if (rv == 0.0 || !isfinite(rv)) S.done = isfinite(rv) ? K_BREAKDOWN : K_NONFINITE;
        else S.alpha = S.rho / rv;
    }
}

// After G2: omega_k, rho_{k+1} = (rh, s) - omega_k (rh, t), beta_k (a zero omega or rho ends the
// solve at the next tests, before beta is used)
__device__ __forceinline__ void pkw_after_g2(KState &S, const double (&tot)[4], double &rho_next) {
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        S.done = K_NONFINITE;
        return;
    }
    S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
    rho_next = tot[2] - S.omega * tot[3];
    S.beta = (S.omega != 0.0 && S.rho != 0.0) ? (rho_next / S.rho) * (S.alpha / S.omega) : 0.0;
}

// ---------------------------------------------------------------------------------
// One system: one tile per block
// ---------------------------------------------------------------------------------

template <typename V>
__global__ void __launch_bounds__(PKW_BLOCK, PKW_MIN_BLOCKS) pkw_solve(PkwArgs<V> P) {
    constexpr bool F64 = std::is_same<V, double>::value;
    extern __shared__ __align__(16) unsigned char pkw_dyn[];
    V *xw = reinterpret_cast<V *>(pkw_dyn);   // the window of the vector being multiplied
    __shared__ KState S;
    __shared__ double s_rho_next;
    __shared__ int s_sc;                       // scale of the split inner products (FP64 solve)
    __shared__ double s_tot[4];
    __shared__ BTile T;
    __shared__ PkWin Wn;
    if (P.active && !P.active[0]) return;
    const KVecs<V> &K = P.K;
    if (threadIdx.x == 0) { T = P.tiles[blockIdx.x]; Wn = P.win[blockIdx.x]; s_sc = 0; }
    __syncthreads();
    const int64_t rb = T.r_begin, re = T.r_end, lo = Wn.lo, hi = Wn.hi;
    const int64_t G = gridDim.x;
    const int w = threadIdx.x >> 5;
    uint32_t nbar = 0;
    bool ok = true;
    for (int32_t k = 0;; ++k) {
        V *const p_old = (k & 1) ? K.p : P.p2, *const v_old = (k & 1) ? K.v : P.v2;
        V *const p_new = (k & 1) ? P.p2 : K.p, *const v_new = (k & 1) ? P.v2 : K.v;
        const int sc = s_sc;
        // ---- A_k
        {
            DotAcc<df64> acc[2];
            DotAcc<double> acc0[2];
            pkw_a_window<V, PKW_BLOCK>(K, xw, lo, hi, rb, re, k, k ? S.alpha : 0.0, k ? S.omega : 0.0, k ? S.beta : 0.0,
                                       p_old, v_old, p_new, sc, acc[0], acc0[0]);
            __syncthreads();
            pkw_a_spmv<V, PKW_BLOCK>(K, xw, lo, rb, re, P.n, k, v_new, sc, acc[1], acc0[1]);
            const bool d64 = F64 && k == 0;
            if (d64) pkw_block_partial<PKW_BLOCK, DotAcc<double>, 2>(acc0, P.part, G, blockIdx.x, xw);
            else pkw_block_partial<PKW_BLOCK, DotAcc<df64>, 2>(acc, P.part, G, blockIdx.x, xw);
            if (!(ok = pk1_sync(P.bar, nbar))) break;
            if (w < 2) {
                const double x = d64 ? pkw_warp_sum<false>(P.part, w, G, 0, G) : pkw_warp_sum<true>(P.part, w, G, 0, G);
                if ((threadIdx.x & 31) == 0) s_tot[w] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const double f = F64 ? ldexp(1.0, sc) : 1.0;   // sums of split products carry 2^-2sc
                int scn = s_sc;
                pkw_after_g1(S, k, s_tot[0] * f * f, s_tot[1] * f * f, s_rho_next, P.rtol ? P.rtol[0] : P.rtol0, P.maxit,
                             P.stall, F64, scn);
                s_sc = scn;
            }
            __syncthreads();
            if (S.done != K_RUNNING) break;
        }
        // ---- B_k
        {
            const int scb = s_sc;
            DotAcc<df64> acc[4];
            pkw_b_window<V, PKW_BLOCK>(K, xw, lo, hi, rb, re, S.alpha, v_new);
            __syncthreads();
            pkw_b_spmv<V, PKW_BLOCK>(K, xw, lo, rb, re, P.n, scb, acc);
            pkw_block_partial<PKW_BLOCK, DotAcc<df64>, 4>(acc, P.part, G, blockIdx.x, xw);
            if (!(ok = pk1_sync(P.bar, nbar))) break;
            if (w < 4) {
                const double x = pkw_warp_sum<true>(P.part, w, G, 0, G);
                if ((threadIdx.x & 31) == 0) s_tot[w] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const double f = F64 ? ldexp(1.0, scb) : 1.0;
                double tot[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) tot[q] = s_tot[q] * f * f;
                double rn = 0.0;
                pkw_after_g2(S, tot, rn);
                s_rho_next = rn;
            }
            __syncthreads();
            if (S.done != K_RUNNING) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        KState F = S;
        if (!ok) F.done = K_TIMEOUT;
        *P.st = F;
    }
}

// ---------------------------------------------------------------------------------
// A batch: tiles dealt to blocks, every block keeps the states of its tiles' systems
// ---------------------------------------------------------------------------------

constexpr int PKWB_MAXT = 48;   // tiles per block

// After a barrier: for each owned tile whose system runs, warp (tile mod warps) adds the NV
// partials of all tiles of that system (pkw_warp_sum) and lane 0 calls upd(tile, sums).
template <int NV, typename U>
__device__ __forceinline__ void pkwb_sums(const double *part, int64_t ntiles, int nt, const KState *st, const BTile *tl,
                                          bool df, U &&upd) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < nt; t += PKWB_BLOCK / 32) {
        if (st[t].done != K_RUNNING) continue;
        double x[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            x[k] = df ? pkw_warp_sum<true>(part, k, ntiles, tl[t].tile0, tl[t].ntiles_inst)
                      : pkw_warp_sum<false>(part, k, ntiles, tl[t].tile0, tl[t].ntiles_inst);
        if (lane == 0) upd(t, x);
    }
    __syncthreads();
}

template <typename V>
__global__ void __launch_bounds__(PKWB_BLOCK, PKWB_MIN_BLOCKS) pkwb_solve(PkwArgs<V> P) {
    constexpr bool F64 = std::is_same<V, double>::value;
    extern __shared__ __align__(16) unsigned char pkw_dyn[];
    V *xw = reinterpret_cast<V *>(pkw_dyn);
    __shared__ KState s_st[PKWB_MAXT];
    __shared__ BTile s_tl[PKWB_MAXT];
    __shared__ PkWin s_win[PKWB_MAXT];
    __shared__ double s_rn[PKWB_MAXT];   // rho_{k+1} of each owned tile's system
    __shared__ int s_sc[PKWB_MAXT];      // scale of its split inner products (FP64 solve)
    const int64_t G = gridDim.x;
    if (P.ntiles > G * PKWB_MAXT) {   // the host keeps to the limit; every block leaves at once
        if (blockIdx.x == 0 && threadIdx.x == 0) P.bar->err = 2;
        return;
    }
    const int nt = int64_t(blockIdx.x) < P.ntiles ? int((P.ntiles - blockIdx.x + G - 1) / G) : 0;
    const KVecs<V> &K = P.K;
    for (int t = threadIdx.x; t < nt; t += PKWB_BLOCK) {
        const int64_t tile = blockIdx.x + int64_t(t) * G;
        const BTile Tt = P.tiles[tile];
        s_tl[t] = Tt;
        s_win[t] = P.win[tile];
        KState &S = s_st[t];
        S.done = (!P.active || P.active[Tt.inst]) ? K_RUNNING : K_CONVERGED;
        S.iter = 0; S.last_improve = 0; S.maxit = P.maxit; S.stall = P.stall; S.ticket = 0u;
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0; S.scratch[0] = S.scratch[1] = 0.0;
        S.rho = S.rr = S.rr0 = S.best_rr = S.tol2 = S.stall_rr = 0.0;
        s_rn[t] = 0.0;
        s_sc[t] = 0;
    }
    __syncthreads();
    auto running = [&]() {
        int a = 0;
        for (int t = 0; t < nt; ++t) a |= (s_st[t].done == K_RUNNING);
        return a;
    };
    uint32_t nbar = 0, live = 0;
    bool ok = true;
    for (int32_t k = 0;; ++k) {
        V *const p_old = (k & 1) ? K.p : P.p2, *const v_old = (k & 1) ? K.v : P.v2;
        V *const p_new = (k & 1) ? P.p2 : K.p, *const v_new = (k & 1) ? P.v2 : K.v;
        const bool d64 = F64 && k == 0;
        // ---- A_k, tile by tile
        for (int t = 0; t < nt; ++t) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &Tt = s_tl[t];
            const PkWin Wt = s_win[t];
            const KState &S = s_st[t];
            DotAcc<df64> acc[2];
            DotAcc<double> acc0[2];
            __syncthreads();   // the previous tile's readers of the window are done
            pkw_a_window<V, PKWB_BLOCK>(K, xw, Wt.lo, Wt.hi, Tt.r_begin, Tt.r_end, k, k ? S.alpha : 0.0, k ? S.omega : 0.0,
                                        k ? S.beta : 0.0, p_old, v_old, p_new, s_sc[t], acc[0], acc0[0]);
            __syncthreads();
            pkw_a_spmv<V, PKWB_BLOCK>(K, xw, Wt.lo, Tt.r_begin, Tt.r_end, P.n, k, v_new, s_sc[t], acc[1], acc0[1]);
            const int64_t tile = blockIdx.x + int64_t(t) * G;
            if (d64) pkw_block_partial<PKWB_BLOCK, DotAcc<double>, 2>(acc0, P.part, P.ntiles, tile, xw);
            else pkw_block_partial<PKWB_BLOCK, DotAcc<df64>, 2>(acc, P.part, P.ntiles, tile, xw);
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
        pkwb_sums<2>(P.part, P.ntiles, nt, s_st, s_tl, !d64, [&](int t, const double *tot) {
            const double f = F64 ? ldexp(1.0, s_sc[t]) : 1.0;
            int scn = s_sc[t];
            pkw_after_g1(s_st[t], k, tot[0] * f * f, tot[1] * f * f, s_rn[t], P.rtol ? P.rtol[s_tl[t].inst] : P.rtol0,
                         P.maxit, P.stall, F64, scn);
            s_sc[t] = scn;
        });
        // ---- B_k, tile by tile
        for (int t = 0; t < nt; ++t) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &Tt = s_tl[t];
            const PkWin Wt = s_win[t];
            DotAcc<df64> acc[4];
            __syncthreads();
            pkw_b_window<V, PKWB_BLOCK>(K, xw, Wt.lo, Wt.hi, Tt.r_begin, Tt.r_end, s_st[t].alpha, v_new);
            __syncthreads();
            pkw_b_spmv<V, PKWB_BLOCK>(K, xw, Wt.lo, Tt.r_begin, Tt.r_end, P.n, s_sc[t], acc);
            pkw_block_partial<PKWB_BLOCK, DotAcc<df64>, 4>(acc, P.part, P.ntiles, blockIdx.x + int64_t(t) * G, xw);
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
        pkwb_sums<4>(P.part, P.ntiles, nt, s_st, s_tl, true, [&](int t, const double *tot) {
            const double f = F64 ? ldexp(1.0, s_sc[t]) : 1.0;
            double tt[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) tt[q] = tot[q] * f * f;
            pkw_after_g2(s_st[t], tt, s_rn[t]);
        });
    }
    for (int t = threadIdx.x; t < nt; t += PKWB_BLOCK) {
        if (blockIdx.x + int64_t(t) * G != s_tl[t].tile0) continue;
        KState F = s_st[t];
        if (!ok) F.done = K_TIMEOUT;
        P.st[s_tl[t].inst] = F;
    }
}

// Window of each tile: the smallest and largest column its rows touch, widened to the tile and
// rounded to whole thread row groups.  One block per tile.
template <typename V>
__global__ void pkw_window_kernel(KVecs<V> K, int64_t n, const BTile *tiles, PkWin *win) {
    __shared__ int64_t s_lo[8], s_hi[8];
    const BTile T = tiles[blockIdx.x];
    int64_t lo = T.r_begin, hi = T.r_end;
    for (int64_t r = T.r_begin + threadIdx.x; r < T.r_end; r += blockDim.x) {
        const SliceMeta M = K.meta[r / SLICE];
        const int lane = int(r % SLICE);
        for (int c = 0; c < M.ncol; ++c) {
            int64_t col;
            if (M.off_base >= 0) col = r + K.slice_off[M.off_base + c];
            else col = r >= n ? r : K.col_idx[M.col_base + int64_t(c) * SLICE + lane];   // as pkw_cols
            lo = col < lo ? col : lo;
            hi = col + 1 > hi ? col + 1 : hi;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < int(blockDim.x >> 5); ++q) { lo = s_lo[q] < lo ? s_lo[q] : lo; hi = s_hi[q] > hi ? s_hi[q] : hi; }
        if (lo > s_lo[0]) lo = s_lo[0];
        if (hi < s_hi[0]) hi = s_hi[0];
        constexpr int R = VecT<V>::R;
        lo = lo / R * R;
        hi = (hi + R - 1) / R * R;
        if (hi > K.n_pad) hi = K.n_pad;
        win[blockIdx.x] = PkWin{lo, hi};
    }
}

}  // namespace egfem
