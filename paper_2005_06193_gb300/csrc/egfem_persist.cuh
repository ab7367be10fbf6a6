// egfem_persist.cuh -- BiCGStab (van der Vorst 1992) on the Jacobi-scaled system as ONE
// persistent, cooperatively launched kernel per solve.
//
// The graph-captured iteration (egfem_krylov.cuh) launches five kernels per iteration, and
// each pays a launch ramp and a tail in which most SMs idle (ncu on a 1M-row system: the SMs
// are busy for 70 % of kry_t's duration).  Here every thread keeps the same R rows through
// all phases of all iterations; the phases that need other rows' values (the two operator
// applications) or a global sum (the inner products) are separated by a grid barrier:
//
//   A : v = A p,                        (rh, v)          -> alpha      barrier (+ sum)
//   B1: s = r - alpha v                                                barrier
//   B2: t = A s,                        (t, s), (t, t)   -> omega      barrier (+ sum)
//   C : x += alpha p + omega s, r = s - omega t, (rh, r), (r, r) -> beta, test   barrier (+ sum)
//   D : p = r + beta (p - omega v)                                     barrier
//
// Every block sums the per-block partials itself, in one fixed order, so all blocks hold
// bitwise-identical scalars and take the same branches; block 0 alone writes the final state.
// Partials rotate over three slots, so no slot is rewritten before every block has read it.
//
// The barrier is an arrival counter and a generation word.  The cooperative launch guarantees
// that all blocks are resident (the host sizes the grid from the occupancy calculator), so
// every wait ends; each wait is bounded all the same (PK_WAIT_NS of %globaltimer), after which
// the block raises the error word, the other blocks leave their waits, and the solve ends with
// K_TIMEOUT instead of hanging.
//
// Vectors written during the launch are read with plain loads, ordered by the barriers; the
// operator, its index data and the right-hand side are read-only for the launch and use the
// non-coherent path.
//
// Double-float (df64) vectors take compensated arithmetic in the operator application: the
// difference x_c - x_i by TwoSum of the high words, the product with the FP32 operator value
// split exactly by an FMA, and the running sum by TwoSum with the low words accumulated apart
// (as in the Dot2 inner product), normalised once per row; vector updates use the "sloppy"
// double-float addition (TwoSum of the high words, plain sum of the low words; Hida, Li &
// Bailey 2001), whose error is below 2^-44 of the operands.
#pragma once

#include "egfem_batch.cuh"
#include "egfem_krylov.cuh"

namespace egfem {

struct PGrid {
    uint32_t count;     // blocks arrived at the current barrier
    uint32_t gen;       // barriers completed
    int32_t err;        // nonzero: a wait ran out; every block leaves
    int32_t pad;
};

constexpr unsigned long long PK_WAIT_NS = 2000000000ull;   // longest wait at one barrier

__device__ __forceinline__ unsigned long long pk_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier; false when it failed (a wait ran out here or in another block).
__device__ __forceinline__ bool pk_sync(PGrid *g, uint32_t &gen, unsigned long long limit_ns = PK_WAIT_NS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t target = gen + 1u;
        int ok = 1;
        __threadfence();
        const uint32_t arrived = atomicAdd(&g->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&g->count, 0u);
            __threadfence();
            atomicExch(&g->gen, target);
        } else {
            const volatile uint32_t *vg = &g->gen;
            const volatile int32_t *ve = &g->err;
            const unsigned long long t0 = pk_clock_ns();
            uint32_t spins = 0;
            while (*vg != target) {
                if (*ve) { ok = 0; break; }
                if ((++spins & 255u) == 0u && pk_clock_ns() - t0 > limit_ns) {
                    atomicExch(&g->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ok && *(const volatile int32_t *)&g->err) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    gen += 1u;
    return s_ok != 0;
}

// Loads of vectors written during the launch: plain (weak, L1-cached) loads.  The barrier's
// release/acquire pattern (bar.sync, then a gpu-scope fence around the arrival atomic and the
// generation read) orders every write before a barrier before every load after it, so these
// loads see the current values; the non-coherent path (__ldg) is not used for them.
__device__ __forceinline__ double ldc1(const double *p) { return *p; }
__device__ __forceinline__ df64 ldc1(const df64 *p) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    return {t.x, t.y};
}
template <typename V>
__device__ __forceinline__ Pack<V> ldcv(const V *p) {
    Pack<V> o;
    if constexpr (std::is_same<V, df64>::value) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o.v[0] = {t.x, t.y}; o.v[1] = {t.z, t.w};
    } else {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        o.v[0] = t.x; o.v[1] = t.y;
    }
    return o;
}

// sloppy double-float arithmetic for the vector updates
__device__ __forceinline__ df64 dfs_add(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 dfs_sub(df64 a, df64 b) { return dfs_add(a, df_neg(b)); }

template <typename V> struct PkOps;
template <> struct PkOps<double> {
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
};
template <> struct PkOps<df64> {
    static __device__ __forceinline__ df64 add(df64 a, df64 b) { return dfs_add(a, b); }
    static __device__ __forceinline__ df64 sub(df64 a, df64 b) { return dfs_sub(a, b); }
};

// y[r0 .. r0+R) = A x for the R rows at r0; xi = x at those rows
template <typename V>
__device__ __forceinline__ Pack<V> pk_spmv(const KVecs<V> &K, int64_t r0, const V *x, const Pack<V> &xi) {
    constexpr int R = VecT<V>::R;
    using M_t = typename VecT<V>::mat;
    const SliceMeta M = K.meta[r0 / SLICE];
    const int lane = int(r0 % SLICE);
    Pack<V> y;
    M_t a0[R];
    ldm(K.A + M.col_base + lane, a0);
    if constexpr (std::is_same<V, df64>::value) {
        // difference form: column 0 holds the row sum s_i
        float hi[R], lo[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            hi[j] = __fmul_rn(a0[j], xi.v[j].hi);
            lo[j] = __fmaf_rn(a0[j], xi.v[j].lo, __fmaf_rn(a0[j], xi.v[j].hi, -hi[j]));
        }
        for (int c = 1; c < M.ncol; ++c) {
            const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
            M_t a[R];
            ldm(K.A + q, a);
            int32_t col[R];
            row_cols(K, M, r0, q, c, col);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const df64 xc = ldc1(x + col[j]);
                // d = xc - xi: TwoSum of the high words, low words added with its error
                const float dh = __fsub_rn(xc.hi, xi.v[j].hi);
                const float bb = __fsub_rn(dh, xc.hi);
                const float eh = __fadd_rn(__fsub_rn(xc.hi, __fsub_rn(dh, bb)), __fsub_rn(-xi.v[j].hi, bb));
                const float dl = __fadd_rn(__fsub_rn(xc.lo, xi.v[j].lo), eh);
                // a d: exact product of the high word, the rest by FMA
                const float p = __fmul_rn(a[j], dh);
                const float e = __fmaf_rn(a[j], dl, __fmaf_rn(a[j], dh, -p));
                // running sum: TwoSum of the high words, errors into the low word
                const float t = __fadd_rn(hi[j], p);
                const float z = __fsub_rn(t, hi[j]);
                const float err = __fadd_rn(__fsub_rn(hi[j], __fsub_rn(t, z)), __fsub_rn(p, z));
                lo[j] = __fadd_rn(lo[j], __fadd_rn(err, e));
                hi[j] = t;
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) y.v[j] = df_fast_two_sum(hi[j], lo[j]);
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) y.v[j] = a0[j] * xi.v[j];
        for (int c = 1; c < M.ncol; ++c) {
            const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
            M_t a[R];
            ldm(K.A + q, a);
            int32_t col[R];
            row_cols(K, M, r0, q, c, col);
#pragma unroll
            for (int j = 0; j < R; ++j) y.v[j] = fma(a[j], ldc1(x + col[j]), y.v[j]);
        }
    }
    return y;
}

// block sums of NV values -> part[(slot * 2 + k) * gridDim.x + blockIdx.x]
template <int NV>
__device__ __forceinline__ void pk_partials(const double (&val)[NV], double *part, int slot) {
    __shared__ double sh[2][KRY_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double x = warp_sum(val[k]);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (int q = 0; q < KRY_BLOCK / 32; ++q) x += sh[k][q];
            part[(slot * 2 + k) * gridDim.x + blockIdx.x] = x;
        }
    }
}

// grid totals of a slot, summed in the same order by every block (after a barrier)
template <int NV>
__device__ __forceinline__ void pk_totals(const double *part, int slot, double (&tot)[NV]) {
    __shared__ double s_tot[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < NV) {
        double x = 0.0;
        for (int q = lane; q < int(gridDim.x); q += 32) x += __ldcg(&part[(slot * 2 + w) * gridDim.x + q]);
        x = warp_sum(x);
        if (lane == 0) s_tot[w] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s_tot[k];
}

#define PK_LOOP(K) \
    for (int64_t r0 = (int64_t(blockIdx.x) * KRY_BLOCK + threadIdx.x) * VecT<V>::R; r0 < (K).n_pad; \
         r0 += int64_t(gridDim.x) * KRY_BLOCK * VecT<V>::R)

constexpr int32_t K_TIMEOUT = 6;   // a grid-barrier wait ran out (KDone extension)

// Resident blocks per SM the persistent kernels are compiled for (register budget): the
// double-float loops fit 40 registers, the FP64 ones 48.
template <typename V> struct PkMinBlocks { static constexpr int value = 5; };
template <> struct PkMinBlocks<df64> { static constexpr int value = 6; };

// BiCGStab scalars of one system, kept in shared memory (block-uniform; registers are
// left to the row loops).
struct TileState {
    double rho, alpha, omega, beta, rr, rr0, tol2, best_rr, stall_rr;
    int32_t iter, last_improve, done, inst;
};

// Convergence / failure tests after the (rh, r), (r, r) reduction, then beta and rho.
__device__ __forceinline__ void pk_after_c(TileState &S, double rho1, double rr, int32_t maxit, int32_t stall) {
    S.iter += 1;
    S.rr = rr;
    if (rr < 0.81 * S.best_rr) { S.best_rr = rr; S.last_improve = S.iter; }
    // a diverged iteration stops before it overflows; a guarded solve gives up once its
    // residual is 1000 times the initial one
    const double blowup = stall > 0 ? 1e6 : 1e24;
    if (!isfinite(rho1) || !isfinite(rr) || rr > blowup * S.rr0) S.done = K_NONFINITE;
    else if (rr <= S.tol2) S.done = K_CONVERGED;
    else if (rho1 == 0.0 || S.omega == 0.0) S.done = K_BREAKDOWN;
    else if (S.iter >= maxit) S.done = K_MAXIT;
    else if (stall > 0 && S.best_rr <= S.stall_rr && S.iter - S.last_improve >= stall) S.done = K_STAGNATED;
    else {
        S.beta = (rho1 / S.rho) * (S.alpha / S.omega);
        S.rho = rho1;
    }
}

// The whole solve: x = 0 start, BiCGStab until (r, r) <= rtol^2 (b, b), a breakdown, the
// iteration cap, divergence or (stall > 0) stagnation.  K.part needs 6 * gridDim.x doubles.
template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK, PkMinBlocks<V>::value) kry_persistent(KVecs<V> K, PGrid *bar, double rtol, int32_t maxit,
                                                            int32_t stall) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    __shared__ TileState S;
    uint32_t gen = 0;

    // setup: x = v = 0, r = rh = p = b, rho = (b, b)
    {
        double acc[1] = {0.0};
        Pack<V> z;
#pragma unroll
        for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
        PK_LOOP(K) {
            const Pack<V> b = ldv(K.b + r0);
            stv(K.x + r0, z); stv(K.v + r0, z);
            stv(K.r + r0, b); stv(K.rh + r0, b); stv(K.p + r0, b);
#pragma unroll
            for (int j = 0; j < R; ++j) acc[0] += to_d(b.v[j]) * to_d(b.v[j]);
        }
        pk_partials<1>(acc, K.part, 0);
    }
    const bool ok0 = pk_sync(bar, gen);
    double tot1[1], tot2[2];
    pk_totals<1>(K.part, 0, tot1);
    if (threadIdx.x == 0) {
        const double rr0 = tot1[0];
        S.rr0 = S.rho = S.rr = S.best_rr = rr0;
        S.tol2 = rtol * rtol * rr0;
        S.stall_rr = 4e-6 * rr0;   // the stagnation guard waits for a 500x reduction
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0;
        S.iter = 0; S.last_improve = 0; S.inst = 0;
        S.done = !ok0 ? K_TIMEOUT : (rr0 == 0.0) ? K_CONVERGED : (!isfinite(rr0) ? K_NONFINITE : (maxit <= 0 ? K_MAXIT : K_RUNNING));
    }
    __syncthreads();

    while (S.done == K_RUNNING) {
        // A: v = A p, (rh, v)
        {
            DotAcc<V> a;
            PK_LOOP(K) {
                const Pack<V> p = ldcv(K.p + r0);
                const Pack<V> y = pk_spmv(K, r0, K.p, p);
                stv(K.v + r0, y);
                const Pack<V> rh = ldcv(K.rh + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) a.add(rh.v[j], y.v[j]);
            }
            const double acc[1] = {a.value()};
            pk_partials<1>(acc, K.part, 1);
        }
        if (!pk_sync(bar, gen)) { if (threadIdx.x == 0) S.done = K_TIMEOUT; break; }
        pk_totals<1>(K.part, 1, tot1);
        if (threadIdx.x == 0) {
            if (tot1[0] == 0.0 || !isfinite(tot1[0])) S.done = isfinite(tot1[0]) ? K_BREAKDOWN : K_NONFINITE;
            else S.alpha = S.rho / tot1[0];
        }
        __syncthreads();
        if (S.done != K_RUNNING) break;

        // B1: s = r - alpha v
        {
            const V al = cvt<V>(S.alpha);
            PK_LOOP(K) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> s;
#pragma unroll
                for (int j = 0; j < R; ++j) s.v[j] = Op::sub(r.v[j], al * v.v[j]);
                stv(K.s + r0, s);
            }
        }
        if (!pk_sync(bar, gen)) { if (threadIdx.x == 0) S.done = K_TIMEOUT; break; }

        // B2: t = A s, (t, s), (t, t)
        {
            DotAcc<V> ts, tt;
            PK_LOOP(K) {
                const Pack<V> s = ldcv(K.s + r0);
                const Pack<V> y = pk_spmv(K, r0, K.s, s);
                stv(K.t + r0, y);
#pragma unroll
                for (int j = 0; j < R; ++j) { ts.add(y.v[j], s.v[j]); tt.add(y.v[j], y.v[j]); }
            }
            const double acc[2] = {ts.value(), tt.value()};
            pk_partials<2>(acc, K.part, 2);
        }
        if (!pk_sync(bar, gen)) { if (threadIdx.x == 0) S.done = K_TIMEOUT; break; }
        pk_totals<2>(K.part, 2, tot2);
        if (threadIdx.x == 0) {
            if (!isfinite(tot2[0]) || !isfinite(tot2[1])) S.done = K_NONFINITE;
            else S.omega = tot2[1] == 0.0 ? 0.0 : tot2[0] / tot2[1];
        }
        __syncthreads();
        if (S.done != K_RUNNING) break;

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        {
            const V al = cvt<V>(S.alpha), om = cvt<V>(S.omega);
            DotAcc<V> rh_r, r_r;
            PK_LOOP(K) {
                const Pack<V> s = ldcv(K.s + r0), p = ldcv(K.p + r0), t = ldcv(K.t + r0), rh = ldcv(K.rh + r0);
                Pack<V> x = ldcv(K.x + r0), r;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    x.v[j] = Op::add(x.v[j], Op::add(al * p.v[j], om * s.v[j]));
                    r.v[j] = Op::sub(s.v[j], om * t.v[j]);
                    rh_r.add(rh.v[j], r.v[j]);
                    r_r.add(r.v[j], r.v[j]);
                }
                stv(K.x + r0, x);
                stv(K.r + r0, r);
            }
            const double acc[2] = {rh_r.value(), r_r.value()};
            pk_partials<2>(acc, K.part, 0);
        }
        if (!pk_sync(bar, gen)) { if (threadIdx.x == 0) S.done = K_TIMEOUT; break; }
        pk_totals<2>(K.part, 0, tot2);
        if (threadIdx.x == 0) pk_after_c(S, tot2[0], tot2[1], maxit, stall);
        __syncthreads();
        if (S.done != K_RUNNING) break;

        // D: p = r + beta (p - omega v)
        {
            const V be = cvt<V>(S.beta), om = cvt<V>(S.omega);
            PK_LOOP(K) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> p = ldcv(K.p + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) p.v[j] = Op::add(r.v[j], be * Op::sub(p.v[j], om * v.v[j]));
                stv(K.p + r0, p);
            }
        }
        if (!pk_sync(bar, gen)) { if (threadIdx.x == 0) S.done = K_TIMEOUT; break; }
    }
    __syncthreads();

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        KState &Q = *K.st;
        Q.rho = S.rho; Q.alpha = S.alpha; Q.omega = S.omega; Q.beta = S.beta;
        Q.rr = S.rr; Q.rr0 = S.rr0; Q.tol2 = S.tol2; Q.best_rr = S.best_rr; Q.stall_rr = S.stall_rr;
        Q.iter = S.iter; Q.maxit = maxit; Q.done = S.done; Q.last_improve = S.last_improve; Q.stall = stall;
    }
}

#undef PK_LOOP

// Self-test of the barrier's bounded wait: blocks with index >= arrive leave without
// arriving, so with arrive < gridDim.x the barrier cannot complete and the waiting blocks
// must give up after limit_ns.  ok[b] = 1 when block b passed the barrier, 0 when it gave up,
// -1 when it did not arrive.
__global__ void pk_barrier_selftest(PGrid *g, int32_t arrive, unsigned long long limit_ns, int32_t *ok) {
    uint32_t gen = 0;
    if (int32_t(blockIdx.x) >= arrive) {
        if (threadIdx.x == 0) ok[blockIdx.x] = -1;
        return;
    }
    const bool passed = pk_sync(g, gen, limit_ns);
    if (threadIdx.x == 0) ok[blockIdx.x] = passed ? 1 : 0;
}


// ---------------------------------------------------------------------------------
// Batched persistent solve: every instance of a batch (block-diagonal operator) iterates in
// one cooperative launch, with the same five phases and barriers as the single solve.
//
// Block b owns tiles b, b + G, b + 2G, ... (G = gridDim.x, at most PKB_MAXT per block).
// After each reduction barrier, a warp of every block that owns a tile of instance k sums
// k's tile partials in tile order, so all such blocks hold bitwise-identical scalars for k
// and take the same branches; the scalars live in shared memory, one record per owned
// tile.  A finished instance's tiles are skipped.  The loop ends when no block owns a
// running tile: each block posts its running-tile count after the last phase of an
// iteration and every block sums the counts after the barrier.  The owner of an
// instance's first tile writes the instance's final state.
// ---------------------------------------------------------------------------------

constexpr int PKB_MAXT = 64;

template <typename V>
struct PkBatch {
    KVecs<V> K;               // vectors and operator of the whole batch
    const BTile *tiles;
    int64_t ntiles;
    KState *st;               // [instances] final states
    double *part;             // [6 * ntiles + gridDim.x]: 3 slots x 2 values x tiles, then running counts
    const uint8_t *active;    // [instances] instances to solve
    const double *rtol;       // [instances]
    PGrid *bar;
    int32_t maxit, stall;
};

// block sums of NV values for one tile -> part[(slot * 2 + k) * ntiles + tile]
template <int NV>
__device__ __forceinline__ void pkb_tile_partial(const double (&val)[NV], double *part, int slot, int64_t ntiles,
                                                 int64_t tile) {
    __shared__ double sh[2][KRY_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // the previous tile's reader of sh is done
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double x = warp_sum(val[k]);
        if (lane == 0) sh[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (int q = 0; q < KRY_BLOCK / 32; ++q) x += sh[k][q];
            part[(slot * 2 + k) * ntiles + tile] = x;
        }
    }
}

// instance totals of every owned tile's instance: tot[t][k] (after a barrier)
template <typename V, int NV>
__device__ __forceinline__ void pkb_totals(const PkBatch<V> &B, int slot, int nt, const TileState *ts,
                                           double (*tot)[2]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < nt; t += KRY_BLOCK / 32) {
        if (ts[t].done != K_RUNNING) continue;
        const BTile T = B.tiles[blockIdx.x + int64_t(t) * gridDim.x];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (int q = lane; q < T.ntiles_inst; q += 32) x += __ldcg(&B.part[(slot * 2 + k) * B.ntiles + T.tile0 + q]);
            x = warp_sum(x);
            if (lane == 0) tot[t][k] = x;
        }
    }
    __syncthreads();
}

#define PKB_TILES(nt) for (int t = 0; t < (nt); ++t)
#define PKB_ROWS(T) \
    for (int64_t r0 = (T).r_begin + int64_t(threadIdx.x) * VecT<V>::R; r0 < (T).r_end; r0 += int64_t(KRY_BLOCK) * VecT<V>::R)

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK, PkMinBlocks<V>::value) kb_persistent(PkBatch<V> B) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    __shared__ TileState ts[PKB_MAXT];
    __shared__ double tot[PKB_MAXT][2];
    __shared__ double s_run;
    const int64_t G = gridDim.x;
    const int nt = blockIdx.x < B.ntiles ? int((B.ntiles - blockIdx.x + G - 1) / G) : 0;
    const KVecs<V> &K = B.K;
    uint32_t gen = 0;
    bool failed = false;

    for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
        const BTile T = B.tiles[blockIdx.x + int64_t(t) * G];
        TileState &S = ts[t];
        S.rho = S.rr = S.rr0 = S.tol2 = S.best_rr = S.stall_rr = 0.0;
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0;
        S.iter = 0; S.last_improve = 0; S.inst = T.inst;
        S.done = B.active[T.inst] ? K_RUNNING : K_CONVERGED;
    }
    __syncthreads();

    // setup: x = v = 0, r = rh = p = b, rho = (b, b)
    {
        Pack<V> z;
#pragma unroll
        for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            const int64_t tile = blockIdx.x + int64_t(t) * G;
            const BTile T = B.tiles[tile];
            double acc[1] = {0.0};
            PKB_ROWS(T) {
                const Pack<V> b = ldv(K.b + r0);
                stv(K.x + r0, z); stv(K.v + r0, z);
                stv(K.r + r0, b); stv(K.rh + r0, b); stv(K.p + r0, b);
#pragma unroll
                for (int j = 0; j < R; ++j) acc[0] += to_d(b.v[j]) * to_d(b.v[j]);
            }
            pkb_tile_partial<1>(acc, B.part, 0, B.ntiles, tile);
        }
    }
    if (!pk_sync(B.bar, gen)) failed = true;
    pkb_totals<V, 1>(B, 0, nt, ts, tot);
    for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
        TileState &S = ts[t];
        if (S.done != K_RUNNING) continue;
        const double x = tot[t][0], rt = B.rtol[S.inst];
        S.rho = S.rr = S.rr0 = S.best_rr = x;
        S.tol2 = rt * rt * x;
        S.stall_rr = 4e-6 * x;   // the stagnation guard waits for a 500x reduction
        S.done = (x == 0.0) ? K_CONVERGED : (!isfinite(x) ? K_NONFINITE : (B.maxit <= 0 ? K_MAXIT : K_RUNNING));
    }
    __syncthreads();

    while (!failed) {
        // A: v = A p, (rh, v)
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            const int64_t tile = blockIdx.x + int64_t(t) * G;
            const BTile T = B.tiles[tile];
            DotAcc<V> a;
            PKB_ROWS(T) {
                const Pack<V> p = ldcv(K.p + r0);
                const Pack<V> y = pk_spmv(K, r0, K.p, p);
                stv(K.v + r0, y);
                const Pack<V> rh = ldcv(K.rh + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) a.add(rh.v[j], y.v[j]);
            }
            const double acc[1] = {a.value()};
            pkb_tile_partial<1>(acc, B.part, 1, B.ntiles, tile);
        }
        if (!pk_sync(B.bar, gen)) { failed = true; break; }
        pkb_totals<V, 1>(B, 1, nt, ts, tot);
        for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
            TileState &S = ts[t];
            if (S.done != K_RUNNING) continue;
            const double x = tot[t][0];
            if (x == 0.0 || !isfinite(x)) S.done = isfinite(x) ? K_BREAKDOWN : K_NONFINITE;
            else S.alpha = S.rho / x;
        }
        __syncthreads();

        // B1: s = r - alpha v
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            const BTile T = B.tiles[blockIdx.x + int64_t(t) * G];
            const V al = cvt<V>(ts[t].alpha);
            PKB_ROWS(T) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> s;
#pragma unroll
                for (int j = 0; j < R; ++j) s.v[j] = Op::sub(r.v[j], al * v.v[j]);
                stv(K.s + r0, s);
            }
        }
        if (!pk_sync(B.bar, gen)) { failed = true; break; }

        // B2: t = A s, (t, s), (t, t)
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            const int64_t tile = blockIdx.x + int64_t(t) * G;
            const BTile T = B.tiles[tile];
            DotAcc<V> q_ts, q_tt;
            PKB_ROWS(T) {
                const Pack<V> s = ldcv(K.s + r0);
                const Pack<V> y = pk_spmv(K, r0, K.s, s);
                stv(K.t + r0, y);
#pragma unroll
                for (int j = 0; j < R; ++j) { q_ts.add(y.v[j], s.v[j]); q_tt.add(y.v[j], y.v[j]); }
            }
            const double acc[2] = {q_ts.value(), q_tt.value()};
            pkb_tile_partial<2>(acc, B.part, 2, B.ntiles, tile);
        }
        if (!pk_sync(B.bar, gen)) { failed = true; break; }
        pkb_totals<V, 2>(B, 2, nt, ts, tot);
        for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
            TileState &S = ts[t];
            if (S.done != K_RUNNING) continue;
            if (!isfinite(tot[t][0]) || !isfinite(tot[t][1])) S.done = K_NONFINITE;
            else S.omega = tot[t][1] == 0.0 ? 0.0 : tot[t][0] / tot[t][1];
        }
        __syncthreads();

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            const int64_t tile = blockIdx.x + int64_t(t) * G;
            const BTile T = B.tiles[tile];
            const V al = cvt<V>(ts[t].alpha), om = cvt<V>(ts[t].omega);
            DotAcc<V> rh_r, r_r;
            PKB_ROWS(T) {
                const Pack<V> s = ldcv(K.s + r0), p = ldcv(K.p + r0), tv = ldcv(K.t + r0), rh = ldcv(K.rh + r0);
                Pack<V> x = ldcv(K.x + r0), r;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    x.v[j] = Op::add(x.v[j], Op::add(al * p.v[j], om * s.v[j]));
                    r.v[j] = Op::sub(s.v[j], om * tv.v[j]);
                    rh_r.add(rh.v[j], r.v[j]);
                    r_r.add(r.v[j], r.v[j]);
                }
                stv(K.x + r0, x);
                stv(K.r + r0, r);
            }
            const double acc[2] = {rh_r.value(), r_r.value()};
            pkb_tile_partial<2>(acc, B.part, 0, B.ntiles, tile);
        }
        if (!pk_sync(B.bar, gen)) { failed = true; break; }
        pkb_totals<V, 2>(B, 0, nt, ts, tot);
        for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
            TileState &S = ts[t];
            if (S.done != K_RUNNING) continue;
            pk_after_c(S, tot[t][0], tot[t][1], B.maxit, B.stall);
        }
        __syncthreads();

        // D: p = r + beta (p - omega v); post the running-tile count
        int running = 0;
        PKB_TILES(nt) {
            if (ts[t].done != K_RUNNING) continue;
            ++running;
            const BTile T = B.tiles[blockIdx.x + int64_t(t) * G];
            const V be = cvt<V>(ts[t].beta), om = cvt<V>(ts[t].omega);
            PKB_ROWS(T) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> p = ldcv(K.p + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) p.v[j] = Op::add(r.v[j], be * Op::sub(p.v[j], om * v.v[j]));
                stv(K.p + r0, p);
            }
        }
        if (threadIdx.x == 0) B.part[6 * B.ntiles + blockIdx.x] = double(running);
        if (!pk_sync(B.bar, gen)) { failed = true; break; }
        if (threadIdx.x < 32) {
            double x = 0.0;
            for (int q = threadIdx.x; q < int(G); q += 32) x += __ldcg(&B.part[6 * B.ntiles + q]);
            x = warp_sum(x);
            if (threadIdx.x == 0) s_run = x;
        }
        __syncthreads();
        if (s_run == 0.0) break;
    }

    for (int t = threadIdx.x; t < nt; t += KRY_BLOCK) {
        const int64_t tile = blockIdx.x + int64_t(t) * G;
        const BTile T = B.tiles[tile];
        if (tile != T.tile0) continue;
        const TileState &S = ts[t];
        KState &Q = B.st[T.inst];
        Q.rho = S.rho; Q.alpha = S.alpha; Q.omega = S.omega; Q.beta = S.beta;
        Q.rr = S.rr; Q.rr0 = S.rr0; Q.tol2 = S.tol2; Q.best_rr = S.best_rr; Q.stall_rr = S.stall_rr;
        Q.iter = S.iter; Q.maxit = B.maxit; Q.last_improve = S.last_improve; Q.stall = B.stall;
        Q.done = failed ? K_TIMEOUT : S.done;
        Q.ticket = 0u;
    }
}

#undef PKB_TILES
#undef PKB_ROWS

}  // namespace egfem
