// egfem_persist.cuh -- BiCGStab (van der Vorst 1992) on Jacobi-scaled systems as ONE
// persistent, cooperatively launched kernel per solve, for one system or a batch of
// independent systems (block-diagonal operator, instances of uneven size).
//
// The graph-captured iteration (egfem_krylov.cuh) launches five kernels per iteration, and
// each pays a launch ramp and a tail in which most SMs idle (ncu on a 1M-row system: the SMs
// are busy for 70 % of kry_t's duration).  Here the rows are cut into tiles (row ranges
// inside one system); block b owns tiles b, b + G, b + 2G, ... (G = gridDim.x) for the whole
// solve, and the phases that need other rows' values (the two operator applications) or a
// global sum (the inner products) are separated by grid barriers:
//
//   A : v = A p,                        (rh, v)          -> alpha      barrier (+ sums)
//   B1: s = r - alpha v                                                barrier
//   B2: t = A s,                        (t, s), (t, t)   -> omega      barrier (+ sums)
//   C : x += alpha p + omega s, r = s - omega t, (rh, r), (r, r) -> beta, tests   barrier (+ sums)
//   D : p = r + beta (p - omega v)                                     barrier
//
// Each block writes one partial (double) per owned tile and inner product; double-float
// accumulators are summed within the block in double-float arithmetic on the FP32 pipe
// (GB300 executes FP64 at about 1/58 of the FP32 rate).  No block is singled out at a summing
// barrier: after it, EVERY block sums the partials it needs (all of them for one system,
// pk_solve1; all tiles of each owned tile's system for a batch, pk_solveb) in one fixed order
// and updates its own copy of the BiCGStab state in shared memory.  The copies agree bit for
// bit (same inputs, same order), so the loop ends in all blocks at once, and a barrier costs
// one arrival atomic and one wait -- not the arrival, a last block's sums, fence and release,
// and every block's read of the published scalars (about 7 round trips to L2 against 3).
//
// The barriers count arrivals (pk1_sync: one counter that only grows within a launch;
// pkb_sync: a ring of three 64-bit slots that also count the blocks still owning a running
// system, which ends the batched loop).  The cooperative launch guarantees that all blocks are
// resident (the host sizes the grid from the occupancy calculator), so every wait ends; each
// wait is bounded all the same (PK_WAIT_NS of %globaltimer), after which the block raises the
// error word, the other blocks leave their waits, and the host reports a timeout instead of
// hanging.
//
// Vectors written during the launch are read with plain loads, ordered by the barriers; the
// operator, its index data and the right-hand side are read-only for the launch and use the
// non-coherent path; partials rewritten during the launch are read at L2 (ld.global.cg).
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

constexpr int PK1_BLOCK = 512;  // threads per block of the single-system kernel (2 resident per SM)
constexpr int PKB_BLOCK = 256;  // threads per block of the batched kernel (4 resident per SM)
constexpr int PK_MAXT = 64;     // tiles per block

struct PGrid {
    uint32_t count;     // pk_solve1: arrivals so far in this launch (the k-th barrier ends at k x blocks)
    int32_t err;        // nonzero: a wait ran out (1) or too many tiles (2); every block leaves
    unsigned long long slot[3];   // pk_solveb: barrier k counts on slot k % 3 (arrivals | live blocks << 32)
};

constexpr unsigned long long PK_WAIT_NS = 2000000000ull;   // longest wait at one barrier

__device__ __forceinline__ unsigned long long pk_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t atom_add_acq_rel_gpu(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_relaxed_gpu(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu_u64(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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

// Off-diagonal columns whose operator values, indices and gathered vector entries are
// loaded together before any arithmetic (memory-level parallelism of the latency-bound
// operator application; 6 = the off-diagonal columns of a 2D P1 row).
template <typename V> struct PkChunk { static constexpr int value = 1; };

// y += a (xc - xi) for double-float xc, xi and an FP32 operator value a (compensated)
__device__ __forceinline__ void df_acc_diff(float &hi, float &lo, float a, df64 xc, df64 xi) {
    // d = xc - xi: TwoSum of the high words, low words added with its error
    const float dh = __fsub_rn(xc.hi, xi.hi);
    const float bb = __fsub_rn(dh, xc.hi);
    const float eh = __fadd_rn(__fsub_rn(xc.hi, __fsub_rn(dh, bb)), __fsub_rn(-xi.hi, bb));
    const float dl = __fadd_rn(__fsub_rn(xc.lo, xi.lo), eh);
    // a d: exact product of the high word, the rest by FMA
    const float p = __fmul_rn(a, dh);
    const float e = __fmaf_rn(a, dl, __fmaf_rn(a, dh, -p));
    // running sum: TwoSum of the high words, errors into the low word
    const float t = __fadd_rn(hi, p);
    const float z = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    lo = __fadd_rn(lo, __fadd_rn(err, e));
    hi = t;
}

// y[r0 .. r0+R) = A x for the R rows at r0; xi = x at those rows
template <typename V>
__device__ __forceinline__ Pack<V> pk_spmv(const KVecs<V> &K, int64_t r0, const V *x, const Pack<V> &xi) {
    constexpr int R = VecT<V>::R, CH = PkChunk<V>::value;
    constexpr bool DF = std::is_same<V, df64>::value;
    using M_t = typename VecT<V>::mat;
    const SliceMeta M = K.meta[r0 / SLICE];
    const int lane = int(r0 % SLICE);
    // accumulators: FP64 y, or the double-float pair (hi, lo) in the difference form
    // (column 0 holds the row sum s_i).  The FP64 operator's column 0 is the Jacobi-scaled
    // diagonal, stored as exactly 1 by every builder, so y starts at x_i without a load or a
    // multiply (the same value a0 x_i would give).
    double y64[R];
    float hi[R], lo[R];
    if constexpr (DF) {
        M_t a0[R];
        ldm(K.A + M.col_base + lane, a0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            hi[j] = __fmul_rn(a0[j], xi.v[j].hi);
            lo[j] = __fmaf_rn(a0[j], xi.v[j].lo, __fmaf_rn(a0[j], xi.v[j].hi, -hi[j]));
        }
    } else {
#pragma unroll
        for (int j = 0; j < R; ++j) y64[j] = xi.v[j];
    }
#pragma unroll 4
    for (int c0 = 1; c0 < M.ncol; c0 += CH) {
        M_t a[CH][R];
        int32_t col[CH][R];
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (c0 + k < M.ncol) {
                const int64_t q = M.col_base + int64_t(c0 + k) * SLICE + lane;
                ldm(K.A + q, a[k]);
                row_cols(K, M, r0, q, c0 + k, col[k]);
            }
        V xc[CH][R];
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (c0 + k < M.ncol) {
#pragma unroll
                for (int j = 0; j < R; ++j) xc[k][j] = ldc1(x + col[k][j]);
            }
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (c0 + k < M.ncol) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if constexpr (DF) df_acc_diff(hi[j], lo[j], a[k][j], xc[k][j], xi.v[j]);
                    else y64[j] = fma(a[k][j], xc[k][j], y64[j]);
                }
            }
    }
    Pack<V> y;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if constexpr (DF) y.v[j] = df_fast_two_sum(hi[j], lo[j]);
        else y.v[j] = y64[j];
    }
    return y;
}

// Convergence / failure tests after the (rh, r), (r, r) sums, then beta and rho.
__device__ __forceinline__ void pk_after_c(KState &S, double rho1, double rr, int32_t maxit, int32_t stall) {
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

// ---------------------------------------------------------------------------------
// The solve
// ---------------------------------------------------------------------------------

constexpr int32_t K_TIMEOUT = 6;   // a grid-barrier wait ran out (KDone extension)

// Resident blocks per SM the kernels are compiled for, 64 registers per thread either way, with
// the operator's column loop unrolled 4 times (its loads then issue ahead of the arithmetic).
// Every block sums all partials of a reduction, so for one system fewer, larger blocks shorten
// the sums and the barriers: per iteration, 512 x 2 against 256 x 4 at 66 k / 1 M / 4.2 M rows,
// FP64 24.0 / 87.7 / 265 us against 26.8 / 89.1 / 268, double-float 26.7 / 62.0 / 234 against
// 29.7 / 65.5 / 235 (1024 x 1 loses at 4.2 M rows: 278 / 243).  The batched kernel keeps
// 256 x 4: its blocks hold tiles of uneven instances, and 512 x 2 took the 32-instance P3 batch
// from 123.7 to 109.8 solves/s.
constexpr int PK1_MIN_BLOCKS = 2;
constexpr int PKB_MIN_BLOCKS = 4;

template <typename V>
struct PkArgs {
    KVecs<V> K;               // vectors and operator (K.st and K.part unused)
    const BTile *tiles;       // tiles grouped by system, in row order (each knows its system and first tile)
    int64_t ntiles;
    KState *st;               // [systems] BiCGStab state (final state for the host)
    double *part;             // [2 * ntiles] tile partials
    const uint8_t *active;    // [systems] systems to solve, or null (all)
    const double *rtol;       // [systems] tolerances, or null (rtol0 for all)
    double rtol0;
    PGrid *bar;
    int32_t maxit, stall;
};


__device__ __forceinline__ df64 shfl_xor_df(df64 a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Block sum of NV per-thread accumulators for one tile -> part[k * ntiles + tile].
template <typename V, int NV, int BLOCK>
__device__ __forceinline__ void pk_tile_partial(const DotAcc<V> (&acc)[NV], double *part, int64_t ntiles, int64_t tile) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // the previous tile's readers of the shared arrays are done
    if constexpr (std::is_same<V, df64>::value) {
        // warp and block sums in double-float arithmetic (FP32 pipe), one conversion per tile
        __shared__ float2 shf[2][BLOCK / 32];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            df64 x = df_two_sum(acc[k].hi, acc[k].lo);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = df_add(x, shfl_xor_df(x, o));
            if (lane == 0) shf[k][w] = make_float2(x.hi, x.lo);
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            const int k = threadIdx.x;
            df64 x = {shf[k][0].x, shf[k][0].y};
            for (int q = 1; q < BLOCK / 32; ++q) x = df_add(x, df64{shf[k][q].x, shf[k][q].y});
            part[k * ntiles + tile] = df_to_double(x);
        }
    } else {
        __shared__ double shd[2][BLOCK];
#pragma unroll
        for (int k = 0; k < NV; ++k) shd[k][threadIdx.x] = acc[k].value();
        __syncthreads();
        if (w < NV) {
            double x = 0.0;
#pragma unroll
            for (int q = 0; q < BLOCK / 32; ++q) x += shd[w][lane + 32 * q];
            x = warp_sum(x);
            if (lane == 0) part[w * ntiles + tile] = x;
        }
    }
}

#define PK_TILES(nt) for (int t = 0; t < (nt); ++t)
#define PK_ROWS(T) \
    _Pragma("unroll 1") for (int64_t r0 = (T).r_begin + int64_t(threadIdx.x) * VecT<V>::R; r0 < (T).r_end; r0 += int64_t(PKB_BLOCK) * VecT<V>::R)

// ---------------------------------------------------------------------------------
// One system: every block keeps the solver state
// ---------------------------------------------------------------------------------

// Grid-wide barrier on an arrival counter that only grows within a launch: the k-th barrier
// completes when the counter reaches k x gridDim.x.  No block is singled out, so a barrier is
// one arrival atomic and one wait (two L2 round trips) instead of the arrival, the last
// block's release and the waiters' reads.  false when the wait ran out or another block gave up.
__device__ __forceinline__ bool pk1_sync(PGrid *g, uint32_t &nbar, unsigned long long limit_ns = PK_WAIT_NS) {
    __shared__ int s_ok;
    ++nbar;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t target = nbar * gridDim.x;
        int ok = 1;
        if (atom_add_acq_rel_gpu(&g->count, 1u) + 1u < target) {
            const unsigned long long t0 = pk_clock_ns();
            uint32_t spins = 0;
            while (ld_acquire_gpu(&g->count) < target) {
                if (ld_relaxed_gpu(&g->err)) { ok = 0; break; }
                if ((++spins & 255u) == 0u && pk_clock_ns() - t0 > limit_ns) {
                    atomicExch(&g->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Most blocks the single-system kernel sums over (8 resident blocks on each of 152 SMs; the
// host launches the general kernel beyond it)
constexpr int PK1_MAXG = 8 * 152;

// Sums of NV dot products over the grid, the same in every block: the block's partials go to
// part[k * G + block]; after the barrier every block loads all G partials into shared memory
// (one round of parallel L2 loads), and warp k adds those of value k in one fixed order (lanes
// over partials, then the warp's tree); s_p is the kernel's [2][PK1_MAXG] shared buffer.  One warp per sum keeps the FP64 work of the redundant
// sums small: GB300 retires about two FP64 operations per SM and clock.
template <typename V, int NV>
__device__ __forceinline__ bool pk1_allreduce(const PkArgs<V> &P, const DotAcc<V> (&acc)[NV], uint32_t &nbar,
                                              double (*s_p)[PK1_MAXG], double (&tot)[NV]) {
    __shared__ double s_tot[2];
    const int G = int(gridDim.x);
    pk_tile_partial<V, NV, PK1_BLOCK>(acc, P.part, G, blockIdx.x);
    if (!pk1_sync(P.bar, nbar)) return false;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int q = threadIdx.x; q < G; q += PK1_BLOCK) s_p[k][q] = __ldcg(P.part + int64_t(k) * G + q);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < NV) {
        double x = 0.0;
        for (int q = lane; q < G; q += 32) x += s_p[w][q];
        x = warp_sum(x);
        if (lane == 0) s_tot[w] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s_tot[k];
    return true;
}

#define PK1_ROWS \
    _Pragma("unroll 1") for (int64_t r0 = T.r_begin + int64_t(threadIdx.x) * VecT<V>::R; r0 < T.r_end; r0 += int64_t(PK1_BLOCK) * VecT<V>::R)

// The solve of one system, one tile per block (P.ntiles == gridDim.x), in the phases A, B1,
// B2, C, D above from x = 0 until (r, r) <= rtol^2 (b, b), a breakdown, the iteration cap,
// divergence or (stall > 0) stagnation; every block computes the scalars itself from all
// partials and keeps the state in shared memory.  Block 0 writes the final state to P.st
// (done = K_TIMEOUT when a barrier wait ran out; P.bar->err is then set too).  An inactive
// system (P.active[0] == 0) returns at once.
template <typename V>
__global__ void __launch_bounds__(PK1_BLOCK, PK1_MIN_BLOCKS) pk_solve1(PkArgs<V> P) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    __shared__ KState S;
    __shared__ double s_p[2][PK1_MAXG];   // partials of the sums in progress
    if (P.active && !P.active[0]) return;
    const KVecs<V> &K = P.K;
    __shared__ BTile T;   // the block's rows (in shared memory: fewer live registers in the phases)
    if (threadIdx.x == 0) T = P.tiles[blockIdx.x];
    __syncthreads();
    uint32_t nbar = 0;
    bool ok;
    {
        // setup: x = v = 0, r = rh = p = b, (b, b)
        Pack<V> z;
#pragma unroll
        for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
        DotAcc<V> acc[1];
        PK1_ROWS {
            const Pack<V> b = ldv(K.b + r0);
            stv(K.x + r0, z); stv(K.v + r0, z);
            stv(K.r + r0, b); stv(K.rh + r0, b); stv(K.p + r0, b);
#pragma unroll
            for (int j = 0; j < R; ++j) acc[0].add(b.v[j], b.v[j]);
        }
        double tot[1];
        ok = pk1_allreduce<V, 1>(P, acc, nbar, s_p, tot);
        if (threadIdx.x == 0) {
            const double x = ok ? tot[0] : 0.0, rt = P.rtol ? P.rtol[0] : P.rtol0;
            S.iter = 0; S.last_improve = 0; S.maxit = P.maxit; S.stall = P.stall; S.ticket = 0u;
            S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0; S.scratch[0] = S.scratch[1] = 0.0;
            S.rho = S.rr = S.rr0 = S.best_rr = x;
            S.tol2 = rt * rt * x;
            S.stall_rr = 4e-6 * x;
            S.done = (x == 0.0) ? K_CONVERGED : (!isfinite(x) ? K_NONFINITE : (P.maxit <= 0 ? K_MAXIT : K_RUNNING));
        }
        __syncthreads();
    }

    while (ok && S.done == K_RUNNING) {
        // A: v = A p, (rh, v)
        {
            DotAcc<V> acc[1];
            PK1_ROWS {
                const Pack<V> p = ldcv(K.p + r0);
                const Pack<V> y = pk_spmv(K, r0, K.p, p);
                stv(K.v + r0, y);
                const Pack<V> rh = ldcv(K.rh + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) acc[0].add(rh.v[j], y.v[j]);
            }
            double tot[1];
            if (!(ok = pk1_allreduce<V, 1>(P, acc, nbar, s_p, tot))) break;
            if (threadIdx.x == 0) {
                if (tot[0] == 0.0 || !isfinite(tot[0])) S.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
                else S.alpha = S.rho / tot[0];
            }
            __syncthreads();
            if (S.done != K_RUNNING) break;
        }

        // B1: s = r - alpha v
        const V al = cvt<V>(S.alpha);
        PK1_ROWS {
            const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
            Pack<V> s;
#pragma unroll
            for (int j = 0; j < R; ++j) s.v[j] = Op::sub(r.v[j], al * v.v[j]);
            stv(K.s + r0, s);
        }
        if (!(ok = pk1_sync(P.bar, nbar))) break;

        // B2: t = A s, (t, s), (t, t)
        {
            DotAcc<V> acc[2];
            PK1_ROWS {
                const Pack<V> s = ldcv(K.s + r0);
                const Pack<V> y = pk_spmv(K, r0, K.s, s);
                stv(K.t + r0, y);
#pragma unroll
                for (int j = 0; j < R; ++j) { acc[0].add(y.v[j], s.v[j]); acc[1].add(y.v[j], y.v[j]); }
            }
            double tot[2];
            if (!(ok = pk1_allreduce<V, 2>(P, acc, nbar, s_p, tot))) break;
            if (threadIdx.x == 0) {
                if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
                else S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
            }
            __syncthreads();
            if (S.done != K_RUNNING) break;
        }

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        {
            const V om = cvt<V>(S.omega);
            DotAcc<V> acc[2];
            PK1_ROWS {
                const Pack<V> s = ldcv(K.s + r0), p = ldcv(K.p + r0), tv = ldcv(K.t + r0), rh = ldcv(K.rh + r0);
                Pack<V> x = ldcv(K.x + r0), r;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    x.v[j] = Op::add(x.v[j], Op::add(al * p.v[j], om * s.v[j]));
                    r.v[j] = Op::sub(s.v[j], om * tv.v[j]);
                    acc[0].add(rh.v[j], r.v[j]);
                    acc[1].add(r.v[j], r.v[j]);
                }
                stv(K.x + r0, x);
                stv(K.r + r0, r);
            }
            double tot[2];
            if (!(ok = pk1_allreduce<V, 2>(P, acc, nbar, s_p, tot))) break;
            if (threadIdx.x == 0) pk_after_c(S, tot[0], tot[1], P.maxit, P.stall);
            __syncthreads();
            if (S.done != K_RUNNING) break;
        }

        // D: p = r + beta (p - omega v)
        {
            const V be = cvt<V>(S.beta), om = cvt<V>(S.omega);
            PK1_ROWS {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> p = ldcv(K.p + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) p.v[j] = Op::add(r.v[j], be * Op::sub(p.v[j], om * v.v[j]));
                stv(K.p + r0, p);
            }
        }
        if (!(ok = pk1_sync(P.bar, nbar))) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        KState F = S;
        if (!ok) F.done = K_TIMEOUT;
        *P.st = F;
    }
}

#undef PK1_ROWS

// ---------------------------------------------------------------------------------
// Many systems (a batch): every block keeps the states of its tiles' systems
// ---------------------------------------------------------------------------------

// Barrier number nbar of pk_solveb: thread 0 counts the block on slot nbar % 3 (low word:
// arrivals; high word: blocks that still own a running tile) and waits until all gridDim.x
// blocks have arrived; live = the high word then, the same in every block.  Block 0 clears
// slot (nbar - 1) % 3 after passing: every block has read it before arriving here, and none
// adds to it again before barrier nbar + 2, which needs block 0's next arrival.  false when
// the wait ran out or another block gave up.
__device__ __forceinline__ bool pkb_sync(PGrid *g, uint32_t &nbar, int has_live, uint32_t &live,
                                         unsigned long long limit_ns = PK_WAIT_NS) {
    __shared__ int s_ok;
    __shared__ uint32_t s_live;
    ++nbar;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *sl = &g->slot[nbar % 3u];
        const unsigned long long add = 1ull | (has_live ? (1ull << 32) : 0ull);
        unsigned long long v = atom_add_acq_rel_gpu_u64(sl, add) + add;
        int ok = 1;
        const unsigned long long t0 = pk_clock_ns();
        uint32_t spins = 0;
        while (uint32_t(v & 0xffffffffull) < gridDim.x) {
            if (ld_relaxed_gpu(&g->err)) { ok = 0; break; }
            if ((++spins & 255u) == 0u && pk_clock_ns() - t0 > limit_ns) {
                atomicExch(&g->err, 1);
                ok = 0;
                break;
            }
            __nanosleep(32);
            v = ld_acquire_gpu_u64(sl);
        }
        if (blockIdx.x == 0) st_relaxed_gpu_u64(&g->slot[(nbar + 2u) % 3u], 0ull);
        s_ok = ok;
        s_live = uint32_t(v >> 32);
    }
    __syncthreads();
    live = s_live;
    return s_ok != 0;
}

// The sums of a barrier: for each owned tile whose system runs, warp (tile mod 8) adds the NV
// partials of all tiles of that system in one fixed order (lanes over tiles, then the warp's
// tree), so every block holding a tile of the system computes the same sums, and lane 0 calls
// update(state, system, sums) on the block's copy of the state.
template <typename V, int NV, typename U>
__device__ __forceinline__ void pkb_sums(const PkArgs<V> &P, int nt, KState *st, const BTile *tl, U &&update) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < nt; t += PKB_BLOCK / 32) {
        if (st[t].done != K_RUNNING) continue;
        const int64_t t0 = tl[t].tile0;
        const int32_t n = tl[t].ntiles_inst;
        double x[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int q = lane; q < n; q += 32) a += __ldcg(P.part + k * P.ntiles + t0 + q);
            x[k] = warp_sum(a);
        }
        if (lane == 0) update(st[t], tl[t].inst, x);
    }
    __syncthreads();
}

// The batched solve: every active system from x = 0, BiCGStab until (r, r) <= rtol^2 (b, b),
// a breakdown, the iteration cap, divergence or (stall > 0) stagnation; the phases and their
// arithmetic are pk_solve1's.  Tiles are dealt to blocks round-robin (tile = block + t G); a
// block keeps the state of each owned tile's system in shared memory, computed from all of
// that system's partials, and the loop ends at the first barrier at which no block owns a
// running tile.  The block owning a system's first tile writes its final state to P.st
// (done = K_TIMEOUT when a barrier wait ran out; P.bar->err is then set too).
template <typename V>
__global__ void __launch_bounds__(PKB_BLOCK, PKB_MIN_BLOCKS) pk_solveb(PkArgs<V> P) {
    using Op = PkOps<V>;
    constexpr int R = VecT<V>::R;
    __shared__ KState s_st[PK_MAXT];
    __shared__ BTile s_tl[PK_MAXT];
    const int64_t G = gridDim.x;
    if (P.ntiles > G * PK_MAXT) {   // the host keeps to the limit; every block leaves at once
        if (blockIdx.x == 0 && threadIdx.x == 0) P.bar->err = 2;
        return;
    }
    const int nt = int64_t(blockIdx.x) < P.ntiles ? int((P.ntiles - blockIdx.x + G - 1) / G) : 0;
    const KVecs<V> &K = P.K;
    for (int t = threadIdx.x; t < nt; t += PKB_BLOCK) {
        const BTile T = P.tiles[blockIdx.x + int64_t(t) * G];
        s_tl[t] = T;
        KState &S = s_st[t];
        S.done = (!P.active || P.active[T.inst]) ? K_RUNNING : K_CONVERGED;
        S.iter = 0; S.last_improve = 0; S.maxit = P.maxit; S.stall = P.stall; S.ticket = 0u;
        S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0; S.scratch[0] = S.scratch[1] = 0.0;
        S.rho = S.rr = S.rr0 = S.best_rr = S.tol2 = S.stall_rr = 0.0;
    }
    __syncthreads();
    auto running = [&]() {
        int a = 0;
        for (int t = 0; t < nt; ++t) a |= (s_st[t].done == K_RUNNING);
        return a;
    };
    uint32_t nbar = 0, live = 0;

    // setup: x = v = 0, r = rh = p = b, (b, b)
    {
        Pack<V> z;
#pragma unroll
        for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            DotAcc<V> acc[1];
            PK_ROWS(T) {
                const Pack<V> b = ldv(K.b + r0);
                stv(K.x + r0, z); stv(K.v + r0, z);
                stv(K.r + r0, b); stv(K.rh + r0, b); stv(K.p + r0, b);
#pragma unroll
                for (int j = 0; j < R; ++j) acc[0].add(b.v[j], b.v[j]);
            }
            pk_tile_partial<V, 1, PKB_BLOCK>(acc, P.part, P.ntiles, blockIdx.x + int64_t(t) * G);
        }
    }
    bool ok = pkb_sync(P.bar, nbar, running(), live);
    if (ok && live)
        pkb_sums<V, 1>(P, nt, s_st, s_tl, [&](KState &S, int b, const double *tot) {
            const double x = tot[0], rt = P.rtol ? P.rtol[b] : P.rtol0;
            S.rho = S.rr = S.rr0 = S.best_rr = x;
            S.tol2 = rt * rt * x;
            S.stall_rr = 4e-6 * x;
            S.done = (x == 0.0) ? K_CONVERGED : (!isfinite(x) ? K_NONFINITE : (P.maxit <= 0 ? K_MAXIT : K_RUNNING));
        });

    while (ok && live) {
        // A: v = A p, (rh, v)
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            DotAcc<V> acc[1];
            PK_ROWS(T) {
                const Pack<V> p = ldcv(K.p + r0);
                const Pack<V> y = pk_spmv(K, r0, K.p, p);
                stv(K.v + r0, y);
                const Pack<V> rh = ldcv(K.rh + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) acc[0].add(rh.v[j], y.v[j]);
            }
            pk_tile_partial<V, 1, PKB_BLOCK>(acc, P.part, P.ntiles, blockIdx.x + int64_t(t) * G);
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
        pkb_sums<V, 1>(P, nt, s_st, s_tl, [&](KState &S, int, const double *tot) {
            if (tot[0] == 0.0 || !isfinite(tot[0])) S.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
            else S.alpha = S.rho / tot[0];
        });

        // B1: s = r - alpha v
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            const V al = cvt<V>(s_st[t].alpha);
            PK_ROWS(T) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> s;
#pragma unroll
                for (int j = 0; j < R; ++j) s.v[j] = Op::sub(r.v[j], al * v.v[j]);
                stv(K.s + r0, s);
            }
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;

        // B2: t = A s, (t, s), (t, t)
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            DotAcc<V> acc[2];
            PK_ROWS(T) {
                const Pack<V> s = ldcv(K.s + r0);
                const Pack<V> y = pk_spmv(K, r0, K.s, s);
                stv(K.t + r0, y);
#pragma unroll
                for (int j = 0; j < R; ++j) { acc[0].add(y.v[j], s.v[j]); acc[1].add(y.v[j], y.v[j]); }
            }
            pk_tile_partial<V, 2, PKB_BLOCK>(acc, P.part, P.ntiles, blockIdx.x + int64_t(t) * G);
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
        pkb_sums<V, 2>(P, nt, s_st, s_tl, [&](KState &S, int, const double *tot) {
            if (!isfinite(tot[0]) || !isfinite(tot[1])) S.done = K_NONFINITE;
            else S.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
        });

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            const V al = cvt<V>(s_st[t].alpha), om = cvt<V>(s_st[t].omega);
            DotAcc<V> acc[2];
            PK_ROWS(T) {
                const Pack<V> s = ldcv(K.s + r0), p = ldcv(K.p + r0), tv = ldcv(K.t + r0), rh = ldcv(K.rh + r0);
                Pack<V> x = ldcv(K.x + r0), r;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    x.v[j] = Op::add(x.v[j], Op::add(al * p.v[j], om * s.v[j]));
                    r.v[j] = Op::sub(s.v[j], om * tv.v[j]);
                    acc[0].add(rh.v[j], r.v[j]);
                    acc[1].add(r.v[j], r.v[j]);
                }
                stv(K.x + r0, x);
                stv(K.r + r0, r);
            }
            pk_tile_partial<V, 2, PKB_BLOCK>(acc, P.part, P.ntiles, blockIdx.x + int64_t(t) * G);
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
        pkb_sums<V, 2>(P, nt, s_st, s_tl, [&](KState &S, int, const double *tot) {
            pk_after_c(S, tot[0], tot[1], P.maxit, P.stall);
        });

        // D: p = r + beta (p - omega v)
        PK_TILES(nt) {
            if (s_st[t].done != K_RUNNING) continue;
            const BTile &T = s_tl[t];
            const V be = cvt<V>(s_st[t].beta), om = cvt<V>(s_st[t].omega);
            PK_ROWS(T) {
                const Pack<V> r = ldcv(K.r + r0), v = ldcv(K.v + r0);
                Pack<V> p = ldcv(K.p + r0);
#pragma unroll
                for (int j = 0; j < R; ++j) p.v[j] = Op::add(r.v[j], be * Op::sub(p.v[j], om * v.v[j]));
                stv(K.p + r0, p);
            }
        }
        if (!(ok = pkb_sync(P.bar, nbar, running(), live)) || !live) break;
    }
    for (int t = threadIdx.x; t < nt; t += PKB_BLOCK) {
        if (blockIdx.x + int64_t(t) * G != s_tl[t].tile0) continue;
        KState F = s_st[t];
        if (!ok) F.done = K_TIMEOUT;
        P.st[s_tl[t].inst] = F;
    }
}

#undef PK_TILES
#undef PK_ROWS

// Self-test of the barriers' bounded waits: blocks with index >= arrive leave without
// arriving, so with arrive < gridDim.x the batched solve's barrier (pkb_sync) cannot complete
// and the waiting blocks must give up after limit_ns; when it completes, its live count must
// equal the arrivals, and the single-system barrier (pk1_sync) follows.  ok[b] = 1 when block
// b passed both, 0 when it gave up, -1 when it did not arrive.
__global__ void pk_barrier_selftest(PGrid *g, int32_t arrive, unsigned long long limit_ns, int32_t *ok) {
    uint32_t nb = 0, n1 = 0, live = 0;
    if (int32_t(blockIdx.x) >= arrive) {
        if (threadIdx.x == 0) ok[blockIdx.x] = -1;
        return;
    }
    bool passed = pkb_sync(g, nb, 1, live, limit_ns) && live == uint32_t(arrive);
    passed = passed && pk1_sync(g, n1, limit_ns);
    if (threadIdx.x == 0) ok[blockIdx.x] = passed ? 1 : 0;
}

}  // namespace egfem
