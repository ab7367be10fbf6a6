// egfem_batch.cuh -- batched BiCGStab: many independent instances (meshes of uneven size)
// stored as one block-diagonal operator, iterated together in one launch per kernel.
//
// Every instance owns a contiguous, slice-aligned row range.  The work list is a set of
// tiles, each a row range inside one instance; a persistent grid strides over the tiles.
// Dot products are reduced per tile (fixed order) and then per instance by the last of
// the instance's tiles to finish (one atomic ticket per instance, no waiting), which
// updates that instance's BiCGStab scalars.  An instance that has finished (converged,
// failed, or inactive in this Newton step) skips its tiles, so one captured chunk of
// iterations serves the whole batch while instances finish at different iterations.
#pragma once

#include "egfem_krylov.cuh"

namespace egfem {

struct BTile {
    int64_t r_begin, r_end;   // rows [r_begin, r_end), multiples of the thread row count
    int64_t tile0;            // first tile of this instance
    int32_t inst;             // instance index
    int32_t ntiles_inst;      // tiles of this instance
};

template <typename V>
struct KBatch {
    KVecs<V> K;               // vectors and operator of the whole batch (K.st unused)
    const BTile *tiles;
    int64_t ntiles;
    KState *st;               // [instances]
    double *part;             // [2 * ntiles]
};

__device__ __forceinline__ bool inst_finished(const KState *st) {
    return *(volatile const int32_t *)&st->done != K_RUNNING;
}

// Block-reduce NV values for tile T, store the tile partials, and return true in the block
// that finished the instance's last tile, with tot = the instance totals (tile order).
template <int NV>
__device__ bool tile_reduce(double (&val)[NV], double *part, int64_t ntiles, int64_t tile, const BTile &T, KState *S,
                            double (&tot)[NV]) {
    __shared__ double sh[NV][KRY_BLOCK / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // the previous tile's readers of sh are done
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
            part[k * ntiles + tile] = x;
        }
        __threadfence();
        const uint32_t t = atomicAdd(&S->ticket, 1u);
        last = (t == uint32_t(T.ntiles_inst) - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = 0.0;
        for (int q = threadIdx.x; q < T.ntiles_inst; q += KRY_BLOCK) x += __ldcg(&part[k * ntiles + T.tile0 + q]);
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
    if (threadIdx.x == 0) S->ticket = 0u;
    return true;
}

#define KB_TILES(B) for (int64_t tile = blockIdx.x; tile < (B).ntiles; tile += gridDim.x)
#define KB_ROWS(T) \
    for (int64_t r0 = (T).r_begin + int64_t(threadIdx.x) * VecT<V>::R; r0 < (T).r_end; r0 += int64_t(KRY_BLOCK) * VecT<V>::R)

// per-instance state: active instances start (tol2 set by kb_setup), the others are done
__global__ void kb_init_state(int32_t nb, KState *st, const uint8_t *active, const double *rtol, int32_t maxit,
                              int32_t stall) {
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    KState &S = st[b];
    S.iter = 0; S.maxit = maxit; S.last_improve = 0; S.stall = stall; S.ticket = 0u;
    S.alpha = 1.0; S.omega = 1.0; S.beta = 0.0;
    S.scratch[0] = rtol[b];
    S.done = active[b] ? K_RUNNING : K_CONVERGED;
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_setup(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    Pack<V> z;
#pragma unroll
    for (int j = 0; j < R; ++j) z.v[j] = cvt<V>(0.0);
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        double acc[1] = {0.0};
        KB_ROWS(T) {
            const Pack<V> b = ldv(B.K.b + r0);
            stv(B.K.x + r0, z); stv(B.K.v + r0, z);
            stv(B.K.r + r0, b); stv(B.K.rh + r0, b); stv(B.K.p + r0, b);
#pragma unroll
            for (int j = 0; j < R; ++j) acc[0] += to_d(b.v[j]) * to_d(b.v[j]);
        }
        double tot[1];
        if (tile_reduce<1>(acc, B.part, B.ntiles, tile, T, S, tot) && threadIdx.x == 0) {
            const double rtol = S->scratch[0];
            S->rho = tot[0]; S->rr = tot[0]; S->rr0 = tot[0]; S->best_rr = tot[0];
            S->tol2 = rtol * rtol * tot[0];
            S->stall_rr = 4e-6 * tot[0];
            S->done = (tot[0] == 0.0) ? K_CONVERGED : (!isfinite(tot[0]) ? K_NONFINITE : K_RUNNING);
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_v(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        DotAcc<V> a;
        KB_ROWS(T) {
            const Pack<V> y = sell_rows(B.K, r0, B.K.p);
            stv(B.K.v + r0, y);
            const Pack<V> rh = ldv(B.K.rh + r0);
#pragma unroll
            for (int j = 0; j < R; ++j) a.add(rh.v[j], y.v[j]);
        }
        double acc[1] = {a.value()}, tot[1];
        if (tile_reduce<1>(acc, B.part, B.ntiles, tile, T, S, tot) && threadIdx.x == 0) {
            if (tot[0] == 0.0 || !isfinite(tot[0])) S->done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
            else S->alpha = S->rho / tot[0];
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_s(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        const KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        const V alpha = cvt<V>(S->alpha);
        KB_ROWS(T) {
            const Pack<V> r = ldv(B.K.r + r0), v = ldv(B.K.v + r0);
            Pack<V> s;
#pragma unroll
            for (int j = 0; j < R; ++j) s.v[j] = r.v[j] - alpha * v.v[j];
            stv(B.K.s + r0, s);
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_t(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        DotAcc<V> ts, tt;
        KB_ROWS(T) {
            const Pack<V> y = sell_rows(B.K, r0, B.K.s);
            stv(B.K.t + r0, y);
            const Pack<V> s = ldv(B.K.s + r0);
#pragma unroll
            for (int j = 0; j < R; ++j) { ts.add(y.v[j], s.v[j]); tt.add(y.v[j], y.v[j]); }
        }
        double acc[2] = {ts.value(), tt.value()}, tot[2];
        if (tile_reduce<2>(acc, B.part, B.ntiles, tile, T, S, tot) && threadIdx.x == 0) {
            if (!isfinite(tot[0]) || !isfinite(tot[1])) S->done = K_NONFINITE;
            else S->omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_x(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        const V alpha = cvt<V>(S->alpha), omega = cvt<V>(S->omega);
        DotAcc<V> rho, rr;
        KB_ROWS(T) {
            const Pack<V> s = ldv(B.K.s + r0), p = ldv(B.K.p + r0), t = ldv(B.K.t + r0), rh = ldv(B.K.rh + r0);
            Pack<V> x = ldv(B.K.x + r0), r;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                x.v[j] += alpha * p.v[j] + omega * s.v[j];
                r.v[j] = s.v[j] - omega * t.v[j];
                rho.add(rh.v[j], r.v[j]);
                rr.add(r.v[j], r.v[j]);
            }
            stv(B.K.x + r0, x);
            stv(B.K.r + r0, r);
        }
        double acc[2] = {rho.value(), rr.value()}, tot[2];
        if (tile_reduce<2>(acc, B.part, B.ntiles, tile, T, S, tot) && threadIdx.x == 0) {
            KState &Q = *S;
            Q.iter += 1;
            Q.rr = tot[1];
            if (tot[1] < 0.81 * Q.best_rr) { Q.best_rr = tot[1]; Q.last_improve = Q.iter; }
            const double blowup = Q.stall > 0 ? 1e6 : 1e24;
            if (!isfinite(tot[0]) || !isfinite(tot[1]) || tot[1] > blowup * Q.rr0) Q.done = K_NONFINITE;
            else if (tot[1] <= Q.tol2) Q.done = K_CONVERGED;
            else if (tot[0] == 0.0 || Q.omega == 0.0) Q.done = K_BREAKDOWN;
            else if (Q.iter >= Q.maxit) Q.done = K_MAXIT;
            else if (Q.stall > 0 && Q.best_rr <= Q.stall_rr && Q.iter - Q.last_improve >= Q.stall) Q.done = K_STAGNATED;
            else {
                Q.beta = (tot[0] / Q.rho) * (Q.alpha / Q.omega);
                Q.rho = tot[0];
            }
        }
    }
}

template <typename V>
__global__ void __launch_bounds__(KRY_BLOCK) kb_p(KBatch<V> B) {
    constexpr int R = VecT<V>::R;
    KB_TILES(B) {
        const BTile T = B.tiles[tile];
        const KState *S = B.st + T.inst;
        if (inst_finished(S)) continue;
        const V beta = cvt<V>(S->beta), omega = cvt<V>(S->omega);
        KB_ROWS(T) {
            const Pack<V> r = ldv(B.K.r + r0), v = ldv(B.K.v + r0);
            Pack<V> p = ldv(B.K.p + r0);
#pragma unroll
            for (int j = 0; j < R; ++j) p.v[j] = r.v[j] + beta * (p.v[j] - omega * v.v[j]);
            stv(B.K.p + r0, p);
        }
    }
}

// per-instance sum over free rows of r^2 (tiles in the FP64 row layout, R = 2)
__global__ void __launch_bounds__(KRY_BLOCK) kb_norm2(int64_t ntiles, const BTile *tiles, KState *st, double *part,
                                                      const double *r, const uint8_t *dir, int64_t n, double *out) {
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const BTile T = tiles[tile];
        double acc[1] = {0.0};
        for (int64_t i = T.r_begin + threadIdx.x; i < T.r_end; i += KRY_BLOCK)
            if (i < n && !dir[i]) acc[0] += r[i] * r[i];
        double tot[1];
        if (tile_reduce<1>(acc, part, ntiles, tile, T, st + T.inst, tot) && threadIdx.x == 0) out[T.inst] = tot[0];
    }
}

// u -= lam[inst] x on the rows of instances with mask[inst] set
template <typename V>
__global__ void kb_update(int64_t n, const int32_t *slice_inst, const uint8_t *mask, const double *lam, double *u,
                          const V *x) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = slice_inst[i / SLICE];
    if (mask[b]) u[i] -= lam[b] * to_d(x[i]);
}

#undef KB_TILES
#undef KB_ROWS

}  // namespace egfem
