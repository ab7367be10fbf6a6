// egfem_cluster.cuh -- Jacobi-BiCGStab for one system small enough to live in the distributed
// shared memory of one thread-block cluster (up to 16 CTAs, one per SM).
//
// The grid-wide persistent solve (egfem_persist.cuh) pays, at every one of its five grid
// barriers per iteration, a chain of dependent L2 round trips (arrival atomic, last-block sum,
// fence, release, poll, scalar read): about 30 us per iteration however few rows there are.
// Here the cluster's CTAs own contiguous slice-aligned row ranges; the seven Krylov vectors of
// those rows stay in each CTA's shared memory for the whole solve; the SpMV gathers its
// neighbours' entries from the owning CTA's shared memory (mapa + ld.shared::cluster); and the
// hardware cluster barrier (barrier.cluster.arrive.release / wait.acquire) replaces the grid
// barrier.  Each reduction is two-level: the CTA's partial goes to its own shared memory, and
// after the barrier one warp of every CTA adds the cluster's partials in a fixed order, so
// every CTA computes bit-identical scalars and takes the same decisions -- every CTA executes
// the same sequence of barriers, and no thread ever waits on a flag another CTA sets.  The
// pointwise updates p = r + beta (p - omega v) and s = r - alpha v are formed inside the SpMV
// for the gathered neighbours, which leaves three barriers per iteration instead of five.
//
// The operator (the Jacobi-scaled Jacobian in SELL layout) is read-only during the solve and
// is read from global memory.  Arithmetic and stopping rules are those of pk_solve<double>.
#pragma once

#include "egfem_persist.cuh"

namespace egfem {

constexpr int PKC_BLOCK = 512;          // threads per CTA
constexpr int PKC_WARPS = PKC_BLOCK / 32;
constexpr int PKC_NVEC = 9;             // p and v (two buffers each), s, t, r, rh, x in shared memory
constexpr int PKC_MAX_CLUSTER = 16;     // non-portable cluster size (one GPC holds it)

enum { PV_P0 = 0, PV_P1, PV_V0, PV_V1, PV_S, PV_T, PV_R, PV_RH, PV_X };

struct PkcArgs {
    KVecs<double> K;        // operator, b (rhs) and x (solution out) in global memory
    KState *st;             // final state (written by rank 0)
    int64_t n_pad;          // rows (whole slices)
    int32_t rows_cta;       // rows per CTA (a multiple of SLICE); the last CTA may own fewer
    double rtol;
    int32_t maxit, stall;
};

__device__ __forceinline__ void pkc_cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pkc_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t pkc_nranks() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// a double in CTA `rank`'s shared memory at the offset of `p` in this CTA's
__device__ __forceinline__ double pkc_ld_remote(const double *p, uint32_t rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra));
    return v;
}

// Each warp's sums of NV per-thread values (fixed shuffle order) to buf[k * PKC_WARPS + warp].
template <int NV>
__device__ __forceinline__ void pkc_warp_partial(const double (&x)[NV], double *buf) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double v = warp_sum(x[k]);
        if (lane == 0) buf[k * PKC_WARPS + w] = v;
    }
}

// After a cluster barrier, warp 0 of every CTA: each lane adds its share of the cluster's warp
// partials (entry e = rank * PKC_WARPS + warp, lanes strided, e increasing) and the warp adds
// the lanes in a fixed shuffle order, so every CTA gets bit-identical sums; lane 0 applies
// update(S, tot) to the CTA's shared state and the closing __syncthreads publishes it.  (GB300
// issues about two FP64 operations per clock per SM: scalar work is done once per CTA by one
// warp, not recomputed by every thread.)
template <int NV, typename U>
__device__ __forceinline__ void pkc_reduce_update(const double *buf, uint32_t nranks, KState &S, U &&update) {
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x, ne = nranks * PKC_WARPS;
        double tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double acc = 0.0;
            for (uint32_t e = lane; e < ne; e += 32)
                acc += pkc_ld_remote(buf + k * PKC_WARPS + (e % PKC_WARPS), e / PKC_WARPS);
            tot[k] = warp_sum(acc);
        }
        if (lane == 0) update(S, tot);
    }
    __syncthreads();
}

// The three values (r_j, a_j, b_j) of column j, from this CTA's shared memory or the owner's
struct PkcCol {
    double r, a, b;
};

__device__ __forceinline__ PkcCol pkc_gather(const double *r, const double *va, const double *vb, int64_t col, int64_t base,
                                             int64_t rows_here, int64_t rc) {
    PkcCol c;
    if (col >= base && col < base + rows_here) {
        const int64_t o = col - base;
        c.r = r[o]; c.a = va[o]; c.b = vb[o];
    } else {
        const uint32_t q = uint32_t(col / rc);
        const int64_t o = col - int64_t(q) * rc;
        c.r = pkc_ld_remote(r + o, q); c.a = pkc_ld_remote(va + o, q); c.b = pkc_ld_remote(vb + o, q);
    }
    return c;
}

// y_g = sum_c A_gc z_c for the owned row g, where z_j = f(r_j, a_j, b_j) is formed from the
// stored vectors as it is gathered (z_g, the row's own value, is passed in).  f(r, a, b) is
// r + beta (a - omega b) for p (a = previous p, b = previous v) and r - alpha a for s (a = v);
// every CTA forms a neighbour's z from the same operands in the same order as its owner, so the
// products are those of the stored vector.
template <typename F>
__device__ __forceinline__ double pkc_spmv_row(const KVecs<double> &K, int64_t g, int64_t base, int64_t rows_here,
                                               int64_t rc, double zg, const double *r, const double *va,
                                               const double *vb, F &&f) {
    const SliceMeta M = K.meta[g / SLICE];
    const int lane = int(g % SLICE);
    double y = __ldg(K.A + M.col_base + lane) * zg;
#pragma unroll 4
    for (int c = 1; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const double a = __ldg(K.A + q);
        const int64_t col = M.off_base >= 0 ? g + __ldg(K.slice_off + M.off_base + c) : int64_t(__ldg(K.col_idx + q));
        const PkcCol z = pkc_gather(r, va, vb, col, base, rows_here, rc);
        y = fma(a, f(z.r, z.a, z.b), y);
    }
    return y;
}

#define PKC_ROWS for (int64_t l = threadIdx.x; l < rows_here; l += PKC_BLOCK)

// The solve: x = 0 start, BiCGStab until (r, r) <= rtol^2 (b, b), a breakdown, the iteration
// cap, divergence or (stall > 0) stagnation.  One cluster; grid = the cluster.
//
// Per iteration three phases, each ending with a reduction and a cluster barrier:
//   A: p = r + beta (p' - omega v') (own rows; neighbours' formed while gathered),
//      v = A p, (rh, v)                                     -> alpha
//   B: s = r - alpha v (likewise), t = A s, (t, s), (t, t)   -> omega
//   C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r) -> beta, convergence
// p and v alternate between two buffers: phase A reads the previous iteration's (p', v') of
// its neighbours while every CTA writes the new ones to the other buffer.  r is written only
// in phase C, which no CTA reads remotely; s never leaves its CTA.
__global__ void __launch_bounds__(PKC_BLOCK, 1) pkc_solve(PkcArgs P) {
    extern __shared__ double sv[];              // [PKC_NVEC][rows_cta]
    __shared__ double red_0[PKC_WARPS], red_a[PKC_WARPS], red_o[2 * PKC_WARPS], red_r[2 * PKC_WARPS];
    __shared__ KState S;                        // this CTA's copy of the state (warp 0 writes it)
    const uint32_t rank = pkc_rank(), nranks = pkc_nranks();
    const int64_t RC = P.rows_cta;
    const int64_t base = int64_t(rank) * RC;
    const int64_t rows_here = base >= P.n_pad ? 0 : (P.n_pad - base < RC ? P.n_pad - base : RC);
    double *s = sv + PV_S * RC, *t = sv + PV_T * RC, *r = sv + PV_R * RC, *rh = sv + PV_RH * RC, *x = sv + PV_X * RC;
    const KVecs<double> &K = P.K;

    // setup: x = p' = v' = 0, r = rh = b, (b, b)
    double acc0 = 0.0;
    PKC_ROWS {
        const double b = __ldg(K.b + base + l);
        x[l] = 0.0; s[l] = 0.0; t[l] = 0.0;
        sv[PV_P0 * RC + l] = 0.0; sv[PV_P1 * RC + l] = 0.0; sv[PV_V0 * RC + l] = 0.0; sv[PV_V1 * RC + l] = 0.0;
        r[l] = b; rh[l] = b;
        acc0 = fma(b, b, acc0);
    }
    {
        const double a1[1] = {acc0};
        pkc_warp_partial<1>(a1, red_0);
    }
    pkc_cluster_barrier();   // also: every CTA of the cluster has started before any remote access
    pkc_reduce_update<1>(red_0, nranks, S, [&](KState &Q, const double *tot) {
        const double bb = tot[0];
        Q.iter = 0; Q.last_improve = 0; Q.maxit = P.maxit; Q.stall = P.stall; Q.ticket = 0u;
        Q.alpha = 1.0; Q.omega = 1.0; Q.beta = 0.0; Q.scratch[0] = Q.scratch[1] = 0.0;
        Q.rho = Q.rr = Q.rr0 = Q.best_rr = bb;
        Q.tol2 = P.rtol * P.rtol * bb;
        Q.stall_rr = 4e-6 * bb;
        Q.done = (bb == 0.0) ? K_CONVERGED : (!isfinite(bb) ? K_NONFINITE : (P.maxit <= 0 ? K_MAXIT : K_RUNNING));
    });

    int cur = 0;   // buffer of the p, v being formed; 1 - cur holds the previous ones
    while (S.done == K_RUNNING) {
        double *p = sv + (PV_P0 + cur) * RC, *v = sv + (PV_V0 + cur) * RC;
        const double *pp = sv + (PV_P0 + 1 - cur) * RC, *vp = sv + (PV_V0 + 1 - cur) * RC;
        const double be = S.beta, om0 = S.omega;
        auto fp = [be, om0](double rj, double pj, double vj) { return rj + be * (pj - om0 * vj); };

        // A: p, v = A p, (rh, v)
        double acc = 0.0;
        PKC_ROWS {
            const double pg = fp(r[l], pp[l], vp[l]);
            p[l] = pg;
            const double y = pkc_spmv_row(K, base + l, base, rows_here, RC, pg, r, pp, vp, fp);
            v[l] = y;
            acc = fma(rh[l], y, acc);
        }
        {
            const double a1[1] = {acc};
            pkc_warp_partial<1>(a1, red_a);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<1>(red_a, nranks, S, [&](KState &Q, const double *tot) {
            if (tot[0] == 0.0 || !isfinite(tot[0])) Q.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
            else Q.alpha = Q.rho / tot[0];
        });
        if (S.done != K_RUNNING) break;

        // B: s = r - alpha v, t = A s, (t, s), (t, t)
        const double al = S.alpha;
        auto fs = [al](double rj, double vj, double) { return rj - al * vj; };
        double ts = 0.0, tt = 0.0;
        PKC_ROWS {
            const double sg = fs(r[l], v[l], 0.0);
            s[l] = sg;
            const double y = pkc_spmv_row(K, base + l, base, rows_here, RC, sg, r, v, v, fs);
            t[l] = y;
            ts = fma(y, sg, ts);
            tt = fma(y, y, tt);
        }
        {
            const double a2[2] = {ts, tt};
            pkc_warp_partial<2>(a2, red_o);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<2>(red_o, nranks, S, [&](KState &Q, const double *tot) {
            if (!isfinite(tot[0]) || !isfinite(tot[1])) Q.done = K_NONFINITE;
            else Q.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
        });
        if (S.done != K_RUNNING) break;

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        const double om = S.omega;
        double rr1 = 0.0, rr2 = 0.0;
        PKC_ROWS {
            x[l] = x[l] + (al * p[l] + om * s[l]);
            const double rn = s[l] - om * t[l];
            r[l] = rn;
            rr1 = fma(rh[l], rn, rr1);
            rr2 = fma(rn, rn, rr2);
        }
        {
            const double a2[2] = {rr1, rr2};
            pkc_warp_partial<2>(a2, red_r);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<2>(red_r, nranks, S, [&](KState &Q, const double *tot) {
            pk_after_c(Q, tot[0], tot[1], P.maxit, P.stall);
        });
        cur = 1 - cur;
    }

    // results: x of the owned rows, the state from rank 0; the final barrier keeps every
    // CTA's shared memory alive until the last remote read of the partials above is done
    PKC_ROWS K.x[base + l] = x[l];
    if (rank == 0 && threadIdx.x == 0) *P.st = S;
    pkc_cluster_barrier();
}

#undef PKC_ROWS

}  // namespace egfem
