// egfem_cluster.cuh -- Jacobi-BiCGStab for one system small enough to live in the distributed
// shared memory of one thread-block cluster (up to 16 CTAs, one per SM).
//
// The grid-wide persistent solve (egfem_persist.cuh) pays, at every one of its five grid
// barriers per iteration, a chain of dependent L2 round trips (arrival atomic, wait, and at the
// summing barriers one round of partial loads): about 19 us per iteration however few rows
// there are.
// Here the cluster's CTAs own contiguous slice-aligned row ranges; the seven Krylov vectors of
// those rows stay in each CTA's shared memory for the whole solve; the SpMV gathers its
// neighbours' entries from the owning CTA's shared memory (mapa + ld.shared::cluster); and the
// hardware cluster barrier (barrier.cluster.arrive.release / wait.acquire) replaces the grid
// barrier.  Each reduction is two-level: the CTA's partial goes to its own shared memory, and
// after the barrier one warp of every CTA adds the cluster's partials in a fixed order, so
// every CTA computes bit-identical scalars and takes the same decisions -- every CTA executes
// the same sequence of barriers, and no thread ever waits on a flag another CTA sets.
//
// GB300 issues about two FP64 operations per clock per SM, so at these sizes the FP64
// instruction count, not memory or the barriers (about 0.3 us each), sets the time: a
// reduction stores each thread's partial to shared memory and one warp adds only the
// partials of threads that own rows; the pointwise vector updates stay separate phases
// (forming p and s inside the SpMV for each gathered neighbour would save two barriers but
// triple the SpMV's FP64 work).
//
// V = double (the FP64 path) or df64 (the mixed path: double-float vectors, the FP32 operator
// applied in difference form with its row sum in column 0, compensated as in pk_solve1).
//
// The operator (the Jacobi-scaled Jacobian in SELL layout) is read-only during the solve.
// When it fits beside the vectors, each CTA copies its rows of it to shared memory at the
// start (ELL values and column codes naming the owning CTA and offset), and the iterations
// touch no global memory; otherwise it is read from global memory.  Arithmetic and stopping
// rules are those of pk_solve1<double>.
#pragma once

#include "egfem_persist.cuh"

namespace egfem {

constexpr int PKC_BLOCK = 512;          // threads per CTA
constexpr int PKC_NVEC = 7;             // p, v, s, t, r, rh, x in shared memory
constexpr int PKC_MAX_CLUSTER = 16;     // non-portable cluster size (one GPC holds it)

enum { PV_P = 0, PV_V, PV_S, PV_T, PV_R, PV_RH, PV_X };

template <typename V>
struct PkcArgs {
    KVecs<V> K;             // operator, b (rhs) and x (solution out) in global memory
    KState *st;             // final state (written by rank 0)
    int64_t n_pad;          // rows (whole slices)
    int32_t rows_cta;       // rows per CTA (a multiple of SLICE); the last CTA may own fewer
    int32_t op_cols;        // > 0: the operator is copied to shared memory as op_cols ELL columns
    double rtol;
    int32_t maxit, stall;
    const uint8_t *active;  // nullable: the solve does nothing when *active == 0 (graph Newton loop)
    const double *rtol_ptr; // nullable: the tolerance read from device memory instead of rtol
};

// Shared-memory bytes per row: the Krylov vectors, and with the operator copy its ELL values,
// column codes (owning rank << 16 | offset in that CTA) and the row's column count.
template <typename V>
__host__ __device__ constexpr int64_t pkc_row_bytes(int op_cols) {
    return int64_t(PKC_NVEC) * int64_t(sizeof(V)) +
           (op_cols > 0 ? int64_t(op_cols) * int64_t(sizeof(typename VecT<V>::mat) + 4) + 1 : 0);
}

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

// Reduction, first half (before the cluster barrier): every thread stores its NV partials to
// th[k][tid]; after a __syncthreads warp 0 adds those of the nact threads that own rows (lane j
// takes tid = j, j + 32, ... in order, then a fixed shuffle tree) and lane 0 stores the CTA's
// sums to cta[k].
template <int NV>
__device__ __forceinline__ void pkc_cta_partial(const double (&x)[NV], double (*th)[PKC_BLOCK], int nact, double *cta) {
#pragma unroll
    for (int k = 0; k < NV; ++k) th[k][threadIdx.x] = x[k];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int j = threadIdx.x; j < nact; j += 32) a += th[k][j];
            a = warp_sum(a);
            if (threadIdx.x == 0) cta[k] = a;
        }
    }
}

// Second half (after the cluster barrier): warp 0 of every CTA loads the cluster's CTA sums
// (lane q from CTA q) and adds them in a fixed shuffle order, so every CTA gets bit-identical
// totals; lane 0 applies update(S, tot) to the CTA's shared state and the closing
// __syncthreads publishes it to the CTA.
template <int NV, typename U>
__device__ __forceinline__ void pkc_reduce_update(const double *cta, uint32_t nranks, KState &S, U &&update) {
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        double tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = warp_sum(lane < nranks ? pkc_ld_remote(cta + k, lane) : 0.0);
        if (lane == 0) update(S, tot);
    }
    __syncthreads();
}

// a df64 in CTA `rank`'s shared memory (its two words)
__device__ __forceinline__ df64 pkc_ld_remote(const df64 *p, uint32_t rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    df64 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.hi), "=f"(v.lo) : "r"(ra));
    return v;
}

// Row accumulator of the SpMV: FP64 y = a0 x_g + sum a_c x_c, or for df64 the difference form
// y = s_g x_g + sum a_c (x_c - x_g) (column 0 holds the row sum s_g) in a compensated pair.
template <typename V> struct PkcRow;
template <> struct PkcRow<double> {
    double y, xg;
    // column 0 is the Jacobi-scaled diagonal, stored as exactly 1: y starts at x (= a0 x)
    __device__ __forceinline__ PkcRow(double, double x) : y(x), xg(x) {}
    __device__ __forceinline__ void add(double a, double xc) { y = fma(a, xc, y); }
    __device__ __forceinline__ double value() const { return y; }
};
template <> struct PkcRow<df64> {
    float hi, lo;
    df64 xg;
    __device__ __forceinline__ PkcRow(float a0, df64 x) : xg(x) {
        hi = __fmul_rn(a0, x.hi);
        lo = __fmaf_rn(a0, x.lo, __fmaf_rn(a0, x.hi, -hi));
    }
    __device__ __forceinline__ void add(float a, df64 xc) { df_acc_diff(hi, lo, a, xc, xg); }
    __device__ __forceinline__ df64 value() const { return df_fast_two_sum(hi, lo); }
};

// y_g = (A x)_g for the owned row g; x is vector `vec` of the cluster, xg its value at g
template <typename V>
__device__ __forceinline__ V pkc_spmv_row(const KVecs<V> &K, const V *xv, int64_t g, int64_t base, int64_t rows_here,
                                          int64_t rc, V xg) {
    const SliceMeta M = K.meta[g / SLICE];
    const int lane = int(g % SLICE);
    PkcRow<V> y(__ldg(K.A + M.col_base + lane), xg);
#pragma unroll 4
    for (int c = 1; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const auto a = __ldg(K.A + q);
        const int64_t col = M.off_base >= 0 ? g + __ldg(K.slice_off + M.off_base + c) : int64_t(__ldg(K.col_idx + q));
        V xc;
        if (col >= base && col < base + rows_here) {
            xc = xv[col - base];
        } else {
            const uint32_t o = uint32_t(col / rc);
            xc = pkc_ld_remote(xv + (col - int64_t(o) * rc), o);
        }
        y.add(a, xc);
    }
    return y.value();
}

// the same product from the shared-memory copy of the operator (row l of this CTA)
template <typename V, typename M_t>
__device__ __forceinline__ V pkc_spmv_row_smem(const M_t *opv, const uint32_t *opc, const uint8_t *opn, const V *xv,
                                               int64_t l, int64_t rc, uint32_t rank, V xg) {
    PkcRow<V> y(opv[l], xg);
    const int nc = opn[l];
#pragma unroll 4
    for (int c = 1; c < nc; ++c) {
        const uint32_t code = opc[int64_t(c) * rc + l];
        const uint32_t o = code >> 16, off = code & 0xFFFFu;
        const V xc = o == rank ? xv[off] : pkc_ld_remote(xv + off, o);
        y.add(opv[int64_t(c) * rc + l], xc);
    }
    return y.value();
}

#define PKC_ROWS for (int64_t l = threadIdx.x; l < rows_here; l += PKC_BLOCK)

// The solve: x = 0 start, BiCGStab until (r, r) <= rtol^2 (b, b), a breakdown, the iteration
// cap, divergence or (stall > 0) stagnation.  One cluster; grid = the cluster.  The phases and
// their order are those of pk_solve1<double>: A v = A p | B1 s = r - alpha v | B2 t = A s |
// C x, r | D p, with a cluster barrier after each.
template <typename V>
__global__ void __launch_bounds__(PKC_BLOCK, 1) pkc_solve(PkcArgs<V> P) {
    using Op = PkOps<V>;
    using M_t = typename VecT<V>::mat;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sv = reinterpret_cast<V *>(smem_raw);     // [PKC_NVEC][rows_cta]
    __shared__ double th[2][PKC_BLOCK];         // per-thread partials of the reduction in progress
    __shared__ double cta_0[1], cta_a[1], cta_o[2], cta_r[2];
    __shared__ KState S;                        // this CTA's copy of the state (warp 0 writes it)
    // an inactive solve (graph Newton loop, nothing to do) returns at once in every CTA
    if (P.active && !*P.active) return;
    const double rtol = P.rtol_ptr ? *P.rtol_ptr : P.rtol;
    const uint32_t rank = pkc_rank(), nranks = pkc_nranks();
    const int64_t RC = P.rows_cta;
    const int64_t base = int64_t(rank) * RC;
    const int64_t rows_here = base >= P.n_pad ? 0 : (P.n_pad - base < RC ? P.n_pad - base : RC);
    const int nact = int(rows_here < PKC_BLOCK ? rows_here : PKC_BLOCK);   // threads that own rows
    V *p = sv + PV_P * RC, *v = sv + PV_V * RC, *s = sv + PV_S * RC, *t = sv + PV_T * RC;
    V *r = sv + PV_R * RC, *rh = sv + PV_RH * RC, *x = sv + PV_X * RC;
    const KVecs<V> &K = P.K;
    // the operator copy (when P.op_cols > 0): values [op_cols][RC], codes [op_cols][RC], counts [RC]
    const int MC = P.op_cols;
    M_t *opv = reinterpret_cast<M_t *>(sv + PKC_NVEC * RC);
    uint32_t *opc = reinterpret_cast<uint32_t *>(opv + int64_t(MC) * RC);
    uint8_t *opn = reinterpret_cast<uint8_t *>(opc + int64_t(MC) * RC);
    if (MC > 0) {
        PKC_ROWS {
            const int64_t g = base + l;
            const SliceMeta M = K.meta[g / SLICE];
            const int lane = int(g % SLICE);
            opn[l] = uint8_t(M.ncol < MC ? M.ncol : MC);
            for (int c = 0; c < MC; ++c) {
                M_t a = M_t(0);
                uint32_t code = (rank << 16) | uint32_t(l);
                if (c < M.ncol) {
                    const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
                    a = __ldg(K.A + q);
                    const int64_t col = M.off_base >= 0 ? g + __ldg(K.slice_off + M.off_base + c) : int64_t(__ldg(K.col_idx + q));
                    const uint32_t o = uint32_t(col / RC);
                    code = (o << 16) | uint32_t(col - int64_t(o) * RC);
                }
                opv[int64_t(c) * RC + l] = a;
                opc[int64_t(c) * RC + l] = code;
            }
        }
    }
    auto spmv = [&](const V *xv, int64_t l, V xg) -> V {
        return MC > 0 ? pkc_spmv_row_smem<V, M_t>(opv, opc, opn, xv, l, RC, rank, xg)
                      : pkc_spmv_row<V>(K, xv, base + l, base, rows_here, RC, xg);
    };

    // setup: x = v = 0, r = rh = p = b, (b, b)
    DotAcc<V> acc0;
    const V zero = cvt<V>(0.0);
    PKC_ROWS {
        const V b = K.b[base + l];
        x[l] = zero; v[l] = zero; s[l] = zero; t[l] = zero;
        r[l] = b; rh[l] = b; p[l] = b;
        acc0.add(b, b);
    }
    {
        const double a1[1] = {acc0.value()};
        pkc_cta_partial<1>(a1, th, nact, cta_0);
    }
    pkc_cluster_barrier();   // also: every CTA of the cluster has started before any remote access
    pkc_reduce_update<1>(cta_0, nranks, S, [&](KState &Q, const double *tot) {
        const double bb = tot[0];
        Q.iter = 0; Q.last_improve = 0; Q.maxit = P.maxit; Q.stall = P.stall; Q.ticket = 0u;
        Q.alpha = 1.0; Q.omega = 1.0; Q.beta = 0.0; Q.scratch[0] = Q.scratch[1] = 0.0;
        Q.rho = Q.rr = Q.rr0 = Q.best_rr = bb;
        Q.tol2 = rtol * rtol * bb;
        Q.stall_rr = 4e-6 * bb;
        Q.done = (bb == 0.0) ? K_CONVERGED : (!isfinite(bb) ? K_NONFINITE : (P.maxit <= 0 ? K_MAXIT : K_RUNNING));
    });

    while (S.done == K_RUNNING) {
        // A: v = A p, (rh, v)
        DotAcc<V> acc;
        PKC_ROWS {
            const V y = spmv(p, l, p[l]);
            v[l] = y;
            acc.add(rh[l], y);
        }
        {
            const double a1[1] = {acc.value()};
            pkc_cta_partial<1>(a1, th, nact, cta_a);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<1>(cta_a, nranks, S, [&](KState &Q, const double *tot) {
            if (tot[0] == 0.0 || !isfinite(tot[0])) Q.done = isfinite(tot[0]) ? K_BREAKDOWN : K_NONFINITE;
            else Q.alpha = Q.rho / tot[0];
        });
        if (S.done != K_RUNNING) break;

        // B1: s = r - alpha v (every CTA's s is complete before the SpMV gathers it)
        const V al = cvt<V>(S.alpha);
        PKC_ROWS s[l] = Op::sub(r[l], al * v[l]);
        pkc_cluster_barrier();

        // B2: t = A s, (t, s), (t, t)
        DotAcc<V> ts, tt;
        PKC_ROWS {
            const V sl = s[l];
            const V y = spmv(s, l, sl);
            t[l] = y;
            ts.add(y, sl);
            tt.add(y, y);
        }
        {
            const double a2[2] = {ts.value(), tt.value()};
            pkc_cta_partial<2>(a2, th, nact, cta_o);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<2>(cta_o, nranks, S, [&](KState &Q, const double *tot) {
            if (!isfinite(tot[0]) || !isfinite(tot[1])) Q.done = K_NONFINITE;
            else Q.omega = tot[1] == 0.0 ? 0.0 : tot[0] / tot[1];
        });
        if (S.done != K_RUNNING) break;

        // C: x += alpha p + omega s, r = s - omega t, (rh, r), (r, r)
        const V om = cvt<V>(S.omega);
        DotAcc<V> rr1, rr2;
        PKC_ROWS {
            x[l] = Op::add(x[l], Op::add(al * p[l], om * s[l]));
            const V rn = Op::sub(s[l], om * t[l]);
            r[l] = rn;
            rr1.add(rh[l], rn);
            rr2.add(rn, rn);
        }
        {
            const double a2[2] = {rr1.value(), rr2.value()};
            pkc_cta_partial<2>(a2, th, nact, cta_r);
        }
        pkc_cluster_barrier();
        pkc_reduce_update<2>(cta_r, nranks, S, [&](KState &Q, const double *tot) {
            pk_after_c(Q, tot[0], tot[1], P.maxit, P.stall);
        });
        if (S.done != K_RUNNING) break;

        // D: p = r + beta (p - omega v)
        const V be = cvt<V>(S.beta);
        PKC_ROWS p[l] = Op::add(r[l], be * Op::sub(p[l], om * v[l]));
        pkc_cluster_barrier();
    }

    // results: x of the owned rows, the state from rank 0; the final barrier keeps every
    // CTA's shared memory alive until the last remote read of the partials above is done
    PKC_ROWS K.x[base + l] = x[l];
    if (rank == 0 && threadIdx.x == 0) *P.st = S;
    pkc_cluster_barrier();
}

#undef PKC_ROWS

}  // namespace egfem
