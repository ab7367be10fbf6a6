// egfem_kernels.cuh -- device code of the EGFEM Newton hot path (sm_103a).
//
// Layout (built by egfem_build.cpp): rows are grouped in slices of 32 consecutive rows;
// every per-row list (local columns, leaves, fibres, reaction entries) is stored
// column-interleaved within its slice (entry j of row r at base + 32 j + r), so one
// thread per row reads coalesced 32-wide words.  The tensor is row-segmented CSF:
//     row i -> fibres (one per W node m with a nonzero T_imk) -> leaves (k != i, T_imk)
// with the diagonal T_imi = -sum_{k != i} T_imk kept once per fibre.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "egfem_df64.cuh"
#include <climits>

#include "egfem_internal.h"

namespace egfem {

constexpr int CSF_BLOCK = 128;
// Threads per block of the row kernels for MAXC local columns: their per-thread shared arrays
// (up to 16 B per column) keep to 32 KB, below the 48 KB static limit.
template <int MAXC> __host__ __device__ constexpr int csf_block() { return MAXC <= 16 ? CSF_BLOCK : 2048 / MAXC; }
// Resident blocks per SM that the tensor-action kernels are compiled for.  Their per-row fibre
// chains wait on gathers (the W node's nodal values at each fibre start), so resident warps hide
// that latency, but each needs registers for the fibre loaded ahead: for up to 8 local columns
// (2D P1 rows, 16 KB of shared memory per block) ten blocks (48 registers).  Measured at 1024^2
// (nodal pass + kernel, FP64 / mixed): the compiler's choice (56-63 registers, nine blocks, no
// fibre ahead) 355 / 309 us; twelve blocks (40 registers) 340 / 301; ten blocks with the fibre
// ahead 328 / 273; twelve with it 350 / 303.  Wider rows keep the compiler's choice.
template <int MAXC> __host__ __device__ constexpr int csf_min_blocks() { return MAXC <= 8 ? 10 : 1; }

struct CsfArgs {
    int64_t n_rows;
    const SliceMeta *meta;
    const int32_t *col_idx, *col_slot;
    const double *leaf_val;
    const uint8_t *leaf_col;
    const uint32_t *fib_info;
    const double *fib_tdiag;
    const int32_t *fib_m;
    const double *rx_val;
    const uint32_t *rx_info;
    const uint8_t *dir;
    Nonlin nl;
    const double *u;       // [n_rows] input
    const double *d;       // [n_rows] load (Dirichlet rows: boundary values); may be null for J only
    double *r;             // residual out (nullable)
    double *jcsr;          // Jacobian values in CSR order (nullable)
    double *a64;           // D J in SELL order, FP64 (nullable)
    float *a32;            // D J in SELL order, FP32 (nullable)
    double *q64;           // D r (nullable)
    float *q32;            // D r (nullable)
    double *jsell;         // unscaled J in SELL order (nullable)
    double *dinv;          // 1 / J_ii (nullable)
    const int32_t *rx_m;         // W_c index of each reaction entry
    // nodal values of the nonlinearities, evaluated once per W node by wnode_kernel
    // (nullable: then every fibre / reaction entry evaluates g itself)
    const double *wa_val, *wa_gp;   // a_m = kappa_m + g_a((Pi u)_m), g_a'((Pi u)_m)
    const double *wc_val, *wc_gp;   // c_m = g_c((Pi_c u)_m),         g_c'((Pi_c u)_m)
    const float *wa_val32, *wa_gp32;   // FP32 copies of a_m, g_a' (csf_mixed_kernel)
    const float *leaf_val32;           // FP32 copy of leaf_val (csf_mixed_kernel)
    const int32_t *slice_inst;   // batch: instance of each slice (nullable)
    const uint8_t *inst_mask;    // batch: rows of instances with mask 0 are skipped (nullable)
    WShare ws;                   // one tensor for a batch of one mesh (ws.k > 0), else ws.k = 0
    int32_t *status;       // error word (singular diagonal)
};

__device__ __forceinline__ void g_eval(int32_t kind, int32_t p, double scale, double s, double &g, double &gp) {
    if (kind == EGFEM_G_POW) {
        double sp = 1.0;                      // s^(p-1)
        for (int32_t k = 1; k < p; ++k) sp *= s;
        g = scale * sp * s;
        gp = scale * double(p) * sp;
    } else if (kind == EGFEM_G_EXP) {
        g = scale * exp(s);
        gp = g;
    } else {
        g = 0.0;
        gp = 0.0;
    }
}

// (Pi u)_m = u_i + sum_t w_t (u_{c_t} - u_i), the weights w_t summing to one (Sec. 3.2).
__device__ __forceinline__ double interp_du(uint32_t info, const double *du, int stride) {
    const uint32_t kind = (info >> 24) & 0xF;
    const double d0 = du[(info & 0xFF) * stride];
    if (kind == W_VERTEX) return d0;
    const double d1 = du[((info >> 8) & 0xFF) * stride];
    if (kind == W_MID) return 0.5 * (d0 + d1);
    if (kind == W_THIRD) return (2.0 * d0 + d1) * (1.0 / 3.0);
    const double d2 = du[((info >> 16) & 0xFF) * stride];
    return (d0 + d1 + d2) * (1.0 / 3.0);
}

// The row of this thread, and its instance in a batch of one shared mesh (else 0): with a
// shared tensor the blocks take the instances in turn for each range of local rows, so the
// instances that read the same part of the tensor do so close together (from L2).  -1 past the
// end.
template <int BLK>
__device__ __forceinline__ int64_t csf_row(const CsfArgs &A, int32_t &inst) {
    if (A.ws.k > 0) {
        const int32_t lb = int32_t(blockIdx.x) / A.ws.k, b = int32_t(blockIdx.x) % A.ws.k;
        const int64_t lr = int64_t(lb) * BLK + threadIdx.x;
        inst = b;
        return lr < A.ws.rows ? int64_t(b) * A.ws.rows + lr : -1;
    }
    inst = 0;
    return int64_t(blockIdx.x) * BLK + threadIdx.x;
}

// The stride of a node kind, chosen with selects (an indexed read of a kernel argument would
// copy the argument to local memory)
__device__ __forceinline__ int64_t ws_stride(const int64_t (&st)[5], uint32_t info) {
    const uint32_t w = (info >> 24) & 0xF;
    return w == W_VERTEX ? st[W_VERTEX] : w == W_MID ? st[W_MID] : w == W_THIRD ? st[W_THIRD] : w == W_FACE ? st[W_FACE] : 0;
}

// W index of a fibre's node (coefficient space) or a reaction entry's node, for the row's instance
__device__ __forceinline__ int64_t wa_index(const CsfArgs &A, int32_t m, uint32_t info, int32_t inst) {
    return A.ws.k > 0 ? int64_t(m) + ws_stride(A.ws.a, info) * int64_t(inst) : int64_t(m);
}
__device__ __forceinline__ int64_t wc_index(const CsfArgs &A, int32_t m, uint32_t info, int32_t inst) {
    return A.ws.k > 0 ? int64_t(m) + ws_stride(A.ws.c, info) * int64_t(inst) : int64_t(m);
}

// J_{i, c_t} += e * w_t  (the Pi_ml factor of the eliminated Jacobian, Sec. 4)
__device__ __forceinline__ void scatter_pi(uint32_t info, double e, double *J, int stride) {
    const uint32_t kind = (info >> 24) & 0xF;
    const uint32_t c0 = info & 0xFF, c1 = (info >> 8) & 0xFF, c2 = (info >> 16) & 0xFF;
    if (kind == W_VERTEX) { J[c0 * stride] += e; return; }
    // 0.5 e is exact, so the FMA adds the same value as h = 0.5 e, J += h, in one FP64 operation
    if (kind == W_MID) { J[c0 * stride] = fma(0.5, e, J[c0 * stride]); J[c1 * stride] = fma(0.5, e, J[c1 * stride]); return; }
    if (kind == W_THIRD) { const double h = e * (1.0 / 3.0); J[c0 * stride] += 2.0 * h; J[c1 * stride] += h; return; }
    if (kind == W_FACE) { const double h = e * (1.0 / 3.0); J[c0 * stride] += h; J[c1 * stride] += h; J[c2 * stride] += h; }
}

// FP32 variant of scatter_pi
__device__ __forceinline__ void scatter_pi32(uint32_t info, float e, float *J, int stride) {
    const uint32_t kind = (info >> 24) & 0xF;
    const uint32_t c0 = info & 0xFF, c1 = (info >> 8) & 0xFF, c2 = (info >> 16) & 0xFF;
    if (kind == W_VERTEX) { J[c0 * stride] += e; return; }
    if (kind == W_MID) { const float h = 0.5f * e; J[c0 * stride] += h; J[c1 * stride] += h; return; }
    if (kind == W_THIRD) { const float h = e * (1.0f / 3.0f); J[c0 * stride] += 2.0f * h; J[c1 * stride] += h; return; }
    if (kind == W_FACE) { const float h = e * (1.0f / 3.0f); J[c0 * stride] += h; J[c1 * stride] += h; J[c2 * stride] += h; }
}

// double-float variant of scatter_pi: J_{i, c_t} += e * w_t with the weights in double-float
__device__ __forceinline__ void scatter_pi_df(uint32_t info, df64 e, df64 *J, int stride) {
    const uint32_t kind = (info >> 24) & 0xF;
    const uint32_t c0 = info & 0xFF, c1 = (info >> 8) & 0xFF, c2 = (info >> 16) & 0xFF;
    if (kind == W_VERTEX) { J[c0 * stride] = df_acc(J[c0 * stride], e); return; }
    if (kind == W_MID) {
        const df64 h = {__fmul_rn(0.5f, e.hi), __fmul_rn(0.5f, e.lo)};   // exact
        J[c0 * stride] = df_acc(J[c0 * stride], h);
        J[c1 * stride] = df_acc(J[c1 * stride], h);
        return;
    }
    // 1/3 as a float pair (0x3eaaaaab and the rounded remainder), accurate to about 2^-48
    const df64 h = df_mul(e, df64{0.333333343f, -9.93410748e-09f});
    if (kind == W_THIRD) {
        J[c0 * stride] = df_acc(J[c0 * stride], df64{__fmul_rn(2.0f, h.hi), __fmul_rn(2.0f, h.lo)});
        J[c1 * stride] = df_acc(J[c1 * stride], h);
        return;
    }
    if (kind == W_FACE) {
        J[c0 * stride] = df_acc(J[c0 * stride], h);
        J[c1 * stride] = df_acc(J[c1 * stride], h);
        J[c2 * stride] = df_acc(J[c2 * stride], h);
    }
}

// Fused pointwise nonlinearity + residual + Jacobian fill (one thread per row).
// MAXC bounds the local columns of a row; du and J live in shared memory, one column
// of csf_block<MAXC>() entries per local column.
//
// JDF: the Jacobian is accumulated in double-float on the FP32 pipe (J1 = T .2 a per leaf, the
// Pi scatter of D g' per fibre, T_ii a per fibre), from exact splits of the FP64 values
// (split_dbl), and rounded to FP64 once per entry.  The residual, D = T .3 u and everything
// written from them stay FP64.  GB300 retires about two FP64 operations per SM and clock, and
// this kernel is bound by that pipe: the variant takes about a third of its FP64 operations off
// it.  Its entries agree with the FP64 accumulation to about 1e-14 relative; it serves the
// Newton steps' operator (the Jacobian only steers the Newton direction, the residual is exact
// FP64), while egfem_jacobian and the adjoint use the FP64 accumulation.
template <int MAXC, bool JDF>
__global__ void __launch_bounds__(csf_block<MAXC>(), csf_min_blocks<MAXC>()) csf_fused_kernel(CsfArgs A) {
    constexpr int BLK = csf_block<MAXC>();
    __shared__ double s_du[MAXC * BLK];
    __shared__ double s_J[MAXC * BLK];   // FP64 entries, or double-float pairs (JDF)
    const int tid = threadIdx.x;
    int32_t inst;
    const int64_t row = csf_row<BLK>(A, inst);
    if (row < 0 || row >= A.n_rows) return;
    const int64_t sl = row / SLICE;
    const int lane = int(row % SLICE);
    if (A.inst_mask && !A.inst_mask[A.slice_inst[sl]]) return;
    const SliceMeta M = A.meta[sl];
    const double ui = A.u[row];
    const double di = A.d ? A.d[row] : 0.0;
    double *du = s_du + tid, *J = s_J + tid;
    if (A.dir[row]) {
        if (A.r) A.r[row] = ui - di;
        if (A.q64) A.q64[row] = ui - di;
        if (A.q32) A.q32[row] = float(ui - di);
        if (A.dinv) A.dinv[row] = 1.0;
        for (int c = 0; c < M.ncol; ++c) {
            const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
            const double v = (c == 0) ? 1.0 : 0.0;
            if (A.a64) A.a64[q] = v;
            if (A.a32) A.a32[q] = float(v);
            if (A.jcsr && c == 0) A.jcsr[A.col_slot[q]] = 1.0;
            if (A.jsell) A.jsell[q] = v;
        }
        return;
    }
    df64 *Jd = reinterpret_cast<df64 *>(s_J) + tid;
    for (int c = 0; c < M.ncol; ++c) {
        const int32_t g = A.col_idx[M.col_base + int64_t(c) * SLICE + lane];
        du[c * BLK] = A.u[g] - ui;
        if constexpr (JDF) Jd[c * BLK] = df64{0.f, 0.f};
        else J[c * BLK] = 0.0;
    }
    const Nonlin nl = A.nl;
    double r = 0.0, j1d = 0.0, D = 0.0, a = 0.0, gp = 0.0;
    df64 a_df = {0.f, 0.f}, j1d_df = {0.f, 0.f};
    uint32_t info = 0;
    bool j2 = false;
    int f = -1;
    // the next fibre's info and W index are loaded one fibre ahead, so a fibre start waits for one
    // gather (the W node's nodal values) rather than for the index and then the gather
    uint32_t nx_info = 0;
    int32_t nx_m = 0;
    if (M.nfib > 0) { nx_info = __ldg(A.fib_info + M.fib_base + lane); nx_m = __ldg(A.fib_m + M.fib_base + lane); }
    // tensor data are read-only (non-coherent loads); unrolling lets the next leaves' loads
    // issue ahead of this leaf's arithmetic
#pragma unroll 4
    for (int j = 0; j < M.nleaf; ++j) {
        const int64_t q = M.leaf_base + int64_t(j) * SLICE + lane;
        const uint8_t lc = __ldg(A.leaf_col + q);
        const double T = __ldg(A.leaf_val + q);
        if (lc & LEAF_FIBRE_START) {
            if (f >= 0) {
                r += a * D;
                if (j2) {
                    if constexpr (JDF) scatter_pi_df(info, split_dbl(D * gp, 0), Jd, BLK);
                    else scatter_pi(info, D * gp, J, BLK);
                }
            }
            ++f;
            const int64_t fq = M.fib_base + int64_t(f) * SLICE + lane;
            info = nx_info;
            const int32_t mf = nx_m;
            const double td = __ldg(A.fib_tdiag + fq);
            if (f + 1 < M.nfib) { nx_info = __ldg(A.fib_info + fq + SLICE); nx_m = __ldg(A.fib_m + fq + SLICE); }
            // the J2 scatter is tested on integers (an FP64 compare would take an FP64 slot)
            j2 = !nl.picard && ((info >> 24) & 0xF) != W_CONST;
            if (((info >> 24) & 0xF) == W_CONST) {
                a = nl.kappa;
                gp = 0.0;
            } else if (A.wa_val) {
                const int64_t m = wa_index(A, mf, info, inst);
                a = A.wa_val[m];
                gp = A.wa_gp[m];
            } else {
                const double pu = ui + interp_du(info, du, BLK);
                double w;
                g_eval(nl.a_kind, nl.a_pi, nl.a_scale, pu, w, gp);
                a = (nl.kappa_field ? nl.kappa_field[wa_index(A, A.fib_m[fq], info, inst)] : nl.kappa) + w;
            }
            if constexpr (JDF) {
                a_df = split_dbl(a, 0);
                j1d_df = df_acc_prod(j1d_df, split_dbl(td, 0), a_df);
            } else {
                j1d += td * a;
            }
            D = 0.0;
        }
        const int c = lc & LEAF_PAD;
        if (c != LEAF_PAD) {
            D += T * du[c * BLK];
            if constexpr (JDF) Jd[c * BLK] = df_acc_prod(Jd[c * BLK], split_dbl(T, 0), a_df);
            else J[c * BLK] += T * a;
        }
    }
    if (f >= 0) {
        r += a * D;
        if (j2) {
            if constexpr (JDF) scatter_pi_df(info, split_dbl(D * gp, 0), Jd, BLK);
            else scatter_pi(info, D * gp, J, BLK);
        }
    }
    // reaction gamma M^c c, c = c_scale g_c(Pi_c u)
    for (int j = 0; j < M.nrx; ++j) {
        const int64_t q = M.rx_base + int64_t(j) * SLICE + lane;
        const double mv = A.rx_val[q];
        if (mv == 0.0) continue;
        const uint32_t xi = A.rx_info[q];
        double cv, cp;
        if (A.wc_val) {
            const int64_t m = wc_index(A, A.rx_m[q], xi, inst);
            cv = A.wc_val[m];
            cp = A.wc_gp[m];
        } else {
            const double pc = ui + interp_du(xi, du, BLK);
            g_eval(nl.c_kind, nl.c_pi, nl.c_scale, pc, cv, cp);
        }
        r += nl.gamma * mv * cv;
        if (!nl.picard) {
            if constexpr (JDF) scatter_pi_df(xi, split_dbl(nl.gamma * mv * cp, 0), Jd, BLK);
            else scatter_pi(xi, nl.gamma * mv * cp, J, BLK);
        }
    }
    double diag;
    if constexpr (JDF) diag = df_to_double_bits(df_acc(j1d_df, Jd[0]));
    else diag = j1d + J[0];
    const double res = r - di;
    if (A.r) A.r[row] = res;
    double dinv = 0.0;
    if (diag != 0.0) dinv = 1.0 / diag;
    else if (A.status) atomicOr(A.status, 1);
    if (A.dinv) A.dinv[row] = dinv;
    if (A.q64) A.q64[row] = dinv * res;
    if (A.q32) A.q32[row] = float(dinv * res);
    double rowsum = 0.0;
    for (int c = 0; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const int32_t slot = A.col_slot[q];
        double v;
        if constexpr (JDF) v = (c == 0) ? diag : df_to_double_bits(Jd[c * BLK]);
        else v = (c == 0) ? diag : J[c * BLK];
        if (A.jcsr && slot >= 0) A.jcsr[slot] = v;
        if (A.jsell) A.jsell[q] = slot >= 0 ? v : 0.0;
        // the scaled diagonal is stored as exactly 1 (the persistent FP64 solve relies on it)
        const double sv = slot >= 0 ? (c == 0 && dinv != 0.0 ? 1.0 : dinv * v) : 0.0;
        if (A.a64) A.a64[q] = sv;
        if (A.a32) { rowsum += sv; A.a32[q] = float(sv); }
    }
    // the FP32 operator keeps its row sum in column 0 (difference-form SpMV)
    if (A.a32) A.a32[M.col_base + lane] = float(rowsum);
}

// Mixed-precision tensor action for the Newton step of the mixed path (one thread per row):
// the residual r (and D r) in FP64 exactly as csf_fused_kernel computes it, the Jacobian in
// FP32 from the FP32 copies of T, of u's differences and of the nodal values, written only as
// the Jacobi-scaled FP32 solver operator.  Its diagonal uses the exact zero row sums of T
// (J1_ii = -sum of the row's off-diagonal J1 entries), and the row sum kept in column 0 for the
// difference-form operator comes from the same identity -- J1 rows sum to zero, the J2 and
// reaction rows to sum_m D_im g'_m and gamma sum_m M_im g_c'_m (Pi's rows sum to one) --
// summed (compensated) from the contributions exactly as scattered, less the Dirichlet
// columns the operator does not store.  FP64 work per row: the differences of u, one FMA
// per leaf and one per fibre.  Needs wa_val/wa_val32 (or a constant coefficient), wc_val for
// a reaction, leaf_val32, r, q64 and a32.
template <int MAXC>
__global__ void __launch_bounds__(csf_block<MAXC>(), csf_min_blocks<MAXC>()) csf_mixed_kernel(CsfArgs A) {
    constexpr int BLK = csf_block<MAXC>();
    __shared__ double s_du[MAXC * BLK];
    __shared__ float s_du32[MAXC * BLK];
    __shared__ float s_J[MAXC * BLK];
    const int tid = threadIdx.x;
    int32_t inst;
    const int64_t row = csf_row<BLK>(A, inst);
    if (row < 0 || row >= A.n_rows) return;
    const int64_t sl = row / SLICE;
    const int lane = int(row % SLICE);
    if (A.inst_mask && !A.inst_mask[A.slice_inst[sl]]) return;
    const SliceMeta M = A.meta[sl];
    const double ui = A.u[row];
    const double di = A.d ? A.d[row] : 0.0;
    double *du = s_du + tid;
    float *du32 = s_du32 + tid, *J = s_J + tid;
    if (A.dir[row]) {
        A.r[row] = ui - di;
        A.q64[row] = ui - di;
        for (int c = 0; c < M.ncol; ++c) A.a32[M.col_base + int64_t(c) * SLICE + lane] = (c == 0) ? 1.0f : 0.0f;
        return;
    }
    for (int c = 0; c < M.ncol; ++c) {
        const int32_t g = A.col_idx[M.col_base + int64_t(c) * SLICE + lane];
        const double d = A.u[g] - ui;
        du[c * BLK] = d;
        du32[c * BLK] = float(d);
        J[c * BLK] = 0.0f;
    }
    const Nonlin nl = A.nl;
    // FP64: the residual (D, r).  FP32: the Jacobian (D32, J, s1) and its row sum (rs_hi + rs_lo,
    // a compensated sum of the J2 and reaction contributions exactly as scattered)
    double r = 0.0, D = 0.0, a = 0.0;
    float a32 = 0.0f, gp32 = 0.0f, s1 = 0.0f, D32 = 0.0f, rs_hi = 0.0f, rs_lo = 0.0f;
    auto rs_add = [&](float e) {
        const float t = __fadd_rn(rs_hi, e);
        const float z = __fsub_rn(t, rs_hi);
        rs_lo = __fadd_rn(rs_lo, __fadd_rn(__fsub_rn(rs_hi, __fsub_rn(t, z)), __fsub_rn(e, z)));
        rs_hi = t;
    };
    uint32_t info = 0;
    int f = -1;
    // the next fibre's info and W index one fibre ahead, as in csf_fused_kernel
    uint32_t nx_info = 0;
    int32_t nx_m = 0;
    if (M.nfib > 0) { nx_info = __ldg(A.fib_info + M.fib_base + lane); nx_m = __ldg(A.fib_m + M.fib_base + lane); }
    // tensor data are read-only (non-coherent loads); unrolling lets the next leaves' loads
    // issue ahead of this leaf's arithmetic
#pragma unroll 4
    for (int j = 0; j < M.nleaf; ++j) {
        const int64_t q = M.leaf_base + int64_t(j) * SLICE + lane;
        const uint8_t lc = __ldg(A.leaf_col + q);
        if (lc & LEAF_FIBRE_START) {
            if (f >= 0) {
                r += a * D;
                if (gp32 != 0.0f && !nl.picard) {
                    const float e = D32 * gp32;
                    scatter_pi32(info, e, J, BLK);
                    rs_add(e);
                }
            }
            ++f;
            const int64_t fq = M.fib_base + int64_t(f) * SLICE + lane;
            info = nx_info;
            const int32_t mf = nx_m;
            if (f + 1 < M.nfib) { nx_info = __ldg(A.fib_info + fq + SLICE); nx_m = __ldg(A.fib_m + fq + SLICE); }
            if (((info >> 24) & 0xF) == W_CONST) {
                a = nl.kappa;
                a32 = float(nl.kappa);
                gp32 = 0.0f;
            } else {
                const int64_t m = wa_index(A, mf, info, inst);
                a = A.wa_val[m];
                a32 = A.wa_val32[m];
                gp32 = A.wa_gp32[m];
            }
            D = 0.0;
            D32 = 0.0f;
        }
        const int c = lc & LEAF_PAD;
        if (c != LEAF_PAD) {
            D += __ldg(A.leaf_val + q) * du[c * BLK];
            const float T32 = __ldg(A.leaf_val32 + q);
            D32 += T32 * du32[c * BLK];
            const float t = T32 * a32;
            J[c * BLK] += t;
            s1 += t;
        }
    }
    if (f >= 0) {
        r += a * D;
        if (gp32 != 0.0f && !nl.picard) {
            const float e = D32 * gp32;
            scatter_pi32(info, e, J, BLK);
            rs_add(e);
        }
    }
    // reaction gamma M^c c, c = c_scale g_c(Pi_c u)
    for (int j = 0; j < M.nrx; ++j) {
        const int64_t q = M.rx_base + int64_t(j) * SLICE + lane;
        const double mv = A.rx_val[q];
        if (mv == 0.0) continue;
        const int64_t m = wc_index(A, A.rx_m[q], A.rx_info[q], inst);
        r += nl.gamma * mv * A.wc_val[m];
        if (!nl.picard) {
            const float e = float(nl.gamma * mv * A.wc_gp[m]);
            scatter_pi32(A.rx_info[q], e, J, BLK);
            rs_add(e);
        }
    }
    const float diag = J[0] - s1;
    const double res = r - di;
    A.r[row] = res;
    float dinv = 0.0f;
    if (diag != 0.0f) dinv = 1.0f / diag;
    else if (A.status) atomicOr(A.status, 1);
    A.q64[row] = double(dinv) * res;
    for (int c = 1; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const float v = J[c * BLK];
        if (A.col_slot[q] >= 0) {
            A.a32[q] = dinv * v;
        } else {
            A.a32[q] = 0.0f;
            rs_add(-v);
        }
    }
    A.a32[M.col_base + lane] = dinv * (rs_hi + rs_lo);
}

// The exponent e when x = 2^e exactly (a positive normal number with an empty significand), else
// INT_MIN
__device__ __forceinline__ int pow2_exponent(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const int ex = int((b >> 52) & 0x7ffu);
    return ((b & 0x000fffffffffffffull) == 0ull && ex != 0 && ex != 0x7ff && (b >> 63) == 0ull) ? ex - 1023 : INT_MIN;
}

// f x for f = 2^e (e = pow2_exponent(f), INT_MIN when f is no power of two): an exponent shift on
// the integer pipe when x is a normal number and the product stays normal, else one FP64
// multiplication.  Both give the same bits (the product by a power of two is exact there).
__device__ __forceinline__ double mul_pow2(double x, double f, int e) {
    if (e != INT_MIN) {
        const long long b = __double_as_longlong(x);
        const int ex = int((b >> 52) & 0x7ff);
        if (ex != 0 && ex != 0x7ff && ex + e >= 1 && ex + e <= 0x7fe)
            return __longlong_as_double(b + (static_cast<long long>(e) << 52));
    }
    return f * x;
}

// Nodal values of one nonlinearity on its W space (Sec. 3.1 eq. (5), Sec. 3.2), one thread
// per W node, each node evaluated once: val_m = base_m + g((Pi u)_m), gp_m = g'((Pi u)_m),
// with base = kappa (constant, or the field when base_field is set) for the coefficient
// space and 0 for the reaction space.  Every FP64 operation costs a slot of GB300's narrow
// FP64 pipe, so the integer power is written with few: t = s^(p-1), gp = (scale p) t with
// scale p from the host, val = base + (scale t) s; products by powers of two (the midpoint's
// 1/2, and scale or scale p when they are such, e.g. 1 and 2 for w = u^2) are exponent shifts
// on the integer pipe with the same bits (mul_pow2).
__global__ void __launch_bounds__(256) wnode_kernel(int64_t n_w, const uint8_t *kind, const int32_t *sup, const double *u,
                                                    int32_t g_kind, int32_t g_p, double g_scale, double g_scale_p,
                                                    double base, const double *base_field, double *val, double *gp,
                                                    float *val32, float *gp32) {
    const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= n_w) return;
    const uint32_t k = kind[m];
    const double u0 = u[sup[3 * m]];
    double pu;
    if (k == W_VERTEX) pu = u0;
    else if (k == W_MID) pu = mul_pow2(u0 + u[sup[3 * m + 1]], 0.5, -1);
    else if (k == W_THIRD) pu = fma(2.0, u0, u[sup[3 * m + 1]]) * (1.0 / 3.0);
    else pu = (u0 + u[sup[3 * m + 1]] + u[sup[3 * m + 2]]) * (1.0 / 3.0);
    const double b0 = base_field ? base_field[m] : base;
    double v, d;
    if (g_kind == EGFEM_G_POW) {
        double t = 1.0;                       // pu^(p-1)
        if (g_p >= 2) t = pu;
        for (int32_t k = 2; k < g_p; ++k) t *= pu;
        d = g_p == 1 ? g_scale : mul_pow2(t, g_scale_p, pow2_exponent(g_scale_p));
        const double st = mul_pow2(t, g_scale, pow2_exponent(g_scale));
        v = b0 + st * pu;   // this rounding order: the Krylov iteration counts follow a's last bit
    } else {
        double g;
        g_eval(g_kind, g_p, g_scale, pu, g, d);
        v = b0 + g;
    }
    val[m] = v;
    gp[m] = d;
    if (val32) {   // FP32 copies for the mixed-precision Jacobian
        val32[m] = float(v);
        gp32[m] = float(d);
    }
}

// Pointwise nonlinearity alone (Sec. 3.2), one thread per W node.
__global__ void pointwise_kernel(int64_t n_w, const uint8_t *kind, const int32_t *sup, const double *u, Nonlin nl,
                                 double *w, double *wp) {
    const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= n_w) return;
    const uint32_t k = kind[m];
    double pu;
    const double u0 = u[sup[3 * m]];
    if (k == W_VERTEX) pu = u0;
    else if (k == W_MID) pu = 0.5 * (u0 + u[sup[3 * m + 1]]);
    else if (k == W_THIRD) pu = (2.0 * u0 + u[sup[3 * m + 1]]) * (1.0 / 3.0);
    else pu = (u0 + u[sup[3 * m + 1]] + u[sup[3 * m + 2]]) * (1.0 / 3.0);
    double g, gp;
    g_eval(nl.a_kind, nl.a_pi, nl.a_scale, pu, g, gp);
    if (w) w[m] = g;
    if (wp) wp[m] = gp;
}

}  // namespace egfem
