// egfem_mf.cuh -- element-local ("matrix-free") evaluation of the tensor action and the
// Jacobian, the variant beside the CSF operator.
//
// With P1 trial functions the trilinear form factors per cell K (Sec. 3.3):
//     T_imk = sum_K iota^K_m S^K_ik,   iota^K_m = int_K eta_m,   S^K = |K| grad lambda (grad lambda)^T,
// so with a = kappa + g(Pi u) and abar_K = sum_m (iota^K_m / |K|) a_m (S^K carries |K|):
//     r_i  = sum_K abar_K (S^K u)_i - d_i
//     J_ib = sum_K [ abar_K S^K_ib + (S^K u)_i c^K_b ],   c^K_b = sum_m (iota^K_m / |K|) g'(Pi u)_m Pi_mb
// i.e. each cell contributes a scaled stiffness plus a rank-one matrix.  A gradient
// coefficient with W_a = P0 (Sec. 5) has the same form, its one cell node carrying
// g(||grad u_K||^2) and c^K = 2 g' S^K u / |K|.  Pass 1 (one
// thread per cell) evaluates abar_K, S^K u and c^K from the cell's own vertex values and
// stores them; pass 2 (one thread per row, the row's cells from the vertex-to-cell list)
// gathers them into r_i and the row's Jacobian entries in a fixed order (deterministic).
// This needs about 2.5x fewer FP64 operations than the CSF action, whose leaves
// re-expand the factored form.
#pragma once

#include "egfem_kernels.cuh"

namespace egfem {

constexpr int MF_MAXW = 10;   // local W nodes of P3 on a triangle / P2 on a tetrahedron

// Local W nodes of the reference cell: barycentric weights (alpha / p) and
// iota / |K| (closed forms by node kind), uniform over the mesh.
struct MfLocal {
    int32_t nw;                         // local W nodes
    double w[MF_MAXW][4];               // barycentric weights on the cell's vertices
    double iota[MF_MAXW];               // int_K eta_l / |K|
    double mu[MF_MAXW][4];              // int_K lambda_a eta_l / |K| (reaction spaces)
    double mu3[MF_MAXW][4][4];          // int_K lambda_a lambda_b eta_l / |K| (product reaction)
};

struct MfArgs {
    int64_t n_cells, n_rows;
    int32_t dim;
    const int32_t *verts;               // [(dim+1) n_cells]
    const double *S;                    // [(dim+1)(dim+2)/2 n_cells] packed upper triangle, row-major
    const double *vol;                  // [n_cells]
    const int64_t *v2c_ptr;             // [n_rows + 1]
    const int32_t *v2c;                 // cells of each vertex
    double *E;                          // [ne n_cells] abar, S u, c per cell (+ rho, R with loc_c)
    int32_t ne;                         // doubles per cell record: 2 dim + 3, or + (d+1) + (d+1)^2
    MfLocal loc;
    MfLocal loc_c;                      // W_c = I_k, P2 or P3 (nw > 0): the reaction's local nodes
    Nonlin nl;
};

__device__ __forceinline__ int tri_index(int a, int b, int nv) {   // packed upper triangle
    if (a > b) { const int t = a; a = b; b = t; }
    return a * nv - (a * (a - 1)) / 2 + (b - a);
}

// t = base^q for the gradient coefficient.  When 4q is an integer of magnitude <= 8 (the
// minimal surface q = -1/2, the p-Laplacian q = (p - 2)/2 for p = 3/2, 5/2, 3, ...) it is a
// product of square roots and powers of base, which costs far fewer FP64 operations than a
// general power; otherwise pow.  base > 0 whenever q < 0 (the build requires a positive shift).
__device__ __forceinline__ double gradpow_base(double base, double q) {
    const double q4 = 4.0 * q;
    if (q4 == rint(q4) && fabs(q4) <= 8.0) {
        int k = int(q4);
        double r = base;                       // k quarter powers of base
        if (k % 4 == 0) { k /= 4; }
        else if (k % 2 == 0) { r = sqrt(base); k /= 2; }
        else { r = sqrt(sqrt(base)); }
        const int e = k < 0 ? -k : k;
        double t = 1.0;
        for (int i = 0; i < e; ++i) t *= r;
        return k < 0 ? 1.0 / t : t;
    }
    return pow(base, q);
}

// pass 1: per cell abar_K, (S^K u)_a (difference form), c^K_b
template <int DIM>
__global__ void __launch_bounds__(256) mf_cell_kernel(MfArgs M, const double *u) {
    constexpr int NV = DIM + 1, NS = NV * (NV + 1) / 2;
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= M.n_cells) return;
    double uk[NV], S[NS];
#pragma unroll
    for (int a = 0; a < NV; ++a) uk[a] = u[M.verts[c * NV + a]];
#pragma unroll
    for (int q = 0; q < NS; ++q) S[q] = M.S[c * NS + q];
    // (S^K u)_a in difference form (the rows of S^K sum to zero)
    double su[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < NV; ++b)
            if (b != a) t += S[tri_index(a, b, NV)] * (uk[b] - uk[a]);
        su[a] = t;
    }
    // S^K already carries |K|, so the cell weights are iota^K_m / |K| (sum over m: 1)
    double abar = 0.0, cb[NV];
#pragma unroll
    for (int b = 0; b < NV; ++b) cb[b] = 0.0;
    if (M.nl.a_kind == EGFEM_G_NONE) {
        abar = M.nl.kappa;
    } else if (M.nl.a_kind == EGFEM_G_GRADPOW) {
        // W_a = P0 (Sec. 5, gradient nonlinearities): the cell's one W node carries
        // s = ||grad u_K||^2 = u^T S^K u / |K| = sum_a (u_a - u_0) (S^K u)_a / |K|, and
        // ds/du_b = 2 (S^K u)_b / |K|, so c^K = 2 g'(s) S^K u / |K| (a symmetric rank one)
        const double ivol = 1.0 / M.vol[c];
        double sg = 0.0;
#pragma unroll
        for (int a = 1; a < NV; ++a) sg += (uk[a] - uk[0]) * su[a];
        sg = fmax(sg * ivol, 0.0);
        const double base = M.nl.a_shift + sg, q = M.nl.a_preal;
        const double t = gradpow_base(base, q);
        const double g = M.nl.a_scale * t;
        // g' = scale q base^(q-1) = q g / base; at base = 0 (shift 0, so q = 0 or q >= 1) it is
        // scale for q = 1 and 0 otherwise
        const double gp = q == 0.0 ? 0.0 : base > 0.0 ? q * g / base : (q == 1.0 ? M.nl.a_scale : 0.0);
        abar = M.nl.kappa + g;
        const double e = 2.0 * gp * ivol;
#pragma unroll
        for (int b = 0; b < NV; ++b) cb[b] = e * su[b];
    } else {
        for (int l = 0; l < M.loc.nw; ++l) {
            const double io = M.loc.iota[l];
            if (io == 0.0) continue;
            double pu = 0.0;
#pragma unroll
            for (int a = 0; a < NV; ++a) pu += M.loc.w[l][a] * uk[a];
            double g, gp;
            g_eval(M.nl.a_kind, M.nl.a_pi, M.nl.a_scale, pu, g, gp);
            abar += io * (M.nl.kappa + g);
            const double e = io * gp;
#pragma unroll
            for (int b = 0; b < NV; ++b) cb[b] += e * M.loc.w[l][b];
        }
    }
    double *E = M.E + c * M.ne;
    E[0] = abar;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
        E[1 + a] = su[a];
        E[1 + NV + a] = cb[a];
    }
    if (M.nl.c_kind != EGFEM_G_NONE && M.loc_c.nw > 0) {
        // W_c = I_k (Sec. 3.1, Case 3) or P2/P3: M^K_al = |K| mu_la (w_l lambda_a(x_l) for I_k,
        // int_K lambda_a eta_l for a Lagrange space) and c_l = g_c((Pi u)_l), so the cell adds
        // rho_a = gamma |K| sum_l mu_la g_c((Pi u)_l) to row a's residual and
        // R_ab = gamma |K| sum_l mu_la g_c'((Pi u)_l) Pi_lb to its Jacobian; both are evaluated
        // here once per cell and gathered by the row pass
        double rho[NV], R[NV * NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) rho[a] = 0.0;
#pragma unroll
        for (int q = 0; q < NV * NV; ++q) R[q] = 0.0;
        // The product form (decomposition (a), Sec. 5), gamma int c u phi_a = gamma |K| sum_l c_l
        // sum_k mu3_lak u_k, has R_ab = gamma |K| sum_l [c_l mu3_lab + (mu3_la. u) c'_l Pi_lb].
        // The g' terms are left out of the Picard matrix (the product's c_l mu3 term stays).
        const double gv = M.nl.gamma * M.vol[c];
        const bool prod = M.nl.c_product != 0, newton = !M.nl.picard;
        for (int l = 0; l < M.loc_c.nw; ++l) {
            double uq = 0.0;
#pragma unroll
            for (int b = 0; b < NV; ++b) uq += M.loc_c.w[l][b] * uk[b];
            double g, gp;
            g_eval(M.nl.c_kind, M.nl.c_pi, M.nl.c_scale, uq, g, gp);
            const double wg = gv * g, wd = gv * gp;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                double ma = M.loc_c.mu[l][a];
                if (prod) {
                    ma = 0.0;
#pragma unroll
                    for (int k = 0; k < NV; ++k) ma += M.loc_c.mu3[l][a][k] * uk[k];
#pragma unroll
                    for (int b = 0; b < NV; ++b) R[a * NV + b] += wg * M.loc_c.mu3[l][a][b];
                }
                rho[a] += wg * ma;
                if (newton) {
                    const double md = wd * ma;
#pragma unroll
                    for (int b = 0; b < NV; ++b) R[a * NV + b] += md * M.loc_c.w[l][b];
                }
            }
        }
#pragma unroll
        for (int a = 0; a < NV; ++a) E[1 + 2 * NV + a] = rho[a];
#pragma unroll
        for (int q = 0; q < NV * NV; ++q) E[1 + 3 * NV + q] = R[q];
    }
}

// pass 2: per row, gather the cells' contributions; outputs as the CSF kernel's
template <int DIM, int MAXC>
__global__ void __launch_bounds__(csf_block<MAXC>()) mf_row_kernel(MfArgs M, CsfArgs A) {
    constexpr int BLK = csf_block<MAXC>();
    constexpr int NV = DIM + 1, NS = NV * (NV + 1) / 2;
    __shared__ double s_J[MAXC * BLK];
    __shared__ int32_t s_col[MAXC * BLK];
    const int tid = threadIdx.x;
    const int64_t row = int64_t(blockIdx.x) * BLK + tid;
    if (row >= A.n_rows) return;
    const int64_t sl = row / SLICE;
    if (A.inst_mask && !A.inst_mask[A.slice_inst[sl]]) return;
    const int lane = int(row % SLICE);
    const SliceMeta Ms = A.meta[sl];
    const double ui = A.u[row];
    const double di = A.d ? A.d[row] : 0.0;
    double *J = s_J + tid;
    int32_t *C = s_col + tid;
    if (A.dir[row]) {
        if (A.r) A.r[row] = ui - di;
        if (A.q64) A.q64[row] = ui - di;
        if (A.q32) A.q32[row] = float(ui - di);
        if (A.dinv) A.dinv[row] = 1.0;
        for (int c = 0; c < Ms.ncol; ++c) {
            const int64_t q = Ms.col_base + int64_t(c) * SLICE + lane;
            const double v = (c == 0) ? 1.0 : 0.0;
            if (A.a64) A.a64[q] = v;
            if (A.a32) A.a32[q] = float(v);
            if (A.jcsr && c == 0) A.jcsr[A.col_slot[q]] = 1.0;
            if (A.jsell) A.jsell[q] = v;
        }
        return;
    }
    for (int c = 0; c < Ms.ncol; ++c) {
        C[c * BLK] = A.col_idx[Ms.col_base + int64_t(c) * SLICE + lane];
        J[c * BLK] = 0.0;
    }
    const Nonlin nl = A.nl;
    double r = 0.0, diag_extra = 0.0;
    for (int64_t t = M.v2c_ptr[row]; t < M.v2c_ptr[row + 1]; ++t) {
        const int64_t cell = M.v2c[t];
        int32_t vk[NV], lcb[NV];
#pragma unroll
        for (int b = 0; b < NV; ++b) vk[b] = M.verts[cell * NV + b];
        int a = 0;
#pragma unroll
        for (int b = 1; b < NV; ++b) if (vk[b] == row) a = b;
        // the row's local Jacobian column of each of the cell's vertices
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            lcb[b] = 0;
            for (int c = 0; c < Ms.ncol; ++c) if (C[c * BLK] == vk[b]) { lcb[b] = c; break; }
        }
        const double *E = M.E + cell * M.ne;
        const double abar = E[0], su = E[1 + a];
        r += abar * su;
#pragma unroll
        for (int b = 0; b < NV; ++b) {
            const int lc = lcb[b];
            double v = nl.picard ? 0.0 : su * E[1 + NV + b];
            if (b != a) {
                // abar S_ab off the diagonal; on it abar S_aa = -sum_{b != a} abar S_ab
                const double t = abar * M.S[cell * NS + tri_index(a, b, NV)];
                v += t;
                diag_extra -= t;
            }
            J[lc * BLK] += v;
        }
        if (nl.sigma != 0.0) {
            // linear reaction sigma M^K: M_ab = |K| (1 + delta_ab) / ((d+1)(d+2))
            const double m0 = nl.sigma * M.vol[cell] / double((DIM + 1) * (DIM + 2));
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                const double mab = (b == a) ? 2.0 * m0 : m0;
                r += mab * A.u[vk[b]];
                J[lcb[b] * BLK] += mab;
            }
        }
        if (nl.c_kind != EGFEM_G_NONE && M.loc_c.nw > 0) {
            // gamma M^c c with W_c = I_k, P2 or P3 (or the product form): the cell pass's rho_a
            // and R_ab, the latter already without the g' terms for the Picard matrix
            r += E[1 + 2 * NV + a];
#pragma unroll
            for (int b = 0; b < NV; ++b) J[lcb[b] * BLK] += E[1 + 3 * NV + a * NV + b];
        } else if (nl.c_kind != EGFEM_G_NONE) {
            // gamma M^c c with W_c = P1: M_ab = |K| (1 + delta_ab) / ((d+1)(d+2))
            const double m0 = M.vol[cell] / double((DIM + 1) * (DIM + 2));
#pragma unroll
            for (int b = 0; b < NV; ++b) {
                double g, gp;
                g_eval(nl.c_kind, nl.c_pi, nl.c_scale, A.u[vk[b]], g, gp);
                const double mab = (b == a) ? 2.0 * m0 : m0;
                r += nl.gamma * mab * g;
                if (!nl.picard) J[lcb[b] * BLK] += nl.gamma * mab * gp;
            }
        }
    }
    const double diag = J[0] + diag_extra;
    const double res = r - di;
    if (A.r) A.r[row] = res;
    double dinv = 0.0;
    if (diag != 0.0) dinv = 1.0 / diag;
    else if (A.status) atomicOr(A.status, 1);
    if (A.dinv) A.dinv[row] = dinv;
    if (A.q64) A.q64[row] = dinv * res;
    if (A.q32) A.q32[row] = float(dinv * res);
    double rowsum = 0.0;
    for (int c = 0; c < Ms.ncol; ++c) {
        const int64_t q = Ms.col_base + int64_t(c) * SLICE + lane;
        const int32_t slot = A.col_slot[q];
        const double v = (c == 0) ? diag : J[c * BLK];
        if (A.jcsr && slot >= 0) A.jcsr[slot] = v;
        if (A.jsell) A.jsell[q] = slot >= 0 ? v : 0.0;
        const double sv = slot >= 0 ? (c == 0 && dinv != 0.0 ? 1.0 : dinv * v) : 0.0;   // unit diagonal
        rowsum += sv;
        if (A.a64) A.a64[q] = sv;
        if (A.a32) A.a32[q] = float(sv);
    }
    if (A.a32) A.a32[Ms.col_base + lane] = float(rowsum);
}

}  // namespace egfem
