// egfem_internal.h -- data layouts shared by the host build and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/egfem.h"

namespace egfem {

// Rows are processed in slices of SLICE consecutive rows, one thread per row, with
// every per-row array stored column-interleaved inside its slice (SELL-32): entry j of
// the slice's row r sits at base + j * SLICE + r, so a warp's loads are coalesced.
constexpr int SLICE = 32;

// Kinds of W nodes; each fixes the interpolation weights of Pi (Sec. 3.2,
// (Pi)_mj = phi_j(x_m)) on the node's 1-3 supporting P1 vertices.
enum WKind : uint32_t {
    W_CONST = 0,   // no nonlinearity: the coefficient is the constant kappa
    W_VERTEX = 1,  // node at a vertex                          weights {1}
    W_MID = 2,     // edge midpoint                             weights {1/2, 1/2}
    W_THIRD = 3,   // edge point at 1/3 from its first vertex   weights {2/3, 1/3}
    W_FACE = 4     // face / triangle centroid                  weights {1/3, 1/3, 1/3}
};

// Fibre / reaction-entry info word: bits 0-7, 8-15, 16-23 = local columns of the
// supporting vertices (up to 3), bits 24-27 = WKind.
__host__ __device__ inline uint32_t pack_info(uint32_t kind, uint32_t c0, uint32_t c1, uint32_t c2) {
    return (c0 & 0xFF) | ((c1 & 0xFF) << 8) | ((c2 & 0xFF) << 16) | ((kind & 0xF) << 24);
}

// Leaf byte: bits 0-5 local column (LEAF_PAD = padding), bit 7 = first leaf of a fibre.
constexpr uint8_t LEAF_PAD = 0x3F;
constexpr uint8_t LEAF_FIBRE_START = 0x80;

struct SliceMeta {
    int64_t col_base;   // into col_idx / col_slot / J SELL values
    int64_t leaf_base;  // into leaf_val / leaf_col
    int64_t fib_base;   // into fib_info / fib_tdiag / fib_m
    int64_t rx_base;    // into rx_val / rx_info / rx_m
    int64_t off_base;   // uniform slice: into slice_off (column c of row i is i + slice_off[off_base + c]); -1 otherwise
    int32_t ncol, nleaf, nfib, nrx;
};

// Host image of the row-segmented CSF tensor (row i -> fibres by W node m -> leaves by
// trial column k) plus the reaction entries and the Jacobian pattern.
struct HostCSF {
    int64_t n_rows = 0;
    int32_t n_slices = 0;
    int32_t max_cols = 0;
    std::vector<SliceMeta> meta;
    std::vector<int32_t> slice_off;  // column offsets (col - row) of the uniform slices
    std::vector<int32_t> col_idx;    // global P1 node of each local column (pad: the row itself)
    std::vector<int32_t> col_slot;   // CSR slot of each local column (-1: Dirichlet column or pad)
    std::vector<double> leaf_val;    // T_imk for k != i
    std::vector<uint8_t> leaf_col;   // local column of k | fibre-start flag
    std::vector<uint32_t> fib_info;  // Pi support of W node m (local columns) and kind
    std::vector<double> fib_tdiag;   // T_imi = -sum_{k != i} T_imk (exact zero row sums)
    std::vector<int32_t> fib_m;      // global W_a index of the fibre's node
    std::vector<double> rx_val;      // M^c_im (reaction entries)
    std::vector<uint32_t> rx_info;   // Pi_c support of W_c node m
    std::vector<int32_t> rx_m;       // global W_c index
    std::vector<uint8_t> dir;        // per row
    std::vector<int32_t> rowptr;     // Jacobian CSR pattern
    std::vector<int32_t> cols;
};

// One W space: node kinds and supporting P1 vertices (global).
struct HostWSpace {
    int degree = 1;
    int64_t n = 0;
    std::vector<uint8_t> kind;       // WKind per node
    std::vector<int32_t> sup;        // [3 * n] supporting vertices (-1 unused), ordered as the weights
    std::vector<double> coords;      // [dim * n]
};

// Element-local data for the matrix-free operator and the load vector.
struct HostCells {
    int32_t dim = 2;
    int64_t n = 0;
    std::vector<int32_t> verts;      // [(dim+1) * n]
    std::vector<double> vol;         // |K|
    std::vector<double> S;           // [(dim+1)^2 * n]  |K| grad lambda_a . grad lambda_b
    std::vector<int32_t> wa;         // [nloc_a * n] W_a node of each local W node
};

struct DeviceCSF {
    int64_t n_rows = 0;
    int32_t n_slices = 0;
    int32_t max_cols = 0;
    SliceMeta *meta = nullptr;
    int32_t *col_idx = nullptr, *col_slot = nullptr;
    int32_t *slice_off = nullptr;
    int64_t n_uniform = 0;
    double *leaf_val = nullptr;
    uint8_t *leaf_col = nullptr;
    uint32_t *fib_info = nullptr;
    double *fib_tdiag = nullptr;
    int32_t *fib_m = nullptr;
    double *rx_val = nullptr;
    uint32_t *rx_info = nullptr;
    int32_t *rx_m = nullptr;
    uint8_t *dir = nullptr;
    int32_t *rowptr = nullptr, *cols = nullptr;
    int64_t n_colentries = 0, n_leaves = 0, n_fibres = 0, n_rx = 0, nnz = 0;
};

// A batch whose instances all use one mesh, stored with one copy of the tensor (k > 0): instance
// b owns rows [b rows, (b + 1) rows); every instance's slices point at instance 0's leaves,
// fibres and reaction entries, whose W indices are instance 0's: instance b's W index of a
// node of kind w (WKind) is that plus b a[w] (coefficient space) or b c[w] (reaction space).
struct WShare {
    int32_t k;
    int64_t rows;
    int64_t a[5], c[5];
};

// Problem constants passed by value to the kernels.
struct Nonlin {
    int32_t a_kind; int32_t a_pi; double a_scale;
    int32_t c_kind; int32_t c_pi; double c_scale;
    double gamma, kappa;
    const double *kappa_field;   // W_a field or nullptr
    int32_t picard;              // nonzero: the Picard matrix (no g' terms) instead of the Jacobian
    double a_preal, a_shift;     // EGFEM_G_GRADPOW: g = a_scale (a_shift + |grad u|^2)^a_preal
    double sigma;                // linear reaction sigma M u (element-local operator only)
    int32_t c_product;           // reaction gamma int c u phi_i (element-local operator only)
};

// Host-side assembly entry points (egfem_build.cpp).
egfem_status build_wspace(const egfem_mesh &mesh, int degree, HostWSpace &W, std::vector<int32_t> &cell2w,
                          int &nloc, std::string &err);
egfem_status build_csf(const egfem_mesh &mesh, const egfem_problem &prob, const HostWSpace &Wa,
                       const std::vector<int32_t> &cell2wa, int nloc_a, const HostWSpace &Wc,
                       const std::vector<int32_t> &cell2wc, int nloc_c, HostCSF &out, std::string &err);
egfem_status validate_mesh(const egfem_mesh &mesh, std::string &err);
bool share_tensor(HostCSF &H, int32_t k, int64_t rows, WShare &ws);
double basis_integral(int dim, int degree, int kind);   // int_K eta_m / |K| by node kind
void cell_stiffness(const egfem_mesh &mesh, std::vector<double> &vol, std::vector<double> *S);
std::vector<double> cell_centroids(const egfem_mesh &mesh);
int quad_rule(int dim, int k, double bary[][4], double *w);
std::vector<double> quad_points(const egfem_mesh &mesh, int nq, const double bary[][4]);
void set_last_error(const std::string &msg);            // text returned by egfem_last_error()

}  // namespace egfem
