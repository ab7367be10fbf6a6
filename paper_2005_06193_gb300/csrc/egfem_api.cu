// egfem_api.cu -- the C ABI of include/egfem.h: build/upload, the hot-path entry
// points, the Newton driver with captured BiCGStab chunks, and the adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "egfem_internal.h"
#include "egfem_kernels.cuh"
#include "egfem_krylov.cuh"
#include "egfem_batch.cuh"
#include "egfem_mf.cuh"
#include "egfem_persist.cuh"
#include "egfem_window.cuh"
#include "egfem_cluster.cuh"
#include "egfem_gnewton.cuh"

using namespace egfem;

namespace {

thread_local std::string g_last_error;

#define EG_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
            return e_ == cudaErrorMemoryAllocation ? EGFEM_ERR_OOM : EGFEM_ERR_CUDA;                   \
        }                                                                                              \
    } while (0)

#define EG_TRY(expr)                                   \
    do {                                               \
        egfem_status s_ = (expr);                      \
        if (s_ != EGFEM_OK) return s_;                 \
    } while (0)

template <typename T>
egfem_status dalloc(T *&p, size_t n) {
    p = nullptr;
    if (n == 0) return EGFEM_OK;
    EG_CUDA(cudaMalloc((void **)&p, n * sizeof(T)));
    return EGFEM_OK;
}

template <typename T>
egfem_status upload(T *&p, const std::vector<T> &v) {
    EG_TRY(dalloc(p, v.size()));
    if (!v.empty()) EG_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return EGFEM_OK;
}

template <typename V>
struct KWork {
    typename VecT<V>::mat *A = nullptr;   // Jacobi-scaled operator (SELL layout)
    V *b = nullptr, *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
    V *p2 = nullptr, *v2 = nullptr;       // second p / v buffers of the fused double-float iteration
    // persistent solve (pk_solve1): one tile of rows per block
    int g_pk = 0;                         // blocks (0: not available)
    BTile *pk_tiles = nullptr;
    int64_t pk_ntiles = 0;
    double *pk_part = nullptr;            // [4 * pk_ntiles]
    PGrid *bar = nullptr;
    // windowed single-system solve (pkw_solve): one window per tile; 0 bytes: not available
    PkWin *pkw_win = nullptr;
    size_t pkw_smem = 0;
    // windowed batched solve (pkwb_solve): its own tiles (inside instances) and windows
    BTile *pkwb_tiles = nullptr;
    PkWin *pkwb_win = nullptr;
    double *pkwb_part = nullptr;          // [4 * pkwb_ntiles]
    int64_t pkwb_ntiles = 0;
    int pkwb_grid = 0;
    size_t pkwb_smem = 0;                 // 0: not available
    bool pkwb_planned = false;            // planned with the batch layout in place
    // cluster solve (pkc_solve, FP64): CTAs in the cluster (0: not used) and rows per CTA
    int pkc_cluster = 0;
    int32_t pkc_rows = 0;
    int32_t pkc_op = 0;                   // ELL columns of the shared-memory operator copy (0: none)
    size_t pkc_smem = 0;                  // dynamic shared memory per CTA
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    bool ready = false;
    // grid of each iteration kernel: one wave of resident blocks (occupancy x SMs), capped
    // by the work, so the grid-stride loops run without a tail wave
    int g_setup = 1, g_v = 1, g_s = 1, g_t = 1, g_x = 1, g_p = 1, g_vp = 1, g_st = 1, g_xr = 1;
};

}  // namespace

struct egfem_t {
    int device = 0;
    int sms = 148;
    egfem_problem prob{};
    egfem_options opts{};
    egfem_mesh mesh_sizes{};
    int32_t dim = 2;
    int64_t n = 0, nwa = 0, nwc = 0, ncells = 0;
    DeviceCSF csf;
    std::vector<double> wa_coords, wc_coords;
    uint8_t *wa_kind = nullptr, *wc_kind = nullptr;
    int32_t *wa_sup = nullptr, *wc_sup = nullptr;
    double *wa_val = nullptr, *wa_gp = nullptr;   // nodal a_m, g_a' (wnode_kernel)
    double *wc_val = nullptr, *wc_gp = nullptr;   // nodal c_m, g_c'
    float *wa_val32 = nullptr, *wa_gp32 = nullptr;   // FP32 copies (mixed tensor action)
    float *leaf_val32 = nullptr;                     // FP32 copy of the tensor values (mixed)
    bool mixed_ta_ready = false;                     // the FP32 copies above exist
    int32_t *cell_verts = nullptr;
    double *cell_vol = nullptr;
    int64_t *v2c_ptr = nullptr;
    int32_t *v2c = nullptr;
    int64_t *tmap = nullptr;            // SELL position of the transposed entry
    double *adj_b0 = nullptr, *adj_acc = nullptr, *adj_ss = nullptr;   // transposed-solve restarts
    Nonlin nl{};
    double *kappa_field = nullptr;
    // Newton workspace
    double *r = nullptr, *jsell = nullptr, *dinv = nullptr;
    double *part = nullptr;
    KState *st = nullptr;
    KState *h_st = nullptr;             // pinned
    double *scal = nullptr;             // device scalars (norms)
    double *h_scal = nullptr;           // pinned
    uint32_t *ticket = nullptr;
    int32_t *status = nullptr;
    KWork<double> k64;                  // FP64 path (and the rescue of failed mixed steps)
    KWork<df64> k32;                    // mixed path: FP32 operator, double-float vectors
    int64_t n_pad = 0;                  // rows rounded up to whole slices (Krylov vectors)
    int kgrid = 1;                      // blocks of the row kernels (norms)
    int kgrid64 = 1, kgrid32 = 1;       // blocks of the FP64 / FP32 Krylov kernels
    cudaStream_t hs = nullptr;          // internal stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int maxc_tpl = 8;
    int64_t last_graph_launches = 0;    // graph launches of the last BiCGStab solve
    int64_t last_graph_nodes = 0;       // kernels per graph launch of that solve
    int64_t last_krylov_kernels = 0;    // kernels the last BiCGStab solve launched
    bool coop = false;                  // the device supports cooperative launches
    // element-local operator (EGFEM_OP_MATRIX_FREE)
    double *cell_S = nullptr, *cell_E = nullptr;
    MfLocal mf_loc{};
    MfLocal mf_loc_c{};                 // W_c = I_k: the reaction's rule (nw = 0: W_c = P1)
    int32_t mf_ne = 0;                  // doubles per cell record of the element-local operator
    // batch (egfem_batch_build): instance b owns rows [inst_off[b], inst_off[b+1])
    int32_t nb = 0;
    std::vector<int64_t> inst_off;
    WShare ws{};                        // one tensor for a batch of one mesh (ws.k > 0)
    int32_t *slice_inst = nullptr;
    uint8_t *inst_mask = nullptr, *h_mask = nullptr;
    double *inst_eta = nullptr, *h_eta = nullptr;
    double *inst_lam = nullptr, *h_lam = nullptr;
    double *inst_norm2 = nullptr, *h_norm2 = nullptr;
    KState *bst = nullptr, *h_bst = nullptr;
    BTile *tiles = nullptr;
    int64_t ntiles = 0;
    int tile_factor = 0;                // rows per tile = KRY_BLOCK * R * tile_factor (0: not tuned yet)
    int tile_R = 0;
    double *bpart = nullptr;
    cudaGraphExec_t bgraph64 = nullptr, bgraph32 = nullptr;
    PGrid *bbar = nullptr;              // grid barrier of the persistent batched solve
    double *bpart2 = nullptr;           // tile partials of the persistent batched solve
    int bgraph_chunk = 0, bgraph_tiles = 0;
    // graph-resident batched Newton loop (egfem_gnewton.cuh): device state, the instantiated
    // graph and the vectors and path it was captured for
    GNState *gn_state = nullptr;
    egfem_stats *gn_stats = nullptr;
    int32_t *gn_loops = nullptr;
    cudaGraphExec_t gn_exec = nullptr;
    const double *gn_u = nullptr, *gn_d = nullptr;
    int gn_mixed = -1;
    int gn_one = -1;                    // 1: captured for egfem_newton_solve, 0: for the batched solve
    int gn_nodes = 0;                   // kernels one body execution launches
    bool gn_failed = false;             // capture or instantiation failed once: host loop only
    bool gn_used = false;               // the last batched solve ran the graph loop
};

namespace {

// Smallest Krylov forcing term of the mixed path.  Its vectors carry 48-bit significands
// (df64), so the iteration is as stable as in FP64; what limits it is the FP32-rounded
// operator, whose relative perturbation (~6e-8, row sums kept exact) the FP64 Newton
// residual corrects at the next step (iterative refinement).
constexpr double kMixedEtaFloor = 1e-8;
// An FP32 solve whose residual has not fallen by 10% for this many iterations stops (its
// iterate is still applied; the FP64 Newton residual judges it).
constexpr int32_t kMixedStall = 150;

// Fewest rows per block of the single-system persistent solve: below this a grid barrier
// over more blocks costs more than the rows it spreads.
constexpr int32_t kPkBlockRows = 32;

int pick_maxc(int maxc) {
    if (maxc <= 8) return 8;
    if (maxc <= 16) return 16;
    if (maxc <= 32) return 32;
    return 64;
}

template <int DIM>
int launch_mf(egfem_t *h, const CsfArgs &A, cudaStream_t s) {
    MfArgs M{};
    M.n_cells = h->ncells; M.n_rows = h->n; M.dim = DIM;
    M.verts = h->cell_verts; M.S = h->cell_S; M.vol = h->cell_vol; M.v2c_ptr = h->v2c_ptr; M.v2c = h->v2c;
    M.E = h->cell_E; M.ne = h->mf_ne; M.loc = h->mf_loc; M.loc_c = h->mf_loc_c;
    M.nl = A.nl;   // this call's record: it carries the Picard flag
    mf_cell_kernel<DIM><<<unsigned((h->ncells + 255) / 256), 256, 0, s>>>(M, A.u);
    auto grid = [&](int blk) { return unsigned((h->n + blk - 1) / blk); };
    switch (h->maxc_tpl) {
        case 8: mf_row_kernel<DIM, 8><<<grid(csf_block<8>()), csf_block<8>(), 0, s>>>(M, A); break;
        case 16: mf_row_kernel<DIM, 16><<<grid(csf_block<16>()), csf_block<16>(), 0, s>>>(M, A); break;
        case 32: mf_row_kernel<DIM, 32><<<grid(csf_block<32>()), csf_block<32>(), 0, s>>>(M, A); break;
        default: mf_row_kernel<DIM, 64><<<grid(csf_block<64>()), csf_block<64>(), 0, s>>>(M, A); break;
    }
    return 2;
}

// FP32 copies of the tensor values and nodal buffers for csf_mixed_kernel (once per handle).
egfem_status ensure_mixed_tensor(egfem_t *h, cudaStream_t s) {
    if (h->mixed_ta_ready) return EGFEM_OK;
    EG_TRY(dalloc(h->leaf_val32, size_t(std::max<int64_t>(1, h->csf.n_leaves))));
    if (h->csf.n_leaves > 0)
        cast_kernel<double, float><<<unsigned((h->csf.n_leaves + 255) / 256), 256, 0, s>>>(h->csf.n_leaves, h->csf.leaf_val,
                                                                                          h->leaf_val32);
    if (h->wa_val) {
        EG_TRY(dalloc(h->wa_val32, size_t(h->nwa)));
        EG_TRY(dalloc(h->wa_gp32, size_t(h->nwa)));
    }
    EG_CUDA(cudaGetLastError());
    h->mixed_ta_ready = true;
    return EGFEM_OK;
}

// The Newton step of the mixed path needs only r, D r and the FP32 operator: then the
// mixed-precision tensor action (FP32 Jacobian) serves it.
bool mixed_tensor_action(const egfem_t *h, const CsfArgs &A) {
    return h->opts.op == EGFEM_OP_CSF && h->mixed_ta_ready && A.a32 && A.r && A.q64 && !A.a64 && !A.jcsr && !A.jsell &&
           !A.dinv && !A.q32;
}

// Pointwise nonlinearity + residual + Jacobian fill at A.u; returns the kernels launched.
int launch_csf(egfem_t *h, const CsfArgs &A, cudaStream_t s) {
    if (h->opts.op == EGFEM_OP_MATRIX_FREE) return h->dim == 2 ? launch_mf<2>(h, A, s) : launch_mf<3>(h, A, s);
    int launched = 1;
    const bool mix = mixed_tensor_action(h, A);
    // each W node's nonlinearity once (Sec. 3.2), then the tensor action gathers it per fibre
    CsfArgs B = A;
    if (h->wa_val) {
        float *v32 = mix ? h->wa_val32 : nullptr, *g32 = mix ? h->wa_gp32 : nullptr;
        wnode_kernel<<<unsigned((h->nwa + 255) / 256), 256, 0, s>>>(h->nwa, h->wa_kind, h->wa_sup, A.u, h->nl.a_kind, h->nl.a_pi,
                                                                  h->nl.a_scale, h->nl.a_scale * h->nl.a_pi, h->nl.kappa,
                                                                  h->nl.kappa_field, h->wa_val, h->wa_gp, v32, g32);
        B.wa_val = h->wa_val; B.wa_gp = h->wa_gp; B.wa_val32 = v32; B.wa_gp32 = g32;
        ++launched;
    }
    if (h->wc_val) {
        wnode_kernel<<<unsigned((h->nwc + 255) / 256), 256, 0, s>>>(h->nwc, h->wc_kind, h->wc_sup, A.u, h->nl.c_kind, h->nl.c_pi,
                                                                  h->nl.c_scale, h->nl.c_scale * h->nl.c_pi, 0.0, nullptr,
                                                                  h->wc_val, h->wc_gp, nullptr, nullptr);
        B.wc_val = h->wc_val; B.wc_gp = h->wc_gp;
        ++launched;
    }
    // a shared tensor: ws.k blocks per range of local rows, one per instance (csf_row)
    auto grid = [&](int blk) {
        return h->ws.k > 0 ? unsigned((h->ws.rows + blk - 1) / blk * h->ws.k) : unsigned((h->n + blk - 1) / blk);
    };
    if (mix) {
        B.leaf_val32 = h->leaf_val32;
        switch (h->maxc_tpl) {
            case 8: csf_mixed_kernel<8><<<grid(csf_block<8>()), csf_block<8>(), 0, s>>>(B); break;
            case 16: csf_mixed_kernel<16><<<grid(csf_block<16>()), csf_block<16>(), 0, s>>>(B); break;
            case 32: csf_mixed_kernel<32><<<grid(csf_block<32>()), csf_block<32>(), 0, s>>>(B); break;
            default: csf_mixed_kernel<64><<<grid(csf_block<64>()), csf_block<64>(), 0, s>>>(B); break;
        }
        return launched;
    }
    // the Newton steps' evaluations (residual and solver operator) accumulate the Jacobian in
    // double-float; egfem_jacobian (CSR values) and the adjoint (jsell, dinv) in FP64
    if (!A.jcsr && !A.jsell && !A.dinv) {
        switch (h->maxc_tpl) {
            case 8: csf_fused_kernel<8, true><<<grid(csf_block<8>()), csf_block<8>(), 0, s>>>(B); break;
            case 16: csf_fused_kernel<16, true><<<grid(csf_block<16>()), csf_block<16>(), 0, s>>>(B); break;
            case 32: csf_fused_kernel<32, true><<<grid(csf_block<32>()), csf_block<32>(), 0, s>>>(B); break;
            default: csf_fused_kernel<64, true><<<grid(csf_block<64>()), csf_block<64>(), 0, s>>>(B); break;
        }
        return launched;
    }
    switch (h->maxc_tpl) {
        case 8: csf_fused_kernel<8, false><<<grid(csf_block<8>()), csf_block<8>(), 0, s>>>(B); break;
        case 16: csf_fused_kernel<16, false><<<grid(csf_block<16>()), csf_block<16>(), 0, s>>>(B); break;
        case 32: csf_fused_kernel<32, false><<<grid(csf_block<32>()), csf_block<32>(), 0, s>>>(B); break;
        default: csf_fused_kernel<64, false><<<grid(csf_block<64>()), csf_block<64>(), 0, s>>>(B); break;
    }
    return launched;
}

// Largest Krylov forcing term, also the first step's: the option when set, else 0.9 for Newton
// (Eisenstat and Walker's cap for choice 2) and 1e-2 for Picard, whose frozen-coefficient step
// is no Newton direction and needs its linear solves tighter to decrease the residual.
double eta_cap(const egfem_t *h) {
    if (h->opts.eta_max > 0.0) return h->opts.eta_max;
    return h->opts.iteration == EGFEM_ITER_PICARD ? 1e-2 : 0.9;
}

CsfArgs csf_args(egfem_t *h, const double *u, const double *d) {
    CsfArgs A{};
    A.n_rows = h->n;
    A.meta = h->csf.meta;
    A.col_idx = h->csf.col_idx; A.col_slot = h->csf.col_slot;
    A.leaf_val = h->csf.leaf_val; A.leaf_col = h->csf.leaf_col;
    A.fib_info = h->csf.fib_info; A.fib_tdiag = h->csf.fib_tdiag; A.fib_m = h->csf.fib_m;
    A.rx_val = h->csf.rx_val; A.rx_info = h->csf.rx_info; A.rx_m = h->csf.rx_m;
    A.dir = h->csf.dir;
    A.nl = h->nl;
    A.nl.picard = h->opts.iteration == EGFEM_ITER_PICARD;
    A.u = u; A.d = d;
    A.status = h->status;
    A.ws = h->ws;
    return A;
}

template <typename V>
int kgrid_of(const egfem_t *h) { return sizeof(V) == 8 ? h->kgrid64 : h->kgrid32; }

template <typename V>
KVecs<V> kvecs(egfem_t *h, KWork<V> &W) {
    KVecs<V> K{};
    K.n_pad = h->n_pad; K.meta = h->csf.meta; K.col_idx = h->csf.col_idx; K.slice_off = h->csf.slice_off; K.A = W.A;
    K.x = W.x; K.r = W.r; K.rh = W.rh; K.p = W.p; K.v = W.v; K.s = W.s; K.t = W.t; K.b = W.b;
    K.st = h->st; K.part = h->part;
    return K;
}

template <typename V>
int one_wave(const egfem_t *h, const void *func) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, KRY_BLOCK, 0) != cudaSuccess || nb < 1) nb = 1;
    const int64_t work = (h->n_pad + int64_t(KRY_BLOCK) * VecT<V>::R - 1) / (int64_t(KRY_BLOCK) * VecT<V>::R);
    return int(std::max<int64_t>(1, std::min<int64_t>(work, int64_t(nb) * h->sms)));
}

// Cluster solve plan for one system (FP64 or double-float vectors): the rows must fit the Krylov
// vectors of the cluster's
// CTAs in shared memory (PKC_NVEC doubles per row); the cluster size is the smallest power of two
// giving at most kPkcTargetRows rows per CTA (or the krylov_cluster option), and the launch
// configuration must be schedulable (cudaOccupancyMaxActiveClusters).  Leaves W.pkc_cluster = 0
// when any of this fails: the grid-wide persistent solve is used instead.
constexpr int64_t kPkcTargetRows = 128;

template <typename V>
egfem_status pkc_plan(egfem_t *h, KWork<V> &W) {
    W.pkc_cluster = 0;
    if (h->opts.krylov_cluster < 0 || !h->opts.krylov_persistent) return EGFEM_OK;
    int smem_optin = 0;
    EG_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const int64_t static_smem = 12288;  // the kernel's static shared memory (8.4 KB), rounded up
    const int mc = h->csf.max_cols;     // ELL columns of the shared-memory operator copy
    auto rows_max = [&](int op) { return (int64_t(smem_optin) - static_smem) / pkc_row_bytes<V>(op) / SLICE * SLICE; };
    auto rows_for = [&](int64_t c) { return (h->n_pad + c * SLICE - 1) / (c * SLICE) * SLICE; };
    int64_t c = h->opts.krylov_cluster > 0 ? h->opts.krylov_cluster : 1;
    if (h->opts.krylov_cluster == 0)
        while (c < PKC_MAX_CLUSTER && rows_for(c) > kPkcTargetRows) c *= 2;
    if (c > PKC_MAX_CLUSTER || rows_for(c) > rows_max(0)) return EGFEM_OK;
    const int64_t rows = rows_for(c);
    // the operator goes to shared memory when it fits (column codes hold 16-bit offsets)
    const int op = (mc <= 255 && rows <= 65535 && rows <= rows_max(mc)) ? mc : 0;
    const size_t smem = size_t((rows * pkc_row_bytes<V>(op) + 15) / 16 * 16);
    EG_CUDA(cudaFuncSetAttribute((const void *)pkc_solve<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    EG_CUDA(cudaFuncSetAttribute((const void *)pkc_solve<V>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(c); attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(unsigned(c)); cfg.blockDim = dim3(PKC_BLOCK); cfg.dynamicSmemBytes = smem;
    cfg.stream = h->hs; cfg.attrs = attr; cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (const void *)pkc_solve<V>, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return EGFEM_OK;
    }
    W.pkc_cluster = int(c);
    W.pkc_rows = int32_t(rows);
    W.pkc_op = op;
    W.pkc_smem = smem;
    return EGFEM_OK;
}

template <typename V>
egfem_status launch_pkc(egfem_t *h, KWork<V> &W, double rtol, int32_t maxit, int32_t stall,
                        const uint8_t *active = nullptr, const double *rtol_ptr = nullptr) {
    PkcArgs<V> P{};
    P.K = kvecs(h, W);
    P.st = h->st; P.n_pad = h->n_pad; P.rows_cta = W.pkc_rows; P.op_cols = W.pkc_op;
    P.rtol = rtol; P.maxit = maxit; P.stall = stall; P.active = active; P.rtol_ptr = rtol_ptr;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(W.pkc_cluster); attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(unsigned(W.pkc_cluster)); cfg.blockDim = dim3(PKC_BLOCK);
    cfg.dynamicSmemBytes = W.pkc_smem;
    cfg.stream = h->hs; cfg.attrs = attr; cfg.numAttrs = 1;
    EG_CUDA(cudaLaunchKernelEx(&cfg, pkc_solve<V>, P));
    return EGFEM_OK;
}

// Windowed single-system solve plan: each tile's window (its rows and every column they touch)
// must fit the shared memory of a block while all W.pk_ntiles blocks stay resident; leaves
// W.pkw_smem = 0 (the five-barrier pk_solve1 is used) when it does not.
template <typename V>
egfem_status pkw_plan(egfem_t *h, KWork<V> &W) {
    W.pkw_smem = 0;
    if (W.pk_ntiles < 1 || W.pk_ntiles > PK1_MAXG) return EGFEM_OK;
    EG_TRY(dalloc(W.pkw_win, size_t(W.pk_ntiles)));
    pkw_window_kernel<V><<<unsigned(W.pk_ntiles), 256, 0, h->hs>>>(kvecs(h, W), h->n, W.pk_tiles, W.pkw_win);
    EG_CUDA(cudaGetLastError());
    std::vector<PkWin> win(size_t(W.pk_ntiles));
    EG_CUDA(cudaMemcpyAsync(win.data(), W.pkw_win, win.size() * sizeof(PkWin), cudaMemcpyDeviceToHost, h->hs));
    EG_CUDA(cudaStreamSynchronize(h->hs));
    // the halo rows cost their share of the window updates in every iteration: where they
    // outnumber a tile's own rows twice over (3D meshes in lexicographic order: a halo of one
    // grid plane on each side, 9 times the tile on the 64^3 Kuhn mesh), the five-barrier kernel
    // is faster (64^3, FP64: 98 against 70 Newton solves/s)
    // (against the nominal tile length: the last tile is shorter)
    int64_t wmax = 0, halo_max = 0, tile_len = 0;
    std::vector<BTile> tl(static_cast<size_t>(W.pk_ntiles));
    EG_CUDA(cudaMemcpy(tl.data(), W.pk_tiles, tl.size() * sizeof(BTile), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < win.size(); ++t) {
        wmax = std::max(wmax, win[t].hi - win[t].lo);
        halo_max = std::max(halo_max, (win[t].hi - win[t].lo) - (tl[t].r_end - tl[t].r_begin));
        tile_len = std::max(tile_len, tl[t].r_end - tl[t].r_begin);
    }
    if (halo_max > 2 * tile_len && W.pk_ntiles > 1) return EGFEM_OK;
    const size_t smem = std::max(size_t(wmax) * sizeof(V), PKW_STAGE_BYTES);
    int optin = 0;
    EG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (smem == 0 || smem + 4096 > size_t(optin)) return EGFEM_OK;
    EG_CUDA(cudaFuncSetAttribute((const void *)pkw_solve<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)pkw_solve<V>, PKW_BLOCK, smem) != cudaSuccess) {
        cudaGetLastError();
        return EGFEM_OK;
    }
    if (int64_t(nb) * h->sms < W.pk_ntiles) return EGFEM_OK;
    W.pkw_smem = smem;
    return EGFEM_OK;
}

// Windowed batched solve plan: tiles of 1024 to 4096 rows (about four per block, equal within an
// instance), each tile's window in shared memory with every block resident and a halo of at
// most twice the tile; leaves W.pkwb_smem = 0 (pk_solveb is used) when it does not fit.
template <typename V>
egfem_status pkwb_plan(egfem_t *h, KWork<V> &W) {
    W.pkwb_smem = 0;
    if (h->nb < 1) return EGFEM_OK;   // egfem_batch_build sets the layout after the first allocation
    W.pkwb_planned = true;
    if (!h->coop || h->opts.krylov_persistent != 1) return EGFEM_OK;
    int optin = 0;
    EG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const int64_t G0 = int64_t(PKWB_MIN_BLOCKS) * h->sms;
    const int64_t total = h->inst_off[h->nb];
    // rows per tile: about four tiles per block, 1 024 to 4 096 rows.  Tiles of 8 192 rows made an
    // iteration with every instance running 2-7 % faster (fewer tiles per block, smaller halos
    // relative to the tile), but once few instances still iterate each of them is spread over
    // half as many blocks, and the 256-instance P3 solve took 1.60 s against 1.54 s.
    const int64_t target = std::min<int64_t>(4096, std::max<int64_t>(1024, (total + 4 * G0 - 1) / (4 * G0)));
    std::vector<BTile> T;
    for (int32_t b = 0; b < h->nb; ++b) {
        const int64_t t0 = int64_t(T.size());
        const int64_t lo = h->inst_off[b], hi = h->inst_off[b + 1];
        const int64_t nt = std::max<int64_t>(1, (hi - lo + target - 1) / target);
        const int64_t rows = ((hi - lo + nt - 1) / nt + SLICE - 1) / SLICE * SLICE;
        for (int64_t r = lo; r < hi; r += rows) T.push_back(BTile{r, std::min(hi, r + rows), t0, b, 0});
        for (size_t q = size_t(t0); q < T.size(); ++q) T[q].ntiles_inst = int32_t(T.size() - size_t(t0));
    }
    const int64_t nt = int64_t(T.size());
    const int64_t G = std::min<int64_t>(G0, nt);
    if ((nt + G - 1) / G > PKWB_MAXT) return EGFEM_OK;
    for (void *q : {(void *)W.pkwb_tiles, (void *)W.pkwb_win, (void *)W.pkwb_part}) if (q) cudaFree(q);
    W.pkwb_tiles = nullptr; W.pkwb_win = nullptr; W.pkwb_part = nullptr;
    EG_TRY(upload(W.pkwb_tiles, T));
    EG_TRY(dalloc(W.pkwb_win, size_t(nt)));
    EG_TRY(dalloc(W.pkwb_part, size_t(4 * nt)));
    pkw_window_kernel<V><<<unsigned(nt), 256, 0, h->hs>>>(kvecs(h, W), h->n, W.pkwb_tiles, W.pkwb_win);
    EG_CUDA(cudaGetLastError());
    std::vector<PkWin> win(static_cast<size_t>(nt));
    EG_CUDA(cudaMemcpyAsync(win.data(), W.pkwb_win, win.size() * sizeof(PkWin), cudaMemcpyDeviceToHost, h->hs));
    EG_CUDA(cudaStreamSynchronize(h->hs));
    int64_t wmax = 0;
    for (size_t t = 0; t < win.size(); ++t) {
        const int64_t w = win[t].hi - win[t].lo, own = T[t].r_end - T[t].r_begin;
        wmax = std::max(wmax, w);
        if (w - own > 2 * own && T[t].ntiles_inst > 1) return EGFEM_OK;
    }
    const size_t smem = std::max(size_t(wmax) * sizeof(V), PKW_STAGE_BYTES);
    if (smem + 4096 > size_t(optin)) return EGFEM_OK;
    EG_CUDA(cudaFuncSetAttribute((const void *)pkwb_solve<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)pkwb_solve<V>, PKWB_BLOCK, smem) != cudaSuccess) {
        cudaGetLastError();
        return EGFEM_OK;
    }
    if (int64_t(nb) * h->sms < G) return EGFEM_OK;
    W.pkwb_ntiles = nt;
    W.pkwb_grid = int(G);
    W.pkwb_smem = smem;
    return EGFEM_OK;
}

template <typename V>
egfem_status kwork_alloc(egfem_t *h, KWork<V> &W) {
    if (W.ready) {
        if (h->nb > 0 && !W.pkwb_planned) EG_TRY(pkwb_plan<V>(h, W));
        return EGFEM_OK;
    }
    W.g_setup = one_wave<V>(h, (const void *)kry_setup<V>);
    W.g_v = one_wave<V>(h, (const void *)kry_v<V>);
    W.g_s = one_wave<V>(h, (const void *)kry_s<V>);
    W.g_t = one_wave<V>(h, (const void *)kry_t<V>);
    W.g_x = one_wave<V>(h, (const void *)kry_x<V>);
    W.g_p = one_wave<V>(h, (const void *)kry_p<V>);
    EG_TRY(dalloc(W.A, size_t(h->csf.n_colentries)));
    EG_CUDA(cudaMemset(W.A, 0, size_t(h->csf.n_colentries) * sizeof(*W.A)));
    V **vec[] = {&W.b, &W.x, &W.r, &W.rh, &W.p, &W.v, &W.s, &W.t, &W.p2, &W.v2};
    const int nvec = 10;
    for (int k = 0; k < nvec; ++k) {
        EG_TRY(dalloc(*vec[k], size_t(h->n_pad)));
        EG_CUDA(cudaMemset(*vec[k], 0, size_t(h->n_pad) * sizeof(V)));
    }
    if (h->coop) {
        // every block of a cooperative launch must be resident: at most occupancy x SMs; each
        // block owns one contiguous, slice-aligned tile of rows
        int nb = 0, nbb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)pk_solve1<V>, PK1_BLOCK, 0) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbb, (const void *)pk_solveb<V>, PKB_BLOCK, 0) == cudaSuccess &&
            std::min(nb, nbb) >= 1) {
            nb = std::min(nb, nbb);   // the grid of pk_solve1, which pk_solveb (more blocks per SM) also holds
            const int64_t min_rows = (int64_t(h->opts.krylov_block_rows > 0 ? h->opts.krylov_block_rows : kPkBlockRows) +
                                      SLICE - 1) / SLICE * SLICE;
            const int64_t g = std::max<int64_t>(1, std::min<int64_t>(int64_t(std::min(nb, 8)) * h->sms, h->n_pad / min_rows));
            const int64_t rows = (h->n_pad + g * SLICE - 1) / (g * SLICE) * SLICE;
            std::vector<BTile> T;
            for (int64_t r = 0; r < h->n_pad; r += rows) T.push_back(BTile{r, std::min(h->n_pad, r + rows), 0, 0, 0});
            for (BTile &t : T) t.ntiles_inst = int32_t(T.size());
            W.g_pk = int(g);
            W.pk_ntiles = int64_t(T.size());
            EG_TRY(upload(W.pk_tiles, T));
            EG_TRY(dalloc(W.pk_part, size_t(4 * W.pk_ntiles)));
            EG_TRY(dalloc(W.bar, 1));
            EG_CUDA(cudaMemset(W.bar, 0, sizeof(PGrid)));
            EG_TRY(pkw_plan<V>(h, W));
        }
    }
    EG_TRY(pkc_plan<V>(h, W));
    EG_TRY(pkwb_plan<V>(h, W));
    if constexpr (std::is_same<V, df64>::value) {
        W.g_vp = one_wave<V>(h, (const void *)kry_vp<V>);
        W.g_st = one_wave<V>(h, (const void *)kry_st<V>);
        W.g_xr = one_wave<V>(h, (const void *)kry_xr<V>);
    }
    W.ready = true;
    return EGFEM_OK;
}

template <typename V>
void enqueue_iterations(egfem_t *h, KWork<V> &W, int count, cudaStream_t s) {
    KVecs<V> K = kvecs(h, W);
    if constexpr (std::is_same<V, df64>::value) {
        // fused three-kernel iteration; count is even, so every chunk starts on buffer 0
        for (int it = 0; it < count; ++it) {
            V *pi = (it & 1) ? W.p2 : W.p, *vi = (it & 1) ? W.v2 : W.v;
            V *po = (it & 1) ? W.p : W.p2, *vo = (it & 1) ? W.v : W.v2;
            kry_vp<V><<<W.g_vp, KRY_BLOCK, 0, s>>>(K, po, vo, pi, vi);
            kry_st<V><<<W.g_st, KRY_BLOCK, 0, s>>>(K, vo);
            kry_xr<V><<<W.g_xr, KRY_BLOCK, 0, s>>>(K, po, vo);
        }
        return;
    }
    for (int it = 0; it < count; ++it) {
        kry_v<V><<<W.g_v, KRY_BLOCK, 0, s>>>(K);
        kry_s<V><<<W.g_s, KRY_BLOCK, 0, s>>>(K);
        kry_t<V><<<W.g_t, KRY_BLOCK, 0, s>>>(K);
        kry_x<V><<<W.g_x, KRY_BLOCK, 0, s>>>(K);
        kry_p<V><<<W.g_p, KRY_BLOCK, 0, s>>>(K);
    }
}

template <typename V>
int chunk_of(const egfem_t *h) {
    const int c = std::max(1, h->opts.graph_chunk);
    return std::is_same<V, df64>::value ? (c + 1) / 2 * 2 : c;   // fused iterations come in pairs
}

template <typename V>
egfem_status ensure_graph(egfem_t *h, KWork<V> &W) {
    const int chunk = chunk_of<V>(h);
    if (W.graph && W.graph_chunk == chunk) return EGFEM_OK;
    if (W.graph) { cudaGraphExecDestroy(W.graph); W.graph = nullptr; }
    cudaGraph_t g;
    EG_CUDA(cudaStreamBeginCapture(h->hs, cudaStreamCaptureModeThreadLocal));
    enqueue_iterations(h, W, chunk, h->hs);
    EG_CUDA(cudaStreamEndCapture(h->hs, &g));
    cudaError_t e = cudaGraphInstantiate(&W.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { g_last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e); return EGFEM_ERR_CUDA; }
    W.graph_chunk = chunk;
    return EGFEM_OK;
}

// Cooperative launch of pk_solveb over the given tiles and systems.
template <typename V>
egfem_status launch_pk(egfem_t *h, KWork<V> &W, int grid, const BTile *tiles, int64_t ntiles, KState *st, double *part,
                       const uint8_t *active, const double *rtol,
                       double rtol0, PGrid *bar, int32_t maxit, int32_t stall) {
    PkArgs<V> P{};
    P.K = kvecs(h, W);
    P.tiles = tiles; P.ntiles = ntiles; P.st = st; P.part = part;
    P.active = active; P.rtol = rtol; P.rtol0 = rtol0; P.bar = bar; P.maxit = maxit; P.stall = stall;
    void *args[] = {(void *)&P};
    EG_CUDA(cudaMemsetAsync(bar, 0, sizeof(PGrid), h->hs));
    EG_CUDA(cudaLaunchCooperativeKernel((const void *)pk_solveb<V>, dim3(grid), dim3(PKB_BLOCK), args, 0, h->hs));
    return EGFEM_OK;
}

// One system in one cooperative launch of pk_solve1 (one tile per block; every block keeps the
// solver state); active and rtol_ptr as for launch_pk with one system.
template <typename V>
egfem_status launch_pk1(egfem_t *h, KWork<V> &W, double rtol, int32_t maxit, int32_t stall, const uint8_t *active = nullptr,
                        const double *rtol_ptr = nullptr) {
    PkArgs<V> P{};
    P.K = kvecs(h, W);
    P.tiles = W.pk_tiles; P.ntiles = W.pk_ntiles; P.st = h->st;
    P.part = W.pk_part; P.active = active; P.rtol = rtol_ptr; P.rtol0 = rtol; P.bar = W.bar; P.maxit = maxit; P.stall = stall;
    if (W.pk_ntiles < 1 || W.pk_ntiles > PK1_MAXG)   // no rows, or more blocks than it sums: the general kernel
        return launch_pk(h, W, W.g_pk, W.pk_tiles, W.pk_ntiles, h->st, W.pk_part, active, rtol_ptr,
                         rtol, W.bar, maxit, stall);
    if (W.pkw_smem > 0 && h->opts.krylov_persistent != 2) {
        // two reductions per iteration, halo rows recomputed in shared-memory windows
        PkwArgs<V> Q{};
        Q.K = P.K; Q.p2 = W.p2; Q.v2 = W.v2; Q.tiles = W.pk_tiles; Q.win = W.pkw_win; Q.ntiles = W.pk_ntiles; Q.st = h->st;
        Q.part = W.pk_part; Q.active = active; Q.rtol = rtol_ptr; Q.rtol0 = rtol; Q.bar = W.bar; Q.n = h->n; Q.maxit = maxit;
        Q.stall = stall;
        void *qargs[] = {(void *)&Q};
        EG_CUDA(cudaMemsetAsync(W.bar, 0, sizeof(PGrid), h->hs));
        EG_CUDA(cudaLaunchCooperativeKernel((const void *)pkw_solve<V>, dim3(unsigned(W.pk_ntiles)), dim3(PKW_BLOCK), qargs,
                                            W.pkw_smem, h->hs));
        return EGFEM_OK;
    }
    void *args[] = {(void *)&P};
    EG_CUDA(cudaMemsetAsync(W.bar, 0, sizeof(PGrid), h->hs));
    // one block per tile (at most the resident grid W.g_pk)
    EG_CUDA(cudaLaunchCooperativeKernel((const void *)pk_solve1<V>, dim3(unsigned(W.pk_ntiles)), dim3(PK1_BLOCK), args, 0,
                                        h->hs));
    return EGFEM_OK;
}

template <typename V>
egfem_status launch_pk_single(egfem_t *h, KWork<V> &W, double rtol, int32_t maxit, int32_t stall) {
    if (W.pkc_cluster > 0) return launch_pkc<V>(h, W, rtol, maxit, stall);
    return launch_pk1<V>(h, W, rtol, maxit, stall);
}

// Run BiCGStab on W.A x = W.b (already filled) on the internal stream; returns the
// device-state outcome in *done and the iteration count in *iters.
template <typename V>
egfem_status run_bicgstab(egfem_t *h, KWork<V> &W, double rtol, int32_t maxit, int32_t stall, int32_t *done,
                          int32_t *iters) {
    if (h->opts.krylov_persistent && W.g_pk > 0) {
        // the whole solve in one cooperative launch
        EG_TRY(launch_pk_single(h, W, rtol, maxit, stall));
        EG_CUDA(cudaMemcpyAsync(h->h_st, h->st, sizeof(KState), cudaMemcpyDeviceToHost, h->hs));
        PGrid gb{};
        EG_CUDA(cudaMemcpyAsync(&gb, W.bar, sizeof(PGrid), cudaMemcpyDeviceToHost, h->hs));
        EG_CUDA(cudaStreamSynchronize(h->hs));
        h->last_graph_launches = 0;
        h->last_graph_nodes = 0;
        h->last_krylov_kernels = 1;
        *done = h->h_st->done;
        *iters = h->h_st->iter;
        if (gb.err) {
            g_last_error = gb.err == 2 ? "BiCGStab: more tiles than the persistent solve holds per block"
                                       : "BiCGStab: a grid-barrier wait of the persistent solve ran out";
            return gb.err == 2 ? EGFEM_ERR_INVALID_ARG : EGFEM_ERR_TIMEOUT;
        }
        return EGFEM_OK;
    }
    EG_TRY(ensure_graph(h, W));
    KVecs<V> K = kvecs(h, W);
    kry_setup<V><<<W.g_setup, KRY_BLOCK, 0, h->hs>>>(K, rtol, maxit, stall);
    EG_CUDA(cudaGetLastError());
    h->last_graph_launches = 0;
    h->last_graph_nodes = int64_t(std::is_same<V, df64>::value ? 3 : 5) * chunk_of<V>(h);
    for (;;) {
        EG_CUDA(cudaMemcpyAsync(h->h_st, h->st, sizeof(KState), cudaMemcpyDeviceToHost, h->hs));
        EG_CUDA(cudaStreamSynchronize(h->hs));
        if (h->h_st->done != K_RUNNING) break;
        EG_CUDA(cudaGraphLaunch(W.graph, h->hs));
        ++h->last_graph_launches;
    }
    h->last_krylov_kernels = 1 + h->last_graph_launches * h->last_graph_nodes;
    *done = h->h_st->done;
    *iters = h->h_st->iter;
    return EGFEM_OK;
}

egfem_status join_in(egfem_t *h, cudaStream_t user) {
    EG_CUDA(cudaEventRecord(h->ev_in, user));
    EG_CUDA(cudaStreamWaitEvent(h->hs, h->ev_in, 0));
    return EGFEM_OK;
}

egfem_status join_out(egfem_t *h, cudaStream_t user) {
    EG_CUDA(cudaEventRecord(h->ev_out, h->hs));
    EG_CUDA(cudaStreamWaitEvent(user, h->ev_out, 0));
    return EGFEM_OK;
}

egfem_status norm2_free(egfem_t *h, const double *r, double *out_host) {
    norm2_free_kernel<<<h->kgrid, KRY_BLOCK, 0, h->hs>>>(h->n, r, h->csf.dir, h->part, h->ticket, h->scal);
    EG_CUDA(cudaGetLastError());
    EG_CUDA(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->hs));
    EG_CUDA(cudaStreamSynchronize(h->hs));
    *out_host = h->h_scal[0];
    return EGFEM_OK;
}

egfem_status check_status_word(egfem_t *h) {
    int32_t s = 0;
    EG_CUDA(cudaMemcpyAsync(&s, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->hs));
    EG_CUDA(cudaStreamSynchronize(h->hs));
    if (s & 1) { g_last_error = "zero diagonal in the Jacobian"; return EGFEM_ERR_SINGULAR; }
    return EGFEM_OK;
}

template <typename T>
void dfree(T *&p) { if (p) cudaFree((void *)p); p = nullptr; }

// Local nodes of the degree-p Lagrange W space on the reference cell, in the W numbering's
// local order (vertices; edge nodes from the lower to the higher local vertex; face centroids),
// with iota_l = int_K eta_l / |K| and mu_la = int_K lambda_a eta_l / |K|.  mu comes from the
// expansion eta_alpha = prod_j prod_{i < alpha_j} (p lambda_j - i) / (i + 1) integrated
// monomial by monomial, int_K lambda^beta / |K| = d! beta! / (|beta| + d)!.
egfem_status lagrange_local(int d, int p, MfLocal &L) {
    const int nv = d + 1;
    int count = 1;                                  // C(p + d, d) nodes
    for (int i = 1; i <= d; ++i) count = count * (p + i) / i;
    if (count > MF_MAXW) { g_last_error = "element-local operator supports at most 10 local W nodes"; return EGFEM_ERR_UNSUPPORTED; }
    auto fact = [](int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; };
    auto add = [&](const int *alpha, int kind) {
        // eta as a dense polynomial in (lambda_0..lambda_3), exponents 0..4 each
        std::vector<double> poly(625, 0.0), next(625);
        poly[0] = 1.0;
        for (int j = 0; j < nv; ++j)
            for (int i = 0; i < alpha[j]; ++i) {
                std::fill(next.begin(), next.end(), 0.0);
                const int step = (j == 0 ? 1 : j == 1 ? 5 : j == 2 ? 25 : 125);
                for (int e = 0; e < 625; ++e) {
                    if (poly[e] == 0.0) continue;
                    next[e + step] += poly[e] * double(p) / double(i + 1);
                    next[e] -= poly[e] * double(i) / double(i + 1);
                }
                poly.swap(next);
            }
        const int l = L.nw++;
        for (int a = 0; a < 4; ++a) L.w[l][a] = a < nv ? double(alpha[a]) / double(p) : 0.0;
        L.iota[l] = basis_integral(d, p, kind);
        // int_K lambda^beta / |K| for beta = e + extra (exponent vectors)
        auto moment = [&](int a, int b) {
            double m = 0.0;
            for (int e = 0; e < 625; ++e) {
                if (poly[e] == 0.0) continue;
                int ex[4] = {e % 5, (e / 5) % 5, (e / 25) % 5, e / 125};
                if (a >= 0) ex[a] += 1;
                if (b >= 0) ex[b] += 1;
                double num = fact(d);
                int tot = 0;
                for (int j = 0; j < nv; ++j) { num *= fact(ex[j]); tot += ex[j]; }
                m += poly[e] * num / fact(tot + d);
            }
            return m;
        };
        for (int a = 0; a < 4; ++a) {
            L.mu[l][a] = a < nv ? moment(a, -1) : 0.0;
            for (int b = 0; b < 4; ++b) L.mu3[l][a][b] = (a < nv && b < nv) ? moment(a, b) : 0.0;
        }
    };
    for (int a = 0; a < nv; ++a) { int al[4] = {0, 0, 0, 0}; al[a] = p; add(al, W_VERTEX); }
    for (int a = 0; a < nv && p >= 2; ++a)
        for (int b = a + 1; b < nv; ++b)
            for (int t = 1; t < p; ++t) { int al[4] = {0, 0, 0, 0}; al[a] = p - t; al[b] = t; add(al, p == 2 ? W_MID : W_THIRD); }
    if (p == 3)
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                for (int e = b + 1; e < nv; ++e) { int al[4] = {0, 0, 0, 0}; al[a] = al[b] = al[e] = 1; add(al, W_FACE); }
    return EGFEM_OK;
}

// share_k > 1: the mesh is the disjoint union of share_k copies of one mesh of share_rows rows
// (egfem_batch_build), whose tensor is then stored once when the copies' entries agree.
egfem_status build_impl(const egfem_mesh *mesh, const egfem_problem *prob, const egfem_options *opts, egfem_handle *out,
                        int32_t share_k = 0, int64_t share_rows = 0) {
    if (!mesh || !prob || !out) { g_last_error = "null argument"; return EGFEM_ERR_INVALID_ARG; }
    *out = nullptr;
    std::string err;
    egfem_status st = validate_mesh(*mesh, err);
    if (st != EGFEM_OK) { g_last_error = err; return st; }
    auto check_g = [&](int32_t kind, double p, int32_t deg, const char *what) -> egfem_status {
        if (kind < EGFEM_G_NONE || kind > EGFEM_G_GRADPOW) { g_last_error = std::string(what) + ": unknown kind"; return EGFEM_ERR_INVALID_ARG; }
        if (kind == EGFEM_G_POW && (p < 1 || p > 8 || p != std::floor(p))) { g_last_error = std::string(what) + ": exponent must be an integer in 1..8"; return EGFEM_ERR_INVALID_ARG; }
        if (kind == EGFEM_G_GRADPOW) return EGFEM_OK;
        if (kind != EGFEM_G_NONE && (deg < 1 || deg > 3)) { g_last_error = std::string(what) + ": degree must be 1, 2 or 3"; return EGFEM_ERR_INVALID_ARG; }
        return EGFEM_OK;
    };
    if ((prob->a_space != EGFEM_W_LAGRANGE && prob->a_space != EGFEM_W_QUADRATURE) ||
        (prob->c_space != EGFEM_W_LAGRANGE && prob->c_space != EGFEM_W_QUADRATURE)) {
        g_last_error = "unknown W space kind";
        return EGFEM_ERR_INVALID_ARG;
    }
    // quadrature spaces I_k: the rule's point count (0: no such rule)
    double qa_bary[6][4], qa_w[6], qc_bary[6][4], qc_w[6];
    const bool quad_a = prob->a_space == EGFEM_W_QUADRATURE && prob->a_kind != EGFEM_G_NONE;
    const bool quad_c = prob->c_space == EGFEM_W_QUADRATURE && prob->c_kind != EGFEM_G_NONE;
    const int nqa = quad_a ? quad_rule(mesh->dim, prob->a_degree, qa_bary, qa_w) : 0;
    const int nqc = quad_c ? quad_rule(mesh->dim, prob->c_degree, qc_bary, qc_w) : 0;
    if ((quad_a && nqa == 0) || (quad_c && nqc == 0)) {
        g_last_error = "quadrature space I_k: k must be 1..4 on triangles, 1..3 on tetrahedra";
        return EGFEM_ERR_INVALID_ARG;
    }
    if (!quad_a) EG_TRY(check_g(prob->a_kind, prob->a_p, prob->a_degree, "a"));
    else if (prob->a_kind < EGFEM_G_NONE || prob->a_kind > EGFEM_G_GRADPOW ||
             (prob->a_kind == EGFEM_G_POW && (prob->a_p < 1 || prob->a_p > 8 || prob->a_p != std::floor(prob->a_p)))) {
        g_last_error = "a: unknown kind or exponent";
        return EGFEM_ERR_INVALID_ARG;
    }
    if (!quad_c) {
        EG_TRY(check_g(prob->c_kind, prob->c_p, prob->c_degree, "c"));
    } else if (prob->c_kind < EGFEM_G_NONE || prob->c_kind > EGFEM_G_EXP ||
               (prob->c_kind == EGFEM_G_POW && (prob->c_p < 1 || prob->c_p > 8 || prob->c_p != std::floor(prob->c_p)))) {
        g_last_error = "c: unknown kind or exponent";
        return EGFEM_ERR_INVALID_ARG;
    }
    if (prob->c_kind == EGFEM_G_GRADPOW) { g_last_error = "c: the gradient nonlinearity is a coefficient"; return EGFEM_ERR_INVALID_ARG; }
    const bool gradc = prob->a_kind == EGFEM_G_GRADPOW;
    // a Lagrange W_c of degree 2 or 3 (evaluated by the element-local operator)
    const bool lag_c = !quad_c && prob->c_kind != EGFEM_G_NONE && (prob->c_degree > 1 || prob->c_product);
    if (prob->c_product && prob->c_kind == EGFEM_G_NONE) { g_last_error = "c_product needs a reaction nonlinearity"; return EGFEM_ERR_INVALID_ARG; }
    if (!std::isfinite(prob->sigma)) { g_last_error = "sigma must be finite"; return EGFEM_ERR_INVALID_ARG; }
    if (gradc) {
        // (shift + s)^q on s = ||grad u||^2 >= 0: finite with its derivative at s = 0 when
        // shift > 0, or when shift = 0 and q is 0 or at least 1
        const double q = prob->a_p, sh = prob->a_shift;
        if (!quad_a && prob->a_degree != 0) { g_last_error = "a: the gradient coefficient lives in W_a = P0 (a_degree 0) or I_k"; return EGFEM_ERR_INVALID_ARG; }
        if (!std::isfinite(q) || !std::isfinite(sh) || sh < 0.0 || (sh == 0.0 && q != 0.0 && q < 1.0)) {
            g_last_error = "a: gradient exponent/shift must give a finite (shift + s)^q and derivative at s = 0";
            return EGFEM_ERR_INVALID_ARG;
        }
    }
    std::unique_ptr<egfem_t> h(new egfem_t());
    egfem_default_options(&h->opts);
    if (opts) h->opts = *opts;
    if (h->opts.precision != EGFEM_PREC_FP64 && h->opts.precision != EGFEM_PREC_MIXED) { g_last_error = "bad precision"; return EGFEM_ERR_INVALID_ARG; }
    if (h->opts.op != EGFEM_OP_CSF && h->opts.op != EGFEM_OP_MATRIX_FREE) { g_last_error = "unknown operator variant"; return EGFEM_ERR_INVALID_ARG; }
    if ((gradc || quad_a || quad_c || lag_c || prob->sigma != 0.0 || prob->c_product) && h->opts.op != EGFEM_OP_MATRIX_FREE) {
        // the P0 and I_k forms are multiples of the cell stiffness S^K, and the reaction forms
        // on I_k or P2/P3 and the linear mass term are per-cell products: the element-local
        // operator evaluates them without a stored tensor
        g_last_error = "the gradient coefficient, quadrature spaces, W_c of degree > 1 and sigma need the element-local operator (EGFEM_OP_MATRIX_FREE)";
        return EGFEM_ERR_UNSUPPORTED;
    }
    h->prob = *prob;
    h->dim = mesh->dim; h->n = mesh->n_nodes; h->ncells = mesh->n_cells;
    EG_CUDA(cudaGetDevice(&h->device));
    EG_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
    int coop = 0;
    EG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    h->coop = coop != 0;
    // W spaces
    HostWSpace Wa, Wc;
    std::vector<int32_t> c2wa, c2wc;
    int nla = 0, nlc = 0;
    // With the gradient coefficient or a quadrature space the stored CSF is that of the
    // constant coefficient (without that reaction): it fixes the Jacobian's pattern and the
    // Krylov layout (both the P1 graph), while the element-local kernels evaluate the
    // nonlinearity on its own space.
    egfem_problem layout_prob = *prob;
    const bool mf_a = gradc || quad_a;
    if (mf_a) { layout_prob.a_kind = EGFEM_G_NONE; layout_prob.a_degree = 1; }
    const bool mf_c = quad_c || lag_c;
    if (mf_c) { layout_prob.c_kind = EGFEM_G_NONE; layout_prob.c_degree = 1; }
    st = build_wspace(*mesh, layout_prob.a_kind != EGFEM_G_NONE ? layout_prob.a_degree : 1, Wa, c2wa, nla, err);
    if (st != EGFEM_OK) { g_last_error = err; return st; }
    st = build_wspace(*mesh, layout_prob.c_kind != EGFEM_G_NONE ? layout_prob.c_degree : 1, Wc, c2wc, nlc, err);
    if (st != EGFEM_OK) { g_last_error = err; return st; }
    h->nwa = Wa.n; h->nwc = Wc.n;
    h->wa_coords = Wa.coords; h->wc_coords = Wc.coords;
    if (quad_a) { h->nwa = mesh->n_cells * nqa; h->wa_coords = quad_points(*mesh, nqa, qa_bary); }   // W_a = I_k
    else if (gradc) { h->nwa = mesh->n_cells; h->wa_coords = cell_centroids(*mesh); }             // W_a = P0
    if (quad_c) { h->nwc = mesh->n_cells * nqc; h->wc_coords = quad_points(*mesh, nqc, qc_bary); }  // W_c = I_k
    if (lag_c) {                                                                                 // W_c = P2, P3
        HostWSpace Wh;
        std::vector<int32_t> c2wh;
        int nlh = 0;
        st = build_wspace(*mesh, prob->c_degree, Wh, c2wh, nlh, err);
        if (st != EGFEM_OK) { g_last_error = err; return st; }
        h->nwc = Wh.n; h->wc_coords = Wh.coords;
    }
    HostCSF H;
    st = build_csf(*mesh, layout_prob, Wa, c2wa, nla, Wc, c2wc, nlc, H, err);
    if (st != EGFEM_OK) { g_last_error = err; return st; }
    h->maxc_tpl = pick_maxc(H.max_cols);
    // transpose map: SELL position of (k, i) for every (i, local column c -> k)
    std::vector<int64_t> tmap(H.col_idx.size(), -1);
    {
        const int64_t n = H.n_rows;
        for (int32_t s = 0; s < H.n_slices; ++s) {
            const SliceMeta &M = H.meta[s];
            for (int c = 0; c < M.ncol; ++c)
                for (int r = 0; r < SLICE; ++r) {
                    const int64_t i = int64_t(s) * SLICE + r;
                    if (i >= n) continue;
                    const int64_t q = M.col_base + int64_t(c) * SLICE + r;
                    const int32_t k = H.col_idx[q];
                    if (H.col_slot[q] < 0 && c != 0) continue;
                    const SliceMeta &Mk = H.meta[k / SLICE];
                    const int rk = k % SLICE;
                    for (int ck = 0; ck < Mk.ncol; ++ck) {
                        const int64_t qk = Mk.col_base + int64_t(ck) * SLICE + rk;
                        if (H.col_idx[qk] == i) { tmap[q] = qk; break; }
                    }
                }
        }
    }
    if (share_k > 1 && h->opts.batch_share) share_tensor(H, share_k, share_rows, h->ws);   // else h->ws.k stays 0
    DeviceCSF &D = h->csf;
    D.n_rows = H.n_rows; D.n_slices = H.n_slices; D.max_cols = H.max_cols;
    D.n_colentries = int64_t(H.col_idx.size()); D.n_leaves = int64_t(H.leaf_val.size());
    D.n_fibres = int64_t(H.fib_info.size()); D.n_rx = int64_t(H.rx_val.size()); D.nnz = H.rowptr.back();
    EG_TRY(upload(D.meta, H.meta));
    EG_TRY(upload(D.col_idx, H.col_idx)); EG_TRY(upload(D.col_slot, H.col_slot));
    EG_TRY(upload(D.slice_off, H.slice_off.empty() ? std::vector<int32_t>(1, 0) : H.slice_off));
    for (const SliceMeta &M : H.meta) D.n_uniform += M.off_base >= 0;
    EG_TRY(upload(D.leaf_val, H.leaf_val)); EG_TRY(upload(D.leaf_col, H.leaf_col));
    EG_TRY(upload(D.fib_info, H.fib_info)); EG_TRY(upload(D.fib_tdiag, H.fib_tdiag)); EG_TRY(upload(D.fib_m, H.fib_m));
    EG_TRY(upload(D.rx_val, H.rx_val)); EG_TRY(upload(D.rx_info, H.rx_info)); EG_TRY(upload(D.rx_m, H.rx_m));
    EG_TRY(upload(D.dir, H.dir)); EG_TRY(upload(D.rowptr, H.rowptr)); EG_TRY(upload(D.cols, H.cols));
    EG_TRY(upload(h->tmap, tmap));
    EG_TRY(upload(h->wa_kind, Wa.kind)); EG_TRY(upload(h->wa_sup, Wa.sup));
    if (prob->a_kind != EGFEM_G_NONE && !mf_a) { EG_TRY(dalloc(h->wa_val, size_t(h->nwa))); EG_TRY(dalloc(h->wa_gp, size_t(h->nwa))); }
    if (prob->c_kind != EGFEM_G_NONE && !mf_c) {
        EG_TRY(upload(h->wc_kind, Wc.kind)); EG_TRY(upload(h->wc_sup, Wc.sup));
        EG_TRY(dalloc(h->wc_val, size_t(h->nwc))); EG_TRY(dalloc(h->wc_gp, size_t(h->nwc)));
    }
    // cells and vertex -> cell incidence for the load vector
    {
        const int nv = mesh->dim + 1;
        std::vector<int32_t> cv(mesh->cells, mesh->cells + mesh->n_cells * nv);
        std::vector<double> vol, S;
        const bool mf = h->opts.op == EGFEM_OP_MATRIX_FREE;
        cell_stiffness(*mesh, vol, mf ? &S : nullptr);
        std::vector<int64_t> ptr(mesh->n_nodes + 1, 0);
        for (int64_t c = 0; c < mesh->n_cells; ++c) for (int a = 0; a < nv; ++a) ptr[cv[c * nv + a] + 1]++;
        for (int64_t v = 0; v < mesh->n_nodes; ++v) ptr[v + 1] += ptr[v];
        std::vector<int32_t> lst(ptr.back());
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t c = 0; c < mesh->n_cells; ++c) for (int a = 0; a < nv; ++a) lst[fill[cv[c * nv + a]]++] = int32_t(c);
        EG_TRY(upload(h->cell_verts, cv)); EG_TRY(upload(h->cell_vol, vol));
        EG_TRY(upload(h->v2c_ptr, ptr)); EG_TRY(upload(h->v2c, lst));
        if (mf) {
            // per cell: S^K = |K| grad lambda_a . grad lambda_b (packed upper triangle)
            const int d = mesh->dim;
            EG_TRY(upload(h->cell_S, S));
            h->mf_ne = 2 * d + 3 + (mf_c ? (d + 1) + (d + 1) * (d + 1) : 0);
            EG_TRY(dalloc(h->cell_E, size_t(mesh->n_cells) * size_t(h->mf_ne)));
            // local W nodes of the reference cell in the W numbering's local order
            MfLocal &L = h->mf_loc;
            L = MfLocal{};
            if (quad_a && !gradc) {
                // I_k: the rule's points and weights (w_l / |K|, summing to 1)
                for (int l = 0; l < nqa; ++l) {
                    for (int a = 0; a < 4; ++a) L.w[l][a] = a < nv ? qa_bary[l][a] : 0.0;
                    L.iota[l] = qa_w[l];
                }
                L.nw = nqa;
            } else if (prob->a_kind != EGFEM_G_NONE && !gradc) {
                EG_TRY(lagrange_local(d, prob->a_degree, L));
            }
            MfLocal &Lc = h->mf_loc_c;
            Lc = MfLocal{};
            if (quad_c) {
                // I_k: M_al / |K| = (w_l / |K|) lambda_a(x_l)
                for (int l = 0; l < nqc; ++l) {
                    for (int a = 0; a < 4; ++a) {
                        Lc.w[l][a] = a < nv ? qc_bary[l][a] : 0.0;
                        Lc.mu[l][a] = qc_w[l] * Lc.w[l][a];
                    }
                    for (int a = 0; a < 4; ++a)
                        for (int b = 0; b < 4; ++b) Lc.mu3[l][a][b] = qc_w[l] * Lc.w[l][a] * Lc.w[l][b];
                    Lc.iota[l] = qc_w[l];
                }
                Lc.nw = nqc;
            } else if (lag_c) {
                EG_TRY(lagrange_local(d, prob->c_degree, Lc));
            }
        }
    }
    h->nl.a_kind = prob->a_kind; h->nl.a_pi = gradc ? 0 : int32_t(prob->a_p); h->nl.a_scale = prob->a_scale;
    h->nl.a_preal = prob->a_p; h->nl.a_shift = gradc ? prob->a_shift : 0.0;
    h->nl.c_kind = prob->c_kind; h->nl.c_pi = int32_t(prob->c_p); h->nl.c_scale = prob->c_scale;
    h->nl.gamma = prob->gamma; h->nl.kappa = prob->kappa; h->nl.kappa_field = nullptr;
    h->nl.sigma = prob->sigma;
    h->nl.c_product = prob->c_product ? 1 : 0;
    // workspace
    h->n_pad = int64_t(H.n_slices) * SLICE;
    auto grid_for = [&](int64_t per_block) {
        return int(std::max<int64_t>(1, std::min<int64_t>((h->n_pad + per_block - 1) / per_block, int64_t(h->sms) * 8)));
    };
    h->kgrid = grid_for(KRY_BLOCK);
    h->kgrid64 = grid_for(KRY_BLOCK * VecT<double>::R);
    h->kgrid32 = grid_for(KRY_BLOCK * VecT<float>::R);
    EG_TRY(dalloc(h->r, size_t(h->n)));
    EG_TRY(dalloc(h->part, size_t(2 * std::max<int64_t>(int64_t(h->sms) * 8, std::max(h->kgrid, std::max(h->kgrid64, h->kgrid32))))));
    EG_TRY(dalloc(h->scal, 8));
    EG_TRY(dalloc(h->ticket, 1)); EG_CUDA(cudaMemset(h->ticket, 0, sizeof(uint32_t)));
    EG_TRY(dalloc(h->status, 1)); EG_CUDA(cudaMemset(h->status, 0, sizeof(int32_t)));
    EG_TRY(dalloc(h->st, 1)); EG_CUDA(cudaMemset(h->st, 0, sizeof(KState)));
    EG_CUDA(cudaMallocHost((void **)&h->h_st, sizeof(KState)));
    EG_CUDA(cudaMallocHost((void **)&h->h_scal, 8 * sizeof(double)));
    EG_CUDA(cudaStreamCreateWithFlags(&h->hs, cudaStreamNonBlocking));
    EG_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    EG_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    if (h->opts.precision == EGFEM_PREC_MIXED) EG_TRY(kwork_alloc(h.get(), h->k32));
    else EG_TRY(kwork_alloc(h.get(), h->k64));
    EG_CUDA(cudaDeviceSynchronize());
    *out = h.release();
    return EGFEM_OK;
}

}  // namespace

namespace {

// Single-system graph Newton loop (egfem_gnewton.cuh with one instance): the body is the
// controller, the persistent or cluster BiCGStab with its tolerance and activity read from
// device memory, the controller, u -= x, the tensor action and the free-row norm, the
// controller and the revert.  Kept for later calls with the same vectors and path.
template <typename V>
egfem_status gn_build_one(egfem_t *h, KWork<V> &W, double *d_u, const double *d_d) {
    constexpr bool mixed = std::is_same<V, df64>::value;
    if (h->gn_exec && h->gn_u == d_u && h->gn_d == d_d && h->gn_mixed == int(mixed) && h->gn_one == 1) return EGFEM_OK;
    if (h->gn_exec) { cudaGraphExecDestroy(h->gn_exec); h->gn_exec = nullptr; }
    if (h->nb > 0) return EGFEM_ERR_UNSUPPORTED;   // a batch handle solves through the batched loop
    if (!h->gn_state) {
        EG_TRY(dalloc(h->gn_state, 1));
        EG_TRY(dalloc(h->gn_stats, 1));
        EG_TRY(dalloc(h->gn_loops, 1));
        EG_TRY(dalloc(h->inst_mask, 1));
        EG_TRY(dalloc(h->inst_eta, 1));
        EG_TRY(dalloc(h->inst_lam, 1));
    }
    if (!W.bar && W.pkc_cluster == 0) return EGFEM_ERR_UNSUPPORTED;
    cudaGraph_t g = nullptr;
    EG_CUDA(cudaGraphCreate(&g, 0));
    cudaError_t e = cudaSuccess;
    cudaGraphConditionalHandle cond{};
    cudaGraphNodeParams np{};
    cudaGraphNode_t node = nullptr;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->hs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        g_last_error = std::string("graph Newton loop: ") + cudaGetErrorString(e);
        return EGFEM_ERR_CUDA;
    }
    GNArgs G{};
    G.nb = 1; G.state = h->gn_state; G.stats = h->gn_stats; G.mask = h->inst_mask; G.eta_out = h->inst_eta;
    G.lam = h->inst_lam; G.kst = h->st; G.norm2 = h->scal; G.loops = h->gn_loops;
    G.kerr = W.pkc_cluster > 0 ? nullptr : &W.bar->err;
    G.max_loops = gn_max_loops(h->opts.newton_maxit); G.newton_maxit = h->opts.newton_maxit;
    G.fixed_eta = h->opts.fixed_eta; G.mixed = int(mixed);
    G.eta_max = eta_cap(h); G.eta_min = h->opts.eta_min; G.eta_floor = mixed ? kMixedEtaFloor : 0.0; G.cond = cond;
    const unsigned gu = unsigned((h->n + 255) / 256);
    const int32_t stall = mixed ? kMixedStall : 0;
    int nodes = 0;
    egfem_status st = EGFEM_OK;
    gn_pre<<<1, 32, 0, h->hs>>>(G);
    if (W.pkc_cluster > 0) st = launch_pkc<V>(h, W, 0.0, h->opts.krylov_maxit, stall, h->inst_mask, h->inst_eta);
    else st = launch_pk1<V>(h, W, 0.0, h->opts.krylov_maxit, stall, h->inst_mask, h->inst_eta);
    gn_mid<<<1, 32, 0, h->hs>>>(G);
    gn_update_one<V><<<gu, 256, 0, h->hs>>>(h->n, h->inst_mask, h->inst_lam, d_u, W.x);
    CsfArgs A = csf_args(h, d_u, d_d);
    A.r = h->r; A.q64 = h->k64.b;
    if (mixed) A.a32 = h->k32.A;
    else A.a64 = h->k64.A;
    nodes += launch_csf(h, A, h->hs);
    if (mixed) { cast_kernel<double, df64><<<gu, 256, 0, h->hs>>>(h->n, h->k64.b, h->k32.b); ++nodes; }
    norm2_free_kernel<<<h->kgrid, KRY_BLOCK, 0, h->hs>>>(h->n, h->r, h->csf.dir, h->part, h->ticket, h->scal);
    gn_post<<<1, 32, 0, h->hs>>>(G);
    gn_update_one<V><<<gu, 256, 0, h->hs>>>(h->n, h->inst_mask, h->inst_lam, d_u, W.x);
    nodes += 7;
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(h->hs, &body);
    if (st == EGFEM_OK && e == cudaSuccess) e = cudaGetLastError();
    if (st == EGFEM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->gn_exec, g, 0);
    cudaGraphDestroy(g);
    if (st != EGFEM_OK || e != cudaSuccess) {
        if (e != cudaSuccess) g_last_error = std::string("graph Newton loop: ") + cudaGetErrorString(e);
        cudaGetLastError();
        h->gn_exec = nullptr;
        return st != EGFEM_OK ? st : EGFEM_ERR_CUDA;
    }
    h->gn_u = d_u; h->gn_d = d_d; h->gn_mixed = int(mixed); h->gn_nodes = nodes; h->gn_one = 1;
    return EGFEM_OK;
}

// Run it from the host driver's state after the first evaluation; false when unavailable.  On a
// hand-back (handed_back) the current step awaits its FP64 redo: rbefore is its starting norm
// and eta its forcing term.
template <typename V>
bool gn_run_one(egfem_t *h, KWork<V> &W, double *d_u, const double *d_d, double &rn, double &rprev, double &eta,
                double target, egfem_stats &S, bool &handed_back, double &rbefore) {
    handed_back = false;
    if (!h->opts.newton_graph || h->gn_failed || !h->opts.krylov_persistent || h->nb > 0) return false;
    if (W.g_pk <= 0 && W.pkc_cluster <= 0) return false;
    if (gn_build_one<V>(h, W, d_u, d_d) != EGFEM_OK) { h->gn_failed = true; return false; }
    GNState G{rn, rprev, rn, target, eta, 1.0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h->gn_state, &G, sizeof(GNState), cudaMemcpyHostToDevice, h->hs) != cudaSuccess ||
        cudaMemcpyAsync(h->gn_stats, &S, sizeof(egfem_stats), cudaMemcpyHostToDevice, h->hs) != cudaSuccess ||
        cudaMemsetAsync(h->gn_loops, 0, sizeof(int32_t), h->hs) != cudaSuccess ||
        cudaGraphLaunch(h->gn_exec, h->hs) != cudaSuccess) {
        cudaGetLastError();
        h->gn_failed = true;
        return false;
    }
    int32_t loops = 0;
    cudaMemcpyAsync(&G, h->gn_state, sizeof(GNState), cudaMemcpyDeviceToHost, h->hs);
    cudaMemcpyAsync(&S, h->gn_stats, sizeof(egfem_stats), cudaMemcpyDeviceToHost, h->hs);
    cudaMemcpyAsync(&loops, h->gn_loops, sizeof(int32_t), cudaMemcpyDeviceToHost, h->hs);
    if (cudaStreamSynchronize(h->hs) != cudaSuccess) return true;   // the caller's next CUDA call reports it
    rn = G.rn; rprev = G.rprev; eta = G.eta; rbefore = G.rbefore;
    handed_back = G.host != 0;
    S.kernel_launches += int64_t(loops) * h->gn_nodes;
    h->gn_used = true;
    return true;
}

}  // namespace

extern "C" {

egfem_status egfem_selftest_grid_barrier(int32_t blocks, int32_t arrive, double wait_ms, int32_t *ok_host,
                                         int32_t *err_host) {
    if (blocks < 1 || blocks > 64 || arrive < 0 || arrive > blocks || !(wait_ms > 0.0) || wait_ms > 2000.0 || !ok_host) {
        g_last_error = "selftest_grid_barrier: blocks in 1..64, arrive in 0..blocks, 0 < wait_ms <= 2000, ok_host set";
        return EGFEM_ERR_INVALID_ARG;
    }
    PGrid *g = nullptr;
    int32_t *ok = nullptr;
    EG_TRY(dalloc(g, 1));
    egfem_status st = EGFEM_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
        st = EGFEM_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc((void **)&ok, sizeof(int32_t) * size_t(blocks));
    if (e != cudaSuccess) fail(e, "cudaMalloc");
    if (st == EGFEM_OK && (e = cudaMemset(g, 0, sizeof(PGrid))) != cudaSuccess) fail(e, "cudaMemset");
    if (st == EGFEM_OK) {
        unsigned long long limit = (unsigned long long)(wait_ms * 1e6);
        if (arrive == blocks) {
            void *args[] = {(void *)&g, (void *)&arrive, (void *)&limit, (void *)&ok};
            e = cudaLaunchCooperativeKernel((const void *)pk_barrier_selftest, dim3(blocks), dim3(64), args, 0, nullptr);
        } else {
            pk_barrier_selftest<<<blocks, 64>>>(g, arrive, limit, ok);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) fail(e, "launch");
    }
    if (st == EGFEM_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) fail(e, "cudaDeviceSynchronize");
    if (st == EGFEM_OK && (e = cudaMemcpy(ok_host, ok, sizeof(int32_t) * size_t(blocks), cudaMemcpyDeviceToHost)) != cudaSuccess)
        fail(e, "cudaMemcpy");
    if (st == EGFEM_OK && err_host && (e = cudaMemcpy(err_host, &g->err, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        fail(e, "cudaMemcpy");
    cudaFree(ok);
    cudaFree(g);
    return st;
}

void egfem_default_options(egfem_options *o) {
    if (!o) return;
    o->newton_rtol = 1e-10;
    o->newton_atol = 0.0;
    o->newton_maxit = 50;
    o->eta_max = 0.0;   // the library's cap: eta_cap()
    o->eta_min = 1e-12;
    o->krylov_maxit = 100000;
    o->precision = EGFEM_PREC_FP64;
    o->op = EGFEM_OP_CSF;
    o->graph_chunk = 32;
    o->fixed_eta = 0;
    o->krylov_persistent = 1;
    o->iteration = EGFEM_ITER_NEWTON;
    o->krylov_block_rows = 0;
    o->krylov_cluster = 0;
    o->newton_graph = 1;
    o->batch_share = 1;
}

egfem_status egfem_build(const egfem_mesh *mesh, const egfem_problem *prob, const egfem_options *opts, egfem_handle *out) {
    try {
        return build_impl(mesh, prob, opts, out);
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return EGFEM_ERR_OOM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return EGFEM_ERR_INVALID_ARG;
    }
}

void egfem_destroy(egfem_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->hs) cudaStreamSynchronize(h->hs);
    DeviceCSF &D = h->csf;
    dfree(D.meta); dfree(D.col_idx); dfree(D.col_slot); dfree(D.slice_off); dfree(D.leaf_val); dfree(D.leaf_col);
    dfree(D.fib_info); dfree(D.fib_tdiag); dfree(D.fib_m); dfree(D.rx_val); dfree(D.rx_info); dfree(D.rx_m);
    dfree(D.dir); dfree(D.rowptr); dfree(D.cols);
    dfree(h->cell_S); dfree(h->cell_E);
    dfree(h->tmap); dfree(h->wa_kind); dfree(h->wa_sup); dfree(h->cell_verts); dfree(h->cell_vol);
    dfree(h->wc_kind); dfree(h->wc_sup); dfree(h->wa_val); dfree(h->wa_gp); dfree(h->wc_val); dfree(h->wc_gp);
    dfree(h->wa_val32); dfree(h->wa_gp32); dfree(h->leaf_val32);
    dfree(h->v2c_ptr); dfree(h->v2c); dfree(h->kappa_field);
    dfree(h->r); dfree(h->jsell); dfree(h->dinv); dfree(h->part); dfree(h->scal); dfree(h->ticket); dfree(h->status); dfree(h->st);
    for (KWork<double> *W : {&h->k64}) {
        if (W->graph) cudaGraphExecDestroy(W->graph);
        dfree(W->A); dfree(W->b); dfree(W->x); dfree(W->r); dfree(W->rh); dfree(W->p); dfree(W->v); dfree(W->s); dfree(W->t);
        dfree(W->p2); dfree(W->v2); dfree(W->bar); dfree(W->pk_tiles); dfree(W->pk_part); dfree(W->pkw_win);
        dfree(W->pkwb_tiles); dfree(W->pkwb_win); dfree(W->pkwb_part);
    }
    for (KWork<df64> *W : {&h->k32}) {
        if (W->graph) cudaGraphExecDestroy(W->graph);
        dfree(W->A); dfree(W->b); dfree(W->x); dfree(W->r); dfree(W->rh); dfree(W->p); dfree(W->v); dfree(W->s); dfree(W->t);
        dfree(W->p2); dfree(W->v2); dfree(W->bar); dfree(W->pk_tiles); dfree(W->pk_part); dfree(W->pkw_win);
        dfree(W->pkwb_tiles); dfree(W->pkwb_win); dfree(W->pkwb_part);
    }
    dfree(h->adj_b0); dfree(h->adj_acc); dfree(h->adj_ss);
    dfree(h->slice_inst); dfree(h->inst_mask); dfree(h->inst_eta); dfree(h->inst_lam); dfree(h->inst_norm2);
    dfree(h->bst); dfree(h->tiles); dfree(h->bpart); dfree(h->bbar); dfree(h->bpart2);
    if (h->gn_exec) cudaGraphExecDestroy(h->gn_exec);
    dfree(h->gn_state); dfree(h->gn_stats); dfree(h->gn_loops);
    if (h->bgraph64) cudaGraphExecDestroy(h->bgraph64);
    if (h->bgraph32) cudaGraphExecDestroy(h->bgraph32);
    for (void *q : {(void *)h->h_mask, (void *)h->h_eta, (void *)h->h_lam, (void *)h->h_norm2, (void *)h->h_bst})
        if (q) cudaFreeHost(q);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->hs) cudaStreamDestroy(h->hs);
    delete h;
}

egfem_status egfem_set_options(egfem_handle h, const egfem_options *opts) {
    if (!h || !opts) return EGFEM_ERR_INVALID_ARG;
    if (opts->precision != h->opts.precision || opts->op != h->opts.op) {
        g_last_error = "precision and operator are fixed at build";
        return EGFEM_ERR_INVALID_ARG;
    }
    h->opts = *opts;
    // the graph Newton loop bakes the options in: capture it again at the next batched solve
    if (h->gn_exec) { cudaGraphExecDestroy(h->gn_exec); h->gn_exec = nullptr; }
    h->gn_failed = false;
    return EGFEM_OK;
}

egfem_status egfem_sizes(egfem_handle h, int64_t *n_nodes, int64_t *n_wa, int64_t *n_wc, int64_t *jac_rows, int64_t *jac_nnz) {
    if (!h) return EGFEM_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = h->n;
    if (n_wa) *n_wa = h->nwa;
    if (n_wc) *n_wc = h->nwc;
    if (jac_rows) *jac_rows = h->n;
    if (jac_nnz) *jac_nnz = h->csf.nnz;
    return EGFEM_OK;
}

egfem_status egfem_tensor_storage(egfem_handle h, int64_t *bytes, int32_t *share_count) {
    if (!h) return EGFEM_ERR_INVALID_ARG;
    const DeviceCSF &D = h->csf;
    if (bytes)
        *bytes = D.n_leaves * int64_t(sizeof(double) + sizeof(uint8_t)) +
                 D.n_fibres * int64_t(sizeof(uint32_t) + sizeof(double) + sizeof(int32_t)) +
                 D.n_rx * int64_t(sizeof(double) + sizeof(uint32_t) + sizeof(int32_t));
    if (share_count) *share_count = h->ws.k;
    return EGFEM_OK;
}

egfem_status egfem_w_coords(egfem_handle h, int32_t which, double *coords_host) {
    if (!h || !coords_host || (which != 0 && which != 1)) return EGFEM_ERR_INVALID_ARG;
    const std::vector<double> &c = which == 0 ? h->wa_coords : h->wc_coords;
    std::memcpy(coords_host, c.data(), c.size() * sizeof(double));
    return EGFEM_OK;
}

egfem_status egfem_jacobian_pattern(egfem_handle h, const int32_t **d_rowptr, const int32_t **d_cols) {
    if (!h) return EGFEM_ERR_INVALID_ARG;
    if (d_rowptr) *d_rowptr = h->csf.rowptr;
    if (d_cols) *d_cols = h->csf.cols;
    return EGFEM_OK;
}

egfem_status egfem_set_kappa(egfem_handle h, const double *d_kappa, egfem_stream stream) {
    if (!h) return EGFEM_ERR_INVALID_ARG;
    if (d_kappa && h->opts.op == EGFEM_OP_MATRIX_FREE) {
        g_last_error = "a kappa field needs the CSF operator";
        return EGFEM_ERR_UNSUPPORTED;
    }
    if (d_kappa && h->nl.a_kind == EGFEM_G_GRADPOW) {
        g_last_error = "a kappa field is not available with the gradient coefficient";
        return EGFEM_ERR_UNSUPPORTED;
    }
    EG_CUDA(cudaSetDevice(h->device));
    if (!d_kappa) { h->nl.kappa_field = nullptr; return EGFEM_OK; }
    if (!h->kappa_field) EG_TRY(dalloc(h->kappa_field, size_t(h->nwa)));
    EG_CUDA(cudaMemcpyAsync(h->kappa_field, d_kappa, size_t(h->nwa) * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    h->nl.kappa_field = h->kappa_field;
    return EGFEM_OK;
}

egfem_status egfem_pointwise(egfem_handle h, const double *d_u, double *d_w, double *d_wprime, egfem_stream stream) {
    if (!h || !d_u) return EGFEM_ERR_INVALID_ARG;
    if (h->nl.a_kind == EGFEM_G_GRADPOW || h->prob.a_space == EGFEM_W_QUADRATURE) {
        g_last_error = "the gradient coefficient and I_k are evaluated per cell inside the element-local operator";
        return EGFEM_ERR_UNSUPPORTED;
    }
    EG_CUDA(cudaSetDevice(h->device));
    const unsigned grid = unsigned((h->nwa + 255) / 256);
    pointwise_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(h->nwa, h->wa_kind, h->wa_sup, d_u, h->nl, d_w, d_wprime);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_residual(egfem_handle h, const double *d_u, const double *d_d, double *d_r, egfem_stream stream) {
    if (!h || !d_u || !d_d || !d_r) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    CsfArgs A = csf_args(h, d_u, d_d);
    A.r = d_r;
    launch_csf(h, A, (cudaStream_t)stream);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_jacobian(egfem_handle h, const double *d_u, double *d_vals, egfem_stream stream) {
    if (!h || !d_u || !d_vals) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    CsfArgs A = csf_args(h, d_u, nullptr);
    A.jcsr = d_vals;
    launch_csf(h, A, (cudaStream_t)stream);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_spmv(egfem_handle h, const double *d_vals, const double *d_x, double *d_y, egfem_stream stream) {
    if (!h || !d_vals || !d_x || !d_y) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    csr_spmv_kernel<<<unsigned((h->n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(h->n, h->csf.rowptr, h->csf.cols, d_vals, d_x, d_y);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_bicgstab(egfem_handle h, const double *d_vals, const double *d_rhs, double *d_x, double rtol,
                            int32_t maxit, int32_t *iters, egfem_stream stream) {
    if (!h || !d_vals || !d_rhs || !d_x || rtol < 0 || maxit < 0) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    EG_TRY(join_in(h, (cudaStream_t)stream));
    EG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int32_t), h->hs));
    int32_t done = 0, it = 0;
    const unsigned g = unsigned((h->n + 255) / 256);
    if (h->opts.precision == EGFEM_PREC_MIXED) {
        EG_TRY(kwork_alloc(h, h->k32));
        csr_to_sell_kernel<df64><<<g, 256, 0, h->hs>>>(h->n, h->csf.meta, h->csf.col_slot, d_vals, d_rhs, h->k32.A, h->k32.b,
                                                        h->status);
        EG_CUDA(cudaGetLastError());
        EG_TRY(check_status_word(h));
        EG_TRY(run_bicgstab(h, h->k32, rtol, maxit, 0, &done, &it));
        cast_kernel<df64, double><<<g, 256, 0, h->hs>>>(h->n, h->k32.x, d_x);
    } else {
        EG_TRY(kwork_alloc(h, h->k64));
        csr_to_sell_kernel<double><<<g, 256, 0, h->hs>>>(h->n, h->csf.meta, h->csf.col_slot, d_vals, d_rhs, h->k64.A, h->k64.b,
                                                          h->status);
        EG_CUDA(cudaGetLastError());
        EG_TRY(check_status_word(h));
        EG_TRY(run_bicgstab(h, h->k64, rtol, maxit, 0, &done, &it));
        EG_CUDA(cudaMemcpyAsync(d_x, h->k64.x, size_t(h->n) * sizeof(double), cudaMemcpyDeviceToDevice, h->hs));
    }
    EG_CUDA(cudaGetLastError());
    EG_TRY(join_out(h, (cudaStream_t)stream));
    if (iters) *iters = it;
    if (done == K_CONVERGED) return EGFEM_OK;
    if (done == K_MAXIT || done == K_STAGNATED) return EGFEM_ERR_NOT_CONVERGED;
    if (done == K_BREAKDOWN) return EGFEM_ERR_BREAKDOWN;
    return EGFEM_ERR_NONFINITE;
}

egfem_status egfem_newton_solve(egfem_handle h, double *d_u, const double *d_d, egfem_stats *stats, egfem_stream stream) {
    if (!h || !d_u || !d_d) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    const auto t0 = std::chrono::steady_clock::now();
    egfem_stats S;
    std::memset(&S, 0, sizeof(S));
    const bool mixed = h->opts.precision == EGFEM_PREC_MIXED;
    if (mixed) EG_TRY(kwork_alloc(h, h->k64));   // FP64 rescue of failed FP32 solves
    EG_TRY(join_in(h, (cudaStream_t)stream));
    EG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int32_t), h->hs));
    // residual, Jacobi-scaled Jacobian and right-hand side at u (both precisions when mixed)
    // residual and solver operator at u: the FP64 operator (need64, and always in FP64 mode),
    // else only the FP32 one from the mixed-precision tensor action
    bool have64 = false;
    if (mixed && h->opts.op == EGFEM_OP_CSF) EG_TRY(ensure_mixed_tensor(h, h->hs));
    auto eval = [&](double *rn, bool need64 = false) -> egfem_status {
        CsfArgs A = csf_args(h, d_u, d_d);
        A.r = h->r;
        A.q64 = h->k64.b;
        have64 = !mixed || need64;
        if (have64) A.a64 = h->k64.A;
        if (mixed) A.a32 = h->k32.A;
        S.kernel_launches += launch_csf(h, A, h->hs) + 1 + (mixed ? 1 : 0);
        if (mixed) cast_kernel<double, df64><<<unsigned((h->n + 255) / 256), 256, 0, h->hs>>>(h->n, h->k64.b, h->k32.b);
        EG_CUDA(cudaGetLastError());
        double n2;
        EG_TRY(norm2_free(h, h->r, &n2));
        *rn = std::sqrt(n2);
        return EGFEM_OK;
    };
    const unsigned g = unsigned((h->n + 255) / 256);
    auto update = [&](bool fp32, double lam) -> egfem_status {   // u -= lam x
        if (fp32) newton_update_kernel<df64><<<g, 256, 0, h->hs>>>(h->n, d_u, h->k32.x, lam);
        else newton_update_kernel<double><<<g, 256, 0, h->hs>>>(h->n, d_u, h->k64.x, lam);
        EG_CUDA(cudaGetLastError());
        S.kernel_launches += 1;
        return EGFEM_OK;
    };
    double rn;
    egfem_status status = eval(&rn);
    if (status != EGFEM_OK) return status;
    const double r0 = rn;
    S.res0 = r0;
    const double target = std::max(h->opts.newton_rtol * r0, h->opts.newton_atol);
    double eta = eta_cap(h), rprev = rn;
    int k = 0;
    status = EGFEM_OK;
    // the Newton loop on the device (damping included); the host loop below resumes from its state
    h->gn_used = false;
    bool resume64 = false;   // the graph handed back its current step for the FP64 redo
    double rb_resume = rn;
    if (rn > target && std::isfinite(rn)) {
        bool back = false;
        const bool ran = mixed ? gn_run_one<df64>(h, h->k32, d_u, d_d, rn, rprev, eta, target, S, back, rb_resume)
                               : gn_run_one<double>(h, h->k64, d_u, d_d, rn, rprev, eta, target, S, back, rb_resume);
        if (!ran && h->opts.newton_graph == 2) {
            g_last_error = "graph Newton loop required (newton_graph = 2) but unavailable: " + g_last_error;
            status = EGFEM_ERR_UNSUPPORTED;
        } else if (ran) {
            EG_CUDA(cudaGetLastError());
            k = S.newton_iters;
            const egfem_status ws = check_status_word(h);   // a zero Jacobi diagonal on the way
            if (ws != EGFEM_OK) status = ws;
            else if (S.status != EGFEM_OK) {
                status = egfem_status(S.status);
                if (status == EGFEM_ERR_NOT_CONVERGED)
                    g_last_error = k >= h->opts.newton_maxit ? "Newton iteration cap"
                                                             : "Newton step failed to decrease the residual after 6 halvings";
            } else if (back || rn > target) {
                // residual and operator at the current u for the host loop: the undone step
                // of a hand-back (its FP64 redo follows), or the graph's loop cap
                status = eval(&rn);
                resume64 = back;
            }
        }
    }
    while (status == EGFEM_OK) {
        if (!std::isfinite(rn)) { status = EGFEM_ERR_NONFINITE; break; }
        if (rn <= target) break;
        if (k >= h->opts.newton_maxit) { status = EGFEM_ERR_NOT_CONVERGED; g_last_error = "Newton iteration cap"; break; }
        egfem_status ws = check_status_word(h);
        if (ws != EGFEM_OK) { status = ws; break; }
        // Eisenstat-Walker forcing term (choice 2, gamma = 0.9, alpha = 2), safeguarded; a step
        // resumed from the graph keeps its forcing term and starting norm
        if (k > 0 && !h->opts.fixed_eta && !resume64) {
            double e = 0.9 * (rn / rprev) * (rn / rprev);
            const double sg = 0.9 * eta * eta;
            if (sg > 0.1) e = std::max(e, sg);
            eta = std::min(eta_cap(h), e);
            eta = std::max(eta, 0.5 * target / rn);
        }
        eta = std::max(eta, h->opts.eta_min);
        bool fp32 = mixed && !resume64, stepped = false;
        const double rbefore = resume64 ? rb_resume : rn;
        int32_t its_step = k < EGFEM_HIST ? S.krylov_hist[k] : 0;   // the graph's share of this step
        resume64 = false;
        while (!stepped) {
            int32_t done = 0, it = 0;
            if (!fp32 && !have64) {   // an FP64 rescue needs the FP64 operator at this u
                status = eval(&rn, true);
                if (status != EGFEM_OK) break;
            }
            if (fp32) status = run_bicgstab(h, h->k32, std::max(eta, kMixedEtaFloor), h->opts.krylov_maxit, kMixedStall, &done, &it);
            else status = run_bicgstab(h, h->k64, eta, h->opts.krylov_maxit, 0, &done, &it);
            if (status != EGFEM_OK) break;
            S.kernel_launches += h->last_krylov_kernels;
            S.krylov_iters += it;
            its_step += it;
            const bool failed = done == K_NONFINITE || (done == K_BREAKDOWN && it == 0) || (fp32 && done == K_BREAKDOWN);
            if (failed) {
                if (fp32) { fp32 = false; ++S.fp64_rescues; continue; }
                status = done == K_NONFINITE ? EGFEM_ERR_NONFINITE : EGFEM_ERR_BREAKDOWN;
                break;
            }
            status = update(fp32, 1.0);
            if (status != EGFEM_OK) break;
            status = eval(&rn);
            if (status != EGFEM_OK) break;
            // damping (the paper's remark on damped iterations, Sec. 4): halve the step while
            // the FP64 residual norm fails to decrease sufficiently (Armijo test, <= 6 halvings)
            double lam = 1.0;
            for (int bt = 0; bt < 6 && !(rn <= (1.0 - 1e-4 * lam) * rbefore); ++bt) {
                status = update(fp32, -0.5 * lam);   // step length lam -> lam / 2
                if (status != EGFEM_OK) break;
                lam *= 0.5;
                status = eval(&rn);
                if (status != EGFEM_OK) break;
            }
            if (status != EGFEM_OK) break;
            if (rn < rbefore) { stepped = true; break; }
            // no step length decreases the residual: undo the step
            status = update(fp32, -lam);
            if (status == EGFEM_OK) status = eval(&rn);
            if (status != EGFEM_OK) break;
            if (fp32) { fp32 = false; ++S.fp64_rescues; continue; }
            status = EGFEM_ERR_NOT_CONVERGED;
            g_last_error = "Newton step failed to decrease the residual after 6 halvings";
            break;
        }
        if (k < EGFEM_HIST) S.krylov_hist[k] = its_step;
        if (!stepped) break;
        ++k;
        rprev = rbefore;
        if (k - 1 < EGFEM_HIST) S.res_hist[k - 1] = rn;
    }
    S.newton_iters = k;
    S.res_final = rn;
    S.status = status;
    S.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    egfem_status js = join_out(h, (cudaStream_t)stream);
    if (stats) *stats = S;
    return status != EGFEM_OK ? status : js;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Adjoint and load vectors
// ---------------------------------------------------------------------------------

namespace {

// AT[tmap[q]] = J[q] * dinv[col(q)]  (the transpose, Jacobi-scaled by its own diagonal)
template <typename M_t>
__global__ void transpose_scaled_kernel(int64_t n, const SliceMeta *meta, const int32_t *col_idx, const int64_t *tmap,
                                        const double *jsell, const double *dinv, M_t *AT) {
    const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const SliceMeta M = meta[row / SLICE];
    const int lane = int(row % SLICE);
    for (int c = 0; c < M.ncol; ++c) {
        const int64_t q = M.col_base + int64_t(c) * SLICE + lane;
        const int64_t t = tmap[q];
        if (t < 0) continue;
        AT[t] = (c == 0 && dinv[row] != 0.0) ? M_t(1) : M_t(jsell[q] * dinv[col_idx[q]]);   // unit diagonal
    }
}

template <typename V>
__global__ void adjoint_rhs_kernel(int64_t n, const double *g, const uint8_t *dir, const double *dinv, V *b) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = cvt<V>(dir[i] ? 0.0 : g[i] * dinv[i]);
}

// res = b0 - A x with the solver's FP64 operator (SELL layout), and per slice of 32 rows the sum
// of res^2 in one fixed order (16 threads of 2 rows each, then a fixed shuffle tree): the true
// residual of the transposed solve.  x = null: res = b0 (the norms of the right-hand side).
__global__ void __launch_bounds__(256) adj_resid_kernel(KVecs<double> K, const double *b0, const double *x, double *res,
                                                       double *slice_ss) {
    const int64_t r0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2;
    double ss = 0.0;
    if (r0 < K.n_pad) {
        const Pack<double> bb = ldv(b0 + r0);
        Pack<double> o = bb;
        if (x) {
            const Pack<double> y = sell_rows(K, r0, x);
            o.v[0] = bb.v[0] - y.v[0];
            o.v[1] = bb.v[1] - y.v[1];
        }
        if (res) stv(res + r0, o);
        ss = o.v[0] * o.v[0] + o.v[1] * o.v[1];
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    if ((threadIdx.x & 15) == 0 && r0 < K.n_pad) slice_ss[r0 / SLICE] = ss;
}

__global__ void add_into_kernel(int64_t n, const double *x, double *acc) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) acc[i] += x[i];
}

// grad_kappa_m -= lambda_i sum_k T_imk (u_k - u_i)   (sum_k T_imk = 0)
__global__ void grad_kappa_kernel(int64_t n_rows, const SliceMeta *meta, const int32_t *col_idx, const double *leaf_val,
                                  const uint8_t *leaf_col, const uint32_t *fib_info, const int32_t *fib_m, const uint8_t *dir,
                                  const double *u, const double *lam, double *grad, WShare ws) {
    const int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= n_rows || dir[row]) return;
    const int64_t inst = ws.k > 0 ? row / ws.rows : 0;   // a shared tensor's W indices are instance 0's
    const double li = lam[row];
    if (li == 0.0) return;
    const SliceMeta M = meta[row / SLICE];
    const int lane = int(row % SLICE);
    const double ui = u[row];
    double D = 0.0;
    int f = -1;
    for (int j = 0; j < M.nleaf; ++j) {
        const int64_t q = M.leaf_base + int64_t(j) * SLICE + lane;
        const uint8_t lc = leaf_col[q];
        if (lc & LEAF_FIBRE_START) {
            if (f >= 0) {
                const int64_t fq = M.fib_base + int64_t(f) * SLICE + lane;
                if (((fib_info[fq] >> 24) & 0xF) != W_CONST) atomicAdd(&grad[fib_m[fq] + ws_stride(ws.a, fib_info[fq]) * inst], -li * D);
            }
            ++f;
            D = 0.0;
        }
        const int c = lc & LEAF_PAD;
        if (c != LEAF_PAD) D += leaf_val[q] * (u[col_idx[M.col_base + int64_t(c) * SLICE + lane]] - ui);
    }
    if (f >= 0) {
        const int64_t fq = M.fib_base + int64_t(f) * SLICE + lane;
        if (((fib_info[fq] >> 24) & 0xF) != W_CONST) atomicAdd(&grad[fib_m[fq] + ws_stride(ws.a, fib_info[fq]) * inst], -li * D);
    }
}

__global__ void load_cellwise_kernel(int64_t n, int dim, const int64_t *v2c_ptr, const int32_t *v2c, const double *vol,
                                     const uint8_t *dir, const double *f, double *d) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (dir[i]) { d[i] = 0.0; return; }
    double s = 0.0;
    for (int64_t t = v2c_ptr[i]; t < v2c_ptr[i + 1]; ++t) { const int32_t c = v2c[t]; s += f[c] * vol[c]; }
    d[i] = s / double(dim + 1);
}

__global__ void load_cellwise_t_kernel(int64_t nc, int dim, const int32_t *cv, const double *vol, const uint8_t *dir,
                                       const double *lam, double *g) {
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double s = 0.0;
    for (int a = 0; a <= dim; ++a) { const int32_t v = cv[c * (dim + 1) + a]; if (!dir[v]) s += lam[v]; }
    g[c] = s * vol[c] / double(dim + 1);
}

template <typename V>
egfem_status batch_tiles(egfem_t *h, int factor);
template <typename V>
egfem_status run_batch_bicgstab(egfem_t *h, KWork<V> &W, cudaGraphExec_t &G, int32_t stall, int64_t *launches);

template <typename V>
egfem_status adjoint_solve(egfem_t *h, KWork<V> &W, const double *d_u, const double *d_g, double *d_lambda, egfem_stats *S) {
    if (!h->jsell) EG_TRY(dalloc(h->jsell, size_t(h->csf.n_colentries)));
    if (!h->dinv) EG_TRY(dalloc(h->dinv, size_t(h->n)));
    EG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int32_t), h->hs));
    CsfArgs A = csf_args(h, d_u, nullptr);
    A.nl.picard = 0;   // the adjoint needs the true Jacobian
    A.jsell = h->jsell; A.dinv = h->dinv;
    launch_csf(h, A, h->hs);
    EG_CUDA(cudaGetLastError());
    EG_TRY(check_status_word(h));
    const unsigned g = unsigned((h->n + 255) / 256);
    using M_t = typename VecT<V>::mat;
    EG_CUDA(cudaMemsetAsync(W.A, 0, size_t(h->csf.n_colentries) * sizeof(M_t), h->hs));
    transpose_scaled_kernel<M_t><<<g, 256, 0, h->hs>>>(h->n, h->csf.meta, h->csf.col_idx, h->tmap, h->jsell, h->dinv, W.A);
    if (VecT<V>::diff) rowsum_form_kernel<M_t><<<g, 256, 0, h->hs>>>(h->n, h->csf.meta, W.A);
    adjoint_rhs_kernel<V><<<g, 256, 0, h->hs>>>(h->n, d_g, h->csf.dir, h->dinv, W.b);
    EG_CUDA(cudaGetLastError());
    // True-residual restarts.  With the right-hand side as shadow residual, the inner products
    // of the transposed system lose their digits within a few hundred iterations (measured at
    // 512^2: (rh, r) at 1e-11 of |rh||r| after 100 iterations, at the rounding level after 700),
    // so the recursive residual drifts from b - A x (a 275-fold gap at the 1e-13 target) and
    // BiCGStab can end in an exact breakdown.  Each round therefore forms the true residual
    // res = b - A lambda in FP64, solves A delta = res afresh (new shadow residual) for the
    // instances above the target, and adds delta; an instance is done when its true residual is
    // below kAdjTol of its right-hand side, or when a round no longer halves it: the FP64 floor
    // of evaluating b - A lambda, about eps |A| |lambda|, which lies above 1e-13 |b| when lambda
    // is much larger than b (at 512^2: about 1e-12 |b|).  The first solve asks for kAdjTol1 of
    // the recursive residual, which is below that floor already.
    static_assert(std::is_same<V, double>::value, "the transposed solve is FP64");
    constexpr double kAdjTol = 1e-13, kAdjTol1 = 1e-12;
    constexpr int kAdjRounds = 5;
    const int64_t nsl = h->n_pad / SLICE;
    if (!h->adj_b0) {
        EG_TRY(dalloc(h->adj_b0, size_t(h->n_pad)));
        EG_TRY(dalloc(h->adj_acc, size_t(h->n_pad)));
        EG_TRY(dalloc(h->adj_ss, size_t(nsl)));
    }
    const int32_t ninst = h->nb > 0 ? h->nb : 1;
    auto inst_slices = [&](int32_t b, int64_t &s0, int64_t &s1) {
        s0 = h->nb > 0 ? h->inst_off[b] / SLICE : 0;
        s1 = h->nb > 0 ? (h->inst_off[b + 1] + SLICE - 1) / SLICE : nsl;
    };
    std::vector<double> ss(static_cast<size_t>(nsl)), bb(static_cast<size_t>(ninst), 0.0), rr(static_cast<size_t>(ninst), 0.0);
    const unsigned gr = unsigned((h->n_pad / 2 + 255) / 256);
    KVecs<V> K = kvecs(h, W);
    auto inst_sums = [&](std::vector<double> &out) -> egfem_status {
        EG_CUDA(cudaMemcpyAsync(ss.data(), h->adj_ss, size_t(nsl) * sizeof(double), cudaMemcpyDeviceToHost, h->hs));
        EG_CUDA(cudaStreamSynchronize(h->hs));
        for (int32_t b = 0; b < ninst; ++b) {
            int64_t s0, s1;
            inst_slices(b, s0, s1);
            double t = 0.0;
            for (int64_t q = s0; q < s1; ++q) t += ss[size_t(q)];
            out[size_t(b)] = t;
        }
        return EGFEM_OK;
    };
    EG_CUDA(cudaMemcpyAsync(h->adj_b0, W.b, size_t(h->n_pad) * sizeof(double), cudaMemcpyDeviceToDevice, h->hs));
    EG_CUDA(cudaMemsetAsync(h->adj_acc, 0, size_t(h->n_pad) * sizeof(double), h->hs));
    adj_resid_kernel<<<gr, 256, 0, h->hs>>>(K, h->adj_b0, nullptr, nullptr, h->adj_ss);
    EG_CUDA(cudaGetLastError());
    EG_TRY(inst_sums(bb));
    std::vector<uint8_t> todo(static_cast<size_t>(ninst), 1);
    std::vector<double> rtol(static_cast<size_t>(ninst), kAdjTol1), rprev(static_cast<size_t>(ninst), 0.0);
    int32_t it_total = 0;
    bool nonfinite = false, met = false;
    for (int round = 0; round < kAdjRounds; ++round) {
        int32_t done = 0, it = 0;
        if (h->nb > 0) {
            // a batch: every instance runs its own BiCGStab (own scalars and convergence test), as
            // its single-instance adjoint would; one joint BiCGStab on the block-diagonal system
            // shares its scalars across instances and needs more iterations (2044 against at most
            // about 1300 for 16 instances at 512^2)
            if (!h->tile_factor) EG_TRY(batch_tiles<V>(h, 4));
            for (int32_t b = 0; b < h->nb; ++b) { h->h_mask[b] = todo[size_t(b)]; h->h_eta[b] = rtol[size_t(b)]; }
            EG_CUDA(cudaMemsetAsync(W.x, 0, size_t(h->n_pad) * sizeof(double), h->hs));
            int64_t launches = 0;
            EG_TRY(run_batch_bicgstab(h, W, h->bgraph64, 0, &launches));
            S->kernel_launches += launches;
            for (int32_t b = 0; b < h->nb; ++b) {
                if (!todo[size_t(b)]) continue;
                const KState &Q = h->h_bst[b];
                it = std::max(it, Q.iter);
                if (Q.done == K_NONFINITE) nonfinite = true;
            }
        } else {
            EG_TRY(run_bicgstab(h, W, rtol[0], h->opts.krylov_maxit, 0, &done, &it));
            S->kernel_launches += h->last_krylov_kernels;
            if (done == K_NONFINITE) nonfinite = true;
        }
        it_total += it;
        if (nonfinite) break;
        // lambda += delta; res = b0 - A lambda becomes the next right-hand side
        add_into_kernel<<<unsigned((h->n_pad + 255) / 256), 256, 0, h->hs>>>(h->n_pad, W.x, h->adj_acc);
        adj_resid_kernel<<<gr, 256, 0, h->hs>>>(K, h->adj_b0, h->adj_acc, W.b, h->adj_ss);
        EG_CUDA(cudaGetLastError());
        S->kernel_launches += 2;
        EG_TRY(inst_sums(rr));
        met = true;
        for (int32_t b = 0; b < ninst; ++b) {
            if (!todo[size_t(b)]) continue;
            const double lim = kAdjTol * kAdjTol * bb[size_t(b)];
            // done: below the target, or the round did not halve the true residual (the floor)
            const bool floor = round > 0 && rr[size_t(b)] > 0.25 * rprev[size_t(b)];
            todo[size_t(b)] = !(rr[size_t(b)] <= lim || floor);
            rprev[size_t(b)] = rr[size_t(b)];
            if (todo[size_t(b)]) {
                met = false;
                rtol[size_t(b)] = std::min(0.5, kAdjTol * std::sqrt(bb[size_t(b)] / rr[size_t(b)]));
            }
        }
        if (met) break;
    }
    double bsum = 0.0, rsum = 0.0;
    for (int32_t b = 0; b < ninst; ++b) { bsum += bb[size_t(b)]; rsum += rr[size_t(b)]; }
    S->res0 = std::sqrt(bsum);
    S->res_final = std::sqrt(rsum);
    S->krylov_iters += it_total;
    S->kernel_launches += 4;
    if (nonfinite) return EGFEM_ERR_NONFINITE;
    cast_kernel<V, double><<<g, 256, 0, h->hs>>>(h->n, h->adj_acc, d_lambda);
    EG_CUDA(cudaGetLastError());
    // rounds exhausted while still improving: the iterate is kept; it counts as converged within
    // 1e3 x the target
    for (int32_t b = 0; b < ninst && !met; ++b)
        if (todo[size_t(b)] && !(rr[size_t(b)] <= 1e6 * kAdjTol * kAdjTol * bb[size_t(b)])) {
            g_last_error = "adjoint: the transposed solve did not reach its tolerance";
            return EGFEM_ERR_NOT_CONVERGED;
        }
    return EGFEM_OK;
}

template <typename V>
egfem_status profile_impl(egfem_t *h, KWork<V> &W, const double *d_u, const double *d_d, int32_t reps, egfem_profile *out,
                          cudaStream_t user) {
    EG_TRY(join_in(h, user));
    cudaEvent_t e0, e1;
    EG_CUDA(cudaEventCreate(&e0));
    EG_CUDA(cudaEventCreate(&e1));
    const double vb = double(sizeof(V)), mb = double(sizeof(typename VecT<V>::mat));
    const double N = double(h->n), CE = double(h->csf.n_colentries), L = double(h->csf.n_leaves);
    const double F = double(h->csf.n_fibres), RX = double(h->csf.n_rx), SM = double(h->csf.n_slices) * sizeof(SliceMeta);
    auto timeit = [&](const char *name, double bytes, double flops, int fp64, auto launch) -> egfem_status {
        const int k = out->count;
        if (k >= EGFEM_PROF_MAX) return EGFEM_OK;
        launch();  // warm
        EG_CUDA(cudaEventRecord(e0, h->hs));
        for (int r = 0; r < reps; ++r) launch();
        EG_CUDA(cudaEventRecord(e1, h->hs));
        EG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        EG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        std::snprintf(out->name[k], sizeof(out->name[k]), "%s", name);
        out->ms[k] = double(ms) / reps;
        out->bytes[k] = bytes;
        out->flops[k] = flops;
        out->fp64[k] = fp64;
        out->count = k + 1;
        return EGFEM_OK;
    };
    CsfArgs A = csf_args(h, d_u, d_d);
    A.r = h->r;
    EG_TRY(kwork_alloc(h, h->k64));
    A.q64 = h->k64.b;
    if (std::is_same<V, double>::value) A.a64 = (double *)W.A;
    else A.a32 = (float *)W.A;
    // nodal pass: per W node its kind and support, the value and derivative written (u counted
    // with the rows); fused kernel: leaves (value + column byte), fibres (info, diagonal, W index),
    // reaction entries (value, info, W index), the nodal values read once, local columns
    // (index + CSR slot) and the operator written, u/d/r/q once each
    const double NWA = h->wa_val ? double(h->nwa) : 0.0, NWC = h->wc_val ? double(h->nwc) : 0.0;
    double csf_bytes = (NWA + NWC) * (1 + 12 + 2 * 16) + L * 9 + F * (NWA > 0 ? 16 : 12) + RX * (NWC > 0 ? 16 : 12) +
                       CE * (8 + mb) + N * (8 + 8 + 8 + 8 + 1) + SM;
    if (h->opts.op == EGFEM_OP_MATRIX_FREE) {
        // cells: vertices, packed S, |K|, the per-cell record written and read back;
        // rows: vertex-to-cell lists, local columns and the outputs
        const double NC = double(h->ncells), nv = h->dim + 1, ns = nv * (nv + 1) / 2, ne = double(h->mf_ne);
        csf_bytes = NC * (4 * nv + 8 * ns + 8 + 2 * 8 * ne) + N * (8 + 4 * 2 * nv) + CE * (8 + mb) + N * (8 + 8 + 8 + 8 + 1) + SM;
    }
    // FP64 operations: 2 per leaf (D and J1), per fibre the residual, diagonal and J2 scatter
    // (6; 12 when g is evaluated per fibre), 4 per reaction entry, 2 per local column, and
    // the nodal pass (interpolation and g, about 6 per node)
    // (a tensor shared by the ws.k instances of a batch is read once from DRAM but applied to
    // every instance: its bytes count once, its operations ws.k times)
    const double KS = h->ws.k > 0 ? double(h->ws.k) : 1.0;
    double csf_flops = KS * (L * 4 + F * (NWA > 0 ? 6 : 12) + RX * (NWC > 0 ? 4 : 10)) + CE * 2 + (NWA + NWC) * 6;
    if (h->opts.op == EGFEM_OP_MATRIX_FREE) {
        // cell pass: S u in difference form (3 per off-diagonal pair), then per local W node
        // the interpolation, g and the c^K update (4 nv + 6; the gradient coefficient: 3 nv and
        // the power, counted as 12); row pass, per (row, cell) pair: r and the nv Jacobian
        // entries (6 nv + 2)
        const double NC = double(h->ncells), nv = h->dim + 1;
        const double nw = h->nl.a_kind == EGFEM_G_GRADPOW ? 0.0 : double(h->mf_loc.nw);
        const double coef = h->nl.a_kind == EGFEM_G_GRADPOW ? 3 * nv + 12 : nw * (4 * nv + 6);
        // reaction: P1 W_c, 6 per vertex in the row pass; I_k, P2, P3, per local node
        // nv + 6 + 3 nv + 2 nv^2 in the cell pass and nv + 1 per (row, cell) pair; the linear
        // term sigma M, 3 per vertex of each (row, cell) pair
        const double react_row = (h->nl.c_kind == EGFEM_G_NONE ? 0.0 : h->mf_loc_c.nw > 0 ? nv + 1 : 6 * nv) +
                                 (h->nl.sigma != 0.0 ? 3 * nv : 0.0);
        const double react_cell = h->nl.c_kind != EGFEM_G_NONE && h->mf_loc_c.nw > 0
                                      ? double(h->mf_loc_c.nw) * (4 * nv + 6 + 2 * nv * nv) : 0.0;
        csf_flops = NC * (3 * nv * (nv - 1) + coef + react_cell) + NC * nv * (6 * nv + 2 + react_row);
    }
    const char *ta_name = h->opts.op == EGFEM_OP_MATRIX_FREE ? "tensor_action_mf" : "csf_fused";
    if (!std::is_same<V, double>::value && h->opts.op == EGFEM_OP_CSF) {
        // mixed path: the mixed-precision tensor action (FP64 residual, FP32 Jacobian).  Nodal
        // pass as above plus the FP32 copies written; leaves: FP64 and FP32 value + column byte;
        // fibres: info + W index; nodal values read once (FP64 value, FP32 value and
        // derivative); local columns: index + slot read, FP32 operator written; u/d/r/q.
        // FP64 operations: 2 per leaf (D), 3 per fibre (residual, row sum), 4 per reaction
        // entry, 1 per local column (difference), 6 per node.
        EG_TRY(ensure_mixed_tensor(h, h->hs));
        ta_name = "csf_mixed";
        csf_bytes = (NWA + NWC) * (1 + 12 + 2 * 16) + NWA * 8 + L * 13 + F * 8 + NWA * 16 + RX * 16 + NWC * 16 +
                    CE * (8 + 4) + N * (8 + 8 + 8 + 8 + 1) + SM;
        csf_flops = KS * (L * 2 + F * 3 + RX * 4) + CE * 1 + (NWA + NWC) * 6;
    }
    EG_TRY(timeit(ta_name, csf_bytes, csf_flops, 1, [&] { launch_csf(h, A, h->hs); }));
    if (!std::is_same<V, double>::value)
        cast_kernel<double, V><<<unsigned((h->n + 255) / 256), 256, 0, h->hs>>>(h->n, h->k64.b, W.b);
    KVecs<V> K = kvecs(h, W);
    const bool persistent = h->opts.krylov_persistent && W.g_pk > 0;
    if (!persistent) {   // state for the iteration kernels: set up, one iteration
        kry_setup<V><<<W.g_setup, KRY_BLOCK, 0, h->hs>>>(K, 0.0, 1 << 30, 0);
        enqueue_iterations(h, W, 1, h->hs);
    }
    EG_CUDA(cudaGetLastError());
    const int fp = std::is_same<V, double>::value ? 1 : 0;
    auto run = [&](const char *name, double bytes, double flops, auto kern, int kg) -> egfem_status {
        EG_CUDA(cudaMemsetAsync(&h->st->done, 0, sizeof(int32_t), h->hs));
        EG_TRY(timeit(name, bytes, flops, fp, [&] { kern<<<kg, KRY_BLOCK, 0, h->hs>>>(K); }));
        int32_t done = 0;
        EG_CUDA(cudaMemcpy(&done, &h->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (done != K_RUNNING) out->ms[out->count - 1] = NAN;
        return EGFEM_OK;
    };
    // column indices are read only in non-uniform slices
    double ce_nonuni = 0;
    {
        std::vector<SliceMeta> hm(size_t(h->csf.n_slices));
        EG_CUDA(cudaMemcpy(hm.data(), h->csf.meta, hm.size() * sizeof(SliceMeta), cudaMemcpyDeviceToHost));
        for (const SliceMeta &M : hm) if (M.off_base < 0) ce_nonuni += double(M.ncol) * SLICE;
    }
    if (persistent) {
        // persistent solve: a fixed number of iterations (rtol 0), reported per iteration.  Per
        // row and iteration: A reads p, rh, writes v; B1 reads r, v, writes s; B2 reads s, writes
        // t; C reads s, p, t, rh, x, writes x, r; D reads r, v, p, writes p (19 vector passes);
        // the operator is read twice.
        const int32_t iters = 40;
        cudaError_t le = cudaSuccess;
        const bool cl = W.pkc_cluster > 0;
        // windowed solve (pkw_solve): per row and iteration A reads s, t, p, v (window) and x, b,
        // writes x, r, p, v; B reads r, v (window) and b, writes s, t (15 vector passes); the
        // updates take 12 FP64 flops per row, the inner products run on the FP32 pipe
        const bool win = !cl && W.pkw_smem > 0 && h->opts.krylov_persistent != 2 && W.pk_ntiles <= PK1_MAXG;
        // the FP64 operator's unit diagonal is neither read nor multiplied (column 0 of each row)
        const double CEo = std::is_same<V, double>::value ? CE - N : CE;
        const double kbytes = 2 * (CEo * mb + ce_nonuni * 4 + SM) + (win ? 15 : 19) * N * vb;
        const double kflops = 4 * CEo + (win && fp ? 12 : 22) * N;
        EG_TRY(timeit(cl ? "kry_cluster" : (win ? "kry_window" : "kry_persistent"), kbytes, kflops, fp, [&] {
            if (launch_pk_single(h, W, 0.0, iters, 0) != EGFEM_OK) le = cudaErrorLaunchFailure;
        }));
        EG_CUDA(le);
        int32_t done = 0;
        EG_CUDA(cudaMemcpy(&done, &h->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost));
        out->ms[out->count - 1] = (done == K_MAXIT) ? out->ms[out->count - 1] / iters : NAN;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return join_out(h, user);
    }
    if constexpr (std::is_same<V, df64>::value) {
        // fused iteration: per row, kry_vp reads r, p, v, rh and writes p, v; kry_st reads r, v and
        // writes t; kry_xr reads r, v, p, t, rh, x and writes x, r (gathered neighbours counted once)
        auto runf = [&](const char *name, double bytes, double flops, auto launch) -> egfem_status {
            EG_CUDA(cudaMemsetAsync(&h->st->done, 0, sizeof(int32_t), h->hs));
            EG_TRY(timeit(name, bytes, flops, 0, launch));
            int32_t done = 0;
            EG_CUDA(cudaMemcpy(&done, &h->st->done, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (done != K_RUNNING) out->ms[out->count - 1] = NAN;
            return EGFEM_OK;
        };
        EG_TRY(runf("kry_vp", CE * mb + ce_nonuni * 4 + 6 * N * vb + SM, 2 * CE + 6 * N,
                    [&] { kry_vp<V><<<W.g_vp, KRY_BLOCK, 0, h->hs>>>(K, W.p2, W.v2, W.p, W.v); }));
        EG_TRY(runf("kry_st", CE * mb + ce_nonuni * 4 + 3 * N * vb + SM, 2 * CE + 6 * N,
                    [&] { kry_st<V><<<W.g_st, KRY_BLOCK, 0, h->hs>>>(K, W.v2); }));
        EG_TRY(runf("kry_xr", 8 * N * vb, 12 * N, [&] { kry_xr<V><<<W.g_xr, KRY_BLOCK, 0, h->hs>>>(K, W.p2, W.v2); }));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return join_out(h, user);
    }
    EG_TRY(run("kry_v", CE * mb + ce_nonuni * 4 + 3 * N * vb + SM, 2 * CE + 2 * N, kry_v<V>, W.g_v));
    EG_TRY(run("kry_s", 3 * N * vb, 2 * N, kry_s<V>, W.g_s));
    EG_TRY(run("kry_t", CE * mb + ce_nonuni * 4 + 2 * N * vb + SM, 2 * CE + 4 * N, kry_t<V>, W.g_t));
    EG_TRY(run("kry_x", 7 * N * vb, 10 * N, kry_x<V>, W.g_x));
    EG_TRY(run("kry_p", 4 * N * vb, 4 * N, kry_p<V>, W.g_p));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return join_out(h, user);
}

}  // namespace

extern "C" {

egfem_status egfem_adjoint(egfem_handle h, const double *d_u, const double *d_dJdu, double *d_lambda, double *d_grad_kappa,
                           egfem_stats *stats, egfem_stream stream) {
    if (!h || !d_u || !d_dJdu || !d_lambda) return EGFEM_ERR_INVALID_ARG;
    if (d_grad_kappa && (h->nl.a_kind == EGFEM_G_GRADPOW || h->prob.a_space == EGFEM_W_QUADRATURE)) {
        g_last_error = "dJ/dkappa is not available with the gradient coefficient or I_k";
        return EGFEM_ERR_UNSUPPORTED;
    }
    EG_CUDA(cudaSetDevice(h->device));
    egfem_stats S;
    std::memset(&S, 0, sizeof(S));
    EG_TRY(join_in(h, (cudaStream_t)stream));
    // The transposed solve is FP64 in both precisions: it must reach 1e-13, and refinement
    // with the FP32 operator contracts only by about kappa * 6e-8 per sweep (16 instances at
    // 512^2: 4611 double-float iterations against 1868 FP64 ones).
    egfem_status st = kwork_alloc(h, h->k64);
    if (st == EGFEM_OK) st = adjoint_solve(h, h->k64, d_u, d_dJdu, d_lambda, &S);
    if (st == EGFEM_OK && d_grad_kappa) {
        EG_CUDA(cudaMemsetAsync(d_grad_kappa, 0, size_t(h->nwa) * sizeof(double), h->hs));
        grad_kappa_kernel<<<unsigned((h->n + 255) / 256), 256, 0, h->hs>>>(h->n, h->csf.meta, h->csf.col_idx, h->csf.leaf_val,
                                                                          h->csf.leaf_col, h->csf.fib_info, h->csf.fib_m, h->csf.dir, d_u, d_lambda,
                                                                          d_grad_kappa, h->ws);
        EG_CUDA(cudaGetLastError());
    }
    S.status = st;
    if (stats) *stats = S;
    egfem_status js = join_out(h, (cudaStream_t)stream);
    return st != EGFEM_OK ? st : js;
}

egfem_status egfem_load_cellwise(egfem_handle h, const double *d_f, double *d_d, egfem_stream stream) {
    if (!h || !d_f || !d_d) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    load_cellwise_kernel<<<unsigned((h->n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(h->n, h->dim, h->v2c_ptr, h->v2c,
                                                                                           h->cell_vol, h->csf.dir, d_f, d_d);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_load_cellwise_transpose(egfem_handle h, const double *d_lam, double *d_g, egfem_stream stream) {
    if (!h || !d_lam || !d_g) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    load_cellwise_t_kernel<<<unsigned((h->ncells + 255) / 256), 256, 0, (cudaStream_t)stream>>>(h->ncells, h->dim, h->cell_verts,
                                                                                                  h->cell_vol, h->csf.dir, d_lam, d_g);
    EG_CUDA(cudaGetLastError());
    return EGFEM_OK;
}

egfem_status egfem_profile_kernels(egfem_handle h, const double *d_u, const double *d_d, int32_t reps, egfem_profile *out,
                                   egfem_stream stream) {
    if (!h || !d_u || !d_d || !out || reps < 1) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    std::memset(out, 0, sizeof(*out));
    const bool mixed = h->opts.precision == EGFEM_PREC_MIXED;
    return mixed ? profile_impl(h, h->k32, d_u, d_d, reps, out, (cudaStream_t)stream)
                 : profile_impl(h, h->k64, d_u, d_d, reps, out, (cudaStream_t)stream);
}

const char *egfem_status_string(egfem_status s) {
    switch (s) {
        case EGFEM_OK: return "EGFEM_OK";
        case EGFEM_ERR_INVALID_ARG: return "EGFEM_ERR_INVALID_ARG";
        case EGFEM_ERR_MESH: return "EGFEM_ERR_MESH";
        case EGFEM_ERR_CUDA: return "EGFEM_ERR_CUDA";
        case EGFEM_ERR_OOM: return "EGFEM_ERR_OOM";
        case EGFEM_ERR_NOT_CONVERGED: return "EGFEM_ERR_NOT_CONVERGED";
        case EGFEM_ERR_BREAKDOWN: return "EGFEM_ERR_BREAKDOWN";
        case EGFEM_ERR_SINGULAR: return "EGFEM_ERR_SINGULAR";
        case EGFEM_ERR_NONFINITE: return "EGFEM_ERR_NONFINITE";
        case EGFEM_ERR_TIMEOUT: return "EGFEM_ERR_TIMEOUT";
        case EGFEM_ERR_UNSUPPORTED: return "EGFEM_ERR_UNSUPPORTED";
    }
    return "EGFEM_ERR_UNKNOWN";
}

const char *egfem_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

void egfem::set_last_error(const std::string &msg) { g_last_error = msg; }

extern "C" {

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batched solves: many instances as one block-diagonal operator (egfem_batch_*)
// ---------------------------------------------------------------------------------

namespace {

template <typename V>
egfem_status batch_tiles(egfem_t *h, int factor) {
    // about `factor` tiles per block of the persistent solve: the target tile size is the
    // batch's rows over (blocks x factor), and each instance is cut into equal slice-aligned
    // tiles near that size, so blocks get nearly equal work whatever the instance sizes
    constexpr int R = VecT<V>::R;
    int nbk = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, (const void *)pk_solveb<V>, PKB_BLOCK, 0) != cudaSuccess || nbk < 1)
        nbk = 1;
    const int64_t blocks = int64_t(std::min(nbk, 8)) * h->sms;
    const int64_t target = std::max<int64_t>(SLICE, (h->inst_off[h->nb] + blocks * factor - 1) / (blocks * factor));
    std::vector<BTile> T;
    for (int32_t b = 0; b < h->nb; ++b) {
        const int64_t t0 = int64_t(T.size());
        const int64_t lo = h->inst_off[b], hi = h->inst_off[b + 1];
        const int64_t nt = std::max<int64_t>(1, (hi - lo + target / 2) / target);
        const int64_t rows = ((hi - lo + nt - 1) / nt + SLICE - 1) / SLICE * SLICE;
        for (int64_t r = lo; r < hi; r += rows) T.push_back(BTile{r, std::min(hi, r + rows), t0, b, 0});
        for (size_t q = size_t(t0); q < T.size(); ++q) T[q].ntiles_inst = int32_t(T.size() - size_t(t0));
    }
    dfree(h->tiles);
    dfree(h->bpart);
    dfree(h->bpart2);
    EG_TRY(upload(h->tiles, T));
    EG_TRY(dalloc(h->bpart2, size_t(2 * T.size())));
    h->ntiles = int64_t(T.size());
    // 3 slots x 2 values per tile, then one running count per block of the persistent solve
    EG_TRY(dalloc(h->bpart, size_t(6 * h->ntiles + int64_t(h->sms) * 8)));
    h->tile_factor = factor;
    h->tile_R = R;
    if (h->bgraph64) { cudaGraphExecDestroy(h->bgraph64); h->bgraph64 = nullptr; }
    if (h->bgraph32) { cudaGraphExecDestroy(h->bgraph32); h->bgraph32 = nullptr; }
    return EGFEM_OK;
}

template <typename V>
KBatch<V> kbatch(egfem_t *h, KWork<V> &W) {
    KBatch<V> B{};
    B.K = kvecs(h, W);
    B.tiles = h->tiles; B.ntiles = h->ntiles; B.st = h->bst; B.part = h->bpart;
    return B;
}

template <typename V>
int bgrid(const egfem_t *h) { return int(std::max<int64_t>(1, std::min<int64_t>(h->ntiles, int64_t(h->sms) * 8))); }

template <typename V>
void enqueue_batch_iterations(egfem_t *h, KWork<V> &W, int count, cudaStream_t s) {
    const KBatch<V> B = kbatch(h, W);
    const int g = bgrid<V>(h);
    for (int it = 0; it < count; ++it) {
        kb_v<V><<<g, KRY_BLOCK, 0, s>>>(B);
        kb_s<V><<<g, KRY_BLOCK, 0, s>>>(B);
        kb_t<V><<<g, KRY_BLOCK, 0, s>>>(B);
        kb_x<V><<<g, KRY_BLOCK, 0, s>>>(B);
        kb_p<V><<<g, KRY_BLOCK, 0, s>>>(B);
    }
}

template <typename V>
egfem_status batch_graph(egfem_t *h, KWork<V> &W, cudaGraphExec_t &G) {
    const int chunk = std::max(1, h->opts.graph_chunk);
    if (G && h->bgraph_chunk == chunk) return EGFEM_OK;
    if (G) { cudaGraphExecDestroy(G); G = nullptr; }
    cudaGraph_t g;
    EG_CUDA(cudaStreamBeginCapture(h->hs, cudaStreamCaptureModeThreadLocal));
    enqueue_batch_iterations(h, W, chunk, h->hs);
    EG_CUDA(cudaStreamEndCapture(h->hs, &g));
    cudaError_t e = cudaGraphInstantiate(&G, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { g_last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e); return EGFEM_ERR_CUDA; }
    h->bgraph_chunk = chunk;
    return EGFEM_OK;
}

// Blocks of the persistent batched solve: resident blocks (occupancy x SMs), capped by the
// tiles; 0 when that solve cannot run (no cooperative launch, option off, or more than
// PK_MAXT tiles per block at the current tile size).
template <typename V>
const KWork<V> &kwork_of(const egfem_t *h);
template <>
const KWork<double> &kwork_of<double>(const egfem_t *h) { return h->k64; }
template <>
const KWork<df64> &kwork_of<df64>(const egfem_t *h) { return h->k32; }

template <typename V>
int pk_batch_grid(const egfem_t *h) {
    if (kwork_of<V>(h).pkwb_smem > 0 && h->opts.krylov_persistent == 1) return kwork_of<V>(h).pkwb_grid;   // windowed
    if (!h->coop || !h->opts.krylov_persistent || h->ntiles < 1) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)pk_solveb<V>, PKB_BLOCK, 0) != cudaSuccess || nb < 1)
        return 0;
    const int64_t g = std::min<int64_t>(h->ntiles, std::min<int64_t>(int64_t(nb), 8) * h->sms);
    if ((h->ntiles + g - 1) / g > PK_MAXT) return 0;
    return int(g);
}

template <typename V>
egfem_status launch_batch_persistent(egfem_t *h, KWork<V> &W, int grid, int32_t maxit, int32_t stall) {
    if (!h->bbar) EG_TRY(dalloc(h->bbar, 1));
    if (W.pkwb_smem > 0 && h->opts.krylov_persistent == 1) {
        // two reductions per iteration, each tile's halo recomputed in a shared-memory window
        PkwArgs<V> Q{};
        Q.K = kvecs(h, W); Q.p2 = W.p2; Q.v2 = W.v2; Q.tiles = W.pkwb_tiles; Q.win = W.pkwb_win;
        Q.ntiles = W.pkwb_ntiles; Q.st = h->bst; Q.part = W.pkwb_part; Q.active = h->inst_mask; Q.rtol = h->inst_eta;
        Q.rtol0 = 0.0; Q.bar = h->bbar; Q.n = h->n; Q.maxit = maxit; Q.stall = stall;
        void *qargs[] = {(void *)&Q};
        EG_CUDA(cudaMemsetAsync(h->bbar, 0, sizeof(PGrid), h->hs));
        EG_CUDA(cudaLaunchCooperativeKernel((const void *)pkwb_solve<V>, dim3(unsigned(W.pkwb_grid)), dim3(PKWB_BLOCK),
                                            qargs, W.pkwb_smem, h->hs));
        return EGFEM_OK;
    }
    return launch_pk(h, W, grid, h->tiles, h->ntiles, h->bst, h->bpart2,
                     h->inst_mask, h->inst_eta, 0.0, h->bbar, maxit, stall);
}

// BiCGStab for every instance with h_mask set (tolerance h_eta): one persistent launch
// for the whole batch when available, else graph-captured iteration kernels; returns with
// h_bst holding every instance's final state.
template <typename V>
egfem_status run_batch_bicgstab(egfem_t *h, KWork<V> &W, cudaGraphExec_t &G, int32_t stall, int64_t *launches) {
    EG_CUDA(cudaMemcpyAsync(h->inst_mask, h->h_mask, size_t(h->nb), cudaMemcpyHostToDevice, h->hs));
    EG_CUDA(cudaMemcpyAsync(h->inst_eta, h->h_eta, size_t(h->nb) * sizeof(double), cudaMemcpyHostToDevice, h->hs));
    const int pg = pk_batch_grid<V>(h);
    if (pg > 0) {
        EG_TRY(launch_batch_persistent(h, W, pg, h->opts.krylov_maxit, stall));
        EG_CUDA(cudaMemcpyAsync(h->h_bst, h->bst, size_t(h->nb) * sizeof(KState), cudaMemcpyDeviceToHost, h->hs));
        PGrid gb{};
        EG_CUDA(cudaMemcpyAsync(&gb, h->bbar, sizeof(PGrid), cudaMemcpyDeviceToHost, h->hs));
        EG_CUDA(cudaStreamSynchronize(h->hs));
        *launches += 1;
        if (gb.err) {
            g_last_error = gb.err == 2 ? "batched BiCGStab: more tiles than the persistent solve holds per block"
                                       : "batched BiCGStab: a grid-barrier wait of the persistent solve ran out";
            return gb.err == 2 ? EGFEM_ERR_INVALID_ARG : EGFEM_ERR_TIMEOUT;
        }
        return EGFEM_OK;
    }
    EG_TRY(batch_graph(h, W, G));
    kb_init_state<<<(h->nb + 127) / 128, 128, 0, h->hs>>>(h->nb, h->bst, h->inst_mask, h->inst_eta, h->opts.krylov_maxit, stall);
    const KBatch<V> B = kbatch(h, W);
    kb_setup<V><<<bgrid<V>(h), KRY_BLOCK, 0, h->hs>>>(B);
    EG_CUDA(cudaGetLastError());
    *launches += 2;
    for (;;) {
        EG_CUDA(cudaMemcpyAsync(h->h_bst, h->bst, size_t(h->nb) * sizeof(KState), cudaMemcpyDeviceToHost, h->hs));
        EG_CUDA(cudaStreamSynchronize(h->hs));
        bool running = false;
        for (int32_t b = 0; b < h->nb && !running; ++b) running = h->h_bst[b].done == K_RUNNING;
        if (!running) break;
        EG_CUDA(cudaGraphLaunch(G, h->hs));
        *launches += 5 * int64_t(std::max(1, h->opts.graph_chunk));
    }
    return EGFEM_OK;
}

// Time a few batched BiCGStab iterations for each tile size and keep the fastest
// (the project's autotuner; it runs once per handle, on the first batched solve).  With
// the persistent solve, a tile size is a candidate only if no block owns more than
// PK_MAXT tiles.
template <typename V>
egfem_status autotune_tiles(egfem_t *h, KWork<V> &W) {
    cudaEvent_t e0, e1;
    EG_CUDA(cudaEventCreate(&e0));
    EG_CUDA(cudaEventCreate(&e1));
    int best = 1;
    float best_ms = 1e30f;
    for (int f : {1, 2, 4, 8}) {
        EG_TRY(batch_tiles<V>(h, f));
        for (int32_t b = 0; b < h->nb; ++b) { h->h_mask[b] = 1; h->h_eta[b] = 0.0; }
        EG_CUDA(cudaMemcpyAsync(h->inst_mask, h->h_mask, size_t(h->nb), cudaMemcpyHostToDevice, h->hs));
        EG_CUDA(cudaMemcpyAsync(h->inst_eta, h->h_eta, size_t(h->nb) * sizeof(double), cudaMemcpyHostToDevice, h->hs));
        float ms = 0;
        const int pg = pk_batch_grid<V>(h);
        if (h->coop && h->opts.krylov_persistent) {
            if (pg == 0) continue;   // too many tiles per block at this size
            // setup + 2 iterations (warm), then setup + 8 iterations; the difference is 6 iterations
            EG_TRY(launch_batch_persistent(h, W, pg, 2, 0));
            EG_CUDA(cudaEventRecord(e0, h->hs));
            EG_TRY(launch_batch_persistent(h, W, pg, 2, 0));
            EG_CUDA(cudaEventRecord(e1, h->hs));
            EG_CUDA(cudaEventSynchronize(e1));
            float ms2 = 0;
            EG_CUDA(cudaEventElapsedTime(&ms2, e0, e1));
            EG_CUDA(cudaEventRecord(e0, h->hs));
            EG_TRY(launch_batch_persistent(h, W, pg, 8, 0));
            EG_CUDA(cudaEventRecord(e1, h->hs));
            EG_CUDA(cudaEventSynchronize(e1));
            EG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms -= ms2;
        } else {
            kb_init_state<<<(h->nb + 127) / 128, 128, 0, h->hs>>>(h->nb, h->bst, h->inst_mask, h->inst_eta, 1 << 30, 0);
            const KBatch<V> B = kbatch(h, W);
            kb_setup<V><<<bgrid<V>(h), KRY_BLOCK, 0, h->hs>>>(B);
            enqueue_batch_iterations(h, W, 2, h->hs);   // warm
            EG_CUDA(cudaEventRecord(e0, h->hs));
            enqueue_batch_iterations(h, W, 6, h->hs);
            EG_CUDA(cudaEventRecord(e1, h->hs));
            EG_CUDA(cudaEventSynchronize(e1));
            EG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (ms < best_ms) { best_ms = ms; best = f; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return batch_tiles<V>(h, best);
}

egfem_status batch_norms(egfem_t *h) {
    kb_norm2<<<int(std::max<int64_t>(1, std::min<int64_t>(h->ntiles, int64_t(h->sms) * 8))), KRY_BLOCK, 0, h->hs>>>(
        h->ntiles, h->tiles, h->bst, h->bpart, h->r, h->csf.dir, h->n, h->inst_norm2);
    EG_CUDA(cudaGetLastError());
    EG_CUDA(cudaMemcpyAsync(h->h_norm2, h->inst_norm2, size_t(h->nb) * sizeof(double), cudaMemcpyDeviceToHost, h->hs));
    EG_CUDA(cudaStreamSynchronize(h->hs));
    return EGFEM_OK;
}

// Capture the body of the graph-resident batched Newton loop (see egfem_gnewton.cuh) for the
// vectors d_u, d_d and the FP64 (V = double) or mixed (V = df64) path, under a conditional
// WHILE node; the graph is kept for later calls with the same vectors and path.
template <typename V>
egfem_status gn_build(egfem_t *h, KWork<V> &W, double *d_u, const double *d_d, int pg) {
    constexpr bool mixed = std::is_same<V, df64>::value;
    if (h->gn_exec && h->gn_u == d_u && h->gn_d == d_d && h->gn_mixed == int(mixed) && h->gn_one == 0) return EGFEM_OK;
    if (h->gn_exec) { cudaGraphExecDestroy(h->gn_exec); h->gn_exec = nullptr; }
    if (!h->bbar) EG_TRY(dalloc(h->bbar, 1));   // no allocation may happen inside the capture
    if (!h->gn_state) {
        EG_TRY(dalloc(h->gn_state, size_t(std::max<int32_t>(h->nb, 1))));
        EG_TRY(dalloc(h->gn_stats, size_t(h->nb)));
        EG_TRY(dalloc(h->gn_loops, 1));
    }
    cudaGraph_t g = nullptr;
    EG_CUDA(cudaGraphCreate(&g, 0));
    egfem_status st = EGFEM_OK;
    cudaError_t e = cudaSuccess;
    cudaGraphConditionalHandle cond{};
    cudaGraphNodeParams np{};
    cudaGraphNode_t node = nullptr;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->hs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        g_last_error = std::string("graph Newton loop: ") + cudaGetErrorString(e);
        return EGFEM_ERR_CUDA;
    }
    GNArgs G{};
    G.nb = h->nb; G.state = h->gn_state; G.stats = h->gn_stats; G.mask = h->inst_mask; G.eta_out = h->inst_eta;
    G.lam = h->inst_lam; G.kst = h->bst; G.norm2 = h->inst_norm2; G.loops = h->gn_loops;
    G.kerr = &h->bbar->err;
    G.max_loops = gn_max_loops(h->opts.newton_maxit); G.newton_maxit = h->opts.newton_maxit;
    G.fixed_eta = h->opts.fixed_eta; G.mixed = int(mixed);
    G.eta_max = eta_cap(h); G.eta_min = h->opts.eta_min; G.eta_floor = mixed ? kMixedEtaFloor : 0.0; G.cond = cond;
    const unsigned gu = unsigned((h->n + 255) / 256);
    int nodes = 0;
    gn_pre<<<1, 256, 0, h->hs>>>(G);
    st = launch_batch_persistent(h, W, pg, h->opts.krylov_maxit, mixed ? kMixedStall : 0);
    gn_mid<<<1, 256, 0, h->hs>>>(G);
    kb_update<V><<<gu, 256, 0, h->hs>>>(h->n, h->slice_inst, h->inst_mask, h->inst_lam, d_u, W.x);
    CsfArgs A = csf_args(h, d_u, d_d);
    A.r = h->r; A.q64 = h->k64.b;
    if (mixed) A.a32 = h->k32.A;   // the FP64 redo, which needs the FP64 operator, is the host loop's
    else A.a64 = h->k64.A;
    A.slice_inst = h->slice_inst; A.inst_mask = h->inst_mask;
    nodes += launch_csf(h, A, h->hs);
    if (mixed) { cast_kernel<double, df64><<<gu, 256, 0, h->hs>>>(h->n, h->k64.b, h->k32.b); ++nodes; }
    kb_norm2<<<int(std::max<int64_t>(1, std::min<int64_t>(h->ntiles, int64_t(h->sms) * 8))), KRY_BLOCK, 0, h->hs>>>(
        h->ntiles, h->tiles, h->bst, h->bpart, h->r, h->csf.dir, h->n, h->inst_norm2);
    gn_post<<<1, 256, 0, h->hs>>>(G);
    kb_update<V><<<gu, 256, 0, h->hs>>>(h->n, h->slice_inst, h->inst_mask, h->inst_lam, d_u, W.x);
    nodes += 7;
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(h->hs, &body);
    if (st == EGFEM_OK && e == cudaSuccess) e = cudaGetLastError();
    if (st == EGFEM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->gn_exec, g, 0);
    cudaGraphDestroy(g);
    if (st != EGFEM_OK || e != cudaSuccess) {
        if (e != cudaSuccess) g_last_error = std::string("graph Newton loop: ") + cudaGetErrorString(e);
        cudaGetLastError();
        h->gn_exec = nullptr;
        return st != EGFEM_OK ? st : EGFEM_ERR_CUDA;
    }
    h->gn_u = d_u; h->gn_d = d_d; h->gn_mixed = int(mixed); h->gn_nodes = nodes; h->gn_one = 0;
    return EGFEM_OK;
}

// Run the graph-resident Newton loop from the host driver's state (after its first residual
// evaluation) and take its state back: instances it handed back (resume64: their current step
// awaits the FP64 redo, from rbefore with forcing term eta), and any it did not finish, continue
// in the host loop.  Returns false when the graph is unavailable (the host loop then does
// everything).
template <typename V>
bool gn_run(egfem_t *h, KWork<V> &W, double *d_u, const double *d_d, std::vector<double> &rn, std::vector<double> &rprev,
            std::vector<double> &eta, const std::vector<double> &target, std::vector<int32_t> &st,
            std::vector<egfem_stats> &S, std::vector<double> &rbefore, std::vector<int> &resume64, int64_t *launches) {
    if (!h->opts.newton_graph || h->gn_failed) return false;
    const int pg = pk_batch_grid<V>(h);
    if (pg <= 0) return false;
    if (gn_build<V>(h, W, d_u, d_d, pg) != EGFEM_OK) { h->gn_failed = true; return false; }
    h->gn_used = true;
    const int nb = h->nb;
    std::vector<GNState> G(nb);
    for (int b = 0; b < nb; ++b) G[b] = GNState{rn[b], rprev[b], rn[b], target[b], eta[b], 1.0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h->gn_state, G.data(), sizeof(GNState) * size_t(nb), cudaMemcpyHostToDevice, h->hs) != cudaSuccess ||
        cudaMemcpyAsync(h->gn_stats, S.data(), sizeof(egfem_stats) * size_t(nb), cudaMemcpyHostToDevice, h->hs) != cudaSuccess ||
        cudaMemsetAsync(h->gn_loops, 0, sizeof(int32_t), h->hs) != cudaSuccess ||
        cudaGraphLaunch(h->gn_exec, h->hs) != cudaSuccess) {
        cudaGetLastError();
        h->gn_failed = true;
        return false;
    }
    int32_t loops = 0;
    cudaMemcpyAsync(G.data(), h->gn_state, sizeof(GNState) * size_t(nb), cudaMemcpyDeviceToHost, h->hs);
    cudaMemcpyAsync(S.data(), h->gn_stats, sizeof(egfem_stats) * size_t(nb), cudaMemcpyDeviceToHost, h->hs);
    cudaMemcpyAsync(&loops, h->gn_loops, sizeof(int32_t), cudaMemcpyDeviceToHost, h->hs);
    if (cudaStreamSynchronize(h->hs) != cudaSuccess) return true;   // the caller's next CUDA call reports it
    for (int b = 0; b < nb; ++b) {
        rn[b] = G[b].rn; rprev[b] = G[b].rprev; eta[b] = G[b].eta; rbefore[b] = G[b].rbefore;
        resume64[b] = G[b].host != 0;
        st[b] = S[b].status;
    }
    *launches += int64_t(loops) * h->gn_nodes;
    return true;
}

egfem_status batch_newton(egfem_t *h, double *d_u, const double *d_d, egfem_stats *stats) {
    const int nb = h->nb;
    const bool mixed = h->opts.precision == EGFEM_PREC_MIXED;
    EG_TRY(kwork_alloc(h, h->k64));
    if (mixed) EG_TRY(kwork_alloc(h, h->k32));
    if (!h->tile_factor) {
        // tune on the operator at the initial state
        CsfArgs A0 = csf_args(h, d_u, d_d);
        A0.r = h->r; A0.a64 = h->k64.A; A0.q64 = h->k64.b;
        if (mixed) A0.a32 = h->k32.A;
        launch_csf(h, A0, h->hs);
        if (mixed) cast_kernel<double, df64><<<unsigned((h->n + 255) / 256), 256, 0, h->hs>>>(h->n, h->k64.b, h->k32.b);
        // the tile autotuner times the five-barrier batched solve; the windowed one plans its own tiles
        if (mixed) EG_TRY(h->k32.pkwb_smem > 0 ? batch_tiles<df64>(h, 4) : autotune_tiles<df64>(h, h->k32));
        else EG_TRY(h->k64.pkwb_smem > 0 ? batch_tiles<double>(h, 4) : autotune_tiles<double>(h, h->k64));
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<egfem_stats> S(nb);
    for (auto &x : S) std::memset(&x, 0, sizeof(x));
    std::vector<double> rn(nb), rprev(nb), rbefore(nb), target(nb), eta(nb, eta_cap(h)), lam(nb, 1.0);
    std::vector<int> active(nb, 0), fp32(nb, 0), pending(nb, 0), resume64(nb, 0);
    std::vector<int32_t> st(nb, EGFEM_OK);
    int64_t launches = 0;
    // evaluate residual/operator for instances with mask m
    // mixed path: the residual in FP64 and the FP32 operator (csf_mixed_kernel); the FP64 operator
    // is formed only for the instances whose step is redone in FP64 (eval64 below)
    if (mixed && h->opts.op == EGFEM_OP_CSF) EG_TRY(ensure_mixed_tensor(h, h->hs));
    auto eval = [&](const std::vector<int> &m) -> egfem_status {
        for (int b = 0; b < nb; ++b) h->h_mask[b] = uint8_t(m[b]);
        EG_CUDA(cudaMemcpyAsync(h->inst_mask, h->h_mask, size_t(nb), cudaMemcpyHostToDevice, h->hs));
        CsfArgs A = csf_args(h, d_u, d_d);
        A.r = h->r; A.q64 = h->k64.b;
        if (mixed) A.a32 = h->k32.A;
        else A.a64 = h->k64.A;
        A.slice_inst = h->slice_inst; A.inst_mask = h->inst_mask;
        launches += launch_csf(h, A, h->hs) + 1 + (mixed ? 1 : 0);
        if (mixed) cast_kernel<double, df64><<<unsigned((h->n + 255) / 256), 256, 0, h->hs>>>(h->n, h->k64.b, h->k32.b);
        EG_CUDA(cudaGetLastError());
        EG_TRY(batch_norms(h));
        for (int b = 0; b < nb; ++b) if (m[b]) rn[b] = std::sqrt(h->h_norm2[b]);
        return EGFEM_OK;
    };
    // the FP64 operator (and D r) at the current u for instances with mask m: the FP64 redo of a
    // mixed step
    auto eval64 = [&](const std::vector<int> &m) -> egfem_status {
        for (int b = 0; b < nb; ++b) h->h_mask[b] = uint8_t(m[b]);
        EG_CUDA(cudaMemcpyAsync(h->inst_mask, h->h_mask, size_t(nb), cudaMemcpyHostToDevice, h->hs));
        CsfArgs A = csf_args(h, d_u, d_d);
        A.r = h->r; A.q64 = h->k64.b; A.a64 = h->k64.A;
        A.slice_inst = h->slice_inst; A.inst_mask = h->inst_mask;
        launches += launch_csf(h, A, h->hs);
        EG_CUDA(cudaGetLastError());
        return EGFEM_OK;
    };
    // u -= lam_b x_b for instances with mask m, x from the FP32 (p32) or FP64 workspace
    auto update = [&](const std::vector<int> &m, const std::vector<double> &l, bool p32) -> egfem_status {
        for (int b = 0; b < nb; ++b) { h->h_mask[b] = uint8_t(m[b]); h->h_lam[b] = l[b]; }
        EG_CUDA(cudaMemcpyAsync(h->inst_mask, h->h_mask, size_t(nb), cudaMemcpyHostToDevice, h->hs));
        EG_CUDA(cudaMemcpyAsync(h->inst_lam, h->h_lam, size_t(nb) * sizeof(double), cudaMemcpyHostToDevice, h->hs));
        const unsigned g = unsigned((h->n + 255) / 256);
        if (p32) kb_update<df64><<<g, 256, 0, h->hs>>>(h->n, h->slice_inst, h->inst_mask, h->inst_lam, d_u, h->k32.x);
        else kb_update<double><<<g, 256, 0, h->hs>>>(h->n, h->slice_inst, h->inst_mask, h->inst_lam, d_u, h->k64.x);
        EG_CUDA(cudaGetLastError());
        ++launches;
        return EGFEM_OK;
    };
    std::vector<int> all(nb, 1);
    EG_TRY(eval(all));
    for (int b = 0; b < nb; ++b) {
        S[b].res0 = rn[b];
        target[b] = std::max(h->opts.newton_rtol * rn[b], h->opts.newton_atol);
        rprev[b] = rn[b];
    }
    // the Newton loop on the device (damping included); the host loop below finishes what it hands back
    h->gn_used = false;
    const bool ran = mixed ? gn_run<df64>(h, h->k32, d_u, d_d, rn, rprev, eta, target, st, S, rbefore, resume64, &launches)
                           : gn_run<double>(h, h->k64, d_u, d_d, rn, rprev, eta, target, st, S, rbefore, resume64, &launches);
    if (!ran && h->opts.newton_graph == 2) {
        g_last_error = "graph Newton loop required (newton_graph = 2) but unavailable: " + g_last_error;
        return EGFEM_ERR_UNSUPPORTED;
    }
    if (ran) {
        EG_CUDA(cudaGetLastError());
        std::vector<int> left(nb, 0);
        bool any = false;
        for (int b = 0; b < nb; ++b) {
            left[b] = st[b] == EGFEM_OK && !(rn[b] <= target[b]);
            any = any || left[b];
        }
        if (any) EG_TRY(eval(left));   // their residual and operator at the current u
    }
    for (int step = 0; step <= h->opts.newton_maxit; ++step) {
        bool any = false;
        for (int b = 0; b < nb; ++b) {
            active[b] = 0;
            if (st[b] != EGFEM_OK) continue;
            if (!std::isfinite(rn[b])) { st[b] = EGFEM_ERR_NONFINITE; continue; }
            if (rn[b] <= target[b]) continue;
            if (S[b].newton_iters >= h->opts.newton_maxit) { st[b] = EGFEM_ERR_NOT_CONVERGED; continue; }
            active[b] = 1;
            any = true;
            if (resume64[b]) {   // the graph's step, handed back for its FP64 redo
                fp32[b] = 0;
                resume64[b] = 0;
                continue;
            }
            if (S[b].newton_iters > 0 && !h->opts.fixed_eta) {
                double e = 0.9 * (rn[b] / rprev[b]) * (rn[b] / rprev[b]);
                const double sg = 0.9 * eta[b] * eta[b];
                if (sg > 0.1) e = std::max(e, sg);
                eta[b] = std::max(std::min(eta_cap(h), e), 0.5 * target[b] / rn[b]);
            }
            eta[b] = std::max(eta[b], h->opts.eta_min);
            fp32[b] = mixed ? 1 : 0;
            rbefore[b] = rn[b];
        }
        if (!any) break;
        // up to two passes: FP32 for the mixed path, then FP64 for the instances it failed
        for (int pass = 0; pass < 2; ++pass) {
            const bool p32 = mixed && pass == 0;
            bool todo = false;
            for (int b = 0; b < nb; ++b) {
                pending[b] = active[b] && (fp32[b] == (p32 ? 1 : 0));
                h->h_mask[b] = uint8_t(pending[b]);
                h->h_eta[b] = p32 ? std::max(eta[b], kMixedEtaFloor) : eta[b];
                todo = todo || pending[b];
            }
            if (!todo) continue;
            if (mixed && !p32) {
                // the FP64 operator of the instances redone in FP64 (the mixed evaluations skip it)
                std::vector<int> redo(pending.begin(), pending.end());
                EG_TRY(eval64(redo));
                for (int b = 0; b < nb; ++b) h->h_mask[b] = uint8_t(pending[b]);
            }
            if (p32) EG_TRY(run_batch_bicgstab(h, h->k32, h->bgraph32, kMixedStall, &launches));
            else EG_TRY(run_batch_bicgstab(h, h->k64, h->bgraph64, 0, &launches));
            std::vector<int> ok(nb, 0);
            for (int b = 0; b < nb; ++b) {
                if (!pending[b]) continue;
                const KState &K = h->h_bst[b];
                S[b].krylov_iters += K.iter;
                if (S[b].newton_iters < EGFEM_HIST) S[b].krylov_hist[S[b].newton_iters] += K.iter;
                const bool failed = K.done == K_NONFINITE || (K.done == K_BREAKDOWN && (p32 || K.iter == 0));
                if (failed) {
                    if (p32) { fp32[b] = 0; ++S[b].fp64_rescues; }
                    else { st[b] = K.done == K_NONFINITE ? EGFEM_ERR_NONFINITE : EGFEM_ERR_BREAKDOWN; active[b] = 0; }
                    continue;
                }
                ok[b] = 1;
                lam[b] = 1.0;
            }
            EG_TRY(update(ok, lam, p32));
            EG_TRY(eval(ok));
            // damping: halve the step of every instance whose residual fails the Armijo test
            for (int bt = 0; bt < 6; ++bt) {
                std::vector<int> bad(nb, 0);
                std::vector<double> dl(nb, 0.0);
                bool anybad = false;
                for (int b = 0; b < nb; ++b)
                    if (ok[b] && !(rn[b] <= (1.0 - 1e-4 * lam[b]) * rbefore[b])) { bad[b] = 1; dl[b] = -0.5 * lam[b]; anybad = true; }
                if (!anybad) break;
                EG_TRY(update(bad, dl, p32));
                for (int b = 0; b < nb; ++b) if (bad[b]) lam[b] *= 0.5;
                EG_TRY(eval(bad));
            }
            std::vector<int> undo(nb, 0);
            bool anyundo = false;
            for (int b = 0; b < nb; ++b) {
                if (!ok[b]) continue;
                if (rn[b] < rbefore[b]) {
                    ++S[b].newton_iters;
                    if (S[b].newton_iters - 1 < EGFEM_HIST) S[b].res_hist[S[b].newton_iters - 1] = rn[b];
                    rprev[b] = rbefore[b];
                    active[b] = 0;   // stepped
                    continue;
                }
                undo[b] = 1;
                anyundo = true;
            }
            if (anyundo) {
                // no step length decreased the residual: step back by the applied length
                std::vector<double> back(nb, 0.0);
                for (int b = 0; b < nb; ++b) back[b] = -lam[b];
                EG_TRY(update(undo, back, p32));
                EG_TRY(eval(undo));
                for (int b = 0; b < nb; ++b) {
                    if (!undo[b]) continue;
                    if (p32) { fp32[b] = 0; ++S[b].fp64_rescues; }
                    else { st[b] = EGFEM_ERR_NOT_CONVERGED; active[b] = 0; }
                }
            }
        }
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    egfem_status worst = EGFEM_OK;
    for (int b = 0; b < nb; ++b) {
        if (st[b] == EGFEM_OK && !(rn[b] <= target[b])) st[b] = EGFEM_ERR_NOT_CONVERGED;
        S[b].status = st[b];
        S[b].res_final = rn[b];
        S[b].solve_ms = ms;
        S[b].kernel_launches = launches;
        if (st[b] != EGFEM_OK && worst == EGFEM_OK) worst = egfem_status(st[b]);
    }
    if (stats) std::memcpy(stats, S.data(), sizeof(egfem_stats) * size_t(nb));
    return worst;
}

}  // namespace

extern "C" {

egfem_status egfem_batch_build(int32_t count, const egfem_mesh *meshes, const egfem_problem *prob, const egfem_options *opts,
                               egfem_handle *out) {
    if (count < 1 || !meshes || !prob || !out) { g_last_error = "bad batch arguments"; return EGFEM_ERR_INVALID_ARG; }
    try {
        const int32_t dim = meshes[0].dim;
        std::vector<int64_t> off(size_t(count) + 1, 0), coff(size_t(count) + 1, 0);
        for (int32_t b = 0; b < count; ++b) {
            const egfem_mesh &m = meshes[b];
            if (m.dim != dim) { g_last_error = "all batch meshes must share one dimension"; return EGFEM_ERR_INVALID_ARG; }
            std::string err;
            egfem_status st = validate_mesh(m, err);
            if (st != EGFEM_OK) { g_last_error = "instance " + std::to_string(b) + ": " + err; return st; }
            off[b + 1] = off[b] + (m.n_nodes + SLICE - 1) / SLICE * SLICE;
            coff[b + 1] = coff[b] + m.n_cells;
        }
        const int64_t N = off[count], C = coff[count];
        if (N >= (int64_t(1) << 31) - 1) { g_last_error = "batch too large for int32 node indices"; return EGFEM_ERR_INVALID_ARG; }
        // disjoint union; the padding nodes of each instance belong to no cell and are Dirichlet
        std::vector<double> X(size_t(N) * dim, 0.0);
        std::vector<int32_t> cells(size_t(C) * (dim + 1));
        std::vector<uint8_t> dir(size_t(N), 1);
        for (int32_t b = 0; b < count; ++b) {
            const egfem_mesh &m = meshes[b];
            std::memcpy(&X[size_t(off[b]) * dim], m.coords, sizeof(double) * size_t(m.n_nodes) * dim);
            for (int64_t v = 0; v < m.n_nodes; ++v) dir[size_t(off[b] + v)] = m.dirichlet ? (m.dirichlet[v] ? 1 : 0) : 0;
            for (int64_t c = 0; c < m.n_cells * (dim + 1); ++c) cells[size_t(coff[b] * (dim + 1) + c)] = int32_t(m.cells[c] + off[b]);
        }
        // one mesh for every instance (byte for byte): the tensor can be stored once
        bool same = count > 1;
        for (int32_t b = 1; b < count && same; ++b) {
            const egfem_mesh &m = meshes[b], &m0 = meshes[0];
            same = m.n_nodes == m0.n_nodes && m.n_cells == m0.n_cells &&
                   std::memcmp(&X[size_t(off[b]) * dim], &X[0], sizeof(double) * size_t(m.n_nodes) * dim) == 0 &&
                   std::memcmp(&dir[size_t(off[b])], &dir[0], size_t(m.n_nodes)) == 0 &&
                   std::memcmp(m.cells, m0.cells, sizeof(int32_t) * size_t(m.n_cells) * (dim + 1)) == 0;
        }
        egfem_mesh U{dim, N, C, X.data(), cells.data(), dir.data()};
        egfem_status st = build_impl(&U, prob, opts, out, same ? count : 0, same ? off[1] : 0);
        if (st != EGFEM_OK) return st;
        egfem_t *h = *out;
        h->nb = count;
        h->inst_off = off;
        std::vector<int32_t> si(size_t(h->csf.n_slices));
        for (int32_t b = 0; b < count; ++b)
            for (int64_t sl = off[b] / SLICE; sl < off[b + 1] / SLICE; ++sl) si[size_t(sl)] = b;
        auto fail = [&](egfem_status e) { egfem_destroy(h); *out = nullptr; return e; };
        if ((st = upload(h->slice_inst, si)) != EGFEM_OK) return fail(st);
        if ((st = dalloc(h->inst_mask, size_t(count))) != EGFEM_OK) return fail(st);
        if ((st = dalloc(h->inst_eta, size_t(count))) != EGFEM_OK) return fail(st);
        if ((st = dalloc(h->inst_lam, size_t(count))) != EGFEM_OK) return fail(st);
        if ((st = dalloc(h->inst_norm2, size_t(count))) != EGFEM_OK) return fail(st);
        if ((st = dalloc(h->bst, size_t(count))) != EGFEM_OK) return fail(st);
        if (cudaMemset(h->bst, 0, sizeof(KState) * size_t(count)) != cudaSuccess) return fail(EGFEM_ERR_CUDA);
        if (cudaMallocHost((void **)&h->h_mask, size_t(count)) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_eta, sizeof(double) * size_t(count)) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_lam, sizeof(double) * size_t(count)) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_norm2, sizeof(double) * size_t(count)) != cudaSuccess ||
            cudaMallocHost((void **)&h->h_bst, sizeof(KState) * size_t(count)) != cudaSuccess)
            return fail(EGFEM_ERR_OOM);
        return EGFEM_OK;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return EGFEM_ERR_OOM;
    }
}

egfem_status egfem_batch_layout(egfem_handle h, int32_t *count, int64_t *offsets) {
    if (!h) return EGFEM_ERR_INVALID_ARG;
    if (count) *count = h->nb;
    if (offsets) std::memcpy(offsets, h->inst_off.data(), sizeof(int64_t) * h->inst_off.size());
    return EGFEM_OK;
}

egfem_status egfem_batch_newton_solve(egfem_handle h, double *d_u, const double *d_d, egfem_stats *stats, egfem_stream stream) {
    if (!h || !d_u || !d_d || h->nb < 1) return EGFEM_ERR_INVALID_ARG;
    EG_CUDA(cudaSetDevice(h->device));
    EG_TRY(join_in(h, (cudaStream_t)stream));
    egfem_status st = batch_newton(h, d_u, d_d, stats);
    egfem_status js = join_out(h, (cudaStream_t)stream);
    return st != EGFEM_OK ? st : js;
}

}  // extern "C"
