// egfem_noalloc.cu -- the free-row residual norm with its scratch in static device memory.
//
// Some callers cannot call cudaMalloc when they need this number: applications that hand
// all device memory to their own pool up front, or real-time loops where cudaMalloc's
// implicit device synchronisation and latency are not acceptable.  This entry point
// computes sum_{i : dirichlet[i] == 0} r_i^2 (the quantity of the Newton convergence test)
// by a deterministic two-stage reduction: repeatable from call to call, but not bit-identical
// to the handle's own norm, which partitions the rows differently (the two agree to rounding).
// Its block partials and completion ticket live in a file-scope __device__ array that
// exists as soon as the library is loaded (every GPU that loads it holds the array until
// the process exits).  It allocates nothing and needs no handle.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "egfem_internal.h"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int64_t NA_ROWS_PER_BLOCK = int64_t(NA_BLOCK) * 64;   // rows reduced by one block
constexpr int NA_MAX_BLOCKS = 8192;                              // block partials in the scratch

// scratch: NA_MAX_BLOCKS doubles of block partials, then the 32-bit completion ticket
// (kept 256-byte aligned at the front of its own 256-byte slot)
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 32];

// Set-up once per device context: the host-side name of the array is not a device address,
// so the kernel receives the address that cudaGetSymbolAddress returns with the device
// current.  The address is cached with the id of the context it belongs to: after a
// cudaDeviceReset the module is loaded into a new context (new id) and the address is looked
// up again instead of reusing one that may now be unmapped or belong to another allocation.
// The two driver calls come through the runtime's entry-point query, so the library does not
// link the driver library itself.
std::mutex g_na_mutex;
constexpr int NA_MAX_DEVICES = 64;
struct NaSlot { double *ptr; unsigned long long ctx_id; };
NaSlot g_na[NA_MAX_DEVICES] = {};

typedef CUresult (*NaCtxGetCurrent)(CUcontext *);
typedef CUresult (*NaCtxGetId)(CUcontext, unsigned long long *);

// id of the calling thread's current context; false when it cannot be read (no context yet,
// or the driver does not offer the query), in which case nothing is cached
bool na_current_ctx_id(unsigned long long &id) {
    static NaCtxGetCurrent get_cur = nullptr;
    static NaCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<NaCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<NaCtxGetId>(f);
    });
    if (!get_cur || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, &id) == CUDA_SUCCESS;
}

// device address of the scratch array in the current device's context
egfem_status na_scratch(int dev, double *&scratch) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long id = 0;
    const bool have_id = na_current_ctx_id(id);
    if (have_id && g_na[dev].ptr && g_na[dev].ctx_id == id) {
        scratch = g_na[dev].ptr;
        return EGFEM_OK;
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        egfem::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return EGFEM_ERR_CUDA;
    }
    scratch = static_cast<double *>(p);
    unsigned long long id2 = 0;   // the lookup above creates the context if none was current
    g_na[dev] = na_current_ctx_id(id2) ? NaSlot{scratch, id2} : NaSlot{nullptr, 0ull};
    return EGFEM_OK;
}

__device__ __forceinline__ double na_warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block b sums rows [b * NA_ROWS_PER_BLOCK, (b + 1) * NA_ROWS_PER_BLOCK) into
// scratch[b]; the last block to finish adds the partials in block order.
__global__ void __launch_bounds__(NA_BLOCK) noalloc_norm2_kernel(int64_t n, const double *r, const uint8_t *dir,
                                                                 double *scratch, double *out) {
    __shared__ double sh[NA_BLOCK / 32];
    __shared__ bool last;
    uint32_t *ticket = reinterpret_cast<uint32_t *>(scratch + NA_MAX_BLOCKS);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t lo = int64_t(blockIdx.x) * NA_ROWS_PER_BLOCK;
    const int64_t hi = lo + NA_ROWS_PER_BLOCK < n ? lo + NA_ROWS_PER_BLOCK : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += NA_BLOCK)
        if (!dir[i]) acc += r[i] * r[i];
    acc = na_warp_sum(acc);
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int q = 0; q < NA_BLOCK / 32; ++q) x += sh[q];
        scratch[blockIdx.x] = x;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double x = 0.0;
    for (int q = threadIdx.x; q < int(gridDim.x); q += NA_BLOCK) x += __ldcg(&scratch[q]);
    x = na_warp_sum(x);
    if (lane == 0) sh[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < NA_BLOCK / 32; ++q) t += sh[q];
        *out = t;
        *ticket = 0u;
    }
}

}  // namespace

extern "C" egfem_status egfem_free_norm2_noalloc(int64_t n, const double *d_r, const uint8_t *d_dirichlet, double *d_out,
                                                 egfem_stream stream) {
    if (n < 1 || !d_r || !d_dirichlet || !d_out) { egfem::set_last_error("null pointer or empty vector"); return EGFEM_ERR_INVALID_ARG; }
    if (n > int64_t(NA_MAX_BLOCKS) * NA_ROWS_PER_BLOCK) {
        egfem::set_last_error("n exceeds the static scratch (at most " + std::to_string(int64_t(NA_MAX_BLOCKS) * NA_ROWS_PER_BLOCK) + " rows)");
        return EGFEM_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) { egfem::set_last_error("no usable current device"); return EGFEM_ERR_CUDA; }
    double *scratch = nullptr;
    const egfem_status st = na_scratch(dev, scratch);
    if (st != EGFEM_OK) return st;
    // the ticket must start at zero: a previous call may have been interrupted
    if (cudaMemsetAsync(scratch + NA_MAX_BLOCKS, 0, sizeof(uint32_t), (cudaStream_t)stream) != cudaSuccess) {
        egfem::set_last_error("cudaMemsetAsync of the ticket failed");
        return EGFEM_ERR_CUDA;
    }
    const unsigned grid = unsigned((n + NA_ROWS_PER_BLOCK - 1) / NA_ROWS_PER_BLOCK);
    noalloc_norm2_kernel<<<grid, NA_BLOCK, 0, (cudaStream_t)stream>>>(n, d_r, d_dirichlet, scratch, d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { egfem::set_last_error(std::string("launch: ") + cudaGetErrorString(e)); return EGFEM_ERR_CUDA; }
    return EGFEM_OK;
}
