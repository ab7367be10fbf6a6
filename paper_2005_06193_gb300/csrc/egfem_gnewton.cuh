// egfem_gnewton.cuh -- the batched Newton loop as one CUDA graph: a conditional WHILE node whose
// body is  control (which instances step, their forcing terms) -> the batched persistent
// BiCGStab -> control (Krylov outcome) -> u -= x -> tensor action + residual norms -> control
// (acceptance) -> revert of rejected steps.  The controller kernels keep every instance's
// Newton state in device memory and clear the loop's condition when no instance has a step to
// take, so a whole batched solve runs without the host.
//
// An instance whose full step fails the sufficient-decrease test, or whose Krylov solve broke
// down, has the step reverted and is handed back (host = 1): the host driver then finishes it
// with step halving and, on the mixed path, an FP64 redo -- the graph only takes full steps.
// A single system uses the same controllers with one instance (nb = 1).
#pragma once

#include "egfem_kernels.cuh"
#include "egfem_krylov.cuh"

namespace egfem {

// Newton state of one instance, device-resident while the graph runs
struct GNState {
    double rn;        // current ||r|| over free rows
    double rprev;     // ||r|| before the last accepted step (Eisenstat-Walker)
    double rbefore;   // ||r|| when the current step started
    double target;    // stop when rn <= target
    double eta;       // forcing term of the current step
    int32_t host;     // 1: handed back to the host driver
    int32_t pad;
};

struct GNArgs {
    int32_t nb;
    GNState *state;
    egfem_stats *stats;          // per instance: status, newton_iters, krylov_iters, histories
    uint8_t *mask;               // instances taking part in the next kernels
    double *eta_out;             // Krylov tolerance per instance
    double *lam;                 // step factor per instance (1: step, -1: revert)
    const KState *kst;           // final Krylov state per instance
    const double *norm2;         // ||r||^2 per instance after the tensor action
    int32_t *loops;              // body executions so far
    int32_t max_loops;
    int32_t newton_maxit, fixed_eta;
    double eta_max, eta_min, eta_floor;
    cudaGraphConditionalHandle cond;
};

// Start of a body: which instances take a step and their forcing terms (Eisenstat-Walker,
// choice 2, safeguarded, as the host driver); no instance left -> the loop ends.
__global__ void gn_pre(GNArgs G) {
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    int any = 0;
    for (int b = threadIdx.x; b < G.nb; b += blockDim.x) {
        GNState &S = G.state[b];
        egfem_stats &T = G.stats[b];
        G.mask[b] = 0;
        if (S.host || T.status != EGFEM_OK) continue;
        if (!isfinite(S.rn)) { T.status = EGFEM_ERR_NONFINITE; continue; }
        if (S.rn <= S.target) continue;
        if (T.newton_iters >= G.newton_maxit) { T.status = EGFEM_ERR_NOT_CONVERGED; continue; }
        double eta = S.eta;
        if (T.newton_iters > 0 && !G.fixed_eta) {
            double e = 0.9 * (S.rn / S.rprev) * (S.rn / S.rprev);
            const double sg = 0.9 * eta * eta;
            if (sg > 0.1) e = fmax(e, sg);
            eta = fmax(fmin(G.eta_max, e), 0.5 * S.target / S.rn);
        }
        eta = fmax(eta, G.eta_min);
        S.eta = eta;
        S.rbefore = S.rn;
        G.eta_out[b] = fmax(eta, G.eta_floor);
        G.mask[b] = 1;
        any = 1;
    }
    if (any) atomicOr(&s_any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t k = ++*G.loops;
        if (!s_any || k > G.max_loops) cudaGraphSetConditional(G.cond, 0);
    }
}

// After the Krylov solve: count its iterations; a breakdown or non-finite solve hands the
// instance back (the host redoes it, in FP64 on the mixed path); the others step by x.
__global__ void gn_mid(GNArgs G) {
    for (int b = threadIdx.x; b < G.nb; b += blockDim.x) {
        if (!G.mask[b]) continue;
        const KState &K = G.kst[b];
        egfem_stats &T = G.stats[b];
        T.krylov_iters += K.iter;
        if (T.newton_iters < EGFEM_HIST) T.krylov_hist[T.newton_iters] += K.iter;
        if (K.done == K_NONFINITE || K.done == K_BREAKDOWN) {
            G.state[b].host = 1;
            G.mask[b] = 0;
            continue;
        }
        G.lam[b] = 1.0;
    }
}

// After the tensor action at u - x: accept the step on sufficient decrease (the host driver's
// Armijo test with step length 1); otherwise keep the mask with lam = -1 so that the following
// update reverts it, and hand the instance back.
__global__ void gn_post(GNArgs G) {
    for (int b = threadIdx.x; b < G.nb; b += blockDim.x) {
        if (!G.mask[b]) continue;
        GNState &S = G.state[b];
        egfem_stats &T = G.stats[b];
        const double rn = sqrt(G.norm2[b]);
        if (rn <= (1.0 - 1e-4) * S.rbefore) {
            if (T.newton_iters < EGFEM_HIST) T.res_hist[T.newton_iters] = rn;
            T.newton_iters += 1;
            S.rprev = S.rbefore;
            S.rn = rn;
            G.mask[b] = 0;
        } else {
            S.host = 1;
            G.lam[b] = -1.0;
        }
    }
}

// u -= lam x on every row when the single system's mask is set (the graph loop's step and
// revert for one system)
template <typename V>
__global__ void gn_update_one(int64_t n, const uint8_t *mask, const double *lam, double *u, const V *x) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n && *mask) u[i] -= *lam * to_d(x[i]);
}

}  // namespace egfem
