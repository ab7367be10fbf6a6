// egfem_gnewton.cuh -- the Newton loop as one CUDA graph: a conditional WHILE node whose body is
// control (which instances start a step, their forcing terms) -> the persistent BiCGStab ->
// control (Krylov outcome, pending step halvings) -> u -= lam x -> tensor action + residual
// norms -> control (sufficient decrease) -> undo of failed steps.  The controller kernels keep
// every instance's Newton state in device memory and clear the loop's condition when no
// instance has work left, so a whole solve, damping included, runs without the host.
//
// The damping is the host driver's (Sec. 4's remark on damped iterations): a step whose
// residual fails the sufficient-decrease test is halved, one body execution per halving (the
// solve is skipped for it), at most six times; a step that still does not decrease the residual
// is undone.  On the mixed path such a step, or an FP32 Krylov breakdown, is handed back
// (host = 1) for the host driver's FP64 redo of the same step; in FP64 it ends the instance
// with an error status, as in the host driver.  A single system uses the same controllers with
// one instance (nb = 1).
#pragma once

#include "egfem_kernels.cuh"
#include "egfem_krylov.cuh"
#include "egfem_persist.cuh"

namespace egfem {

// Newton state of one instance, device-resident while the graph runs
struct GNState {
    double rn;        // current ||r|| over free rows
    double rprev;     // ||r|| before the last accepted step (Eisenstat-Walker)
    double rbefore;   // ||r|| when the current step started
    double target;    // stop when rn <= target
    double eta;       // forcing term of the current step
    double lam;       // step length applied in the current step
    int32_t host;     // 1: handed back to the host driver (FP64 redo of the current step)
    int32_t bt;       // halvings of the current step so far
    int32_t pending;  // 1: a halving is due in the next body execution
    int32_t pad;
};

struct GNArgs {
    int32_t nb;
    GNState *state;
    egfem_stats *stats;          // per instance: status, newton_iters, krylov_iters, histories
    uint8_t *mask;               // instances taking part in the next kernels
    double *eta_out;             // Krylov tolerance per instance
    double *lam;                 // increment factor per instance: u -= lam x
    const KState *kst;           // final Krylov state per instance
    const double *norm2;         // ||r||^2 per instance after the tensor action
    const int32_t *kerr;         // nonzero: a grid-barrier wait of the persistent solve ran out (nullable)
    int32_t *loops;              // body executions so far
    int32_t max_loops;
    int32_t newton_maxit, fixed_eta, mixed;
    double eta_max, eta_min, eta_floor;
    cudaGraphConditionalHandle cond;
};

constexpr int GN_MAX_HALVINGS = 6;

// Body executions a solve can need: at most 1 + GN_MAX_HALVINGS per Newton step, and a last
// one that finds nothing to do
inline int32_t gn_max_loops(int32_t newton_maxit) { return (1 + GN_MAX_HALVINGS) * newton_maxit + 2; }

// Start of a body: which instances start a step and their forcing terms (Eisenstat-Walker,
// choice 2, safeguarded, as the host driver); instances with a halving due keep the loop going
// without a solve; no instance left -> the loop ends.
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
        if (S.pending) { any = 1; continue; }
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

// After the Krylov solve: count its iterations and start the step with length 1; a non-finite
// solve, or a breakdown before the first iteration (any breakdown in FP32), fails the step --
// handed back for the FP64 redo on the mixed path, an error status in FP64.  An instance with a
// halving due takes it now: u -= (-lam / 2) x.
__global__ void gn_mid(GNArgs G) {
    for (int b = threadIdx.x; b < G.nb; b += blockDim.x) {
        GNState &S = G.state[b];
        egfem_stats &T = G.stats[b];
        if (!G.mask[b]) {
            if (S.pending && !S.host && T.status == EGFEM_OK) {
                S.pending = 0;
                G.lam[b] = -0.5 * S.lam;
                S.lam *= 0.5;
                S.bt += 1;
                G.mask[b] = 1;
            }
            continue;
        }
        const KState &K = G.kst[b];
        if (K.done == K_TIMEOUT || (G.kerr && *G.kerr)) {
            T.status = EGFEM_ERR_TIMEOUT;
            G.mask[b] = 0;
            continue;
        }
        T.krylov_iters += K.iter;
        if (T.newton_iters < EGFEM_HIST) T.krylov_hist[T.newton_iters] += K.iter;
        if (K.done == K_NONFINITE || (K.done == K_BREAKDOWN && (G.mixed || K.iter == 0))) {
            if (G.mixed) { S.host = 1; T.fp64_rescues += 1; }
            else T.status = K.done == K_NONFINITE ? EGFEM_ERR_NONFINITE : EGFEM_ERR_BREAKDOWN;
            G.mask[b] = 0;
            continue;
        }
        G.lam[b] = 1.0;
        S.lam = 1.0;
        S.bt = 0;
    }
}

// After the tensor action at the trial point: accept on sufficient decrease (the host driver's
// Armijo test for step length lam), else schedule a halving; after the last halving accept any
// decrease, else undo the step (the mask stays set with lam = -lam for the update that follows).
__global__ void gn_post(GNArgs G) {
    for (int b = threadIdx.x; b < G.nb; b += blockDim.x) {
        if (!G.mask[b]) continue;
        GNState &S = G.state[b];
        egfem_stats &T = G.stats[b];
        const double rn = sqrt(G.norm2[b]);
        const bool armijo = rn <= (1.0 - 1e-4 * S.lam) * S.rbefore;
        if (!armijo && S.bt < GN_MAX_HALVINGS) {
            S.pending = 1;
            G.mask[b] = 0;
            continue;
        }
        if (armijo || rn < S.rbefore) {
            if (T.newton_iters < EGFEM_HIST) T.res_hist[T.newton_iters] = rn;
            T.newton_iters += 1;
            S.rprev = S.rbefore;
            S.rn = rn;
            G.mask[b] = 0;
            continue;
        }
        G.lam[b] = -S.lam;
        if (G.mixed) { S.host = 1; T.fp64_rescues += 1; }
        else T.status = EGFEM_ERR_NOT_CONVERGED;
    }
}

// u -= lam x on every row when the single system's mask is set (the graph loop's step, its
// halvings and its undo for one system)
template <typename V>
__global__ void gn_update_one(int64_t n, const uint8_t *mask, const double *lam, double *u, const V *x) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n && *mask) u[i] -= *lam * to_d(x[i]);
}

}  // namespace egfem
