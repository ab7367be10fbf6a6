/*
 * egfem.h -- C ABI of the GB300 (sm_103a) EGFEM Newton hot path.
 *
 * The library implements the online phase of the extended group finite element
 * method (Tolle & Marheineke, arXiv 2005.06193) for the model problem
 *
 *     -div((kappa + w) grad u) + gamma c = d   in Omega,      u = u_D on Gamma,
 *     w = a_scale * g_a(Pi_a u)  in W_a (P1, P2 or P3),   c = c_scale * g_c(Pi_c u) in W_c,
 *
 * which is Sec. 2.1 eq. (1) with b(u) = u, the coefficient a = kappa + w and the
 * reaction gamma c, on a conforming triangle (2D) or tetrahedron (3D) mesh with P1
 * trial functions (Sec. 5: "linear finite elements in all of the examples").
 *
 * Every Newton step runs, on the GPU:
 *   - the pointwise nonlinearity w = g(Pi u) at the W nodes (Sec. 3.1 eq. (5), Sec. 3.2);
 *   - the trilinear tensor action r_i = sum_{m,k} T_imk (kappa + w)_m u_k + gamma (M^c c)_i - d_i
 *     with T_imk = int eta_m grad phi_k . grad phi_i (Sec. 3.3 eq. (7), Example 4.1);
 *   - the Jacobian of Sec. 4 with its identity blocks eliminated,
 *     J = (T ._2 a) + (T ._3 u) diag(g_a') Pi_a + gamma M^c diag(g_c') Pi_c,
 *     written into a fixed CSR pattern (the P1 adjacency of the mesh);
 *   - a Jacobi-preconditioned BiCGStab solve of J delta = r and the update u <- u - delta.
 *
 * Conventions shared by all calls
 *   - Device pointers (prefix d_) are caller-owned CUDA device memory on the device that
 *     was current at egfem_build; host pointers are only read during the call.
 *   - Vectors are contiguous float64 in node order of the mesh (P1) or of the W space.
 *   - Dirichlet rows: r_i = u_i - d_i, J row i = e_i, and the Dirichlet columns of free
 *     rows are zero (Sec. 2.1: the first N_D basis functions carry the boundary data).
 *     The load vector d therefore carries the Dirichlet values u_D on Dirichlet rows.
 *   - Every call is asynchronous on the given stream unless stated otherwise; calls that
 *     return convergence information synchronise that stream.
 *   - Errors are returned, never raised: no call aborts the process.  A status of
 *     EGFEM_ERR_CUDA means a CUDA runtime call failed; egfem_last_error() describes it.
 */
#ifndef EGFEM_H
#define EGFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct egfem_t *egfem_handle;
typedef struct CUstream_st *egfem_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    EGFEM_OK = 0,
    EGFEM_ERR_INVALID_ARG = 1,   /* a pointer, size or option is out of range            */
    EGFEM_ERR_MESH = 2,          /* malformed mesh: bad index, degenerate cell, ...      */
    EGFEM_ERR_CUDA = 3,          /* a CUDA runtime call failed                            */
    EGFEM_ERR_OOM = 4,           /* device or host allocation failed                      */
    EGFEM_ERR_NOT_CONVERGED = 5, /* Newton or Krylov iteration cap reached                */
    EGFEM_ERR_BREAKDOWN = 6,     /* BiCGStab breakdown (rho = 0 or omega = 0)             */
    EGFEM_ERR_SINGULAR = 7,      /* zero Jacobi diagonal                                   */
    EGFEM_ERR_NONFINITE = 8,     /* NaN or Inf in a residual norm                          */
    EGFEM_ERR_TIMEOUT = 9,       /* a bounded device-side wait ran out                    */
    EGFEM_ERR_UNSUPPORTED = 10   /* a valid request this build does not implement         */
} egfem_status;

/* Nonlinearities are a closed set: a host function pointer cannot run on the device. */
typedef enum {
    EGFEM_G_NONE = 0,  /* no nonlinear term                        */
    EGFEM_G_POW = 1,   /* g(s) = s^p  (p a positive integer <= 8)  */
    EGFEM_G_EXP = 2,   /* g(s) = e^s                               */
    EGFEM_G_GRADPOW = 3 /* coefficient only: g = (a_shift + ||grad u||^2)^a_p (any real
                           a_p), the gradient nonlinearities of the p-Laplace and minimal-
                           surface examples (Sec. 5); needs a_degree = 0 (W_a = P0, one node
                           per cell, which carries the cell's constant gradient exactly) and
                           the element-local operator (EGFEM_OP_MATRIX_FREE)              */
} egfem_g_kind;

typedef enum {
    EGFEM_PREC_FP64 = 0,   /* every operator value, vector and reduction in FP64          */
    EGFEM_PREC_MIXED = 1   /* FP32 Jacobian values and Krylov vectors (compensated dot
                              sums); FP64 residual, norm, Newton update (iterative
                              refinement).  A Newton step whose FP32 solve diverges or
                              fails to decrease the FP64 residual is redone in FP64. */
} egfem_precision;

typedef enum {
    EGFEM_ITER_NEWTON = 0,     /* Newton: the full Jacobian of Sec. 4                       */
    EGFEM_ITER_PICARD = 1      /* Picard (Sec. 4, Example 4.1): the frozen-coefficient matrix
                                  T .2 a(u^n), the reaction on the right-hand side; linear
                                  convergence to the same discrete solution               */
} egfem_iteration;

typedef enum {
    EGFEM_OP_CSF = 0,          /* T stored as row-segmented compressed sparse fibres        */
    EGFEM_OP_MATRIX_FREE = 1   /* element-local evaluation: T_imk = sum_K iota^K_m S^K_ik   */
} egfem_operator;

/* Mesh (host arrays, copied by egfem_build). Sec. 2.1: conforming simplicial partition. */
typedef struct {
    int32_t dim;                /* 2: triangles, 3: tetrahedra                            */
    int64_t n_nodes;            /* number of P1 nodes (vertices)                          */
    int64_t n_cells;            /* number of cells                                        */
    const double *coords;       /* [n_nodes * dim], node coordinates                      */
    const int32_t *cells;       /* [n_cells * (dim + 1)], vertex indices of each cell    */
    const uint8_t *dirichlet;   /* [n_nodes], nonzero marks a Dirichlet node             */
} egfem_mesh;

/* Problem: -div((kappa + a_scale g_a(Pi_a u)) grad u) + gamma c_scale g_c(Pi_c u) + sigma u = d. */
typedef struct {
    int32_t a_kind;      /* egfem_g_kind of the coefficient nonlinearity            */
    double a_p;          /* exponent for EGFEM_G_POW (integer) and EGFEM_G_GRADPOW (real) */
    double a_scale;
    int32_t a_degree;    /* Lagrange degree of W_a: 1 (GFEM), 2 or 3; 0 (P0) for GRADPOW */
    int32_t c_kind;      /* egfem_g_kind of the reaction nonlinearity               */
    double c_p;
    double c_scale;
    int32_t c_degree;    /* Lagrange degree of W_c: 1 (GFEM), 2 or 3 (3D: 2; degrees > 1
                            need EGFEM_OP_MATRIX_FREE), or k of I_k (c_space)          */
    double gamma;        /* reaction coefficient                                     */
    double kappa;        /* constant part of the coefficient                         */
    double a_shift;      /* EGFEM_G_GRADPOW: the shift added to ||grad u||^2 (else unused) */
    int32_t a_space;     /* egfem_w_space of W_a (a_degree is then k of I_k)          */
    int32_t c_space;     /* egfem_w_space of W_c                                      */
    double sigma;        /* linear reaction sigma int u phi_i = sigma (M u)_i, M the P1 mass
                            matrix (the M u term of the superconductivity decomposition (b),
                            Sec. 5); nonzero needs EGFEM_OP_MATRIX_FREE                   */
    int32_t c_product;   /* nonzero: the reaction is gamma int c u phi_i = gamma M3 : (u x c), with
                            the trilinear mass form M3_imk = int eta_m phi_k phi_i on W_c
                            (decomposition (a) of the superconductivity example, Sec. 5);
                            needs EGFEM_OP_MATRIX_FREE                                  */
} egfem_problem;

/* The approximation space W of a nonlinearity (Sec. 3.1).  EGFEM_W_QUADRATURE is Case 3's
 * I_k: the basis w_l delta_{x_l} on the points of a symmetric degree-k quadrature rule of
 * every cell (triangle: k = 1..4 with 1, 3, 4, 6 points; tetrahedron: k = 1..3 with 1, 4, 5
 * points), so that T_ilk = w_l grad phi_k(x_l) . grad phi_i(x_l) and M_il = w_l phi_i(x_l),
 * and the EGFEM reproduces the standard Galerkin approach integrated by that rule.  Its
 * nodes are never shared (n_wa = points x n_cells, numbered cell by cell); it needs the
 * element-local operator (EGFEM_OP_MATRIX_FREE). */
typedef enum {
    EGFEM_W_LAGRANGE = 0,
    EGFEM_W_QUADRATURE = 1
} egfem_w_space;

typedef struct {
    double newton_rtol;      /* stop when ||r||_2 <= newton_rtol * ||r(u0)||_2 (default 1e-10) */
    double newton_atol;      /* ... or ||r||_2 <= newton_atol (default 0)                     */
    int32_t newton_maxit;    /* Newton step cap (default 50)                                  */
    double eta_max;          /* largest Krylov forcing term, and the first step's; 0 (default):
                                0.9 for Newton (the cap Eisenstat and Walker give for choice
                                2), 1e-2 for Picard                                           */
    double eta_min;          /* smallest Krylov forcing term (default 1e-12; mixed: 1e-6)     */
    int32_t krylov_maxit;    /* BiCGStab iteration cap per Newton step (default 100000)       */
    int32_t precision;       /* egfem_precision (default EGFEM_PREC_FP64)                    */
    int32_t op;              /* egfem_operator  (default EGFEM_OP_CSF)                       */
    int32_t graph_chunk;     /* BiCGStab iterations per captured CUDA graph (default 32)     */
    int32_t fixed_eta;       /* nonzero: use eta_max for every step (no Eisenstat-Walker; set
                                eta_max to the wanted constant term)                          */
    int32_t krylov_persistent; /* nonzero (default): each BiCGStab solve is one cooperative
                                  launch with grid barriers; for one system it takes two grid
                                  reductions per iteration, each block holding its rows' stencil
                                  window in shared memory, where the windows fit (1: default);
                                  2: the five-barrier form instead; 0: graph-captured iteration
                                  kernels (graph_chunk iterations per graph launch)          */
    int32_t iteration;       /* egfem_iteration of egfem_newton_solve / batch solve and the
                                matrix egfem_jacobian returns (default EGFEM_ITER_NEWTON);
                                egfem_adjoint always uses the Newton Jacobian               */
    int32_t krylov_block_rows; /* single-system persistent solve: fewest rows per block (rounded
                                  up to 32); the grid is min(rows / this, resident blocks).
                                  0 (default) picks the library's value; read at the first
                                  solve of a handle                                          */
    int32_t krylov_cluster;  /* single-system solve (FP64 or mixed) in one thread-block cluster (the Krylov
                                vectors in distributed shared memory; systems up to about
                                16 x 3904 rows): 0 (default) when it fits, with the cluster
                                size chosen by the library; 1..16 that cluster size; -1
                                never.  Read at the first solve of a handle                   */
    int32_t newton_graph;    /* nonzero (default): egfem_newton_solve and egfem_batch_newton_solve
                                run their Newton loop as one CUDA graph (a conditional WHILE
                                node over controller kernels, the persistent or cluster
                                BiCGStab, the update and the tensor action), step halving
                                included; a step that needs the FP64 redo of the mixed path is
                                finished by the host loop (needs krylov_persistent).
                                0: the host loop only; 2: the graph loop is required (the
                                solve returns EGFEM_ERR_UNSUPPORTED where it is unavailable) */
    int32_t batch_share;     /* egfem_batch_build: nonzero (default): when every instance has
                                the same mesh (nodes, coordinates, cells and Dirichlet flags
                                equal byte for byte) the tensor's leaves, fibres and reaction
                                entries are stored once and read by every instance (their W
                                indices offset per instance by the kernels); 0: one copy per
                                instance.  The results are the same bit for bit         */
} egfem_options;

#define EGFEM_HIST 64
typedef struct {
    int32_t status;                    /* egfem_status of the solve                      */
    int32_t newton_iters;              /* Newton steps taken                             */
    int64_t krylov_iters;              /* BiCGStab iterations summed over all steps      */
    double res0;                       /* ||r(u0)||_2 over free rows (FP64)              */
    double res_final;                  /* final ||r||_2 (FP64)                           */
    double res_hist[EGFEM_HIST];       /* ||r||_2 after each Newton step (FP64)          */
    int32_t krylov_hist[EGFEM_HIST];   /* BiCGStab iterations of each Newton step        */
    double solve_ms;                   /* wall time of the solve (host clock)            */
    int64_t kernel_launches;           /* kernels of this library launched by the call,
                                          graph nodes included                          */
    int32_t fp64_rescues;              /* mixed precision: Newton steps whose FP32 Krylov
                                          solve failed and was redone in FP64           */
} egfem_stats;

#define EGFEM_PROF_MAX 8
/* Per-kernel timing of one Newton step's kernels (egfem_profile_kernels). */
typedef struct {
    int32_t count;                          /* kernels filled in                          */
    char name[EGFEM_PROF_MAX][24];          /* kernel name                                */
    double ms[EGFEM_PROF_MAX];              /* mean duration of one launch, CUDA events   */
    double bytes[EGFEM_PROF_MAX];           /* algorithmic DRAM bytes of one launch       */
    double flops[EGFEM_PROF_MAX];           /* algorithmic floating-point ops of one launch */
    int32_t fp64[EGFEM_PROF_MAX];           /* 1 when the kernel computes in FP64         */
} egfem_profile;

/* Fill *opts with the defaults listed above. */
void egfem_default_options(egfem_options *opts);

/* Offline phase (Sec. 5: "computed ... in an offline phase"): number the W spaces,
 * integrate the element quantities, assemble T (and M^c) in the layout selected by
 * opts->op, build the Jacobian pattern, and upload everything to the current device.
 * mesh, prob and opts are host structs read during the call; *out receives a handle
 * that owns all device memory it allocates (free with egfem_destroy).
 * Errors: INVALID_ARG (null pointer, unsupported degree/dim), MESH (index out of
 * range, zero-volume cell), OOM, CUDA. */
egfem_status egfem_build(const egfem_mesh *mesh, const egfem_problem *prob, const egfem_options *opts,
                         egfem_handle *out);

/* Release every device and host allocation of h (NULL is accepted). */
void egfem_destroy(egfem_handle h);

/* Replace the solver options of h (precision and op must equal those given at build). */
egfem_status egfem_set_options(egfem_handle h, const egfem_options *opts);

/* Sizes: P1 nodes, W_a nodes, W_c nodes, rows and nonzeros of the Jacobian pattern. */
egfem_status egfem_sizes(egfem_handle h, int64_t *n_nodes, int64_t *n_wa, int64_t *n_wc,
                         int64_t *jac_rows, int64_t *jac_nnz);

/* Device bytes of the stored tensor T (Sec. 3.2: leaves, fibres) and of the reaction entries
 * M^c, and the number of batch instances that read one copy of them (0: not shared; see
 * egfem_options.batch_share).  Either output may be NULL. */
egfem_status egfem_tensor_storage(egfem_handle h, int64_t *bytes, int32_t *share_count);

/* Host copy of the W-space node coordinates ([n * dim]); which = 0: W_a, 1: W_c. */
egfem_status egfem_w_coords(egfem_handle h, int32_t which, double *coords_host);

/* Device pointers to the fixed Jacobian CSR pattern (owned by h; int32, sorted columns
 * per row, Dirichlet rows hold only their diagonal). */
egfem_status egfem_jacobian_pattern(egfem_handle h, const int32_t **d_rowptr, const int32_t **d_cols);

/* Optional spatially varying kappa on W_a (Sec. 3.3 coefficient field): d_kappa holds
 * n_wa values (copied); NULL restores the constant prob->kappa. */
egfem_status egfem_set_kappa(egfem_handle h, const double *d_kappa, egfem_stream stream);

/* Pointwise nonlinearity (Sec. 3.2, f = g(Pi u)): d_w[m] = a_scale g_a((Pi_a u)_m) and
 * d_wprime[m] = its derivative, for all n_wa nodes. Either output may be NULL. */
egfem_status egfem_pointwise(egfem_handle h, const double *d_u, double *d_w, double *d_wprime,
                             egfem_stream stream);

/* Residual (Sec. 4 EGFEM root, u-block): d_r[n_nodes] from d_u[n_nodes] and load d_d[n_nodes].
 * Always FP64, evaluated as sum_{m,k} T_imk a_m (u_k - u_i) (equal to the plain form
 * because sum_k T_imk = 0). */
egfem_status egfem_residual(egfem_handle h, const double *d_u, const double *d_d, double *d_r,
                            egfem_stream stream);

/* Jacobian values (Sec. 4, identity blocks eliminated) into the CSR pattern: d_vals[jac_nnz], FP64. */
egfem_status egfem_jacobian(egfem_handle h, const double *d_u, double *d_vals, egfem_stream stream);

/* y = J x with J given by CSR values d_vals in the handle's pattern (FP64). */
egfem_status egfem_spmv(egfem_handle h, const double *d_vals, const double *d_x, double *d_y, egfem_stream stream);

/* Jacobi-preconditioned BiCGStab (van der Vorst 1992) on J x = rhs, J from CSR values
 * d_vals (FP64); x out: solution (the iteration starts from x = 0).  The system is scaled
 * by D = diag(J)^{-1} on the left and the iteration stops at ||D(rhs - J x)|| <=
 * rtol ||D rhs||.  A handle built with EGFEM_PREC_MIXED iterates in FP32 (the operator and
 * vectors rounded once) with FP64 dot sums.  Synchronises the stream.  *iters receives
 * the iteration count.  Errors: NOT_CONVERGED (maxit), BREAKDOWN, NONFINITE, SINGULAR. */
egfem_status egfem_bicgstab(egfem_handle h, const double *d_vals, const double *d_rhs, double *d_x,
                            double rtol, int32_t maxit, int32_t *iters, egfem_stream stream);

/* Newton's method (Sec. 4): d_u in: u0 (must satisfy the Dirichlet data), out: solution.
 * Synchronises the stream.  stats may be NULL. */
egfem_status egfem_newton_solve(egfem_handle h, double *d_u, const double *d_d, egfem_stats *stats,
                                egfem_stream stream);

/* Time each kernel of the Newton step at state d_u, load d_d: the tensor-action / Jacobian
 * kernels ("csf_fused": the nodal pass plus the fused CSF kernel, or "tensor_action_mf"), and
 * the BiCGStab solve -- "kry_persistent" (one cooperative launch running 40 iterations, reported
 * per iteration) when krylov_persistent is set, else the iteration kernels -- each launched reps
 * times back to back on the handle's stream between two CUDA events.  Alongside, the
 * algorithmic bytes and flops of one launch (or iteration): operator and vectors counted once
 * per pass.  Synchronises the stream. */
egfem_status egfem_profile_kernels(egfem_handle h, const double *d_u, const double *d_d, int32_t reps,
                                   egfem_profile *out, egfem_stream stream);

/* Adjoint of a functional j(u*) of the converged solution (implicit function theorem;
 * motivated by the repeated forward/backward solves of optimal control, Sec. 6):
 *   J(u*)^T lambda = dj/du  on free rows, lambda = 0 on Dirichlet rows;
 *   dj/dd_i = lambda_i (free rows);  dj/dkappa_m = -sum_{i,k} lambda_i T_imk u_k.
 * The Jacobi-scaled transposed system (D J^T) lambda = D dj/du is solved by FP64 Jacobi-
 * BiCGStab in either precision of the handle, with true-residual restarts: each round forms
 * res = D dj/du - D J^T lambda in FP64 and solves for the correction with a fresh shadow
 * residual, until ||res|| <= 1e-13 ||D dj/du|| or a round no longer halves ||res|| (its FP64
 * floor, about eps |D J^T| |lambda|), at most 5 rounds; on a batch handle every instance
 * runs its own BiCGStab (own scalars, convergence test and rounds) within one persistent
 * launch per round.  stats->res0 and stats->res_final receive ||D dj/du|| and the final true
 * ||res|| (over all instances), stats->krylov_iters the iterations of all rounds.
 * EGFEM_ERR_NOT_CONVERGED when the rounds end above 1e-10 relative while still improving.
 * d_dJdu[n_nodes] in; d_lambda[n_nodes] out; d_grad_kappa[n_wa] out (may be NULL).
 * Synchronises the stream. */
egfem_status egfem_adjoint(egfem_handle h, const double *d_u, const double *d_dJdu, double *d_lambda,
                           double *d_grad_kappa, egfem_stats *stats, egfem_stream stream);

/* Batched offline phase: count independent instances (meshes of one dimension and any
 * sizes, one shared problem definition) assembled as one block-diagonal operator.
 * Instance b owns the rows [offsets[b], offsets[b+1]) of every batch vector (see
 * egfem_batch_layout); each instance's range is padded to a multiple of 32 rows with
 * padding rows that belong to no cell and behave as Dirichlet rows (u = d there).  The
 * single-instance calls (residual, Jacobian, ...) act on the whole batch.  No paper
 * passage: batching is a serving pattern layered on the method. */
egfem_status egfem_batch_build(int32_t count, const egfem_mesh *meshes, const egfem_problem *prob,
                               const egfem_options *opts, egfem_handle *out);

/* Instance count and row offsets ([count + 1], host) of a batch handle. */
egfem_status egfem_batch_layout(egfem_handle h, int32_t *count, int64_t *offsets);

/* Newton's method for every instance of a batch at once: each BiCGStab kernel launch
 * serves all instances still iterating (per-instance scalars, convergence and damping);
 * tile sizes are chosen by timing on the first call.  stats: [count] per-instance
 * results (may be NULL).  Returns the first non-OK instance status, if any.
 * Synchronises the stream. */
egfem_status egfem_batch_newton_solve(egfem_handle h, double *d_u, const double *d_d, egfem_stats *stats,
                                      egfem_stream stream);

/* Load vector of a cellwise constant source: d_i = sum_{K owns i} f_K |K| / (dim + 1)
 * (exact integral of f phi_i), Dirichlet rows set to 0.  d_f[n_cells] in, d_d[n_nodes] out. */
egfem_status egfem_load_cellwise(egfem_handle h, const double *d_f, double *d_d, egfem_stream stream);

/* Transpose of egfem_load_cellwise: d_g[K] = |K|/(dim+1) sum_{i in K, i free} d_lam[i]. */
egfem_status egfem_load_cellwise_transpose(egfem_handle h, const double *d_lam, double *d_g, egfem_stream stream);

/* Host-only inspection of the offline assembly (no device work, no CUDA call): runs the
 * same W-space numbering and tensor assembly as egfem_build and returns the stored
 * trilinear form as COO triplets (i, m, k, T_imk), including the per-fibre diagonal
 * T_imi.  Call with I == NULL to get the count in *count; then with arrays of that size.
 * m indexes the W_a space (or is -1 for the constant-coefficient stiffness when
 * prob->a_kind == EGFEM_G_NONE).  Used to check the assembly against an independent
 * quadrature on machines without a GPU.  *n_wa (optional) receives the W_a size and
 * wa_coords (optional, [n_wa * dim]) the W_a node coordinates. */
egfem_status egfem_inspect_tensor(const egfem_mesh *mesh, const egfem_problem *prob, int64_t *count,
                                  int64_t *I, int64_t *M, int64_t *K, double *V, int64_t *n_wa, double *wa_coords);

/* Self-test of the bounded device-side wait of the persistent BiCGStab solve (no handle).
 * Launches `blocks` blocks (1..64) of which the first `arrive` (0..blocks) enter the batched
 * solve's grid barrier and then, if it completed with every block counted as live, the
 * single-system solve's barrier.  With arrive == blocks the launch is cooperative and every
 * block must pass both; with arrive < blocks the first barrier cannot complete and each waiting
 * block gives up after wait_ms milliseconds (0 < wait_ms <= 2000) and raises the barriers' error
 * word.  ok_host (host, [blocks]) receives 1 for a block that passed, 0 for one that gave up, -1
 * for one that did not arrive; *err_host (host, optional) the error word.  Synchronous;
 * allocates and frees its own device memory (under 0.5 KB).  Errors: EGFEM_ERR_INVALID_ARG for sizes out of range,
 * EGFEM_ERR_CUDA for a failed launch.  The paper has no counterpart: this checks the
 * library's own failure handling. */
egfem_status egfem_selftest_grid_barrier(int32_t blocks, int32_t arrive, double wait_ms, int32_t *ok_host,
                                         int32_t *err_host);

/* Sum of squares of d_r over the rows whose d_dirichlet entry is 0 (the quantity of the
 * Newton convergence test), written to the device scalar *d_out, for callers that cannot
 * allocate device memory when they need it (an application that reserves all device
 * memory for its own pool, or a real-time loop that cannot afford cudaMalloc's implicit
 * synchronisation).  It allocates nothing and needs no handle: its block partials and
 * completion ticket live in a fixed static device array of 65.8 KB that every GPU which
 * loads the library holds until the process exits.  At most 134,217,728 rows
 * (8192 blocks of 16384 rows); larger n returns EGFEM_ERR_INVALID_ARG.  The first call
 * on a device (and the first after a cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  The sum is deterministic from call to call but is not bit-identical to the
 * handle's own norm (different row partition; they agree to rounding).  All calls share the
 * one array: calls that overlap on the GPU (different streams, or host threads) race, and
 * may write a wrong sum or leave *d_out unwritten (stale), because one call's ticket reset
 * can hide another call's last block; order the calls, for example on one stream.  The
 * ticket is reset at the start of every call.  Asynchronous on stream.  The paper has no counterpart: this is a deployment variant of the library's
 * own residual-norm reduction. */
egfem_status egfem_free_norm2_noalloc(int64_t n, const double *d_r, const uint8_t *d_dirichlet, double *d_out,
                                      egfem_stream stream);

/* Human-readable name of a status code (static storage). */
const char *egfem_status_string(egfem_status s);

/* Description of the last CUDA or validation error seen by this thread (static storage). */
const char *egfem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EGFEM_H */
