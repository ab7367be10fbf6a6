/*
 * egfem_oracle.c -- FP64 CPU oracle for the EGFEM Newton hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares no
 * code, header, table or constant with the CUDA library: it builds its own basis
 * functions, quadrature rules, degree-of-freedom numbering and operators from the
 * paper's definitions, written as plain loops in the paper's order.
 *
 * What it computes (Tolle & Marheineke, "Extended Group Finite Element Method"):
 *   model problem  -div((kappa + a_nl(u)) grad u) + gamma c_nl(u) = d,  u = u_D on the boundary
 *   (Sec. 2.1 eq. (1) with b(u) = u, a = kappa + w, c = gamma * c_nl; Dirichlet only).
 *
 *   SGA   (Sec. 2.1 eqs. (3), (4); Sec. 4 SGA root (8) and Newton):
 *         r_i  = sum_K int_K (kappa + g_a(u_h)) grad u_h . grad phi_i + gamma g_c(u_h) phi_i  - d_i
 *         J_il = sum_K int_K (kappa + g_a(u_h)) grad phi_l . grad phi_i
 *                          + g_a'(u_h) phi_l grad u_h . grad phi_i + gamma g_c'(u_h) phi_l phi_i
 *         re-integrated by quadrature at every call.
 *   EGFEM (Sec. 3.1 eq. (5), Sec. 3.2 interpolation operators, Sec. 3.3 eq. (7),
 *          Sec. 4 EGFEM root (9) and its Newton Jacobian):
 *         a = kappa + g_a(Pi_a u),  c = g_c(Pi_c u)   (pointwise, at the W-space nodes)
 *         r_i  = sum_{m,k} T_imk a_m u_k + gamma sum_m M_im c_m - d_i
 *         T_imk = int eta_m grad phi_k . grad phi_i   (trilinear form K_a, Sec. 3.3 / Example 4.1)
 *         M_im  = int eta_m phi_i                     (bilinear form M^c, Sec. 3.3)
 *         Jacobian: the augmented system in z = (u, a, c) has identity blocks for a and c
 *         (Sec. 4); eliminating them gives the Jacobian in u alone
 *         J_il = sum_m T_iml a_m + sum_m (sum_k T_imk u_k) g_a'(Pi_a u)_m (Pi_a)_ml
 *              + gamma sum_m M_im g_c'(Pi_c u)_m (Pi_c)_ml.
 *   Dirichlet rows (Sec. 2.1, first N_D basis functions on Gamma_D):
 *         r_i = u_i - uD_i, J row i = e_i; Dirichlet columns are zero in free rows
 *         (the Newton update vanishes there once u satisfies the boundary data).
 *
 * Reading used for the residual near convergence: the trial functions sum to one, so
 * sum_k grad phi_k = 0 on every element and sum_k T_imk = 0 exactly.  The residual may
 * therefore be evaluated as sum_{m,k} T_imk a_m (u_k - u_i), which equals the plain
 * definition in exact arithmetic but avoids cancelling O(1) terms in FP64 rounding.
 * Both forms are provided (ORC_FORM_PLAIN, ORC_FORM_DIFF) and tests check they agree.
 *
 * Basis: Lagrange nodal basis of degree p on the reference simplex, obtained by
 * inverting the Vandermonde matrix of the monomials at the lattice nodes.
 * Quadrature: collapsed (Duffy) tensor Gauss-Legendre rules, the 1-D nodes found by
 * Newton's method on the Legendre polynomial.
 * Linear solves: banded LU with partial pivoting (the direct solve the paper's
 * backslash performs, Sec. 5) and a Jacobi-preconditioned BiCGStab (van der Vorst,
 * 1992) for large systems.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 3
#define ORC_MAXNB 20   /* P3 in 3D has 20 local basis functions */
#define ORC_MAXQ 512

enum { ORC_G_NONE = 0, ORC_G_POW = 1, ORC_G_EXP = 2, ORC_G_GRADPOW = 3 };
/* ORC_G_GRADPOW: a gradient nonlinearity for the coefficient (Sec. 5, p-Laplace and minimal
 * surface examples): w = a_scale * (a_shift + ||grad u||^2)^a_p, with W_a = P0 (the gradient
 * of a P1 function is constant on each cell, so the W node of a cell carries it exactly). */
enum { ORC_FORM_PLAIN = 0, ORC_FORM_DIFF = 1 };

/* ------------------------------------------------------------------------- */
/* small dense helpers                                                        */
/* ------------------------------------------------------------------------- */

/* Solve A X = B in place (A n x n row-major, B n x nrhs) by Gaussian elimination with
 * partial pivoting.  Returns 0 on success, -1 on a zero pivot. */
static int dense_solve(int n, double *A, int nrhs, double *B) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) { double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            for (int j = 0; j < nrhs; ++j) { double t = B[c * nrhs + j]; B[c * nrhs + j] = B[piv * nrhs + j]; B[piv * nrhs + j] = t; }
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            for (int j = 0; j < nrhs; ++j) B[r * nrhs + j] -= f * B[c * nrhs + j];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        for (int j = 0; j < nrhs; ++j) {
            double s = B[c * nrhs + j];
            for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * B[k * nrhs + j];
            B[c * nrhs + j] = s / A[c * n + c];
        }
    }
    return 0;
}

static double factorial(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

/* ------------------------------------------------------------------------- */
/* Lagrange elements on the reference simplex                                 */
/* ------------------------------------------------------------------------- */

/* Local node order: vertices 0..d, then edge-interior nodes edge by edge (edges
 * (a,b), a<b, lexicographic; nodes ordered from a to b), then face-interior nodes
 * (faces (a,b,c), a<b<c, lexicographic), then cell-interior nodes.  Each node is a
 * barycentric integer vector alpha (sum = p); the node sits at lambda = alpha / p.  */
typedef struct {
    int dim, p, nb;
    int alpha[ORC_MAXNB][ORC_MAXD + 1];
    double coef[ORC_MAXNB * ORC_MAXNB];  /* phi_i = sum_j coef[j*nb+i] mono_j */
    int mono[ORC_MAXNB][ORC_MAXD];       /* monomial exponents in xi_1..xi_d   */
} orc_elem;

static void elem_init(orc_elem *E, int dim, int p) {
    memset(E, 0, sizeof(*E));
    E->dim = dim; E->p = p;
    int nv = dim + 1, nb = 0;
    /* enumerate all alpha with sum p; then order by support size (vertex, edge, face, cell)
     * and within a support size lexicographically by the support, then by position. */
    int all[ORC_MAXNB][ORC_MAXD + 1]; int na = 0;
    if (p == 0) {
        /* P0: a single node at the barycentre */
        for (int j = 0; j <= ORC_MAXD; ++j) E->alpha[0][j] = 0;
        nb = 1;
    } else {
        int a[ORC_MAXD + 1];
        for (a[0] = p; a[0] >= 0; --a[0])
            for (a[1] = p - a[0]; a[1] >= 0; --a[1]) {
                if (dim == 2) { a[2] = p - a[0] - a[1]; memcpy(all[na++], a, sizeof(int) * 3); continue; }
                for (a[2] = p - a[0] - a[1]; a[2] >= 0; --a[2]) { a[3] = p - a[0] - a[1] - a[2]; memcpy(all[na++], a, sizeof(int) * 4); }
            }
    }
    for (int supp = 1; supp <= nv && p > 0; ++supp) {
        /* candidate supports in lexicographic order: iterate over bitmasks sorted lexicographically */
        int masks[16]; int nm = 0;
        for (int s = 1; s < (1 << nv); ++s) if (__builtin_popcount(s) == supp) masks[nm++] = s;
        /* sort masks by the lexicographic order of their member lists */
        for (int x = 0; x < nm; ++x)
            for (int y = x + 1; y < nm; ++y) {
                int lx[4], ly[4], cx = 0, cy = 0;
                for (int j = 0; j < nv; ++j) { if (masks[x] >> j & 1) lx[cx++] = j; if (masks[y] >> j & 1) ly[cy++] = j; }
                int swap = 0;
                for (int j = 0; j < supp; ++j) { if (lx[j] != ly[j]) { swap = lx[j] > ly[j]; break; } }
                if (swap) { int t = masks[x]; masks[x] = masks[y]; masks[y] = t; }
            }
        for (int mi = 0; mi < nm; ++mi) {
            /* nodes with exactly this support, ordered by decreasing weight of the first member */
            for (int k = 0; k < na; ++k) {
                int s = 0; for (int j = 0; j < nv; ++j) if (all[k][j]) s |= 1 << j;
                if (s != masks[mi]) continue;
                memcpy(E->alpha[nb++], all[k], sizeof(int) * (ORC_MAXD + 1));
            }
        }
    }
    E->nb = nb;
    /* monomials xi^e with |e| <= p */
    int nm = 0, e[3];
    for (int deg = 0; deg <= p; ++deg)
        for (e[0] = deg; e[0] >= 0; --e[0]) {
            if (dim == 2) { E->mono[nm][0] = e[0]; E->mono[nm][1] = deg - e[0]; ++nm; continue; }
            for (e[1] = deg - e[0]; e[1] >= 0; --e[1]) { E->mono[nm][0] = e[0]; E->mono[nm][1] = e[1]; E->mono[nm][2] = deg - e[0] - e[1]; ++nm; }
        }
    /* Vandermonde V[i][j] = mono_j(node_i); coef = V^{-1} so that phi_i(node_k) = delta_ik */
    double V[ORC_MAXNB * ORC_MAXNB], C[ORC_MAXNB * ORC_MAXNB];
    for (int i = 0; i < nb; ++i) {
        double xi[3];
        for (int d = 0; d < dim; ++d) xi[d] = (p == 0) ? 1.0 / (dim + 1) : (double)E->alpha[i][d + 1] / p;
        for (int j = 0; j < nb; ++j) {
            double v = 1.0;
            for (int d = 0; d < dim; ++d) v *= pow(xi[d], E->mono[j][d]);
            V[i * nb + j] = v;
        }
    }
    for (int i = 0; i < nb; ++i) for (int j = 0; j < nb; ++j) C[i * nb + j] = (i == j);
    dense_solve(nb, V, nb, C);          /* C = V^{-1}: column i holds the coefficients of phi_i */
    memcpy(E->coef, C, sizeof(double) * nb * nb);
}

/* values and reference gradients of all basis functions at reference point xi */
static void elem_eval(const orc_elem *E, const double *xi, double *val, double *grad) {
    int nb = E->nb, dim = E->dim;
    double mv[ORC_MAXNB], mg[ORC_MAXNB][ORC_MAXD];
    for (int j = 0; j < nb; ++j) {
        double v = 1.0;
        for (int d = 0; d < dim; ++d) v *= pow(xi[d], E->mono[j][d]);
        mv[j] = v;
        for (int d = 0; d < dim; ++d) {
            int ed = E->mono[j][d];
            if (ed == 0) { mg[j][d] = 0.0; continue; }
            double g = ed * pow(xi[d], ed - 1);
            for (int d2 = 0; d2 < dim; ++d2) if (d2 != d) g *= pow(xi[d2], E->mono[j][d2]);
            mg[j][d] = g;
        }
    }
    for (int i = 0; i < nb; ++i) {
        double v = 0.0, g[3] = {0, 0, 0};
        for (int j = 0; j < nb; ++j) {
            double c = E->coef[j * nb + i];
            v += c * mv[j];
            for (int d = 0; d < dim; ++d) g[d] += c * mg[j][d];
        }
        if (val) val[i] = v;
        if (grad) for (int d = 0; d < dim; ++d) grad[i * dim + d] = g[d];
    }
}

/* ------------------------------------------------------------------------- */
/* Quadrature: collapsed Gauss-Legendre on the reference simplex              */
/* ------------------------------------------------------------------------- */

/* q-point Gauss-Legendre rule on [0,1] (Newton iteration on P_q). */
static void gauss_legendre01(int q, double *x, double *w) {
    for (int i = 0; i < q; ++i) {
        double z = cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            if (q == 1) { p1 = z; p0 = 1.0; }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   /* = (2/((1-z^2)P'^2)) / 2 */
    }
}

/* Rule on the reference simplex {xi >= 0, sum xi <= 1} with q points per direction.
 * 2D: xi1 = s, xi2 = t (1-s), weight (1-s).  3D: xi1 = s, xi2 = t (1-s),
 * xi3 = r (1-s)(1-t), weight (1-s)^2 (1-t).  Weights sum to the reference volume 1/d!. */
static int simplex_rule(int dim, int q, double *pts, double *wts) {
    double x[64], w[64];
    gauss_legendre01(q, x, w);
    int n = 0;
    if (dim == 2) {
        for (int a = 0; a < q; ++a) for (int b = 0; b < q; ++b) {
            double s = x[a], t = x[b];
            pts[2 * n] = s; pts[2 * n + 1] = t * (1 - s);
            wts[n++] = w[a] * w[b] * (1 - s);
        }
    } else {
        for (int a = 0; a < q; ++a) for (int b = 0; b < q; ++b) for (int c = 0; c < q; ++c) {
            double s = x[a], t = x[b], r = x[c];
            pts[3 * n] = s; pts[3 * n + 1] = t * (1 - s); pts[3 * n + 2] = r * (1 - s) * (1 - t);
            wts[n++] = w[a] * w[b] * w[c] * (1 - s) * (1 - s) * (1 - t);
        }
    }
    return n;
}

/* Symmetric rules of degree k on the reference simplex, the rules behind the quadrature
 * spaces I_k (Sec. 3.1, Case 3; the paper cites Dunavant's symmetric Gaussian rules for the
 * triangle).  Each rule is a union of orbits of barycentric points under vertex permutation,
 * with the orbit parameters and weights in closed form:
 *   triangle    k = 1: centroid;  k = 2: (2/3, 1/6, 1/6);  k = 3: centroid (weight -27/48) and
 *               (3/5, 1/5, 1/5) (25/48);  k = 4: (1-2a, a, a) for the two roots
 *               a = (8 - sqrt 10 +- sqrt(38 - 44 sqrt(2/5))) / 18, weights
 *               (620 +- sqrt(213125 - 53320 sqrt 10)) / 3720;
 *   tetrahedron k = 1: centroid;  k = 2: (1-3a, a, a, a), a = (5 - sqrt 5) / 20, weights 1/4;
 *               k = 3: centroid (-4/5) and (1/2, 1/6, 1/6, 1/6) (9/20).
 * Weights are given relative to the simplex volume and scaled here to sum to 1/d!.
 * Points are returned in reference coordinates xi_j = lambda_j (j = 1..d).  Returns the
 * number of points, or -1 for a degree this table does not hold. */
static int orbit_push(int dim, const double *lam, double w, double *pts, double *wts, int n) {
    /* every distinct permutation of lam[0..dim] */
    int nv = dim + 1, perm[4];
    double seen[24][4];
    int ns = 0;
    for (int i = 0; i < nv; ++i) perm[i] = i;
    for (;;) {
        double b[4];
        for (int i = 0; i < nv; ++i) b[i] = lam[perm[i]];
        int dup = 0;
        for (int t = 0; t < ns && !dup; ++t) {
            int same = 1;
            for (int i = 0; i < nv; ++i) same &= seen[t][i] == b[i];
            dup = same;
        }
        if (!dup) {
            for (int i = 0; i < nv; ++i) seen[ns][i] = b[i];
            ++ns;
            for (int j = 1; j <= dim; ++j) pts[(size_t)n * dim + j - 1] = b[j];
            wts[n++] = w;
        }
        /* next permutation (lexicographic) */
        int i = nv - 2;
        while (i >= 0 && perm[i] > perm[i + 1]) --i;
        if (i < 0) break;
        int j = nv - 1;
        while (perm[j] < perm[i]) --j;
        int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        for (int l = i + 1, r = nv - 1; l < r; ++l, --r) { t = perm[l]; perm[l] = perm[r]; perm[r] = t; }
    }
    return n;
}

static int sym_rule(int dim, int k, double *pts, double *wts) {
    int n = 0;
    if (dim == 2) {
        if (k == 1) { double l[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3}; n = orbit_push(2, l, 1.0, pts, wts, n); }
        else if (k == 2) { double l[3] = {2.0 / 3, 1.0 / 6, 1.0 / 6}; n = orbit_push(2, l, 1.0 / 3, pts, wts, n); }
        else if (k == 3) {
            double c[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3}, l[3] = {0.6, 0.2, 0.2};
            n = orbit_push(2, c, -27.0 / 48.0, pts, wts, n);
            n = orbit_push(2, l, 25.0 / 48.0, pts, wts, n);
        } else if (k == 4) {
            double r = sqrt(38.0 - 44.0 * sqrt(0.4)), q = sqrt(213125.0 - 53320.0 * sqrt(10.0));
            double a1 = (8.0 - sqrt(10.0) + r) / 18.0, a2 = (8.0 - sqrt(10.0) - r) / 18.0;
            double l1[3] = {1.0 - 2.0 * a1, a1, a1}, l2[3] = {1.0 - 2.0 * a2, a2, a2};
            n = orbit_push(2, l1, (620.0 + q) / 3720.0, pts, wts, n);
            n = orbit_push(2, l2, (620.0 - q) / 3720.0, pts, wts, n);
        } else return -1;
    } else {
        if (k == 1) { double l[4] = {0.25, 0.25, 0.25, 0.25}; n = orbit_push(3, l, 1.0, pts, wts, n); }
        else if (k == 2) {
            double a = (5.0 - sqrt(5.0)) / 20.0, l[4] = {1.0 - 3.0 * a, a, a, a};
            n = orbit_push(3, l, 0.25, pts, wts, n);
        } else if (k == 3) {
            double c[4] = {0.25, 0.25, 0.25, 0.25}, l[4] = {0.5, 1.0 / 6, 1.0 / 6, 1.0 / 6};
            n = orbit_push(3, c, -0.8, pts, wts, n);
            n = orbit_push(3, l, 0.45, pts, wts, n);
        } else return -1;
    }
    for (int i = 0; i < n; ++i) wts[i] /= (dim == 2 ? 2.0 : 6.0);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Geometry                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    double B[9], Binv[9], vol, x0[3];
} orc_geom;

static void cell_geom(int dim, const double *X, const int *cell, orc_geom *G) {
    const double *p0 = X + (size_t)cell[0] * dim;
    for (int d = 0; d < dim; ++d) G->x0[d] = p0[d];
    for (int c = 0; c < dim; ++c) {
        const double *pc = X + (size_t)cell[c + 1] * dim;
        for (int r = 0; r < dim; ++r) G->B[r * dim + c] = pc[r] - p0[r];
    }
    double A[9], I[9];
    memcpy(A, G->B, sizeof(double) * dim * dim);
    for (int i = 0; i < dim * dim; ++i) I[i] = 0;
    for (int i = 0; i < dim; ++i) I[i * dim + i] = 1;
    double det;
    if (dim == 2) det = G->B[0] * G->B[3] - G->B[1] * G->B[2];
    else det = G->B[0] * (G->B[4] * G->B[8] - G->B[5] * G->B[7])
             - G->B[1] * (G->B[3] * G->B[8] - G->B[5] * G->B[6])
             + G->B[2] * (G->B[3] * G->B[7] - G->B[4] * G->B[6]);
    dense_solve(dim, A, dim, I);
    memcpy(G->Binv, I, sizeof(double) * dim * dim);
    G->vol = fabs(det) / factorial(dim);
}

/* physical gradient g = B^{-T} gref */
static void phys_grad(int dim, const orc_geom *G, const double *gref, double *g) {
    for (int r = 0; r < dim; ++r) {
        double s = 0.0;
        for (int c = 0; c < dim; ++c) s += G->Binv[c * dim + r] * gref[c];
        g[r] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* Global degree-of-freedom numbering for a Lagrange space of degree p        */
/* ------------------------------------------------------------------------- */

/* A lattice node is identified, independently of the element it is seen from, by its
 * barycentric integer coordinates with respect to the global vertices: the sorted list
 * of (global vertex, weight) pairs.  Nodes are numbered in the lexicographic order of
 * these keys.  For p = 0 the single node of a cell is keyed by the cell index. */
typedef struct { int64_t k[8]; int cell, loc; } orc_nodekey;

static int key_cmp(const void *a, const void *b) {
    const orc_nodekey *x = a, *y = b;
    for (int i = 0; i < 8; ++i) { if (x->k[i] < y->k[i]) return -1; if (x->k[i] > y->k[i]) return 1; }
    return 0;
}

typedef struct {
    int p, nloc, n;
    int *cell2dof;     /* [nc * nloc] */
    double *coords;    /* [n * dim]   */
} orc_space;

static void space_free(orc_space *S) { free(S->cell2dof); free(S->coords); memset(S, 0, sizeof(*S)); }

static int space_build(int dim, int nc, const double *X, const int *cells, int p, orc_space *S) {
    orc_elem E; elem_init(&E, dim, p);
    int nl = E.nb;
    size_t total = (size_t)nc * nl;
    orc_nodekey *keys = malloc(sizeof(orc_nodekey) * total);
    if (!keys) return -1;
    for (int c = 0; c < nc; ++c) {
        for (int l = 0; l < nl; ++l) {
            orc_nodekey *K = &keys[(size_t)c * nl + l];
            for (int i = 0; i < 8; ++i) K->k[i] = INT64_MAX;
            K->cell = c; K->loc = l;
            if (p == 0) { K->k[0] = -1; K->k[1] = c; continue; }
            int gv[4], wt[4], cnt = 0;
            for (int j = 0; j <= dim; ++j) if (E.alpha[l][j]) { gv[cnt] = cells[(size_t)c * (dim + 1) + j]; wt[cnt] = E.alpha[l][j]; ++cnt; }
            for (int x = 0; x < cnt; ++x) for (int y = x + 1; y < cnt; ++y)
                if (gv[y] < gv[x]) { int t = gv[x]; gv[x] = gv[y]; gv[y] = t; t = wt[x]; wt[x] = wt[y]; wt[y] = t; }
            for (int x = 0; x < cnt; ++x) { K->k[2 * x] = gv[x]; K->k[2 * x + 1] = wt[x]; }
        }
    }
    qsort(keys, total, sizeof(orc_nodekey), key_cmp);
    S->p = p; S->nloc = nl;
    S->cell2dof = malloc(sizeof(int) * total);
    int n = -1;
    for (size_t t = 0; t < total; ++t) {
        if (t == 0 || key_cmp(&keys[t], &keys[t - 1]) != 0) ++n;
        S->cell2dof[(size_t)keys[t].cell * nl + keys[t].loc] = n;
    }
    S->n = n + 1;
    free(keys);
    S->coords = malloc(sizeof(double) * S->n * dim);
    for (int c = 0; c < nc; ++c) {
        for (int l = 0; l < nl; ++l) {
            int g = S->cell2dof[(size_t)c * nl + l];
            for (int d = 0; d < dim; ++d) {
                double x = 0.0;
                for (int j = 0; j <= dim; ++j) {
                    double lam = (p == 0) ? 1.0 / (dim + 1) : (double)E.alpha[l][j] / p;
                    x += lam * X[(size_t)cells[(size_t)c * (dim + 1) + j] * dim + d];
                }
                S->coords[(size_t)g * dim + d] = x;
            }
        }
    }
    return 0;
}

/* The quadrature space I_k: one node per rule point per cell, never shared between cells
 * (the basis functions w_l delta_{x_l} are discontinuous, Sec. 3.1, Case 3); node c nq + l is
 * the physical image of reference point l on cell c. */
static void space_build_quad(int dim, int nc, const double *X, const int *cells, int nq, const double *qp, orc_space *S) {
    S->p = -1; S->nloc = nq; S->n = nc * nq;
    S->cell2dof = malloc(sizeof(int) * (size_t)nc * nq);
    S->coords = malloc(sizeof(double) * (size_t)S->n * dim);
    for (int c = 0; c < nc; ++c) {
        orc_geom G; cell_geom(dim, X, cells + (size_t)c * (dim + 1), &G);
        for (int l = 0; l < nq; ++l) {
            int g = c * nq + l;
            S->cell2dof[(size_t)c * nq + l] = g;
            for (int r = 0; r < dim; ++r) {
                double x = G.x0[r];
                for (int k = 0; k < dim; ++k) x += G.B[r * dim + k] * qp[l * dim + k];
                S->coords[(size_t)g * dim + r] = x;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Sparse triplet accumulation (COO, sorted and summed)                        */
/* ------------------------------------------------------------------------- */

typedef struct { int64_t i, j, k; double v; } orc_trip;
typedef struct { orc_trip *t; size_t n, cap; } orc_coo;

static void coo_push(orc_coo *C, int64_t i, int64_t j, int64_t k, double v) {
    if (C->n == C->cap) { C->cap = C->cap ? 2 * C->cap : 1024; C->t = realloc(C->t, sizeof(orc_trip) * C->cap); }
    C->t[C->n].i = i; C->t[C->n].j = j; C->t[C->n].k = k; C->t[C->n].v = v; C->n++;
}

static int trip_cmp(const void *a, const void *b) {
    const orc_trip *x = a, *y = b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return 0;
}

/* sort and sum duplicates (entries are kept even when the sum is zero: nothing is dropped) */
static void coo_compress(orc_coo *C) {
    if (!C->n) return;
    qsort(C->t, C->n, sizeof(orc_trip), trip_cmp);
    size_t w = 0;
    for (size_t r = 1; r < C->n; ++r) {
        if (trip_cmp(&C->t[r], &C->t[w]) == 0) C->t[w].v += C->t[r].v;
        else C->t[++w] = C->t[r];
    }
    C->n = w + 1;
}

/* ------------------------------------------------------------------------- */
/* Problem object                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int dim, nv, nc;
    const double *X; const int *cells; const unsigned char *dir;
    int a_kind; double a_p, a_scale; int a_deg;   /* w = a_scale * g(Pi_a u), diffusion coefficient kappa + w */
    int c_kind; double c_p, c_scale; int c_deg;   /* c = c_scale * g(Pi_c u), reaction gamma * M c          */
    double gamma, kappa;
    int qpts;                                      /* Gauss points per direction */
    double a_shift;                                /* ORC_G_GRADPOW: the shift of ||grad u||^2 */
    int a_quad, c_quad;  /* nonzero: W_a / W_c is the quadrature space I_k, k = a_deg / c_deg (Sec. 3.1, Case 3) */
    int rule;            /* > 0: the symmetric degree-`rule` rule for every integral (SGA, load vector,
                            Lagrange-space tensors) instead of the collapsed Gauss rule */
    double sigma;        /* linear reaction sigma * int u phi_i = sigma (M u)_i, M the P1 mass matrix
                            (the M u term of the superconductivity decomposition (b), Sec. 5) */
    int c_product;       /* nonzero: the reaction is gamma int c u phi_i = gamma M3 : (u x c) with the
                            trilinear mass form M3_imk = int eta_m phi_k phi_i (decomposition (a)) */
} orc_spec;

typedef struct {
    orc_spec s;
    orc_elem P1, Ea, Ec;
    orc_space Sa, Sc;
    int nq; double qp[ORC_MAXQ * 3], qw[ORC_MAXQ];
    /* the rules of quadrature spaces (I_k): reference points and weights (sum 1/d!) */
    int aq_n, cq_n; double aq_p[16 * 3], aq_w[16], cq_p[16 * 3], cq_w[16];
    /* basis values tabulated once at the quadrature points (phi: P1, eta_a / eta_c: W spaces)
     * and the constant reference gradients of the P1 basis */
    double *phi_q, *eta_a_q, *eta_c_q, gref1[4 * 3];
    orc_coo T;            /* (i, m, k) -> T_imk over the assembled cells */
    orc_coo M;            /* (i, m, 0) -> M_im                            */
    orc_coo Pa, Pc;       /* (m, j, 0) -> (Pi)_mj                         */
    orc_coo Mu;           /* (i, k, 0) -> int phi_k phi_i (when sigma != 0) */
    orc_coo M3;           /* (i, m, k) -> int eta_m phi_k phi_i (c_product)  */
    double *kappa_field;  /* optional kappa per W_a node (NULL: constant)  */
    int *cell_mask;       /* cells included in the tensor assembly         */
} orc_problem;

/* the coefficient nonlinearity as a function of its argument s (for ORC_G_GRADPOW,
 * s = ||grad u||^2) and its derivative in s */
static double ga_val(const orc_spec *S, double s) {
    if (S->a_kind == ORC_G_GRADPOW) return S->a_scale * pow(S->a_shift + s, S->a_p);
    if (S->a_kind == ORC_G_POW) return S->a_scale * pow(s, S->a_p);
    if (S->a_kind == ORC_G_EXP) return S->a_scale * exp(s);
    return 0.0;
}
static double ga_der(const orc_spec *S, double s) {
    if (S->a_kind == ORC_G_GRADPOW) return (S->a_p == 0.0) ? 0.0 : S->a_scale * S->a_p * pow(S->a_shift + s, S->a_p - 1.0);
    if (S->a_kind == ORC_G_POW) return (S->a_p == 0.0) ? 0.0 : S->a_scale * S->a_p * pow(s, S->a_p - 1.0);
    if (S->a_kind == ORC_G_EXP) return S->a_scale * exp(s);
    return 0.0;
}

static double g_val(int kind, double p, double scale, double s) {
    if (kind == ORC_G_POW) return scale * pow(s, p);
    if (kind == ORC_G_EXP) return scale * exp(s);
    return 0.0;
}
static double g_der(int kind, double p, double scale, double s) {
    if (kind == ORC_G_POW) return (p == 0.0) ? 0.0 : scale * p * pow(s, p - 1.0);
    if (kind == ORC_G_EXP) return scale * exp(s);
    return 0.0;
}

/* Pi_mj = phi_j(x_m): evaluate the P1 basis of a cell holding node m at the node's
 * physical coordinates (barycentric coordinates from x = x0 + B xi). */
static void build_interp(orc_problem *P, const orc_space *S, orc_coo *Pi) {
    int dim = P->s.dim, nl = S->nloc;
    char *seen = calloc(S->n, 1);
    for (int c = 0; c < P->s.nc; ++c) {
        orc_geom G; cell_geom(dim, P->s.X, P->s.cells + (size_t)c * (dim + 1), &G);
        for (int l = 0; l < nl; ++l) {
            int m = S->cell2dof[(size_t)c * nl + l];
            if (seen[m]) continue;
            seen[m] = 1;
            double xi[3], lam[4], dx[3];
            for (int d = 0; d < dim; ++d) dx[d] = S->coords[(size_t)m * dim + d] - G.x0[d];
            for (int r = 0; r < dim; ++r) { xi[r] = 0; for (int q = 0; q < dim; ++q) xi[r] += G.Binv[r * dim + q] * dx[q]; }
            double v[ORC_MAXNB];
            elem_eval(&P->P1, xi, v, NULL);
            for (int j = 0; j <= dim; ++j) lam[j] = v[j];
            for (int j = 0; j <= dim; ++j) coo_push(Pi, m, P->s.cells[(size_t)c * (dim + 1) + j], 0, lam[j]);
        }
    }
    free(seen);
    coo_compress(Pi);
}

/* Local tensors of cell c (Sec. 3.3): Tloc[a][m][b] = int_K eta_m grad phi_b . grad phi_a,
 * Mloc[a][m] = int_K eta_m phi_a, both by quadrature. */
static void local_tensors(const orc_problem *P, int c, const orc_elem *EW, const double *eta_tab, double *Tloc, double *Mloc) {
    int dim = P->s.dim, nv = dim + 1, nw = EW->nb;
    orc_geom G; cell_geom(dim, P->s.X, P->s.cells + (size_t)c * nv, &G);
    double g[4][3];
    for (int a = 0; a < nv; ++a) phys_grad(dim, &G, P->gref1 + a * dim, g[a]);
    if (Tloc) memset(Tloc, 0, sizeof(double) * nv * nw * nv);
    if (Mloc) memset(Mloc, 0, sizeof(double) * nv * nw);
    for (int q = 0; q < P->nq; ++q) {
        double wq = P->qw[q] * factorial(dim) * G.vol;     /* reference weights sum to 1/d! */
        const double *eta = eta_tab + q * ORC_MAXNB, *phi = P->phi_q + q * ORC_MAXNB;
        for (int a = 0; a < nv; ++a)
            for (int m = 0; m < nw; ++m) {
                if (Mloc) Mloc[a * nw + m] += wq * eta[m] * phi[a];
                if (Tloc)
                    for (int b = 0; b < nv; ++b) {
                        double gg = 0.0;
                        for (int d = 0; d < dim; ++d) gg += g[b][d] * g[a][d];
                        Tloc[(a * nw + m) * nv + b] += wq * eta[m] * gg;
                    }
            }
    }
}

/* Local tensors of cell c for a quadrature space (Sec. 3.1, Case 3): with eta_l = w_l delta_{x_l},
 * Tloc[a][l][b] = w_l grad phi_b(x_l) . grad phi_a(x_l) and Mloc[a][l] = w_l phi_a(x_l), w_l the
 * physical weight (reference weight d! |K|). */
static void local_tensors_quad(const orc_problem *P, int c, int nq, const double *qp, const double *qw, double *Tloc, double *Mloc) {
    int dim = P->s.dim, nv = dim + 1;
    orc_geom G; cell_geom(dim, P->s.X, P->s.cells + (size_t)c * nv, &G);
    double g[4][3];
    for (int a = 0; a < nv; ++a) phys_grad(dim, &G, P->gref1 + a * dim, g[a]);
    for (int l = 0; l < nq; ++l) {
        double wl = qw[l] * factorial(dim) * G.vol, phi[ORC_MAXNB];
        elem_eval(&P->P1, qp + l * dim, phi, NULL);
        for (int a = 0; a < nv; ++a) {
            if (Mloc) Mloc[a * nq + l] = wl * phi[a];
            if (Tloc)
                for (int b = 0; b < nv; ++b) {
                    double gg = 0.0;
                    for (int d = 0; d < dim; ++d) gg += g[b][d] * g[a][d];
                    Tloc[(a * nq + l) * nv + b] = wl * gg;
                }
        }
    }
}

/* Trilinear mass form of cell c (decomposition (a) of the superconductivity example, Sec. 5):
 * M3loc[a][m][b] = int_K eta_m phi_b phi_a, by the oracle's quadrature for a Lagrange W and by
 * the delta basis w_l phi_a(x_l) phi_b(x_l) for a quadrature space. */
static void local_mass3(const orc_problem *P, int c, int quad, const orc_elem *EW, const double *eta_tab, int nq,
                        const double *qp, const double *qw, double *M3) {
    int dim = P->s.dim, nv = dim + 1;
    orc_geom G; cell_geom(dim, P->s.X, P->s.cells + (size_t)c * nv, &G);
    if (quad) {
        for (int l = 0; l < nq; ++l) {
            double wl = qw[l] * factorial(dim) * G.vol, phi[ORC_MAXNB];
            elem_eval(&P->P1, qp + l * dim, phi, NULL);
            for (int a = 0; a < nv; ++a)
                for (int b = 0; b < nv; ++b) M3[(a * nq + l) * nv + b] = wl * phi[a] * phi[b];
        }
        return;
    }
    int nw = EW->nb;
    memset(M3, 0, sizeof(double) * nv * nw * nv);
    for (int q = 0; q < P->nq; ++q) {
        double wq = P->qw[q] * factorial(dim) * G.vol;
        const double *eta = eta_tab + q * ORC_MAXNB, *phi = P->phi_q + q * ORC_MAXNB;
        for (int a = 0; a < nv; ++a)
            for (int m = 0; m < nw; ++m)
                for (int b = 0; b < nv; ++b) M3[(a * nw + m) * nv + b] += wq * eta[m] * phi[a] * phi[b];
    }
}

orc_problem *orc_create(const orc_spec *spec, const int *cell_list, int n_cell_list) {
    orc_problem *P = calloc(1, sizeof(orc_problem));
    P->s = *spec;
    int dim = spec->dim, nv = dim + 1;
    elem_init(&P->P1, dim, 1);
    if (P->s.a_deg < 0) P->s.a_deg = 1;
    if (P->s.c_deg < 0) P->s.c_deg = 1;
    /* a quadrature space has no polynomial basis: its element slot holds P0 (unused) */
    elem_init(&P->Ea, dim, P->s.a_quad ? 0 : P->s.a_deg);
    elem_init(&P->Ec, dim, P->s.c_quad ? 0 : P->s.c_deg);
    P->nq = spec->rule > 0 ? sym_rule(dim, spec->rule, P->qp, P->qw) : simplex_rule(dim, spec->qpts, P->qp, P->qw);
    if (P->nq <= 0) { free(P); return NULL; }
    if (P->s.a_quad && (P->aq_n = sym_rule(dim, P->s.a_deg, P->aq_p, P->aq_w)) <= 0) { free(P); return NULL; }
    if (P->s.c_quad && (P->cq_n = sym_rule(dim, P->s.c_deg, P->cq_p, P->cq_w)) <= 0) { free(P); return NULL; }
    P->phi_q = malloc(sizeof(double) * P->nq * ORC_MAXNB);
    P->eta_a_q = malloc(sizeof(double) * P->nq * ORC_MAXNB);
    P->eta_c_q = malloc(sizeof(double) * P->nq * ORC_MAXNB);
    for (int q = 0; q < P->nq; ++q) {
        elem_eval(&P->P1, P->qp + q * dim, P->phi_q + q * ORC_MAXNB, NULL);
        elem_eval(&P->Ea, P->qp + q * dim, P->eta_a_q + q * ORC_MAXNB, NULL);
        elem_eval(&P->Ec, P->qp + q * dim, P->eta_c_q + q * ORC_MAXNB, NULL);
    }
    { double xi0[3] = {0.25, 0.25, 0.25}; elem_eval(&P->P1, xi0, NULL, P->gref1); }
    if (P->s.a_quad) space_build_quad(dim, spec->nc, spec->X, spec->cells, P->aq_n, P->aq_p, &P->Sa);
    else space_build(dim, spec->nc, spec->X, spec->cells, P->s.a_deg, &P->Sa);
    if (P->s.c_quad) space_build_quad(dim, spec->nc, spec->X, spec->cells, P->cq_n, P->cq_p, &P->Sc);
    else space_build(dim, spec->nc, spec->X, spec->cells, P->s.c_deg, &P->Sc);
    build_interp(P, &P->Sa, &P->Pa);
    build_interp(P, &P->Sc, &P->Pc);
    P->cell_mask = calloc(spec->nc, sizeof(int));
    if (cell_list) for (int t = 0; t < n_cell_list; ++t) P->cell_mask[cell_list[t]] = 1;
    else for (int c = 0; c < spec->nc; ++c) P->cell_mask[c] = 1;
    /* assemble T (always) and M (when a reaction term is present) over the selected cells */
    double Tloc[4 * ORC_MAXNB * 4], Mloc[4 * ORC_MAXNB];
    const int nwa = P->Sa.nloc, nwc = P->Sc.nloc;
    for (int c = 0; c < spec->nc; ++c) {
        if (!P->cell_mask[c]) continue;
        const int *cv = spec->cells + (size_t)c * nv;
        if (P->s.a_quad) local_tensors_quad(P, c, P->aq_n, P->aq_p, P->aq_w, Tloc, NULL);
        else local_tensors(P, c, &P->Ea, P->eta_a_q, Tloc, NULL);
        const int *wa = P->Sa.cell2dof + (size_t)c * nwa;
        for (int a = 0; a < nv; ++a)
            for (int m = 0; m < nwa; ++m)
                for (int b = 0; b < nv; ++b)
                    coo_push(&P->T, cv[a], wa[m], cv[b], Tloc[(a * nwa + m) * nv + b]);
        if (spec->c_kind != ORC_G_NONE && spec->c_product) {
            double M3loc[4 * ORC_MAXNB * 4];
            local_mass3(P, c, P->s.c_quad, &P->Ec, P->eta_c_q, P->cq_n, P->cq_p, P->cq_w, M3loc);
            const int *wc = P->Sc.cell2dof + (size_t)c * nwc;
            for (int a = 0; a < nv; ++a)
                for (int m = 0; m < nwc; ++m)
                    for (int b = 0; b < nv; ++b) coo_push(&P->M3, cv[a], wc[m], cv[b], M3loc[(a * nwc + m) * nv + b]);
        } else if (spec->c_kind != ORC_G_NONE) {
            if (P->s.c_quad) local_tensors_quad(P, c, P->cq_n, P->cq_p, P->cq_w, NULL, Mloc);
            else local_tensors(P, c, &P->Ec, P->eta_c_q, NULL, Mloc);
            const int *wc = P->Sc.cell2dof + (size_t)c * nwc;
            for (int a = 0; a < nv; ++a)
                for (int m = 0; m < nwc; ++m)
                    coo_push(&P->M, cv[a], wc[m], 0, Mloc[a * nwc + m]);
        }
    }
    coo_compress(&P->T);
    coo_compress(&P->M);
    coo_compress(&P->M3);
    if (spec->sigma != 0.0) {
        /* the P1 mass matrix by the same quadrature (the P1 element as its own W space) */
        for (int c = 0; c < spec->nc; ++c) {
            if (!P->cell_mask[c]) continue;
            const int *cv = spec->cells + (size_t)c * nv;
            local_tensors(P, c, &P->P1, P->phi_q, NULL, Mloc);
            for (int a = 0; a < nv; ++a)
                for (int m = 0; m < nv; ++m) coo_push(&P->Mu, cv[a], cv[m], 0, Mloc[a * nv + m]);
        }
        coo_compress(&P->Mu);
    }
    return P;
}

void orc_destroy(orc_problem *P) {
    if (!P) return;
    space_free(&P->Sa); space_free(&P->Sc);
    free(P->T.t); free(P->M.t); free(P->Pa.t); free(P->Pc.t); free(P->Mu.t); free(P->M3.t);
    free(P->kappa_field); free(P->cell_mask);
    free(P->phi_q); free(P->eta_a_q); free(P->eta_c_q);
    free(P);
}

void orc_set_kappa_field(orc_problem *P, const double *kappa) {
    free(P->kappa_field); P->kappa_field = NULL;
    if (kappa) { P->kappa_field = malloc(sizeof(double) * P->Sa.n); memcpy(P->kappa_field, kappa, sizeof(double) * P->Sa.n); }
}

/* --- introspection --- */
int orc_space_size(const orc_problem *P, int which) { return which == 0 ? P->Sa.n : P->Sc.n; }
void orc_space_coords(const orc_problem *P, int which, double *out) {
    const orc_space *S = which == 0 ? &P->Sa : &P->Sc;
    memcpy(out, S->coords, sizeof(double) * S->n * P->s.dim);
}
int orc_space_nloc(const orc_problem *P, int which) { return which == 0 ? P->Sa.nloc : P->Sc.nloc; }
void orc_space_cell2dof(const orc_problem *P, int which, int *out) {
    const orc_space *S = which == 0 ? &P->Sa : &P->Sc;
    memcpy(out, S->cell2dof, sizeof(int) * (size_t)P->s.nc * S->nloc);
}
int64_t orc_coo_size(const orc_problem *P, int which) {
    const orc_coo *C = which == 0 ? &P->T : which == 1 ? &P->M : which == 2 ? &P->Pa : &P->Pc;
    return (int64_t)C->n;
}
void orc_coo_export(const orc_problem *P, int which, int64_t *I, int64_t *J, int64_t *K, double *V) {
    const orc_coo *C = which == 0 ? &P->T : which == 1 ? &P->M : which == 2 ? &P->Pa : &P->Pc;
    for (size_t t = 0; t < C->n; ++t) { I[t] = C->t[t].i; J[t] = C->t[t].j; K[t] = C->t[t].k; V[t] = C->t[t].v; }
}
int orc_num_qpts(const orc_problem *P) { return P->nq; }
void orc_ref_rule(const orc_problem *P, double *pts, double *wts) {
    memcpy(pts, P->qp, sizeof(double) * P->nq * P->s.dim);
    memcpy(wts, P->qw, sizeof(double) * P->nq);
}

/* reference-element probes for pin tests */
int orc_ref_basis(int dim, int p, int npts, const double *xi, double *val, double *grad) {
    orc_elem E; elem_init(&E, dim, p);
    for (int t = 0; t < npts; ++t)
        elem_eval(&E, xi + t * dim, val ? val + (size_t)t * E.nb : NULL, grad ? grad + (size_t)t * E.nb * dim : NULL);
    return E.nb;
}
void orc_ref_nodes(int dim, int p, int *alpha) {
    orc_elem E; elem_init(&E, dim, p);
    for (int i = 0; i < E.nb; ++i) for (int j = 0; j <= dim; ++j) alpha[i * (dim + 1) + j] = E.alpha[i][j];
}
int orc_simplex_rule(int dim, int q, double *pts, double *wts) { return simplex_rule(dim, q, pts, wts); }
int orc_sym_rule(int dim, int k, double *pts, double *wts) { return sym_rule(dim, k, pts, wts); }

/* ------------------------------------------------------------------------- */
/* Pointwise nonlinearity (Sec. 3.2): f = g(Pi u) at every W node               */
/* ------------------------------------------------------------------------- */

static void interp_apply(const orc_coo *Pi, int n, const double *u, double *out) {
    for (int m = 0; m < n; ++m) out[m] = 0.0;
    for (size_t t = 0; t < Pi->n; ++t) out[Pi->t[t].i] += Pi->t[t].v * u[Pi->t[t].j];
}

/* ||grad u_h||^2 on cell c (constant for P1) and the P1 basis gradients g[a] */
static double cell_grad2(const orc_problem *P, int c, const double *u, double g[4][3], double gu[3]) {
    int dim = P->s.dim, nv = dim + 1;
    const int *cv = P->s.cells + (size_t)c * nv;
    orc_geom G; cell_geom(dim, P->s.X, cv, &G);
    for (int a = 0; a < nv; ++a) phys_grad(dim, &G, P->gref1 + a * dim, g[a]);
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
        gu[d] = 0.0;
        for (int a = 0; a < nv; ++a) gu[d] += u[cv[a]] * g[a][d];
        s += gu[d] * gu[d];
    }
    return s;
}

void orc_pointwise(const orc_problem *P, const double *u, double *w, double *wprime, double *c, double *cprime) {
    double *pa = malloc(sizeof(double) * P->Sa.n), *pc = malloc(sizeof(double) * P->Sc.n);
    if (P->s.a_kind == ORC_G_GRADPOW) {
        /* W_a = P0 (or I_k): every node of cell c carries ||grad u_h||^2 on c */
        for (int c = 0; c < P->s.nc; ++c) {
            double g[4][3], gu[3];
            double s2 = cell_grad2(P, c, u, g, gu);
            for (int l = 0; l < P->Sa.nloc; ++l) pa[P->Sa.cell2dof[(size_t)c * P->Sa.nloc + l]] = s2;
        }
    } else {
        interp_apply(&P->Pa, P->Sa.n, u, pa);
    }
    interp_apply(&P->Pc, P->Sc.n, u, pc);
    for (int m = 0; m < P->Sa.n; ++m) {
        if (w) w[m] = ga_val(&P->s, pa[m]);
        if (wprime) wprime[m] = ga_der(&P->s, pa[m]);
    }
    for (int m = 0; m < P->Sc.n; ++m) {
        if (c) c[m] = g_val(P->s.c_kind, P->s.c_p, P->s.c_scale, pc[m]);
        if (cprime) cprime[m] = g_der(P->s.c_kind, P->s.c_p, P->s.c_scale, pc[m]);
    }
    free(pa); free(pc);
}

/* ------------------------------------------------------------------------- */
/* EGFEM residual and Jacobian from the assembled tensors                      */
/* ------------------------------------------------------------------------- */

/* r over all nodes; rows whose cells were not all assembled are meaningless (callers
 * that assemble a cell subset read only the rows they asked for). */
void orc_egfem_residual(const orc_problem *P, const double *u, const double *b, const double *uD,
                        int form, double *r) {
    int nv = P->s.nv;
    double *w = malloc(sizeof(double) * P->Sa.n), *c = malloc(sizeof(double) * P->Sc.n);
    orc_pointwise(P, u, w, NULL, c, NULL);
    for (int i = 0; i < nv; ++i) r[i] = 0.0;
    for (size_t t = 0; t < P->T.n; ++t) {
        int64_t i = P->T.t[t].i, m = P->T.t[t].j, k = P->T.t[t].k;
        double a = (P->kappa_field ? P->kappa_field[m] : P->s.kappa) + w[m];
        double uk = (form == ORC_FORM_DIFF) ? (u[k] - u[i]) : u[k];
        r[i] += P->T.t[t].v * a * uk;
    }
    if (P->s.c_kind != ORC_G_NONE)
        for (size_t t = 0; t < P->M.n; ++t) r[P->M.t[t].i] += P->s.gamma * P->M.t[t].v * c[P->M.t[t].j];
    for (size_t t = 0; t < P->Mu.n; ++t) r[P->Mu.t[t].i] += P->s.sigma * P->Mu.t[t].v * u[P->Mu.t[t].j];
    /* product reaction: gamma sum_{m,k} M3_imk c_m u_k */
    for (size_t t = 0; t < P->M3.n; ++t)
        r[P->M3.t[t].i] += P->s.gamma * P->M3.t[t].v * c[P->M3.t[t].j] * u[P->M3.t[t].k];
    for (int i = 0; i < nv; ++i) {
        if (P->s.dir[i]) r[i] = u[i] - (uD ? uD[i] : 0.0);
        else r[i] -= b ? b[i] : 0.0;
    }
    free(w); free(c);
}

/* Iteration matrix as sorted COO (i, l, value); returns the entry count, fills up to cap.
 * picard = 0: the Newton Jacobian (T .2 a) + (T .3 u) diag(g') Pi + gamma M diag(g_c') Pi_c
 * (Sec. 4, identity blocks eliminated).  picard = 1: the frozen-coefficient matrix T .2 a of
 * the Picard iteration (Sec. 4 and Example 4.1: the coefficient is taken at the previous
 * iterate, the reaction term on the right-hand side). */
static int64_t egfem_matrix(const orc_problem *P, const double *u, int picard, int64_t cap, int64_t *I, int64_t *L,
                            double *V) {
    int nv = P->s.nv;
    double *w = malloc(sizeof(double) * P->Sa.n), *wp = malloc(sizeof(double) * P->Sa.n);
    double *c = malloc(sizeof(double) * P->Sc.n), *cp = malloc(sizeof(double) * P->Sc.n);
    orc_pointwise(P, u, w, wp, c, cp);
    orc_coo J = {0};
    /* (T .2 a): J_il += T_iml a_m */
    for (size_t t = 0; t < P->T.n; ++t) {
        int64_t i = P->T.t[t].i, m = P->T.t[t].j, l = P->T.t[t].k;
        double a = (P->kappa_field ? P->kappa_field[m] : P->s.kappa) + w[m];
        coo_push(&J, i, l, 0, P->T.t[t].v * a);
    }
    /* the linear reaction sigma M (a linear term: in the Picard matrix as well) */
    for (size_t t = 0; t < P->Mu.n; ++t) coo_push(&J, P->Mu.t[t].i, P->Mu.t[t].j, 0, P->s.sigma * P->Mu.t[t].v);
    /* (T .3 u) diag(g') Pi: D_im = sum_k T_imk u_k, then J_il += D_im g'_m Pi_ml */
    orc_coo D = {0};
    if (!picard)
        for (size_t t = 0; t < P->T.n; ++t) coo_push(&D, P->T.t[t].i, P->T.t[t].j, 0, P->T.t[t].v * u[P->T.t[t].k]);
    coo_compress(&D);
    /* d(argument of g at node m)/du_l: the interpolation Pi_ml, or for a gradient nonlinearity
     * (W_a = P0) d||grad u_K||^2/du_l = 2 grad u_K . grad phi_l on the cell K of node m */
    orc_coo Pg = {0};
    const orc_coo *Pm = &P->Pa;
    if (P->s.a_kind == ORC_G_GRADPOW) {
        int nvc = P->s.dim + 1;
        for (int c = 0; c < P->s.nc; ++c) {
            double g[4][3], gu[3];
            cell_grad2(P, c, u, g, gu);
            for (int q = 0; q < P->Sa.nloc; ++q) {
                int m = P->Sa.cell2dof[(size_t)c * P->Sa.nloc + q];
                for (int l = 0; l < nvc; ++l) {
                    double t = 0.0;
                    for (int d = 0; d < P->s.dim; ++d) t += gu[d] * g[l][d];
                    coo_push(&Pg, m, P->s.cells[(size_t)c * nvc + l], 0, 2.0 * t);
                }
            }
        }
        coo_compress(&Pg);
        Pm = &Pg;
    }
    size_t *pstart = calloc(P->Sa.n + 1, sizeof(size_t));
    for (size_t t = 0; t < Pm->n; ++t) pstart[Pm->t[t].i + 1]++;
    for (int m = 0; m < P->Sa.n; ++m) pstart[m + 1] += pstart[m];
    for (size_t t = 0; t < D.n; ++t) {
        int64_t i = D.t[t].i, m = D.t[t].j;
        double e = D.t[t].v * wp[m];
        for (size_t q = pstart[m]; q < pstart[m + 1]; ++q) coo_push(&J, i, Pm->t[q].j, 0, e * Pm->t[q].v);
    }
    free(pstart);
    free(Pg.t);
    /* product reaction: gamma (M3 .2 c) (kept by Picard), and gamma (M3 .3 u) diag(c') Pi_c */
    if (P->s.c_product && P->s.c_kind != ORC_G_NONE) {
        for (size_t t = 0; t < P->M3.n; ++t)
            coo_push(&J, P->M3.t[t].i, P->M3.t[t].k, 0, P->s.gamma * P->M3.t[t].v * c[P->M3.t[t].j]);
        if (!picard) {
            orc_coo E = {0};   /* E_im = sum_k M3_imk u_k */
            for (size_t t = 0; t < P->M3.n; ++t) coo_push(&E, P->M3.t[t].i, P->M3.t[t].j, 0, P->M3.t[t].v * u[P->M3.t[t].k]);
            coo_compress(&E);
            size_t *cs = calloc(P->Sc.n + 1, sizeof(size_t));
            for (size_t t = 0; t < P->Pc.n; ++t) cs[P->Pc.t[t].i + 1]++;
            for (int m = 0; m < P->Sc.n; ++m) cs[m + 1] += cs[m];
            for (size_t t = 0; t < E.n; ++t) {
                int64_t i = E.t[t].i, m = E.t[t].j;
                double e = P->s.gamma * E.t[t].v * cp[m];
                for (size_t q = cs[m]; q < cs[m + 1]; ++q) coo_push(&J, i, P->Pc.t[q].j, 0, e * P->Pc.t[q].v);
            }
            free(cs);
            free(E.t);
        }
    }
    /* gamma M diag(g_c') Pi_c */
    if (!picard && P->s.c_kind != ORC_G_NONE && !P->s.c_product) {
        size_t *cs = calloc(P->Sc.n + 1, sizeof(size_t));
        for (size_t t = 0; t < P->Pc.n; ++t) cs[P->Pc.t[t].i + 1]++;
        for (int m = 0; m < P->Sc.n; ++m) cs[m + 1] += cs[m];
        for (size_t t = 0; t < P->M.n; ++t) {
            int64_t i = P->M.t[t].i, m = P->M.t[t].j;
            double e = P->s.gamma * P->M.t[t].v * cp[m];
            for (size_t q = cs[m]; q < cs[m + 1]; ++q) coo_push(&J, i, P->Pc.t[q].j, 0, e * P->Pc.t[q].v);
        }
        free(cs);
    }
    coo_compress(&J);
    /* Dirichlet rows -> identity, Dirichlet columns of free rows -> removed */
    orc_coo Jd = {0};
    for (size_t t = 0; t < J.n; ++t) {
        int64_t i = J.t[t].i, l = J.t[t].j;
        if (P->s.dir[i] || P->s.dir[l]) continue;
        coo_push(&Jd, i, l, 0, J.t[t].v);
    }
    for (int i = 0; i < nv; ++i) if (P->s.dir[i]) coo_push(&Jd, i, i, 0, 1.0);
    coo_compress(&Jd);
    int64_t n = (int64_t)Jd.n;
    for (int64_t t = 0; t < n && t < cap; ++t) { I[t] = Jd.t[t].i; L[t] = Jd.t[t].j; V[t] = Jd.t[t].v; }
    free(J.t); free(D.t); free(Jd.t);
    free(w); free(wp); free(c); free(cp);
    return n;
}

int64_t orc_egfem_jacobian(const orc_problem *P, const double *u, int64_t cap, int64_t *I, int64_t *L, double *V) {
    return egfem_matrix(P, u, 0, cap, I, L, V);
}

int64_t orc_picard_matrix(const orc_problem *P, const double *u, int64_t cap, int64_t *I, int64_t *L, double *V) {
    return egfem_matrix(P, u, 1, cap, I, L, V);
}

/* ------------------------------------------------------------------------- */
/* SGA residual and Jacobian: re-integrated at every call (Sec. 2.1, Sec. 4)   */
/* ------------------------------------------------------------------------- */

static double kappa_at(const orc_problem *P, int c, const double *eta) {
    if (!P->kappa_field) return P->s.kappa;
    if (P->s.a_quad) return NAN;   /* a kappa field on I_k has no values between its nodes */
    const int *wa = P->Sa.cell2dof + (size_t)c * P->Sa.nloc;
    double k = 0.0;
    for (int m = 0; m < P->Ea.nb; ++m) k += P->kappa_field[wa[m]] * eta[m];
    return k;
}

void orc_sga_residual(const orc_problem *P, const double *u, const double *b, const double *uD, int form, double *r) {
    int dim = P->s.dim, nv = dim + 1;
    for (int i = 0; i < P->s.nv; ++i) r[i] = 0.0;
    double g[4][3];
    const double *gref = P->gref1;
    for (int c = 0; c < P->s.nc; ++c) {
        if (!P->cell_mask[c]) continue;
        const int *cv = P->s.cells + (size_t)c * nv;
        orc_geom G; cell_geom(dim, P->s.X, cv, &G);
        for (int a = 0; a < nv; ++a) phys_grad(dim, &G, gref + a * dim, g[a]);
        for (int q = 0; q < P->nq; ++q) {
            double wq = P->qw[q] * factorial(dim) * G.vol;
            const double *phi = P->phi_q + q * ORC_MAXNB, *eta = P->eta_a_q + q * ORC_MAXNB;
            double uh = 0.0;
            for (int a = 0; a < nv; ++a) uh += u[cv[a]] * phi[a];
            /* the coefficient's argument at the quadrature point: u_h, or ||grad u_h||^2 */
            double arg = uh;
            if (P->s.a_kind == ORC_G_GRADPOW) {
                arg = 0.0;
                for (int d = 0; d < dim; ++d) { double gd = 0.0; for (int a = 0; a < nv; ++a) gd += u[cv[a]] * g[a][d]; arg += gd * gd; }
            }
            double coef = kappa_at(P, c, eta) + ga_val(&P->s, arg);
            double reac = (P->s.c_kind != ORC_G_NONE) ? P->s.gamma * g_val(P->s.c_kind, P->s.c_p, P->s.c_scale, uh) : 0.0;
            if (P->s.c_product) reac *= uh;
            reac += P->s.sigma * uh;
            for (int a = 0; a < nv; ++a) {
                double gu = 0.0;
                for (int b2 = 0; b2 < nv; ++b2) {
                    double gg = 0.0;
                    for (int d = 0; d < dim; ++d) gg += g[b2][d] * g[a][d];
                    gu += gg * ((form == ORC_FORM_DIFF) ? (u[cv[b2]] - u[cv[a]]) : u[cv[b2]]);
                }
                r[cv[a]] += wq * (coef * gu + reac * phi[a]);
            }
        }
    }
    for (int i = 0; i < P->s.nv; ++i) {
        if (P->s.dir[i]) r[i] = u[i] - (uD ? uD[i] : 0.0);
        else r[i] -= b ? b[i] : 0.0;
    }
}

int64_t orc_sga_jacobian(const orc_problem *P, const double *u, int64_t cap, int64_t *I, int64_t *L, double *V) {
    int dim = P->s.dim, nv = dim + 1;
    orc_coo J = {0};
    double g[4][3];
    const double *gref = P->gref1;
    for (int c = 0; c < P->s.nc; ++c) {
        if (!P->cell_mask[c]) continue;
        const int *cv = P->s.cells + (size_t)c * nv;
        orc_geom G; cell_geom(dim, P->s.X, cv, &G);
        for (int a = 0; a < nv; ++a) phys_grad(dim, &G, gref + a * dim, g[a]);
        double Jloc[16] = {0};
        for (int q = 0; q < P->nq; ++q) {
            double wq = P->qw[q] * factorial(dim) * G.vol;
            const double *phi = P->phi_q + q * ORC_MAXNB, *eta = P->eta_a_q + q * ORC_MAXNB;
            double uh = 0.0;
            for (int a = 0; a < nv; ++a) uh += u[cv[a]] * phi[a];
            const int gradc = P->s.a_kind == ORC_G_GRADPOW;
            double guh[3] = {0.0, 0.0, 0.0}, arg = uh;
            if (gradc) {
                arg = 0.0;
                for (int d = 0; d < dim; ++d) { for (int a = 0; a < nv; ++a) guh[d] += u[cv[a]] * g[a][d]; arg += guh[d] * guh[d]; }
            }
            double coef = kappa_at(P, c, eta) + ga_val(&P->s, arg);
            double dcoef = ga_der(&P->s, arg);
            double dreac = (P->s.c_kind != ORC_G_NONE) ? P->s.gamma * g_der(P->s.c_kind, P->s.c_p, P->s.c_scale, uh) : 0.0;
            if (P->s.c_product && P->s.c_kind != ORC_G_NONE)   /* d(g(u) u)/du = g'(u) u + g(u) */
                dreac = dreac * uh + P->s.gamma * g_val(P->s.c_kind, P->s.c_p, P->s.c_scale, uh);
            dreac += P->s.sigma;
            for (int a = 0; a < nv; ++a) {
                double gu = 0.0;
                for (int b2 = 0; b2 < nv; ++b2) {
                    double gg = 0.0;
                    for (int d = 0; d < dim; ++d) gg += g[b2][d] * g[a][d];
                    gu += gg * u[cv[b2]];
                }
                for (int l = 0; l < nv; ++l) {
                    double gg = 0.0;
                    for (int d = 0; d < dim; ++d) gg += g[l][d] * g[a][d];
                    /* d coef / d u_l: g'(u_h) phi_l, or g'(s) 2 grad u_h . grad phi_l */
                    double dl = phi[l];
                    if (gradc) { dl = 0.0; for (int d = 0; d < dim; ++d) dl += 2.0 * guh[d] * g[l][d]; }
                    Jloc[a * nv + l] += wq * (coef * gg + dcoef * dl * gu + dreac * phi[l] * phi[a]);
                }
            }
        }
        for (int a = 0; a < nv; ++a) for (int l = 0; l < nv; ++l) coo_push(&J, cv[a], cv[l], 0, Jloc[a * nv + l]);
    }
    coo_compress(&J);
    orc_coo Jd = {0};
    for (size_t t = 0; t < J.n; ++t) {
        int64_t i = J.t[t].i, l = J.t[t].j;
        if (P->s.dir[i] || P->s.dir[l]) continue;
        coo_push(&Jd, i, l, 0, J.t[t].v);
    }
    for (int i = 0; i < P->s.nv; ++i) if (P->s.dir[i]) coo_push(&Jd, i, i, 0, 1.0);
    coo_compress(&Jd);
    int64_t n = (int64_t)Jd.n;
    for (int64_t t = 0; t < n && t < cap; ++t) { I[t] = Jd.t[t].i; L[t] = Jd.t[t].j; V[t] = Jd.t[t].v; }
    free(J.t); free(Jd.t);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Load vector d_i = int f phi_i by the same quadrature                        */
/* ------------------------------------------------------------------------- */

/* physical quadrature points of every cell: xq[(c*nq + q)*dim + d] */
void orc_quad_points(const orc_problem *P, double *xq) {
    int dim = P->s.dim, nv = dim + 1;
    for (int c = 0; c < P->s.nc; ++c) {
        orc_geom G; cell_geom(dim, P->s.X, P->s.cells + (size_t)c * nv, &G);
        for (int q = 0; q < P->nq; ++q)
            for (int r = 0; r < dim; ++r) {
                double x = G.x0[r];
                for (int k = 0; k < dim; ++k) x += G.B[r * dim + k] * P->qp[q * dim + k];
                xq[((size_t)c * P->nq + q) * dim + r] = x;
            }
    }
}

/* b_i = sum_K sum_q w_q |K| f(x_q) phi_i(x_q), f given at the points of orc_quad_points */
void orc_load_vector(const orc_problem *P, const double *fq, double *b) {
    int dim = P->s.dim, nv = dim + 1;
    for (int i = 0; i < P->s.nv; ++i) b[i] = 0.0;
    for (int c = 0; c < P->s.nc; ++c) {
        const int *cv = P->s.cells + (size_t)c * nv;
        orc_geom G; cell_geom(dim, P->s.X, cv, &G);
        for (int q = 0; q < P->nq; ++q) {
            double wq = P->qw[q] * factorial(dim) * G.vol;
            const double *phi = P->phi_q + q * ORC_MAXNB;
            for (int a = 0; a < nv; ++a) b[cv[a]] += wq * fq[(size_t)c * P->nq + q] * phi[a];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Linear algebra: CSR from COO, banded LU, Jacobi BiCGStab                     */
/* ------------------------------------------------------------------------- */

/* Banded LU with partial pivoting (the LAPACK gbtrf/gbtrs scheme): A is n x n with kl
 * sub- and ku super-diagonals, stored densely by rows in a (2kl+ku+1)-wide window
 * (extra kl columns receive fill from row interchanges).  Solves A x = rhs in place. */
int orc_band_solve(int n, int kl, int ku, int64_t nnz, const int64_t *I, const int64_t *L, const double *V, double *x) {
    int w = 2 * kl + ku + 1;                 /* row i stores columns i-kl .. i+kl+ku */
    double *A = calloc((size_t)n * w, sizeof(double));
    if (!A) return -2;
    for (int64_t t = 0; t < nnz; ++t) {
        int64_t off = L[t] - I[t] + kl;
        if (off < 0 || off >= w) { free(A); return -3; }
        A[(size_t)I[t] * w + off] += V[t];
    }
#define AB(i, j) A[(size_t)(i) * w + ((j) - (i) + kl)]
    for (int c = 0; c < n; ++c) {
        int last = c + kl < n - 1 ? c + kl : n - 1;
        int piv = c;
        for (int r = c + 1; r <= last; ++r) if (fabs(AB(r, c)) > fabs(AB(piv, c))) piv = r;
        if (AB(piv, c) == 0.0) { free(A); return -1; }
        int cmax = c + kl + ku < n - 1 ? c + kl + ku : n - 1;
        if (piv != c) {
            for (int j = c; j <= cmax; ++j) { double t = AB(c, j); AB(c, j) = AB(piv, j); AB(piv, j) = t; }
            double t = x[c]; x[c] = x[piv]; x[piv] = t;
        }
        for (int r = c + 1; r <= last; ++r) {
            double f = AB(r, c) / AB(c, c);
            if (f == 0.0) continue;
            for (int j = c; j <= cmax; ++j) AB(r, j) -= f * AB(c, j);
            x[r] -= f * x[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        int cmax = c + kl + ku < n - 1 ? c + kl + ku : n - 1;
        double s = x[c];
        for (int j = c + 1; j <= cmax; ++j) s -= AB(c, j) * x[j];
        x[c] = s / AB(c, c);
    }
#undef AB
    free(A);
    return 0;
}

/* Inner product as ORC_DOT_CHUNKS contiguous partial sums added in chunk order: the same
 * result for any number of OpenMP threads (the chunks, not the threads, fix the order). */
#define ORC_DOT_CHUNKS 64
static double dot(int n, const double *a, const double *b) {
    double part[ORC_DOT_CHUNKS];
#pragma omp parallel for schedule(static)
    for (int c = 0; c < ORC_DOT_CHUNKS; ++c) {
        const int lo = (int)((int64_t)n * c / ORC_DOT_CHUNKS), hi = (int)((int64_t)n * (c + 1) / ORC_DOT_CHUNKS);
        double s = 0;
        for (int i = lo; i < hi; ++i) s += a[i] * b[i];
        part[c] = s;
    }
    double s = 0;
    for (int c = 0; c < ORC_DOT_CHUNKS; ++c) s += part[c];
    return s;
}

/* y = A x, one row at a time (rows split across OpenMP threads; each row summed in order) */
static void csr_matvec(int n, const int64_t *rp, const int64_t *ci, const double *v, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) { double s = 0; for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s += v[t] * x[ci[t]]; y[i] = s; }
}

/* Right-preconditioned BiCGStab (van der Vorst 1992) with M = diag(A)^{-1}.
 * A in sorted COO (row-major).  Stops when ||b - A x|| <= rtol ||b||.  x in: guess. */
/* OpenMP threads of the oracle's parallel loops (results do not depend on it) */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_bicgstab(int n, int64_t nnz, const int64_t *I, const int64_t *L, const double *V,
                 const double *b, double *x, double rtol, int maxit, int *iters, double *relres) {
    int64_t *rp = calloc(n + 1, sizeof(int64_t));
    for (int64_t t = 0; t < nnz; ++t) rp[I[t] + 1]++;
    for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
    double *D = malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) { D[i] = 0; for (int64_t t = rp[i]; t < rp[i + 1]; ++t) if (L[t] == i) D[i] = V[t]; }
    for (int i = 0; i < n; ++i) { if (D[i] == 0.0) { free(rp); free(D); return -4; } D[i] = 1.0 / D[i]; }
    double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n), *p = calloc(n, sizeof(double));
    double *v = calloc(n, sizeof(double)), *s = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    double *ph = malloc(sizeof(double) * n), *sh = malloc(sizeof(double) * n);
    csr_matvec(n, rp, L, V, x, r);
    for (int i = 0; i < n; ++i) { r[i] = b[i] - r[i]; rh[i] = r[i]; }
    double bn = sqrt(dot(n, b, b)), rho = 1, alpha = 1, omega = 1;
    if (bn == 0.0) bn = 1.0;
    int it = 0, status = 1;
    double rn = sqrt(dot(n, r, r));
    if (rn <= rtol * bn) status = 0;
    while (status && it < maxit) {
        double rho1 = dot(n, rh, r);
        if (rho1 == 0.0) { status = -5; break; }
        double beta = (rho1 / rho) * (alpha / omega);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) { p[i] = r[i] + beta * (p[i] - omega * v[i]); ph[i] = D[i] * p[i]; }
        csr_matvec(n, rp, L, V, ph, v);
        double rv = dot(n, rh, v);
        if (rv == 0.0) { status = -5; break; }
        alpha = rho1 / rv;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) { s[i] = r[i] - alpha * v[i]; sh[i] = D[i] * s[i]; }
        csr_matvec(n, rp, L, V, sh, t);
        double tt = dot(n, t, t);
        omega = tt == 0.0 ? 0.0 : dot(n, t, s) / tt;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) { x[i] += alpha * ph[i] + omega * sh[i]; r[i] = s[i] - omega * t[i]; }
        rho = rho1;
        ++it;
        rn = sqrt(dot(n, r, r));
        if (rn <= rtol * bn) status = 0;
        else if (omega == 0.0) { status = -5; break; }
    }
    if (iters) *iters = it;
    if (relres) *relres = rn / bn;
    free(rp); free(D); free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Newton iteration (Sec. 4): u <- u - J(u)^{-1} r(u)                          */
/* ------------------------------------------------------------------------- */

/* method 0 = EGFEM Newton, 1 = SGA Newton, 2 = EGFEM Picard */
static int64_t jac(const orc_problem *P, int method, const double *u, int64_t cap, int64_t *I, int64_t *L, double *V) {
    if (method == 2) return orc_picard_matrix(P, u, cap, I, L, V);
    return method == 0 ? orc_egfem_jacobian(P, u, cap, I, L, V) : orc_sga_jacobian(P, u, cap, I, L, V);
}

static void res(const orc_problem *P, int method, const double *u, const double *b, const double *uD, int form, double *r) {
    if (method != 1) orc_egfem_residual(P, u, b, uD, form, r);
    else orc_sga_residual(P, u, b, uD, form, r);
}

static double norm_free(const orc_problem *P, const double *r) {
    double s = 0.0;
    for (int i = 0; i < P->s.nv; ++i) if (!P->s.dir[i]) s += r[i] * r[i];
    return sqrt(s);
}

/* method 0 = EGFEM Newton, 1 = SGA Newton, 2 = EGFEM Picard (u <- u - A(u)^{-1} r(u) with the
 * frozen-coefficient matrix A = T .2 a(u), i.e. A(u^n) u^{n+1} = b - gamma M c(u^n));
 * solver 0 = banded LU, 1 = BiCGStab(ktol).
 * Stops when ||r||_free <= rtol * ||r(u0)||_free.  hist (optional, maxit+1 doubles)
 * receives the residual norms; iterates (optional, (maxit+1)*nv) the iterates.
 * Returns the number of Newton steps, or a negative code. */
int orc_newton(const orc_problem *P, int method, int solver, const double *b, const double *uD, double *u,
               double rtol, int maxit, double ktol, int form, double *hist, double *iterates, int *krylov_total) {
    int nv = P->s.nv;
    double *r = malloc(sizeof(double) * nv), *d = malloc(sizeof(double) * nv);
    int64_t cap = 0, *I = NULL, *L = NULL; double *V = NULL;
    res(P, method, u, b, uD, form, r);
    double r0 = norm_free(P, r), rn = r0;
    if (hist) hist[0] = r0;
    if (iterates) memcpy(iterates, u, sizeof(double) * nv);
    int k = 0, status = 0, ktot = 0;
    while (rn > rtol * r0 && rn > 0.0) {
        if (k >= maxit) { status = -1; break; }
        int64_t nnz = jac(P, method, u, cap, I, L, V);
        if (nnz > cap) {
            cap = nnz; free(I); free(L); free(V);
            I = malloc(sizeof(int64_t) * cap); L = malloc(sizeof(int64_t) * cap); V = malloc(sizeof(double) * cap);
            nnz = jac(P, method, u, cap, I, L, V);
        }
        memcpy(d, r, sizeof(double) * nv);
        if (solver == 0) {
            int kl = 0, ku = 0;
            for (int64_t t = 0; t < nnz; ++t) { int64_t o = L[t] - I[t]; if (-o > kl) kl = (int)-o; if (o > ku) ku = (int)o; }
            if (orc_band_solve(nv, kl, ku, nnz, I, L, V, d) != 0) { status = -2; break; }
        } else {
            for (int i = 0; i < nv; ++i) d[i] = 0.0;
            int its = 0; double rr = 0;
            int st = orc_bicgstab(nv, nnz, I, L, V, r, d, ktol, 100000, &its, &rr);
            ktot += its;
            if (st != 0) { status = -3; break; }
        }
        for (int i = 0; i < nv; ++i) u[i] -= d[i];
        ++k;
        res(P, method, u, b, uD, form, r);
        rn = norm_free(P, r);
        if (hist) hist[k] = rn;
        if (iterates) memcpy(iterates + (size_t)k * nv, u, sizeof(double) * nv);
        if (!isfinite(rn)) { status = -4; break; }
    }
    if (krylov_total) *krylov_total = ktot;
    free(r); free(d); free(I); free(L); free(V);
    return status == 0 ? k : status;
}

/* ------------------------------------------------------------------------- */
/* Adjoint (implicit function theorem): J^T lambda = dJdu on free rows,         */
/* lambda = 0 on Dirichlet rows.  Gradients of the functional:                 */
/*   d/db_i = lambda_i,  d/dkappa_m = -sum_{i,k} lambda_i T_imk u_k               */
/* ------------------------------------------------------------------------- */

int orc_adjoint(const orc_problem *P, const double *u, const double *dJdu, int solver, double ktol,
                double *lambda, double *grad_kappa) {
    int nv = P->s.nv;
    int64_t nnz = orc_egfem_jacobian(P, u, 0, NULL, NULL, NULL);
    int64_t *I = malloc(sizeof(int64_t) * nnz), *L = malloc(sizeof(int64_t) * nnz);
    double *V = malloc(sizeof(double) * nnz);
    orc_egfem_jacobian(P, u, nnz, I, L, V);
    /* transpose: swap row and column, then re-sort */
    orc_coo Tt = {0};
    for (int64_t t = 0; t < nnz; ++t) coo_push(&Tt, L[t], I[t], 0, V[t]);
    coo_compress(&Tt);
    for (int64_t t = 0; t < nnz; ++t) { I[t] = Tt.t[t].i; L[t] = Tt.t[t].j; V[t] = Tt.t[t].v; }
    free(Tt.t);
    for (int i = 0; i < nv; ++i) lambda[i] = P->s.dir[i] ? 0.0 : dJdu[i];
    int st;
    if (solver == 0) {
        int kl = 0, ku = 0;
        for (int64_t t = 0; t < nnz; ++t) { int64_t o = L[t] - I[t]; if (-o > kl) kl = (int)-o; if (o > ku) ku = (int)o; }
        st = orc_band_solve(nv, kl, ku, nnz, I, L, V, lambda);
    } else {
        double *rhs = malloc(sizeof(double) * nv);
        memcpy(rhs, lambda, sizeof(double) * nv);
        for (int i = 0; i < nv; ++i) lambda[i] = 0.0;
        int its; double rr;
        st = orc_bicgstab(nv, nnz, I, L, V, rhs, lambda, ktol, 100000, &its, &rr);
        free(rhs);
    }
    if (grad_kappa) {
        for (int m = 0; m < P->Sa.n; ++m) grad_kappa[m] = 0.0;
        for (size_t t = 0; t < P->T.n; ++t)
            grad_kappa[P->T.t[t].j] -= lambda[P->T.t[t].i] * P->T.t[t].v * u[P->T.t[t].k];
    }
    free(I); free(L); free(V);
    return st;
}
