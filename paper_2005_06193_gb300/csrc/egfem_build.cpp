// egfem_build.cpp -- offline phase on the host: W-space numbering, element quantities,
// the row-segmented CSF image of the trilinear form and the Jacobian pattern.
//
// Trilinear form (Sec. 3.3 eq. (7), Example 4.1):  T_imk = int eta_m grad phi_k . grad phi_i.
// With P1 trial functions the gradients are constant on a cell K, so
//     T_imk = sum_{K} iota^K_m S^K_ik,   iota^K_m = int_K eta_m,   S^K_ik = |K| grad lambda_i . grad lambda_k,
// and iota^K_m / |K| depends only on the kind of the W node (vertex, edge, face), by the
// barycentric integral int_K lambda^alpha = |K| d! alpha! / (|alpha| + d)!.
// Reaction form (Sec. 3.3):  M^c_im = int eta_m phi_i; for W_c = P1 this is the P1 mass
// matrix |K| (1 + delta_im) / ((d+1)(d+2)) per cell.
//
// Because the P1 basis sums to one, sum_k grad phi_k = 0 on every cell and
// sum_k T_imk = 0 exactly.  The build stores only the off-diagonal leaves k != i and
// one diagonal value per fibre, T_imi := -sum_{k != i} T_imk, so the stored operator has
// exact zero row sums; the kernels then evaluate sum_k T_imk (u_k - u_i), which needs no
// diagonal leaf at all.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "egfem_internal.h"

namespace egfem {

double basis_integral(int dim, int degree, int kind) {
    // int_K eta_m / |K| for the Lagrange node kinds (derived from the barycentric
    // integral above; e.g. 2D P2 edge: 4 int lambda_i lambda_j / |K| = 4 * 2/24 = 1/3).
    const bool edge = (kind == W_MID || kind == W_THIRD);
    if (dim == 2) {
        if (degree == 1) return 1.0 / 3.0;
        if (degree == 2) return kind == W_VERTEX ? 0.0 : 1.0 / 3.0;
        if (degree == 3) return kind == W_VERTEX ? 1.0 / 30.0 : edge ? 3.0 / 40.0 : 9.0 / 20.0;
    } else {
        if (degree == 1) return 1.0 / 4.0;
        if (degree == 2) return kind == W_VERTEX ? -1.0 / 20.0 : 1.0 / 5.0;
        if (degree == 3) return kind == W_VERTEX ? 1.0 / 40.0 : edge ? 0.0 : 9.0 / 40.0;
    }
    return 0.0;
}

egfem_status validate_mesh(const egfem_mesh &m, std::string &err) {
    if (m.dim != 2 && m.dim != 3) { err = "mesh.dim must be 2 or 3"; return EGFEM_ERR_INVALID_ARG; }
    if (m.n_nodes <= 0 || m.n_cells <= 0 || !m.coords || !m.cells) { err = "empty mesh or null arrays"; return EGFEM_ERR_INVALID_ARG; }
    if (m.n_nodes >= (int64_t(1) << 31) - 1) { err = "n_nodes must fit in int32"; return EGFEM_ERR_INVALID_ARG; }
    const int nv = m.dim + 1;
    for (int64_t c = 0; c < m.n_cells; ++c) {
        const int32_t *cv = m.cells + c * nv;
        for (int a = 0; a < nv; ++a) {
            if (cv[a] < 0 || cv[a] >= m.n_nodes) { err = "cell " + std::to_string(c) + " has a vertex index out of range"; return EGFEM_ERR_MESH; }
            for (int b = 0; b < a; ++b)
                if (cv[a] == cv[b]) { err = "cell " + std::to_string(c) + " repeats a vertex"; return EGFEM_ERR_MESH; }
        }
        double B[9];
        for (int k = 0; k < m.dim; ++k)
            for (int r = 0; r < m.dim; ++r) B[r * m.dim + k] = m.coords[int64_t(cv[k + 1]) * m.dim + r] - m.coords[int64_t(cv[0]) * m.dim + r];
        double det = m.dim == 2 ? B[0] * B[3] - B[1] * B[2]
                                : B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) + B[2] * (B[3] * B[7] - B[4] * B[6]);
        if (!std::isfinite(det) || det == 0.0) { err = "cell " + std::to_string(c) + " has zero volume"; return EGFEM_ERR_MESH; }
    }
    return EGFEM_OK;
}

// Cell geometry: |K| and the barycentric gradients (rows of [-1 ... -1; I] B^{-1}).
static void cell_grads(const egfem_mesh &m, int64_t c, double &vol, double g[4][3]) {
    const int d = m.dim, nv = d + 1;
    const int32_t *cv = m.cells + c * nv;
    double B[9], Bi[9];
    for (int k = 0; k < d; ++k)
        for (int r = 0; r < d; ++r) B[r * d + k] = m.coords[int64_t(cv[k + 1]) * d + r] - m.coords[int64_t(cv[0]) * d + r];
    double det;
    if (d == 2) {
        det = B[0] * B[3] - B[1] * B[2];
        Bi[0] = B[3] / det; Bi[1] = -B[1] / det; Bi[2] = -B[2] / det; Bi[3] = B[0] / det;
        vol = std::fabs(det) / 2.0;
    } else {
        det = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) + B[2] * (B[3] * B[7] - B[4] * B[6]);
        Bi[0] = (B[4] * B[8] - B[5] * B[7]) / det; Bi[1] = (B[2] * B[7] - B[1] * B[8]) / det; Bi[2] = (B[1] * B[5] - B[2] * B[4]) / det;
        Bi[3] = (B[5] * B[6] - B[3] * B[8]) / det; Bi[4] = (B[0] * B[8] - B[2] * B[6]) / det; Bi[5] = (B[2] * B[3] - B[0] * B[5]) / det;
        Bi[6] = (B[3] * B[7] - B[4] * B[6]) / det; Bi[7] = (B[1] * B[6] - B[0] * B[7]) / det; Bi[8] = (B[0] * B[4] - B[1] * B[3]) / det;
        vol = std::fabs(det) / 6.0;
    }
    // lambda_j(x) = (B^{-1}(x - x0))_{j-1} for j >= 1: grad lambda_j = row j-1 of B^{-1}
    for (int j = 1; j <= d; ++j)
        for (int r = 0; r < d; ++r) g[j][r] = Bi[(j - 1) * d + r];
    for (int r = 0; r < d; ++r) { double s = 0; for (int j = 1; j <= d; ++j) s += g[j][r]; g[0][r] = -s; }
}

// Per cell |K| and, when S is given, S^K_ab = |K| grad lambda_a . grad lambda_b packed as
// the upper triangle row by row ((d+1)(d+2)/2 values): the P1 stiffness of the cell, which
// is also the trilinear form of a P0 W space, T_iKk = int_K grad phi_k . grad phi_i.
void cell_stiffness(const egfem_mesh &m, std::vector<double> &vol, std::vector<double> *S) {
    const int d = m.dim, nv = d + 1, ns = nv * (nv + 1) / 2;
    vol.assign(size_t(m.n_cells), 0.0);
    if (S) S->assign(size_t(m.n_cells) * ns, 0.0);
    for (int64_t c = 0; c < m.n_cells; ++c) {
        double g[4][3];
        cell_grads(m, c, vol[c], g);
        if (!S) continue;
        int q = 0;
        for (int a = 0; a < nv; ++a)
            for (int b = a; b < nv; ++b) {
                double t = 0;
                for (int r = 0; r < d; ++r) t += g[a][r] * g[b][r];
                (*S)[size_t(c) * ns + q++] = vol[c] * t;
            }
    }
}

// Symmetric quadrature rules of degree k for the quadrature spaces I_k (Sec. 3.1, Case 3):
// Dunavant's triangle rules (k = 1..4) and the tetrahedron rules of degree 1..3, as
// barycentric points with weights relative to the cell volume (summing to 1).  Writes at most
// 6 points into bary / w and returns their number, or 0 for a degree not tabulated.
int quad_rule(int dim, int k, double bary[][4], double *w) {
    int n = 0;
    auto add = [&](double l0, double l1, double l2, double l3, double wt) {
        bary[n][0] = l0; bary[n][1] = l1; bary[n][2] = l2; bary[n][3] = l3; w[n] = wt; ++n;
    };
    auto s21 = [&](double a, double wt) {            // the 3 permutations of (1 - 2a, a, a)
        const double b = 1.0 - 2.0 * a;
        add(b, a, a, 0, wt); add(a, b, a, 0, wt); add(a, a, b, 0, wt);
    };
    auto s31 = [&](double a, double wt) {            // the 4 permutations of (1 - 3a, a, a, a)
        const double b = 1.0 - 3.0 * a;
        add(b, a, a, a, wt); add(a, b, a, a, wt); add(a, a, b, a, wt); add(a, a, a, b, wt);
    };
    if (dim == 2) {
        switch (k) {
            case 1: add(1.0 / 3, 1.0 / 3, 1.0 / 3, 0, 1.0); break;
            case 2: s21(1.0 / 6, 1.0 / 3); break;
            case 3: add(1.0 / 3, 1.0 / 3, 1.0 / 3, 0, -0.5625); s21(0.2, 0.5208333333333333); break;
            case 4: s21(0.445948490915965, 0.223381589678011); s21(0.091576213509771, 0.109951743655322); break;
            default: return 0;
        }
    } else {
        switch (k) {
            case 1: add(0.25, 0.25, 0.25, 0.25, 1.0); break;
            case 2: s31(0.1381966011250105, 0.25); break;
            case 3: add(0.25, 0.25, 0.25, 0.25, -0.8); s31(1.0 / 6, 0.45); break;
            default: return 0;
        }
    }
    return n;
}

// The nodes of I_k: rule point l of cell c is node c * nq + l ([n_cells * nq * dim]).
std::vector<double> quad_points(const egfem_mesh &m, int nq, const double bary[][4]) {
    const int d = m.dim, nv = d + 1;
    std::vector<double> x(size_t(m.n_cells) * nq * d, 0.0);
    for (int64_t c = 0; c < m.n_cells; ++c)
        for (int l = 0; l < nq; ++l)
            for (int a = 0; a < nv; ++a)
                for (int r = 0; r < d; ++r)
                    x[(size_t(c) * nq + l) * d + r] += bary[l][a] * m.coords[int64_t(m.cells[c * nv + a]) * d + r];
    return x;
}

// The nodes of a P0 space: one per cell, at its centroid ([n_cells * dim]).
std::vector<double> cell_centroids(const egfem_mesh &m) {
    const int d = m.dim, nv = d + 1;
    std::vector<double> x(size_t(m.n_cells) * d, 0.0);
    for (int64_t c = 0; c < m.n_cells; ++c)
        for (int a = 0; a < nv; ++a)
            for (int r = 0; r < d; ++r) x[size_t(c) * d + r] += m.coords[int64_t(m.cells[c * nv + a]) * d + r] / double(nv);
    return x;
}

// ---------------------------------------------------------------------------------
// W space: vertices keep their P1 index; edge nodes follow (degree-1 per edge, ordered
// from the lower to the higher global vertex); for degree 3, face centroids last.
// Local order on a cell: vertices, then edges (a,b), a<b lexicographic, each edge's
// nodes from local a to local b, then faces (a,b,c) lexicographic.
// ---------------------------------------------------------------------------------

static inline uint64_t pair_key(uint32_t a, uint32_t b) { return a < b ? (uint64_t(a) << 32) | b : (uint64_t(b) << 32) | a; }

egfem_status build_wspace(const egfem_mesh &m, int p, HostWSpace &W, std::vector<int32_t> &cell2w, int &nloc,
                          std::string &err) {
    const int d = m.dim, nv = d + 1;
    if (p < 1 || p > 3) { err = "W degree must be 1, 2 or 3"; return EGFEM_ERR_INVALID_ARG; }
    const int ned = nv * (nv - 1) / 2;
    const int nfa = (d == 2) ? 1 : 4;
    nloc = nv + ned * (p - 1) + (p == 3 ? nfa : 0);
    W.degree = p;
    // unique edges
    std::vector<uint64_t> ekeys;
    if (p >= 2) {
        ekeys.reserve(size_t(m.n_cells) * ned);
        for (int64_t c = 0; c < m.n_cells; ++c) {
            const int32_t *cv = m.cells + c * nv;
            for (int a = 0; a < nv; ++a)
                for (int b = a + 1; b < nv; ++b) ekeys.push_back(pair_key(cv[a], cv[b]));
        }
        std::sort(ekeys.begin(), ekeys.end());
        ekeys.erase(std::unique(ekeys.begin(), ekeys.end()), ekeys.end());
    }
    // unique faces (3D, p = 3): sorted vertex triples
    struct Tri { int32_t v[3]; bool operator<(const Tri &o) const { return std::lexicographical_compare(v, v + 3, o.v, o.v + 3); }
                 bool operator==(const Tri &o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; } };
    std::vector<Tri> faces;
    if (p == 3 && d == 3) {
        faces.reserve(size_t(m.n_cells) * 4);
        for (int64_t c = 0; c < m.n_cells; ++c) {
            const int32_t *cv = m.cells + c * nv;
            for (int a = 0; a < 4; ++a) for (int b = a + 1; b < 4; ++b) for (int e = b + 1; e < 4; ++e) {
                Tri t{{cv[a], cv[b], cv[e]}}; std::sort(t.v, t.v + 3); faces.push_back(t);
            }
        }
        std::sort(faces.begin(), faces.end());
        faces.erase(std::unique(faces.begin(), faces.end()), faces.end());
    }
    const int64_t NV = m.n_nodes, NE = int64_t(ekeys.size());
    const int64_t NF = (p == 3) ? (d == 2 ? m.n_cells : int64_t(faces.size())) : 0;
    W.n = NV + NE * (p - 1) + NF;
    if (W.n >= (int64_t(1) << 31) - 1) { err = "W space too large for int32 indices"; return EGFEM_ERR_INVALID_ARG; }
    W.kind.assign(W.n, W_VERTEX);
    W.sup.assign(size_t(W.n) * 3, -1);
    W.coords.assign(size_t(W.n) * d, 0.0);
    for (int64_t v = 0; v < NV; ++v) {
        W.sup[3 * v] = int32_t(v);
        for (int r = 0; r < d; ++r) W.coords[v * d + r] = m.coords[v * d + r];
    }
    for (int64_t e = 0; e < NE; ++e) {
        const int32_t lo = int32_t(ekeys[e] >> 32), hi = int32_t(ekeys[e] & 0xFFFFFFFFu);
        for (int t = 0; t < p - 1; ++t) {
            int64_t w = NV + e * (p - 1) + t;
            double wl, wh;
            if (p == 2) { W.kind[w] = W_MID; W.sup[3 * w] = lo; W.sup[3 * w + 1] = hi; wl = wh = 0.5; }
            else if (t == 0) { W.kind[w] = W_THIRD; W.sup[3 * w] = lo; W.sup[3 * w + 1] = hi; wl = 2.0 / 3.0; wh = 1.0 / 3.0; }
            else { W.kind[w] = W_THIRD; W.sup[3 * w] = hi; W.sup[3 * w + 1] = lo; wl = 1.0 / 3.0; wh = 2.0 / 3.0; }
            for (int r = 0; r < d; ++r) W.coords[w * d + r] = wl * m.coords[int64_t(lo) * d + r] + wh * m.coords[int64_t(hi) * d + r];
        }
    }
    auto edge_id = [&](int32_t a, int32_t b) -> int64_t {
        uint64_t k = pair_key(a, b);
        return int64_t(std::lower_bound(ekeys.begin(), ekeys.end(), k) - ekeys.begin());
    };
    auto face_node = [&](int64_t f, const int32_t *v3) {
        int64_t w = NV + NE * (p - 1) + f;
        W.kind[w] = W_FACE;
        int32_t s[3] = {v3[0], v3[1], v3[2]}; std::sort(s, s + 3);
        for (int t = 0; t < 3; ++t) W.sup[3 * w + t] = s[t];
        for (int r = 0; r < d; ++r) {
            double x = 0; for (int t = 0; t < 3; ++t) x += m.coords[int64_t(s[t]) * d + r];
            W.coords[w * d + r] = x / 3.0;
        }
        return w;
    };
    cell2w.assign(size_t(m.n_cells) * nloc, -1);
    for (int64_t c = 0; c < m.n_cells; ++c) {
        const int32_t *cv = m.cells + c * nv;
        int32_t *out = &cell2w[size_t(c) * nloc];
        int l = 0;
        for (int a = 0; a < nv; ++a) out[l++] = cv[a];
        for (int a = 0; a < nv && p >= 2; ++a)
            for (int b = a + 1; b < nv; ++b) {
                int64_t e = edge_id(cv[a], cv[b]);
                if (p == 2) out[l++] = int32_t(NV + e);
                else {
                    // node nearer local a first
                    const bool a_is_lo = cv[a] < cv[b];
                    out[l++] = int32_t(NV + 2 * e + (a_is_lo ? 0 : 1));
                    out[l++] = int32_t(NV + 2 * e + (a_is_lo ? 1 : 0));
                }
            }
        if (p == 3) {
            if (d == 2) out[l++] = int32_t(face_node(c, cv));
            else
                for (int a = 0; a < 4; ++a) for (int b = a + 1; b < 4; ++b) for (int e = b + 1; e < 4; ++e) {
                    Tri t{{cv[a], cv[b], cv[e]}}; std::sort(t.v, t.v + 3);
                    int64_t f = int64_t(std::lower_bound(faces.begin(), faces.end(), t) - faces.begin());
                    out[l++] = int32_t(face_node(f, t.v));
                }
        }
    }
    return EGFEM_OK;
}

// ---------------------------------------------------------------------------------
// CSF assembly, one row (P1 test function) at a time.
// ---------------------------------------------------------------------------------

namespace {

struct RowOut {
    bool dir = false;
    std::vector<int32_t> cols;       // global, self first, then ascending
    std::vector<uint8_t> leafc;
    std::vector<double> leafv;
    std::vector<uint32_t> finfo;
    std::vector<double> ftd;
    std::vector<int32_t> fm;
    std::vector<double> rxv;
    std::vector<uint32_t> rxi;
    std::vector<int32_t> rxm;
    std::vector<int32_t> jrank;      // per local column: rank among free columns in CSR order, -1 if none
    int32_t jnnz = 0;
};

struct Ctx {
    const egfem_mesh *m;
    const egfem_problem *prob;
    const HostWSpace *Wa, *Wc;
    const std::vector<int32_t> *c2wa, *c2wc;
    int nla, nlc;
    std::vector<int64_t> v2c_ptr;
    std::vector<int32_t> v2c;
};

struct Contrib { int32_t m; int32_t k; double v; };

int local_col(const std::vector<int32_t> &cols, int32_t g) {
    for (size_t c = 0; c < cols.size(); ++c) if (cols[c] == g) return int(c);
    return -1;
}

uint32_t info_for(const HostWSpace &W, int32_t w, const std::vector<int32_t> &cols) {
    const uint32_t kind = W.kind[w];
    uint32_t c[3] = {0, 0, 0};
    int nsup = kind == W_VERTEX ? 1 : kind == W_FACE ? 3 : 2;
    for (int t = 0; t < nsup; ++t) c[t] = uint32_t(local_col(cols, W.sup[3 * size_t(w) + t]));
    return pack_info(kind, c[0], c[1], c[2]);
}

void assemble_row(const Ctx &X, int64_t i, RowOut &R) {
    const egfem_mesh &m = *X.m;
    const int d = m.dim, nv = d + 1;
    R = RowOut();
    R.dir = m.dirichlet && m.dirichlet[i];
    // local columns: all vertices of the cells containing i; self first
    std::vector<int32_t> others;
    for (int64_t t = X.v2c_ptr[i]; t < X.v2c_ptr[i + 1]; ++t) {
        const int32_t *cv = m.cells + int64_t(X.v2c[t]) * nv;
        for (int a = 0; a < nv; ++a) if (cv[a] != i) others.push_back(cv[a]);
    }
    std::sort(others.begin(), others.end());
    others.erase(std::unique(others.begin(), others.end()), others.end());
    if (R.dir) {
        R.cols.assign(1, int32_t(i));
        R.jrank.assign(1, 0);
        R.jnnz = 1;
        return;
    }
    R.cols.reserve(others.size() + 1);
    R.cols.push_back(int32_t(i));
    for (int32_t o : others) R.cols.push_back(o);
    // CSR order: free columns sorted by global index
    {
        std::vector<std::pair<int32_t, int>> fc;
        for (size_t c = 0; c < R.cols.size(); ++c)
            if (!(m.dirichlet && m.dirichlet[R.cols[c]])) fc.push_back({R.cols[c], int(c)});
        std::sort(fc.begin(), fc.end());
        R.jrank.assign(R.cols.size(), -1);
        for (size_t r = 0; r < fc.size(); ++r) R.jrank[fc[r].second] = int32_t(r);
        R.jnnz = int32_t(fc.size());
    }
    const egfem_problem &P = *X.prob;
    std::vector<Contrib> acc;
    std::vector<std::pair<int32_t, double>> rx;
    for (int64_t t = X.v2c_ptr[i]; t < X.v2c_ptr[i + 1]; ++t) {
        const int64_t c = X.v2c[t];
        const int32_t *cv = m.cells + c * nv;
        int a = 0;
        while (cv[a] != i) ++a;
        double vol, g[4][3];
        cell_grads(m, c, vol, g);
        double S[4];
        for (int b = 0; b < nv; ++b) {
            double s = 0; for (int r = 0; r < d; ++r) s += g[a][r] * g[b][r];
            S[b] = vol * s;
        }
        if (P.a_kind == EGFEM_G_NONE) {
            for (int b = 0; b < nv; ++b) if (b != a) acc.push_back({-1, cv[b], S[b]});
        } else {
            const int32_t *wl = &(*X.c2wa)[size_t(c) * X.nla];
            for (int l = 0; l < X.nla; ++l) {
                const double iota = basis_integral(d, X.Wa->degree, X.Wa->kind[wl[l]]);
                if (iota == 0.0) continue;
                for (int b = 0; b < nv; ++b) if (b != a) acc.push_back({wl[l], cv[b], iota * S[b]});
            }
        }
        if (P.c_kind != EGFEM_G_NONE) {
            // W_c = P1: M^K_{a,b} = |K| (1 + delta_ab) / ((d+1)(d+2))
            const int32_t *wl = &(*X.c2wc)[size_t(c) * X.nlc];
            for (int b = 0; b < nv; ++b) rx.push_back({wl[b], vol * (a == b ? 2.0 : 1.0) / double((d + 1) * (d + 2))});
        }
    }
    // sum duplicates, ordered by (m, k)
    std::sort(acc.begin(), acc.end(), [](const Contrib &x, const Contrib &y) { return x.m != y.m ? x.m < y.m : x.k < y.k; });
    std::vector<Contrib> T;
    for (const Contrib &e : acc) {
        if (!T.empty() && T.back().m == e.m && T.back().k == e.k) T.back().v += e.v;
        else T.push_back(e);
    }
    // drop leaves that are zero up to rounding (e.g. grad lambda_i . grad lambda_k = 0 on
    // right angles): |T| <= 1e-14 max |T| of the row
    double tmax = 0; for (const Contrib &e : T) tmax = std::max(tmax, std::fabs(e.v));
    const double cut = 1e-14 * tmax;
    size_t s = 0;
    while (s < T.size()) {
        size_t e = s;
        while (e < T.size() && T[e].m == T[s].m) ++e;
        double sum = 0; bool first = true;
        for (size_t q = s; q < e; ++q) {
            if (std::fabs(T[q].v) <= cut) continue;
            uint8_t lc = uint8_t(local_col(R.cols, T[q].k));
            R.leafc.push_back(uint8_t(lc | (first ? LEAF_FIBRE_START : 0)));
            R.leafv.push_back(T[q].v);
            sum += T[q].v;
            first = false;
        }
        if (!first) {
            R.ftd.push_back(-sum);
            R.fm.push_back(T[s].m < 0 ? 0 : T[s].m);
            R.finfo.push_back(T[s].m < 0 ? pack_info(W_CONST, 0, 0, 0) : info_for(*X.Wa, T[s].m, R.cols));
        }
        s = e;
    }
    if (!rx.empty()) {
        std::sort(rx.begin(), rx.end());
        for (size_t q = 0; q < rx.size(); ++q) {
            if (!R.rxm.empty() && R.rxm.back() == rx[q].first) { R.rxv.back() += rx[q].second; continue; }
            R.rxm.push_back(rx[q].first);
            R.rxv.push_back(rx[q].second);
            R.rxi.push_back(info_for(*X.Wc, rx[q].first, R.cols));
        }
    }
}

struct Chunk {
    std::vector<SliceMeta> meta;   // bases relative to the chunk
    std::vector<int32_t> col_idx, col_slot;  // col_slot holds the CSR rank until fixed up
    std::vector<double> leaf_val, fib_tdiag, rx_val;
    std::vector<uint8_t> leaf_col, dir;
    std::vector<uint32_t> fib_info, rx_info;
    std::vector<int32_t> fib_m, rx_m, jnnz;
    int32_t max_cols = 0;
    std::string err;
};

}  // namespace

egfem_status build_csf(const egfem_mesh &m, const egfem_problem &prob, const HostWSpace &Wa,
                       const std::vector<int32_t> &cell2wa, int nloc_a, const HostWSpace &Wc,
                       const std::vector<int32_t> &cell2wc, int nloc_c, HostCSF &out, std::string &err) {
    const int nv = m.dim + 1;
    Ctx X;
    X.m = &m; X.prob = &prob; X.Wa = &Wa; X.Wc = &Wc; X.c2wa = &cell2wa; X.c2wc = &cell2wc; X.nla = nloc_a; X.nlc = nloc_c;
    // vertex -> cell incidence
    X.v2c_ptr.assign(m.n_nodes + 1, 0);
    for (int64_t c = 0; c < m.n_cells; ++c) for (int a = 0; a < nv; ++a) X.v2c_ptr[m.cells[c * nv + a] + 1]++;
    for (int64_t v = 0; v < m.n_nodes; ++v) X.v2c_ptr[v + 1] += X.v2c_ptr[v];
    X.v2c.assign(X.v2c_ptr[m.n_nodes], 0);
    {
        std::vector<int64_t> fill(X.v2c_ptr.begin(), X.v2c_ptr.end() - 1);
        for (int64_t c = 0; c < m.n_cells; ++c) for (int a = 0; a < nv; ++a) X.v2c[fill[m.cells[c * nv + a]]++] = int32_t(c);
    }
    const int64_t n = m.n_nodes;
    const int32_t nslices = int32_t((n + SLICE - 1) / SLICE);
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const int32_t per = (nslices + int32_t(nth) - 1) / int32_t(nth);
    std::vector<Chunk> chunks(nth);
    auto work = [&](unsigned t) {
        Chunk &C = chunks[t];
        const int32_t s0 = int32_t(t) * per, s1 = std::min(nslices, s0 + per);
        RowOut rows[SLICE];
        for (int32_t s = s0; s < s1; ++s) {
            SliceMeta M{};
            M.off_base = -1;
            M.col_base = int64_t(C.col_idx.size()); M.leaf_base = int64_t(C.leaf_val.size());
            M.fib_base = int64_t(C.fib_info.size()); M.rx_base = int64_t(C.rx_val.size());
            for (int r = 0; r < SLICE; ++r) {
                const int64_t i = int64_t(s) * SLICE + r;
                if (i < n) assemble_row(X, i, rows[r]); else rows[r] = RowOut();
                M.ncol = std::max<int32_t>(M.ncol, int32_t(rows[r].cols.size()));
                M.nleaf = std::max<int32_t>(M.nleaf, int32_t(rows[r].leafv.size()));
                M.nfib = std::max<int32_t>(M.nfib, int32_t(rows[r].ftd.size()));
                M.nrx = std::max<int32_t>(M.nrx, int32_t(rows[r].rxv.size()));
            }
            if (M.ncol > 63) { C.err = "a vertex has more than 62 neighbours"; return; }
            C.max_cols = std::max(C.max_cols, M.ncol);
            for (int j = 0; j < M.ncol; ++j)
                for (int r = 0; r < SLICE; ++r) {
                    const int64_t i = int64_t(s) * SLICE + r;
                    const bool has = j < int(rows[r].cols.size());
                    C.col_idx.push_back(has ? rows[r].cols[j] : int32_t(i < n ? i : 0));
                    C.col_slot.push_back(has ? rows[r].jrank[j] : -1);
                }
            for (int j = 0; j < M.nleaf; ++j)
                for (int r = 0; r < SLICE; ++r) {
                    const bool has = j < int(rows[r].leafv.size());
                    C.leaf_val.push_back(has ? rows[r].leafv[j] : 0.0);
                    C.leaf_col.push_back(has ? rows[r].leafc[j] : LEAF_PAD);
                }
            for (int j = 0; j < M.nfib; ++j)
                for (int r = 0; r < SLICE; ++r) {
                    const bool has = j < int(rows[r].ftd.size());
                    C.fib_info.push_back(has ? rows[r].finfo[j] : pack_info(W_CONST, 0, 0, 0));
                    C.fib_tdiag.push_back(has ? rows[r].ftd[j] : 0.0);
                    C.fib_m.push_back(has ? rows[r].fm[j] : 0);
                }
            for (int j = 0; j < M.nrx; ++j)
                for (int r = 0; r < SLICE; ++r) {
                    const bool has = j < int(rows[r].rxv.size());
                    C.rx_val.push_back(has ? rows[r].rxv[j] : 0.0);
                    C.rx_info.push_back(has ? rows[r].rxi[j] : pack_info(W_CONST, 0, 0, 0));
                    C.rx_m.push_back(has ? rows[r].rxm[j] : 0);
                }
            for (int r = 0; r < SLICE; ++r) {
                const int64_t i = int64_t(s) * SLICE + r;
                if (i < n) { C.dir.push_back(rows[r].dir ? 1 : 0); C.jnnz.push_back(rows[r].jnnz); }
            }
            C.meta.push_back(M);
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nth; ++t) th.emplace_back(work, t);
    for (auto &x : th) x.join();
    for (auto &C : chunks) if (!C.err.empty()) { err = C.err; return EGFEM_ERR_MESH; }
    // concatenate
    out = HostCSF();
    out.n_rows = n; out.n_slices = nslices;
    out.rowptr.assign(n + 1, 0);
    int64_t row = 0;
    for (auto &C : chunks) {
        const int64_t cb = int64_t(out.col_idx.size()), lb = int64_t(out.leaf_val.size());
        const int64_t fb = int64_t(out.fib_info.size()), rb = int64_t(out.rx_val.size());
        for (SliceMeta M : C.meta) { M.col_base += cb; M.leaf_base += lb; M.fib_base += fb; M.rx_base += rb; out.meta.push_back(M); }
        out.col_idx.insert(out.col_idx.end(), C.col_idx.begin(), C.col_idx.end());
        out.col_slot.insert(out.col_slot.end(), C.col_slot.begin(), C.col_slot.end());
        out.leaf_val.insert(out.leaf_val.end(), C.leaf_val.begin(), C.leaf_val.end());
        out.leaf_col.insert(out.leaf_col.end(), C.leaf_col.begin(), C.leaf_col.end());
        out.fib_info.insert(out.fib_info.end(), C.fib_info.begin(), C.fib_info.end());
        out.fib_tdiag.insert(out.fib_tdiag.end(), C.fib_tdiag.begin(), C.fib_tdiag.end());
        out.fib_m.insert(out.fib_m.end(), C.fib_m.begin(), C.fib_m.end());
        out.rx_val.insert(out.rx_val.end(), C.rx_val.begin(), C.rx_val.end());
        out.rx_info.insert(out.rx_info.end(), C.rx_info.begin(), C.rx_info.end());
        out.rx_m.insert(out.rx_m.end(), C.rx_m.begin(), C.rx_m.end());
        out.dir.insert(out.dir.end(), C.dir.begin(), C.dir.end());
        for (int32_t k : C.jnnz) { out.rowptr[row + 1] = out.rowptr[row] + k; ++row; }
        out.max_cols = std::max(out.max_cols, C.max_cols);
        C = Chunk();
    }
    if (int64_t(out.rowptr[n]) >= (int64_t(1) << 31) - 1) { err = "Jacobian too large for int32 indices"; return EGFEM_ERR_INVALID_ARG; }
    // uniform slices: every row of the slice sees its local columns at the same offsets
    // (structured meshes away from the boundary), so the solver can form the column index
    // as row + offset and skip reading col_idx
    for (int32_t s = 0; s < nslices; ++s) {
        SliceMeta &M = out.meta[s];
        if (int64_t(s + 1) * SLICE > n) continue;
        bool uni = true;
        for (int j = 0; j < M.ncol && uni; ++j) {
            const int64_t q0 = M.col_base + int64_t(j) * SLICE;
            const int64_t o = int64_t(out.col_idx[q0]) - int64_t(s) * SLICE;
            for (int r = 1; r < SLICE && uni; ++r) uni = int64_t(out.col_idx[q0 + r]) - (int64_t(s) * SLICE + r) == o;
        }
        if (!uni) continue;
        M.off_base = int64_t(out.slice_off.size());
        for (int j = 0; j < M.ncol; ++j) out.slice_off.push_back(int32_t(out.col_idx[M.col_base + int64_t(j) * SLICE] - int64_t(s) * SLICE));
    }
    // CSR slots and column indices
    out.cols.assign(out.rowptr[n], 0);
    for (int32_t s = 0; s < nslices; ++s) {
        const SliceMeta &M = out.meta[s];
        for (int j = 0; j < M.ncol; ++j)
            for (int r = 0; r < SLICE; ++r) {
                const int64_t i = int64_t(s) * SLICE + r;
                const int64_t q = M.col_base + int64_t(j) * SLICE + r;
                if (i >= n || out.col_slot[q] < 0) { out.col_slot[q] = -1; continue; }
                out.col_slot[q] += out.rowptr[i];
                out.cols[out.col_slot[q]] = out.col_idx[q];
            }
    }
    return EGFEM_OK;
}

// A batch of k copies of one mesh (instance b owns the rows [b rows, (b + 1) rows), rows a
// whole number of slices): when the slices of every instance hold instance 0's tensor entries,
// with W indices that differ from instance 0's by b times one stride per node kind and space,
// keep instance 0's leaves, fibres and reaction entries only, point every instance's slices at
// them and return the strides in ws.  Otherwise return false and leave H as it was.  Local
// columns, the Jacobian pattern and the per-row arrays stay per instance.
bool share_tensor(HostCSF &H, int32_t k, int64_t rows, WShare &ws) {
    if (k < 2 || rows <= 0 || rows % SLICE != 0 || H.n_rows != rows * k) return false;
    const int64_t s0 = rows / SLICE;
    int64_t sa[5] = {0, 0, 0, 0, 0}, sc[5] = {0, 0, 0, 0, 0};
    bool ka[5] = {}, kc[5] = {};
    // instance b's W index m against instance 0's m0 for a node of kind w: m - m0 = b stride[w]
    auto stride_ok = [](int64_t *st, bool *known, uint32_t w, int64_t m, int64_t m0, int64_t b) {
        if (w == W_CONST) return true;   // no W node (padding): its index is never read
        const int64_t dm = m - m0;
        if (!known[w]) {
            if (dm % b != 0 || dm < 0) return false;
            st[w] = dm / b;
            known[w] = true;
        }
        return dm == b * st[w];
    };
    for (int64_t b = 1; b < k; ++b)
        for (int64_t l = 0; l < s0; ++l) {
            const SliceMeta &M = H.meta[size_t(b * s0 + l)], &M0 = H.meta[size_t(l)];
            if (M.ncol != M0.ncol || M.nleaf != M0.nleaf || M.nfib != M0.nfib || M.nrx != M0.nrx) return false;
            const size_t nl = size_t(M.nleaf) * SLICE, nf = size_t(M.nfib) * SLICE, nr = size_t(M.nrx) * SLICE;
            if (std::memcmp(H.leaf_val.data() + M.leaf_base, H.leaf_val.data() + M0.leaf_base, nl * sizeof(double)) != 0 ||
                std::memcmp(H.leaf_col.data() + M.leaf_base, H.leaf_col.data() + M0.leaf_base, nl) != 0 ||
                std::memcmp(H.fib_info.data() + M.fib_base, H.fib_info.data() + M0.fib_base, nf * sizeof(uint32_t)) != 0 ||
                std::memcmp(H.fib_tdiag.data() + M.fib_base, H.fib_tdiag.data() + M0.fib_base, nf * sizeof(double)) != 0 ||
                std::memcmp(H.rx_val.data() + M.rx_base, H.rx_val.data() + M0.rx_base, nr * sizeof(double)) != 0 ||
                std::memcmp(H.rx_info.data() + M.rx_base, H.rx_info.data() + M0.rx_base, nr * sizeof(uint32_t)) != 0)
                return false;
            for (size_t q = 0; q < nf; ++q)
                if (!stride_ok(sa, ka, (H.fib_info[M.fib_base + q] >> 24) & 0xF, H.fib_m[M.fib_base + q],
                               H.fib_m[M0.fib_base + q], b))
                    return false;
            for (size_t q = 0; q < nr; ++q)
                if (!stride_ok(sc, kc, (H.rx_info[M.rx_base + q] >> 24) & 0xF, H.rx_m[M.rx_base + q], H.rx_m[M0.rx_base + q], b))
                    return false;
        }
    // instance 0's entries come first (slices are stored in row order)
    const SliceMeta E = H.meta[size_t(s0)];
    H.leaf_val.resize(size_t(E.leaf_base)); H.leaf_col.resize(size_t(E.leaf_base));
    H.fib_info.resize(size_t(E.fib_base)); H.fib_tdiag.resize(size_t(E.fib_base)); H.fib_m.resize(size_t(E.fib_base));
    H.rx_val.resize(size_t(E.rx_base)); H.rx_info.resize(size_t(E.rx_base)); H.rx_m.resize(size_t(E.rx_base));
    H.leaf_val.shrink_to_fit(); H.leaf_col.shrink_to_fit(); H.fib_info.shrink_to_fit(); H.fib_tdiag.shrink_to_fit();
    H.fib_m.shrink_to_fit(); H.rx_val.shrink_to_fit(); H.rx_info.shrink_to_fit(); H.rx_m.shrink_to_fit();
    for (size_t s = size_t(s0); s < H.meta.size(); ++s) {
        const SliceMeta &M0 = H.meta[s % size_t(s0)];
        H.meta[s].leaf_base = M0.leaf_base;
        H.meta[s].fib_base = M0.fib_base;
        H.meta[s].rx_base = M0.rx_base;
    }
    ws = WShare{};
    ws.k = k;
    ws.rows = rows;
    for (int w = 0; w < 5; ++w) { ws.a[w] = sa[w]; ws.c[w] = sc[w]; }
    return true;
}

}  // namespace egfem

// Host-only reconstruction of the stored tensor (see egfem_inspect_tensor in egfem.h).
extern "C" egfem_status egfem_inspect_tensor(const egfem_mesh *mesh, const egfem_problem *prob, int64_t *count,
                                             int64_t *I, int64_t *M, int64_t *K, double *V, int64_t *n_wa,
                                             double *wa_coords) {
    using namespace egfem;
    if (!mesh || !prob || !count) return EGFEM_ERR_INVALID_ARG;
    std::string err;
    egfem_status st = validate_mesh(*mesh, err);
    if (st != EGFEM_OK) return st;
    const bool quad = prob->a_space == EGFEM_W_QUADRATURE;
    if (prob->a_kind == EGFEM_G_GRADPOW || quad) {
        // W_a = P0 or I_k: the form is T_ilk = (w_l / |K|) S^K_ik on the cell K of node l
        // (w_l / |K| = 1 for P0), which the element-local operator reads per cell (no CSF is
        // stored for it); free rows i only, as for the stored tensor
        double bary[6][4], wl[6];
        int nq = 1;
        wl[0] = 1.0;
        if (quad) {
            nq = quad_rule(mesh->dim, prob->a_degree, bary, wl);
            if (nq == 0) return EGFEM_ERR_INVALID_ARG;
        } else if (prob->a_degree != 0) {
            return EGFEM_ERR_INVALID_ARG;
        }
        const int nv = mesh->dim + 1, ns = nv * (nv + 1) / 2;
        std::vector<double> vol, S;
        cell_stiffness(*mesh, vol, &S);
        int64_t cnt = 0;
        for (int64_t c = 0; c < mesh->n_cells; ++c)
            for (int a = 0; a < nv; ++a) {
                const int32_t i = mesh->cells[c * nv + a];
                if (mesh->dirichlet && mesh->dirichlet[i]) continue;
                for (int l = 0; l < nq; ++l)
                    for (int b = 0; b < nv; ++b) {
                        const int lo = std::min(a, b), hi = std::max(a, b);
                        if (I) {
                            I[cnt] = i; M[cnt] = c * nq + l; K[cnt] = mesh->cells[c * nv + b];
                            V[cnt] = wl[l] * S[size_t(c) * ns + lo * nv - (lo * (lo - 1)) / 2 + (hi - lo)];
                        }
                        ++cnt;
                    }
            }
        *count = cnt;
        if (n_wa) *n_wa = mesh->n_cells * nq;
        if (wa_coords) {
            const std::vector<double> x = quad ? quad_points(*mesh, nq, bary) : cell_centroids(*mesh);
            std::memcpy(wa_coords, x.data(), x.size() * sizeof(double));
        }
        return EGFEM_OK;
    }
    HostWSpace Wa, Wc;
    std::vector<int32_t> c2wa, c2wc;
    int nla = 0, nlc = 0;
    st = build_wspace(*mesh, prob->a_kind != EGFEM_G_NONE ? prob->a_degree : 1, Wa, c2wa, nla, err);
    if (st != EGFEM_OK) return st;
    st = build_wspace(*mesh, 1, Wc, c2wc, nlc, err);
    if (st != EGFEM_OK) return st;
    HostCSF H;
    st = build_csf(*mesh, *prob, Wa, c2wa, nla, Wc, c2wc, nlc, H, err);
    if (st != EGFEM_OK) return st;
    int64_t cnt = 0;
    for (int32_t s = 0; s < H.n_slices; ++s) {
        const SliceMeta &Ms = H.meta[s];
        for (int r = 0; r < SLICE; ++r) {
            const int64_t i = int64_t(s) * SLICE + r;
            if (i >= H.n_rows) break;
            int f = -1;
            int32_t m = 0;
            for (int j = 0; j < Ms.nleaf; ++j) {
                const int64_t q = Ms.leaf_base + int64_t(j) * SLICE + r;
                const uint8_t lc = H.leaf_col[q];
                if (lc & LEAF_FIBRE_START) {
                    ++f;
                    const int64_t fq = Ms.fib_base + int64_t(f) * SLICE + r;
                    m = ((H.fib_info[fq] >> 24) & 0xF) == W_CONST ? -1 : H.fib_m[fq];
                    if (I) { I[cnt] = i; M[cnt] = m; K[cnt] = i; V[cnt] = H.fib_tdiag[fq]; }
                    ++cnt;
                }
                const int c = lc & LEAF_PAD;
                if (c == LEAF_PAD) continue;
                if (I) { I[cnt] = i; M[cnt] = m; K[cnt] = H.col_idx[Ms.col_base + int64_t(c) * SLICE + r]; V[cnt] = H.leaf_val[q]; }
                ++cnt;
            }
        }
    }
    *count = cnt;
    if (n_wa) *n_wa = Wa.n;
    if (wa_coords) std::memcpy(wa_coords, Wa.coords.data(), Wa.coords.size() * sizeof(double));
    return EGFEM_OK;
}

