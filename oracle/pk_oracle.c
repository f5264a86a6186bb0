/* pk_oracle.c -- plain, slow, FP64 CPU oracle of the auxiliary-space preconditioned
 * conjugate gradient method for P_k Lagrange discretisations of -div(kappa grad u) = f
 * on tetrahedral meshes (Lee, Leng & Zhang, "A Scalable Auxiliary Space Preconditioner
 * for High-Order Finite Element Methods", 2012).
 *
 * TEST INFRASTRUCTURE ONLY: this library exists to check the CUDA library. Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Each routine names the passage of the paper it follows. Equations are numbered
 * consecutively through the paper: Eq. (1) is the Poisson problem, Eq. (7) the linear
 * system A_h u_h = f_h, Eq. (10) the transfer operators I_P and I_R = I_P^T.
 * Where the paper is silent (PMIS, extended+i interpolation, the colouring, the Krylov
 * details), the routine states the reading it implements.
 *
 * Pins: see the test-suite (closed forms, invariants, brute force). Parity unpinned:
 * the choice of DOF numbering, the colour order and the hash streams are conventions of
 * this project, not of the paper; they are checked only for validity.
 *
 * Compile with -ffp-contract=off so every product and sum rounds as written.
 */
#include "pk_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXLEV 25

struct ocsr {
    int64_t nrows, ncols, nnz;
    int64_t *ptr;
    int32_t *col;
    double *val;
};

typedef struct {
    ocsr *A;          /* level matrix */
    int32_t *colour;  /* JP colouring of A's graph */
    int ncolour;
    uint8_t *strong;  /* strength flags per entry of A */
    int8_t *cf;       /* +1 C, -1 F */
    ocsr *P, *R;      /* interpolation and its transpose (absent on the coarsest) */
    double *l1;       /* row 1-norms */
} olevel;

struct oproblem {
    int k, nloc, dirichlet, source;
    int64_t nv, nt;
    double *xyz;
    int32_t *tets;
    double *kappa;
    int32_t (*mi)[4]; /* local multi-indices */
    double *S;        /* reference tensors S[a][b][m][n] */
    int64_t nedge, nface, nall;
    int64_t *elem_all;  /* all-DOF index of each local node */
    int32_t *elem_dof;  /* compact unknown index or -1 */
    int32_t *elem_vdof; /* compact P1 unknown index of each vertex or -1 */
    int64_t nh, nH;
    int64_t *dof_all;
    double *dof_xyz;
    int64_t *inc_ptr; /* unknown -> incident (tet, local) pairs, tets ascending */
    int32_t *inc_tet, *inc_loc;
    ocsr *Ah, *AH, *Pi, *PiT;
    double *b;
    double *f_all;    /* source 2: f at every P_k node (all-node numbering), else NULL */
    /* setup */
    int have_setup;
    oopts o;
    int32_t *colour_h;
    int ncolour_h;
    double *l1_h;
    int nlev;
    olevel lev[MAXLEV];
    double *chol; /* coarsest Cholesky factor, dense lower, row-major */
    int64_t nc;
};

static void *xmalloc(size_t n) {
    void *p = malloc(n ? n : 1);
    if (!p) {
        fprintf(stderr, "oracle: out of memory (%zu bytes)\n", n);
        abort();
    }
    return p;
}
static void *xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s ? s : 1);
    if (!p) {
        fprintf(stderr, "oracle: out of memory\n");
        abort();
    }
    return p;
}

/* ------------------------------------------------------------------------------------
 * 0. CSR containers
 * ---------------------------------------------------------------------------------- */
static ocsr *csr_alloc(int64_t nrows, int64_t ncols, int64_t nnz) {
    ocsr *a = (ocsr *)xmalloc(sizeof(ocsr));
    a->nrows = nrows;
    a->ncols = ncols;
    a->nnz = nnz;
    a->ptr = (int64_t *)xcalloc((size_t)nrows + 1, sizeof(int64_t));
    a->col = (int32_t *)xmalloc((size_t)nnz * sizeof(int32_t));
    a->val = (double *)xcalloc((size_t)nnz, sizeof(double));
    return a;
}

void orc_csr_free(ocsr *a) {
    if (!a) return;
    free(a->ptr);
    free(a->col);
    free(a->val);
    free(a);
}

void orc_csr_info(const ocsr *a, int64_t *out3) {
    out3[0] = a->nrows;
    out3[1] = a->ncols;
    out3[2] = a->nnz;
}

void orc_csr_copy(const ocsr *a, int64_t *ptr, int32_t *col, double *val) {
    if (ptr) memcpy(ptr, a->ptr, sizeof(int64_t) * (size_t)(a->nrows + 1));
    if (col) memcpy(col, a->col, sizeof(int32_t) * (size_t)a->nnz);
    if (val) memcpy(val, a->val, sizeof(double) * (size_t)a->nnz);
}

ocsr *orc_csr_new(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *ptr,
                  const int32_t *col, const double *val) {
    ocsr *a = csr_alloc(nrows, ncols, nnz);
    memcpy(a->ptr, ptr, sizeof(int64_t) * (size_t)(nrows + 1));
    memcpy(a->col, col, sizeof(int32_t) * (size_t)nnz);
    if (val) memcpy(a->val, val, sizeof(double) * (size_t)nnz);
    return a;
}

/* position of column j in row i, or -1 */
static int64_t csr_find(const ocsr *a, int64_t i, int32_t j) {
    int64_t lo = a->ptr[i], hi = a->ptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a->col[mid] == j) return mid;
        if (a->col[mid] < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* y = A x */
void orc_spmv(const ocsr *a, const double *x, double *y) {
    for (int64_t i = 0; i < a->nrows; ++i) {
        double s = 0.0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) s += a->val[e] * x[a->col[e]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *x, const double *y) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}
static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------------------
 * 1. Counter-based generator: SplitMix64 (Steele, Lea & Flood 2014).
 *    Output i of stream s is mix(s + (i+1) * 0x9E3779B97F4A7C15).
 * ---------------------------------------------------------------------------------- */
static uint64_t sm64(uint64_t stream, uint64_t i) {
    uint64_t z = stream + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Hash streams of the method's random choices (a convention of this project). */
static uint64_t stream_colour(uint64_t seed, int m) { return seed * 64 + (uint64_t)m; }
static uint64_t stream_pmis(uint64_t seed, int l) { return seed * 64 + 32 + (uint64_t)l; }

/* ------------------------------------------------------------------------------------
 * 2. The P_k Lagrange element (Sec. 2: V_h = P^{k,0}, evenly spaced nodes x_i^h).
 *    Local nodes are the multi-indices m in N^4 with |m| = k, at sum_a m_a v_a / k,
 *    in ascending lexicographic order of (m0, m1, m2, m3). The Lagrange basis function
 *    of node m in barycentric coordinates is
 *        phi_m(lambda) = prod_a prod_{j < m_a} (k lambda_a - j) / (j + 1).
 * ---------------------------------------------------------------------------------- */
int orc_nloc(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }

void orc_ref_nodes(int k, int32_t *m4) {
    int c = 0;
    for (int a = 0; a <= k; ++a)
        for (int b = 0; b <= k - a; ++b)
            for (int d = 0; d <= k - a - b; ++d) {
                m4[4 * c + 0] = a;
                m4[4 * c + 1] = b;
                m4[4 * c + 2] = d;
                m4[4 * c + 3] = k - a - b - d;
                ++c;
            }
}

/* coefficients of t^e in p_j(t) = prod_{i<j} (k t - i)/(i+1), e = 0..j */
static void lag_factor(int k, int j, double *c) {
    for (int e = 0; e <= k; ++e) c[e] = 0.0;
    c[0] = 1.0;
    for (int i = 0; i < j; ++i) {
        double nc[8] = {0};
        for (int e = 0; e <= i; ++e) {
            nc[e + 1] += (double)k * c[e] / (double)(i + 1);
            nc[e] -= (double)i * c[e] / (double)(i + 1);
        }
        for (int e = 0; e <= i + 1; ++e) c[e] = nc[e];
    }
}

static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* integral over T of prod_c lambda_c^{g_c}, divided by |T|: 3! g! / (|g| + 3)! */
static double mono_int(const int *g) {
    return 6.0 * fact(g[0]) * fact(g[1]) * fact(g[2]) * fact(g[3]) /
           fact(g[0] + g[1] + g[2] + g[3] + 3);
}

/* Expansion of d phi_m / d lambda_a into monomials: up to 16 terms (exps, coef). */
typedef struct {
    int n;
    int e[64][4];
    double c[64];
} dterms;

static void dphi_terms(int k, const int32_t *m, int a, dterms *t) {
    double cf[4][8], dcf[8];
    for (int b = 0; b < 4; ++b) lag_factor(k, m[b], cf[b]);
    for (int e = 0; e < 8; ++e) dcf[e] = 0.0;
    for (int e = 1; e <= m[a]; ++e) dcf[e - 1] = (double)e * cf[a][e];
    t->n = 0;
    int lim[4];
    for (int b = 0; b < 4; ++b) lim[b] = (b == a) ? (m[a] > 0 ? m[a] - 1 : -1) : m[b];
    if (lim[a] < 0) return; /* derivative identically zero */
    for (int e0 = 0; e0 <= lim[0]; ++e0)
        for (int e1 = 0; e1 <= lim[1]; ++e1)
            for (int e2 = 0; e2 <= lim[2]; ++e2)
                for (int e3 = 0; e3 <= lim[3]; ++e3) {
                    int ee[4] = {e0, e1, e2, e3};
                    double c = 1.0;
                    for (int b = 0; b < 4; ++b) c *= (b == a) ? dcf[ee[b]] : cf[b][ee[b]];
                    if (c == 0.0) continue;
                    int q = t->n++;
                    for (int b = 0; b < 4; ++b) t->e[q][b] = ee[b];
                    t->c[q] = c;
                }
}

/* S[a][b][m][n] = (1/|T|) int_T (d phi_m/d lambda_a)(d phi_n/d lambda_b) dx, exact for any
 * tetrahedron; then the element stiffness of Eq. (7) with piecewise-constant kappa is
 * K_mn = kappa |T| sum_ab (grad lambda_a . grad lambda_b) S[a][b][m][n]. */
void orc_ref_tensor(int k, double *S) {
    int nl = orc_nloc(k);
    int32_t *mi = (int32_t *)xmalloc(sizeof(int32_t) * 4 * (size_t)nl);
    orc_ref_nodes(k, mi);
    dterms *T = (dterms *)xmalloc(sizeof(dterms) * 4 * (size_t)nl);
    for (int m = 0; m < nl; ++m)
        for (int a = 0; a < 4; ++a) dphi_terms(k, mi + 4 * m, a, &T[m * 4 + a]);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int m = 0; m < nl; ++m)
                for (int n = 0; n < nl; ++n) {
                    const dterms *tm = &T[m * 4 + a], *tn = &T[n * 4 + b];
                    double s = 0.0;
                    for (int p = 0; p < tm->n; ++p)
                        for (int q = 0; q < tn->n; ++q) {
                            int g[4];
                            for (int c = 0; c < 4; ++c) g[c] = tm->e[p][c] + tn->e[q][c];
                            s += tm->c[p] * tn->c[q] * mono_int(g);
                        }
                    S[((a * 4 + b) * nl + m) * nl + n] = s;
                }
    free(T);
    free(mi);
}

void orc_basis_eval(int k, const double *lam, double *phi) {
    int nl = orc_nloc(k);
    int32_t mi[35 * 4];
    orc_ref_nodes(k, mi);
    for (int m = 0; m < nl; ++m) {
        double v = 1.0;
        for (int a = 0; a < 4; ++a)
            for (int j = 0; j < mi[4 * m + a]; ++j)
                v *= ((double)k * lam[a] - (double)j) / (double)(j + 1);
        phi[m] = v;
    }
}

/* ------------------------------------------------------------------------------------
 * 3. Geometry of one tetrahedron: J = [x1-x0, x2-x0, x3-x0], |T| = det J / 6,
 *    grad lambda_1..3 = rows of J^{-1}, grad lambda_0 = -(sum of the others).
 * ---------------------------------------------------------------------------------- */
static double tet_geom(const double *x, double G[4][4]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double gl[4][3];
    for (int c = 0; c < 3; ++c) {
        gl[1][c] = inv[0][c];
        gl[2][c] = inv[1][c];
        gl[3][c] = inv[2][c];
        gl[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            G[a][b] = gl[a][0] * gl[b][0] + gl[a][1] * gl[b][1] + gl[a][2] * gl[b][2];
    return det / 6.0;
}

static void element_matrix(int nl, const double *S, double kappa, double vol,
                           double G[4][4], double *K) {
    for (int m = 0; m < nl; ++m)
        for (int n = 0; n < nl; ++n) {
            double s = 0.0;
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) s += G[a][b] * S[((a * 4 + b) * nl + m) * nl + n];
            K[m * nl + n] = kappa * vol * s;
        }
}

void orc_element_stiffness(int k, const double *x12, double kappa, double *K) {
    int nl = orc_nloc(k);
    double *S = (double *)xmalloc(sizeof(double) * 16 * (size_t)nl * (size_t)nl);
    orc_ref_tensor(k, S);
    double G[4][4];
    double vol = tet_geom(x12, G);
    element_matrix(nl, S, kappa, vol, G, K);
    free(S);
}

/* ------------------------------------------------------------------------------------
 * 4. Grundmann-Moeller quadrature on the 3-simplex (Grundmann & Moeller, SIAM J. Numer.
 *    Anal. 15, 1978): degree d = 2s+1, weights for the reference simplex of volume 1/6,
 *        w_i = (-1)^i 2^{-2s} (d+3-2i)^d / (i! (d+3-i)!),   i = 0..s,
 *    at barycentric points (2 beta_c + 1)/(d + 3 - 2i) for beta in N^4, |beta| = s - i.
 *    The paper does not state its load quadrature; this rule is exact to degree 2s+1.
 * ---------------------------------------------------------------------------------- */
int orc_gm_rule(int s, double *lam, double *w, int cap) {
    int d = 2 * s + 1, q = 0;
    for (int i = 0; i <= s; ++i) {
        double wi = ((i & 1) ? -1.0 : 1.0) * pow(2.0, -2.0 * s) * pow((double)(d + 3 - 2 * i), d) /
                    (fact(i) * fact(d + 3 - i));
        int r = s - i;
        for (int b0 = 0; b0 <= r; ++b0)
            for (int b1 = 0; b1 <= r - b0; ++b1)
                for (int b2 = 0; b2 <= r - b0 - b1; ++b2) {
                    int b3 = r - b0 - b1 - b2;
                    if (q < cap) {
                        double den = (double)(d + 3 - 2 * i);
                        lam[4 * q + 0] = (2.0 * b0 + 1.0) / den;
                        lam[4 * q + 1] = (2.0 * b1 + 1.0) / den;
                        lam[4 * q + 2] = (2.0 * b2 + 1.0) / den;
                        lam[4 * q + 3] = (2.0 * b3 + 1.0) / den;
                        w[q] = wi;
                    }
                    ++q;
                }
    }
    return q;
}

/* Manufactured source of Sec. 6's test problem family: with kappa = 1 the solution of
 * Eq. (1) on the unit cube is u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u. */
static double src_sine(const double *x) {
    return 3.0 * M_PI * M_PI * sin(M_PI * x[0]) * sin(M_PI * x[1]) * sin(M_PI * x[2]);
}
static double exact_sine(const double *x) {
    return sin(M_PI * x[0]) * sin(M_PI * x[1]) * sin(M_PI * x[2]);
}

/* ------------------------------------------------------------------------------------
 * 5. DOF map (Sec. 2: nodes x_i^h of V_h; the paper's Fig. 1 numbering is not in the
 *    text, so this project's convention is used): vertices first (by vertex id), then
 *    edges sorted by (min, max) vertex with their k-1 nodes ordered away from the lower
 *    vertex, then faces sorted by their vertex triple with nodes in ascending
 *    lexicographic order of the multi-index over the sorted vertices, then element
 *    interiors by element id in the same order. Homogeneous Dirichlet values (Eq. 1) are
 *    imposed by removing every node on a boundary face; the rest are numbered in order.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int32_t v[3];
    int32_t t;
} facekey;

static int cmp_face(const void *a, const void *b) {
    const facekey *x = (const facekey *)a, *y = (const facekey *)b;
    for (int c = 0; c < 3; ++c)
        if (x->v[c] != y->v[c]) return x->v[c] < y->v[c] ? -1 : 1;
    return (x->t > y->t) - (x->t < y->t);
}

static int64_t find_i64(const int64_t *arr, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (arr[mid] == key) return mid;
        if (arr[mid] < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* rank of composition (p_0..p_{s-1}) (all >= 1, sum k) in ascending lexicographic order */
static int comp_rank(int k, int s, const int *p) {
    int r = 0;
    if (s == 3) {
        for (int a = 1; a <= k - 2; ++a)
            for (int b = 1; b <= k - 1 - a; ++b) {
                int c = k - a - b;
                if (a == p[0] && b == p[1] && c == p[2]) return r;
                ++r;
            }
    } else {
        for (int a = 1; a <= k - 3; ++a)
            for (int b = 1; b <= k - 2 - a; ++b)
                for (int c = 1; c <= k - 1 - a - b; ++c) {
                    int d = k - a - b - c;
                    if (a == p[0] && b == p[1] && c == p[2] && d == p[3]) return r;
                    ++r;
                }
    }
    return -1;
}

static int build_dofmap(oproblem *P) {
    int k = P->k, nl = P->nloc;
    int64_t nv = P->nv, nt = P->nt;
    /* edges */
    int64_t *ek = (int64_t *)xmalloc(sizeof(int64_t) * 6 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        int c = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                int64_t u = P->tets[4 * t + a], v = P->tets[4 * t + b];
                if (u > v) {
                    int64_t w = u;
                    u = v;
                    v = w;
                }
                ek[6 * t + c++] = u * nv + v;
            }
    }
    qsort(ek, (size_t)(6 * nt), sizeof(int64_t), cmp_i64);
    int64_t ne = 0;
    for (int64_t i = 0; i < 6 * nt; ++i)
        if (i == 0 || ek[i] != ek[i - 1]) ek[ne++] = ek[i];
    P->nedge = ne;
    /* faces, with multiplicity to find the boundary */
    facekey *fk = (facekey *)xmalloc(sizeof(facekey) * 4 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int o = 0; o < 4; ++o) {
            int32_t v[3], c = 0;
            for (int a = 0; a < 4; ++a)
                if (a != o) v[c++] = P->tets[4 * t + a];
            qsort(v, 3, sizeof(int32_t), cmp_i32);
            facekey *f = &fk[4 * t + o];
            f->v[0] = v[0];
            f->v[1] = v[1];
            f->v[2] = v[2];
            f->t = (int32_t)t;
        }
    qsort(fk, (size_t)(4 * nt), sizeof(facekey), cmp_face);
    int64_t *fkey = (int64_t *)xmalloc(sizeof(int64_t) * 4 * (size_t)nt); /* unique faces */
    int32_t *fv = (int32_t *)xmalloc(sizeof(int32_t) * 12 * (size_t)nt);
    uint8_t *fbnd = (uint8_t *)xcalloc((size_t)(4 * nt), 1);
    int64_t nf = 0;
    for (int64_t i = 0; i < 4 * nt;) {
        int64_t j = i;
        while (j < 4 * nt && fk[j].v[0] == fk[i].v[0] && fk[j].v[1] == fk[i].v[1] &&
               fk[j].v[2] == fk[i].v[2])
            ++j;
        fv[3 * nf + 0] = fk[i].v[0];
        fv[3 * nf + 1] = fk[i].v[1];
        fv[3 * nf + 2] = fk[i].v[2];
        fbnd[nf] = (j - i == 1);
        fkey[nf] = nf;
        ++nf;
        i = j;
    }
    P->nface = nf;
    int nedof = k - 1, nfdof = (k - 1) * (k - 2) / 2, nidof = (k - 1) * (k - 2) * (k - 3) / 6;
    int64_t off_e = nv, off_f = nv + ne * nedof, off_i = off_f + nf * nfdof;
    P->nall = off_i + nt * nidof;
    uint8_t *bnd = (uint8_t *)xcalloc((size_t)P->nall, 1);
    /* boundary closure: vertices, edges and nodes of boundary faces */
    for (int64_t f = 0; f < nf; ++f) {
        if (!fbnd[f]) continue;
        int32_t *v = &fv[3 * f];
        for (int a = 0; a < 3; ++a) bnd[v[a]] = 1;
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
                int64_t e = find_i64(ek, ne, (int64_t)v[a] * nv + v[b]);
                for (int q = 0; q < nedof; ++q) bnd[off_e + e * nedof + q] = 1;
            }
        for (int q = 0; q < nfdof; ++q) bnd[off_f + f * nfdof + q] = 1;
    }
    if (!P->dirichlet) memset(bnd, 0, (size_t)P->nall);
    /* element -> all-DOF map */
    P->elem_all = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(nt * nl));
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *g = &P->tets[4 * t];
        for (int m = 0; m < nl; ++m) {
            const int32_t *mm = P->mi[m];
            int sup[4], ns = 0;
            for (int a = 0; a < 4; ++a)
                if (mm[a] > 0) sup[ns++] = a;
            int64_t d = -1;
            if (ns == 1) {
                d = g[sup[0]];
            } else if (ns == 2) {
                int a = sup[0], b = sup[1];
                int64_t u = g[a], v = g[b];
                int hi = (v > u) ? b : a;
                if (u > v) {
                    int64_t w = u;
                    u = v;
                    v = w;
                }
                int64_t e = find_i64(ek, ne, u * nv + v);
                d = off_e + e * nedof + (mm[hi] - 1);
            } else if (ns == 3) {
                /* sort the three vertices by global id, carrying multiplicities */
                int idx[3] = {sup[0], sup[1], sup[2]};
                for (int x = 0; x < 3; ++x)
                    for (int y = x + 1; y < 3; ++y)
                        if (g[idx[y]] < g[idx[x]]) {
                            int w = idx[x];
                            idx[x] = idx[y];
                            idx[y] = w;
                        }
                facekey key;
                key.v[0] = g[idx[0]];
                key.v[1] = g[idx[1]];
                key.v[2] = g[idx[2]];
                /* binary search among unique faces */
                int64_t lo = 0, hi = nf - 1, f = -1;
                while (lo <= hi) {
                    int64_t mid = lo + (hi - lo) / 2;
                    int c = 0;
                    for (int z = 0; z < 3 && c == 0; ++z)
                        c = (fv[3 * mid + z] > key.v[z]) - (fv[3 * mid + z] < key.v[z]);
                    if (c == 0) {
                        f = mid;
                        break;
                    }
                    if (c < 0) lo = mid + 1;
                    else hi = mid - 1;
                }
                int p[3] = {mm[idx[0]], mm[idx[1]], mm[idx[2]]};
                d = off_f + f * nfdof + comp_rank(k, 3, p);
            } else {
                int idx[4] = {0, 1, 2, 3};
                for (int x = 0; x < 4; ++x)
                    for (int y = x + 1; y < 4; ++y)
                        if (g[idx[y]] < g[idx[x]]) {
                            int w = idx[x];
                            idx[x] = idx[y];
                            idx[y] = w;
                        }
                int p[4] = {mm[idx[0]], mm[idx[1]], mm[idx[2]], mm[idx[3]]};
                d = off_i + t * nidof + comp_rank(k, 4, p);
            }
            P->elem_all[t * nl + m] = d;
        }
    }
    /* compact numbering of the unknowns */
    int64_t *cmap = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)P->nall);
    int64_t nh = 0;
    for (int64_t d = 0; d < P->nall; ++d) cmap[d] = bnd[d] ? -1 : nh++;
    P->nh = nh;
    P->dof_all = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nh);
    for (int64_t d = 0; d < P->nall; ++d)
        if (cmap[d] >= 0) P->dof_all[cmap[d]] = d;
    P->elem_dof = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(nt * nl));
    for (int64_t i = 0; i < nt * nl; ++i) P->elem_dof[i] = (int32_t)cmap[P->elem_all[i]];
    /* P1 unknowns: the interior vertices, by vertex id */
    int64_t *vmap = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nv);
    int64_t nH = 0;
    for (int64_t v = 0; v < nv; ++v) vmap[v] = bnd[v] ? -1 : nH++;
    P->nH = nH;
    P->elem_vdof = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(4 * nt));
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a) P->elem_vdof[4 * t + a] = (int32_t)vmap[P->tets[4 * t + a]];
    /* node coordinates */
    P->dof_xyz = (double *)xmalloc(sizeof(double) * 3 * (size_t)nh);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            int32_t i = P->elem_dof[t * nl + m];
            if (i < 0) continue;
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int a = 0; a < 4; ++a) s += (double)P->mi[m][a] * P->xyz[3 * P->tets[4 * t + a] + c];
                P->dof_xyz[3 * i + c] = s / (double)k;
            }
        }
    /* incidence: unknown -> (tet, local) in ascending tet order */
    P->inc_ptr = (int64_t *)xcalloc((size_t)nh + 1, sizeof(int64_t));
    for (int64_t i = 0; i < nt * nl; ++i)
        if (P->elem_dof[i] >= 0) P->inc_ptr[P->elem_dof[i] + 1]++;
    for (int64_t i = 0; i < nh; ++i) P->inc_ptr[i + 1] += P->inc_ptr[i];
    P->inc_tet = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)P->inc_ptr[nh]);
    P->inc_loc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)P->inc_ptr[nh]);
    int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nh);
    for (int64_t i = 0; i < nh; ++i) fill[i] = P->inc_ptr[i];
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            int32_t i = P->elem_dof[t * nl + m];
            if (i < 0) continue;
            P->inc_tet[fill[i]] = (int32_t)t;
            P->inc_loc[fill[i]] = m;
            fill[i]++;
        }
    free(fill);
    free(vmap);
    free(cmap);
    free(bnd);
    free(fbnd);
    free(fv);
    free(fkey);
    free(fk);
    free(ek);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * 6. Assembly of Eq. (7): (A_h)_ij = a(phi_j, phi_i), f_i = <f, phi_i>; the P1 matrix
 *    A_H on the same mesh (Sec. 2, auxiliary space V_H); and I_P of Eq. (10) with
 *    c_j^i = psi_j(x_i^h). Every entry sums its element contributions in ascending
 *    element order.
 * ---------------------------------------------------------------------------------- */
static ocsr *build_pattern(const oproblem *P, int p1) {
    int64_t n = p1 ? P->nH : P->nh;
    int nl = p1 ? 4 : P->nloc;
    const int32_t *ed = p1 ? P->elem_vdof : P->elem_dof;
    /* incidence for this space */
    int64_t *iptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < P->nt * nl; ++i)
        if (ed[i] >= 0) iptr[ed[i] + 1]++;
    for (int64_t i = 0; i < n; ++i) iptr[i + 1] += iptr[i];
    int32_t *itet = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)iptr[n]);
    int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) fill[i] = iptr[i];
    for (int64_t t = 0; t < P->nt; ++t)
        for (int m = 0; m < nl; ++m)
            if (ed[t * nl + m] >= 0) itet[fill[ed[t * nl + m]]++] = (int32_t)t;
    int64_t cap = 1 << 20, nnz = 0;
    int32_t *col = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)cap);
    int64_t *ptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    int32_t *buf = NULL;
    int64_t bcap = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t need = (iptr[i + 1] - iptr[i]) * nl;
        if (need > bcap) {
            free(buf);
            bcap = need;
            buf = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)bcap);
        }
        int64_t nb = 0;
        for (int64_t q = iptr[i]; q < iptr[i + 1]; ++q) {
            int64_t t = itet[q];
            for (int m = 0; m < nl; ++m)
                if (ed[t * nl + m] >= 0) buf[nb++] = ed[t * nl + m];
        }
        qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < nb; ++q) {
            if (q > 0 && buf[q] == buf[q - 1]) continue;
            if (nnz == cap) {
                cap *= 2;
                col = (int32_t *)realloc(col, sizeof(int32_t) * (size_t)cap);
                if (!col) abort();
            }
            col[nnz++] = buf[q];
        }
        ptr[i + 1] = nnz;
    }
    free(buf);
    free(fill);
    free(itet);
    free(iptr);
    ocsr *a = (ocsr *)xmalloc(sizeof(ocsr));
    a->nrows = n;
    a->ncols = n;
    a->nnz = nnz;
    a->ptr = ptr;
    a->col = (int32_t *)realloc(col, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    a->val = (double *)xcalloc((size_t)nnz, sizeof(double));
    return a;
}

static void tet_coords(const oproblem *P, int64_t t, double *x12) {
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) x12[3 * a + c] = P->xyz[3 * P->tets[4 * t + a] + c];
}

static void assemble_values(oproblem *P) {
    int nl = P->nloc;
    double *K = (double *)xmalloc(sizeof(double) * (size_t)nl * (size_t)nl);
    memset(P->Ah->val, 0, sizeof(double) * (size_t)P->Ah->nnz);
    memset(P->AH->val, 0, sizeof(double) * (size_t)P->AH->nnz);
    for (int64_t t = 0; t < P->nt; ++t) {
        double x12[12], G[4][4];
        tet_coords(P, t, x12);
        double vol = tet_geom(x12, G);
        element_matrix(nl, P->S, P->kappa[t], vol, G, K);
        for (int m = 0; m < nl; ++m) {
            int32_t i = P->elem_dof[t * nl + m];
            if (i < 0) continue;
            for (int n = 0; n < nl; ++n) {
                int32_t j = P->elem_dof[t * nl + n];
                if (j < 0) continue;
                P->Ah->val[csr_find(P->Ah, i, j)] += K[m * nl + n];
            }
        }
        /* P1: K1_ab = kappa |T| grad lambda_a . grad lambda_b */
        for (int a = 0; a < 4; ++a) {
            int32_t i = P->elem_vdof[4 * t + a];
            if (i < 0) continue;
            for (int b = 0; b < 4; ++b) {
                int32_t j = P->elem_vdof[4 * t + b];
                if (j < 0) continue;
                P->AH->val[csr_find(P->AH, i, j)] += P->kappa[t] * vol * G[a][b];
            }
        }
    }
    free(K);
}

/* Load vector f_i = <f, phi_i> of Eq. (7) by the Grundmann-Moeller rule of degree
 * 2k+3. source 1: the manufactured f, evaluated at the quadrature points; source 2: a
 * caller's f given by its values at the P_k nodes, i.e. f_h = sum_n f_n phi_n (the
 * nodal interpolant, Sec. 2), evaluated at the quadrature points through the basis.
 * The rule is exact for f_h phi_i (degree 2k), so source 2 gives b = M f exactly up to
 * rounding, M the P_k mass matrix. */
static void assemble_load(oproblem *P) {
    int nl = P->nloc, s = P->k + 1;
    double lam[4 * 512], w[512];
    int nq = orc_gm_rule(s, lam, w, 512);
    memset(P->b, 0, sizeof(double) * (size_t)P->nh);
    if (P->source == 0) return;
    double *phiq = (double *)xmalloc(sizeof(double) * (size_t)(nq * nl));
    for (int q = 0; q < nq; ++q) orc_basis_eval(P->k, &lam[4 * q], &phiq[q * nl]);
    for (int64_t t = 0; t < P->nt; ++t) {
        double x12[12], G[4][4];
        tet_coords(P, t, x12);
        double vol = tet_geom(x12, G);
        double fq[512];
        for (int q = 0; q < nq; ++q) {
            if (P->source == 2) {
                double v = 0.0;
                for (int n = 0; n < nl; ++n) v += P->f_all[P->elem_all[t * nl + n]] * phiq[q * nl + n];
                fq[q] = v;
                continue;
            }
            double x[3];
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int a = 0; a < 4; ++a) v += lam[4 * q + a] * x12[3 * a + c];
                x[c] = v;
            }
            fq[q] = src_sine(x);
        }
        for (int m = 0; m < nl; ++m) {
            int32_t i = P->elem_dof[t * nl + m];
            if (i < 0) continue;
            double acc = 0.0;
            for (int q = 0; q < nq; ++q) acc += w[q] * fq[q] * phiq[q * nl + m];
            P->b[i] += 6.0 * vol * acc;
        }
    }
    free(phiq);
}

/* I_P (Eq. 10): row i, column j holds psi_j(x_i^h) = m_a / k for the vertex a of any
 * element containing node i; only interior vertices are columns (V_H within H^1_0). */
static ocsr *build_pi(const oproblem *P) {
    int nl = P->nloc;
    ocsr *a = csr_alloc(P->nh, P->nH, 4 * P->nh);
    int64_t nnz = 0;
    for (int64_t i = 0; i < P->nh; ++i) {
        int64_t t = P->inc_tet[P->inc_ptr[i]];
        int m = P->inc_loc[P->inc_ptr[i]];
        int32_t cj[4];
        double cv[4];
        int c = 0;
        for (int q = 0; q < 4; ++q) {
            int32_t j = P->elem_vdof[4 * t + q];
            if (P->mi[m][q] > 0 && j >= 0) {
                cj[c] = j;
                cv[c] = (double)P->mi[m][q] / (double)P->k;
                ++c;
            }
        }
        for (int x = 0; x < c; ++x)
            for (int y = x + 1; y < c; ++y)
                if (cj[y] < cj[x]) {
                    int32_t tj = cj[x];
                    cj[x] = cj[y];
                    cj[y] = tj;
                    double tv = cv[x];
                    cv[x] = cv[y];
                    cv[y] = tv;
                }
        for (int x = 0; x < c; ++x) {
            a->col[nnz] = cj[x];
            a->val[nnz] = cv[x];
            ++nnz;
        }
        a->ptr[i + 1] = nnz;
    }
    a->nnz = nnz;
    (void)nl;
    return a;
}

oproblem *orc_problem_create(int64_t nv, const double *xyz, int64_t nt, const int32_t *tets,
                             int k, const double *kappa, int source, int dirichlet) {
    if (k < 1 || k > 4 || nv <= 0 || nt <= 0) return NULL;
    oproblem *P = (oproblem *)xcalloc(1, sizeof(oproblem));
    P->k = k;
    P->nloc = orc_nloc(k);
    P->nv = nv;
    P->nt = nt;
    P->source = source;
    P->dirichlet = dirichlet;
    P->xyz = (double *)xmalloc(sizeof(double) * 3 * (size_t)nv);
    memcpy(P->xyz, xyz, sizeof(double) * 3 * (size_t)nv);
    P->tets = (int32_t *)xmalloc(sizeof(int32_t) * 4 * (size_t)nt);
    memcpy(P->tets, tets, sizeof(int32_t) * 4 * (size_t)nt);
    P->kappa = (double *)xmalloc(sizeof(double) * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) P->kappa[t] = kappa ? kappa[t] : 1.0;
    P->mi = (int32_t(*)[4])xmalloc(sizeof(int32_t) * 4 * (size_t)P->nloc);
    orc_ref_nodes(k, &P->mi[0][0]);
    P->S = (double *)xmalloc(sizeof(double) * 16 * (size_t)P->nloc * (size_t)P->nloc);
    orc_ref_tensor(k, P->S);
    build_dofmap(P);
    P->Ah = build_pattern(P, 0);
    P->AH = build_pattern(P, 1);
    P->b = (double *)xcalloc((size_t)P->nh, sizeof(double));
    assemble_values(P);
    assemble_load(P);
    P->Pi = build_pi(P);
    P->PiT = orc_transpose(P->Pi);
    return P;
}

/* Replaces the source by a caller's f at all P_k nodes (f_all[n_all], all-node
 * numbering of the DOF map, boundary nodes included) and re-assembles the load. */
int orc_set_source_nodal(oproblem *P, const double *f_all) {
    if (!P->f_all) P->f_all = (double *)xmalloc(sizeof(double) * (size_t)P->nall);
    memcpy(P->f_all, f_all, sizeof(double) * (size_t)P->nall);
    P->source = 2;
    assemble_load(P);
    return 0;
}

/* Coordinates of all n_all P_k nodes (x = sum_a m_a v_a / k over any element holding
 * the node), in the all-node numbering. */
void orc_problem_nodes(const oproblem *P, double *xyz_all) {
    int nl = P->nloc;
    for (int64_t t = 0; t < P->nt; ++t)
        for (int m = 0; m < nl; ++m) {
            int64_t d = P->elem_all[t * nl + m];
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int a = 0; a < 4; ++a) v += (double)P->mi[m][a] * P->xyz[3 * (int64_t)P->tets[4 * t + a] + c];
                xyz_all[3 * d + c] = v / (double)P->k;
            }
        }
}

int orc_set_kappa(oproblem *P, const double *kappa) {
    for (int64_t t = 0; t < P->nt; ++t) P->kappa[t] = kappa[t];
    assemble_values(P);
    assemble_load(P);
    return 0;
}

static void free_levels(oproblem *P) {
    for (int l = 0; l < P->nlev; ++l) {
        olevel *L = &P->lev[l];
        if (l > 0) orc_csr_free(L->A);
        free(L->colour);
        free(L->strong);
        free(L->cf);
        orc_csr_free(L->P);
        orc_csr_free(L->R);
        free(L->l1);
        memset(L, 0, sizeof(*L));
    }
    P->nlev = 0;
    free(P->chol);
    P->chol = NULL;
    free(P->colour_h);
    P->colour_h = NULL;
    free(P->l1_h);
    P->l1_h = NULL;
    P->have_setup = 0;
}

void orc_problem_free(oproblem *P) {
    if (!P) return;
    free_levels(P);
    free(P->xyz);
    free(P->tets);
    free(P->kappa);
    free(P->mi);
    free(P->S);
    free(P->elem_all);
    free(P->f_all);
    free(P->elem_dof);
    free(P->elem_vdof);
    free(P->dof_all);
    free(P->dof_xyz);
    free(P->inc_ptr);
    free(P->inc_tet);
    free(P->inc_loc);
    orc_csr_free(P->Ah);
    orc_csr_free(P->AH);
    orc_csr_free(P->Pi);
    orc_csr_free(P->PiT);
    free(P->b);
    free(P);
}

void orc_problem_sizes(const oproblem *P, int64_t *o) {
    o[0] = P->nh;
    o[1] = P->nH;
    o[2] = P->Ah->nnz;
    o[3] = P->AH->nnz;
    o[4] = P->Pi->nnz;
    o[5] = P->nall;
    o[6] = P->nedge;
    o[7] = P->nface;
}

const ocsr *orc_problem_matrix(const oproblem *P, int which) {
    return which == 0 ? P->Ah : which == 1 ? P->AH : P->Pi;
}
void orc_problem_rhs(const oproblem *P, double *b) {
    memcpy(b, P->b, sizeof(double) * (size_t)P->nh);
}
void orc_problem_dofs(const oproblem *P, int64_t *dof_all, double *dof_xyz) {
    if (dof_all) memcpy(dof_all, P->dof_all, sizeof(int64_t) * (size_t)P->nh);
    if (dof_xyz) memcpy(dof_xyz, P->dof_xyz, sizeof(double) * 3 * (size_t)P->nh);
}
void orc_problem_elem_dofs(const oproblem *P, int32_t *elem_dof) {
    memcpy(elem_dof, P->elem_dof, sizeof(int32_t) * (size_t)(P->nt * P->nloc));
}

/* ------------------------------------------------------------------------------------
 * 7. Multicolour ordering for the Gauss-Seidel smoothers (the paper's hybrid GS of
 *    Sec. 6.1 is replaced by a multicolour GS). Jones-Plassmann with largest-degree-first
 *    priorities: vertex priority is (degree, hash(stream, i), -i), the degree counting
 *    the off-diagonal entries of the row; each round every uncoloured vertex whose
 *    priority beats all its uncoloured neighbours takes the smallest colour not used by a
 *    neighbour coloured in an earlier round.
 * ---------------------------------------------------------------------------------- */
static int prio_beats(int64_t di, uint64_t hi, int64_t i, int64_t dj, uint64_t hj, int64_t j) {
    /* does vertex i beat vertex j? higher degree wins, then larger hash, then lower index */
    if (di != dj) return di > dj;
    if (hi != hj) return hi > hj;
    return i < j;
}

int orc_colour_jp(int64_t n, const int64_t *ptr, const int32_t *col, uint64_t stream,
                  int32_t *colour) {
    uint64_t *h = (uint64_t *)xmalloc(sizeof(uint64_t) * (size_t)n);
    int64_t *deg = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    uint8_t *pick = (uint8_t *)xmalloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        h[i] = sm64(stream, (uint64_t)i);
        colour[i] = -1;
        deg[i] = 0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) deg[i] += (col[e] != i);
    }
    int64_t left = n;
    int ncol = 0;
    while (left > 0) {
        for (int64_t i = 0; i < n; ++i) {
            pick[i] = 0;
            if (colour[i] >= 0) continue;
            int best = 1;
            for (int64_t e = ptr[i]; e < ptr[i + 1] && best; ++e) {
                int64_t j = col[e];
                if (j == i || colour[j] >= 0) continue;
                if (!prio_beats(deg[i], h[i], i, deg[j], h[j], j)) best = 0;
            }
            pick[i] = (uint8_t)best;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (!pick[i]) continue;
            int c = 0;
            for (;;) {
                int used = 0;
                for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
                    int64_t j = col[e];
                    if (j != i && !pick[j] && colour[j] == c) {
                        used = 1;
                        break;
                    }
                }
                if (!used) break;
                ++c;
            }
            colour[i] = c;
            if (c + 1 > ncol) ncol = c + 1;
            --left;
        }
    }
    free(pick);
    free(deg);
    free(h);
    return ncol;
}

/* ------------------------------------------------------------------------------------
 * 8. Smoothers. Symmetric Gauss-Seidel from a zero initial guess (Algorithm 2.1's
 *    smoother G_h, used as pre- and post-smoother per Remark 2.1, one sweep each as in
 *    Remark 6.1): a forward sweep over the colours 0..C-1 followed by a backward sweep
 *    over C-1..0, each update x_i <- (r_i - sum_{j != i} a_ij x_j) / a_ii.
 *    l1-Jacobi: x <- x + D_l1^{-1} (r - A x) with d_i = sum_j |a_ij|.
 * ---------------------------------------------------------------------------------- */
static void gs_sweep(const ocsr *a, const int32_t *colour, int ncolour, int forward,
                     const double *r, double *x) {
    for (int q = 0; q < ncolour; ++q) {
        int c = forward ? q : ncolour - 1 - q;
        for (int64_t i = 0; i < a->nrows; ++i) {
            if (colour[i] != c) continue;
            double s = r[i], d = 0.0;
            for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
                if (a->col[e] == i) d = a->val[e];
                else s -= a->val[e] * x[a->col[e]];
            }
            x[i] = s / d;
        }
    }
}

void orc_sgs(const ocsr *a, const int32_t *colour, int ncolour, const double *r, double *z) {
    for (int64_t i = 0; i < a->nrows; ++i) z[i] = 0.0;
    gs_sweep(a, colour, ncolour, 1, r, z);
    gs_sweep(a, colour, ncolour, 0, r, z);
}

static double *l1_norms(const ocsr *a) {
    double *d = (double *)xmalloc(sizeof(double) * (size_t)(a->nrows ? a->nrows : 1));
    for (int64_t i = 0; i < a->nrows; ++i) {
        double s = 0.0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) s += fabs(a->val[e]);
        d[i] = s;
    }
    return d;
}

static void l1_step(const ocsr *a, const double *d, const double *r, double *x, int from_zero) {
    int64_t n = a->nrows;
    if (from_zero) {
        for (int64_t i = 0; i < n; ++i) x[i] = r[i] / d[i];
        return;
    }
    double *ax = (double *)xmalloc(sizeof(double) * (size_t)n);
    orc_spmv(a, x, ax);
    for (int64_t i = 0; i < n; ++i) x[i] += (r[i] - ax[i]) / d[i];
    free(ax);
}

/* ------------------------------------------------------------------------------------
 * 9. P1 algebraic multigrid (Sec. 1 and Sec. 6.1: PMIS coarsening and extended+i
 *    interpolation; the paper cites them without formulas).
 *
 *    Strength (Sec. 6.2): j is strong for i iff j != i and -a_ij > theta max_{k!=i}(-a_ik);
 *    if that maximum is <= 0 the row has no strong entries.
 * ---------------------------------------------------------------------------------- */
void orc_strength(const ocsr *a, double theta, uint8_t *strong) {
    for (int64_t i = 0; i < a->nrows; ++i) {
        double mx = 0.0;
        int have = 0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            if (a->col[e] == i) continue;
            double v = -a->val[e];
            if (!have || v > mx) mx = v;
            have = 1;
        }
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            strong[e] = 0;
            if (!have || mx <= 0.0 || a->col[e] == i) continue;
            strong[e] = (-a->val[e] > theta * mx) ? 1 : 0;
        }
    }
}

/* PMIS (De Sterck, Yang & Heys, SIAM J. Matrix Anal. Appl. 27, 2006). Measure of i is
 * the tuple (|S_i^T|, hash(stream, i), i), compared lexicographically, in place of the
 * published |S_i^T| + uniform(0,1). Points with no strong connection either way are F.
 * Each round, every undecided point whose measure beats every undecided point of
 * S_i u S_i^T becomes C; then every undecided point strongly depending on a new C point
 * becomes F. */
static int meas_beats(int64_t mi, uint64_t hi, int64_t i, int64_t mj, uint64_t hj, int64_t j) {
    if (mi != mj) return mi > mj;
    if (hi != hj) return hi > hj;
    return i > j;
}

void orc_pmis(const ocsr *a, const uint8_t *strong, uint64_t stream, int8_t *cf) {
    int64_t n = a->nrows;
    /* transpose of the strength graph: ST row j lists i with j in S_i */
    int64_t *tp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e)
            if (strong[e]) tp[a->col[e] + 1]++;
    for (int64_t i = 0; i < n; ++i) tp[i + 1] += tp[i];
    int32_t *ti = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(tp[n] ? tp[n] : 1));
    int64_t *fl = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) fl[i] = tp[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e)
            if (strong[e]) ti[fl[a->col[e]]++] = (int32_t)i;
    uint64_t *h = (uint64_t *)xmalloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    int64_t *mu = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    uint8_t *newc = (uint8_t *)xcalloc((size_t)n, 1);
    int64_t left = 0;
    for (int64_t i = 0; i < n; ++i) {
        h[i] = sm64(stream, (uint64_t)i);
        mu[i] = tp[i + 1] - tp[i];
        int64_t ns = 0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) ns += strong[e];
        cf[i] = (ns == 0 && mu[i] == 0) ? -1 : 0;
        if (cf[i] == 0) ++left;
    }
    while (left > 0) {
        for (int64_t i = 0; i < n; ++i) {
            newc[i] = 0;
            if (cf[i] != 0) continue;
            int best = 1;
            for (int64_t e = a->ptr[i]; e < a->ptr[i + 1] && best; ++e) {
                int64_t j = a->col[e];
                if (!strong[e] || cf[j] != 0) continue;
                if (!meas_beats(mu[i], h[i], i, mu[j], h[j], j)) best = 0;
            }
            for (int64_t q = tp[i]; q < tp[i + 1] && best; ++q) {
                int64_t j = ti[q];
                if (cf[j] != 0) continue;
                if (!meas_beats(mu[i], h[i], i, mu[j], h[j], j)) best = 0;
            }
            newc[i] = (uint8_t)best;
        }
        for (int64_t i = 0; i < n; ++i)
            if (newc[i]) {
                cf[i] = 1;
                --left;
            }
        for (int64_t i = 0; i < n; ++i) {
            if (cf[i] != 0) continue;
            for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e)
                if (strong[e] && newc[a->col[e]]) {
                    cf[i] = -1;
                    --left;
                    break;
                }
        }
    }
    free(newc);
    free(mu);
    free(h);
    free(fl);
    free(ti);
    free(tp);
}

/* Extended+i interpolation (De Sterck, Falgout, Nolting & Yang, Numer. Linear Algebra
 * Appl. 15, 2008), without truncation. For an F-point i with strong C set C_i^s and
 * strong F set F_i^s,
 *   Chat_i = C_i^s u (union over k in F_i^s of C_k^s),
 * or, with the "+cc" modification (cc = 1; the interpolation of Sec. 1 and Sec. 6.1),
 *   Chat_i = C_i^s u (union over k in F_i^s with C_k^s n C_i^s empty of C_k^s):
 * an F neighbour that already shares a strong C point with i adds no C points of its
 * own; its connections are spread over Chat_i u {i} by the same formula,
 *   abar_kl = a_kl if sign(a_kl) != sign(a_kk) else 0,
 *   d_k = sum_{l in Chat_i u {i}} abar_kl,
 *   atil_ii = a_ii + sum_{n weak, n not in Chat_i} a_in + sum_{k in F_i^s} a_ik abar_ki / d_k,
 *   w_ij = -(a_ij + sum_{k in F_i^s} a_ik abar_kj / d_k) / atil_ii,   j in Chat_i.
 * Reading where the publication is silent: a k with d_k = 0 is lumped (a_ik added to
 * atil_ii). C-points inject. Coarse points are numbered in fine order. */
static double abar(double akl, double akk) {
    if (akk > 0.0) return akl < 0.0 ? akl : 0.0;
    if (akk < 0.0) return akl > 0.0 ? akl : 0.0;
    return akl != 0.0 ? akl : 0.0;
}

static int32_t *coarse_index(int64_t n, const int8_t *cf, int64_t *nc_out) {
    int32_t *ci = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) ci[i] = (cf[i] == 1) ? (int32_t)nc++ : -1;
    *nc_out = nc;
    return ci;
}

static int in_sorted(const int32_t *arr, int64_t n, int32_t v) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (arr[mid] == v) return 1;
        if (arr[mid] < v) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0;
}

/* 1 when k has a strong C point that is also a strong C point of i */
static int shares_strong_c(const ocsr *a, const uint8_t *strong, const int8_t *cf, int64_t i, int64_t k) {
    for (int64_t f = a->ptr[k]; f < a->ptr[k + 1]; ++f) {
        if (!strong[f] || cf[a->col[f]] != 1) continue;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e)
            if (strong[e] && a->col[e] == a->col[f]) return 1;
    }
    return 0;
}

ocsr *orc_extpi(const ocsr *a, const uint8_t *strong, const int8_t *cf, int cc) {
    int64_t n = a->nrows, nc;
    int32_t *ci = coarse_index(n, cf, &nc);
    int64_t cap = 1024, nnz = 0;
    int32_t *pc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)cap);
    double *pv = (double *)xmalloc(sizeof(double) * (size_t)cap);
    int64_t *pp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    int32_t *hat = NULL;
    double *w = NULL;
    int64_t hcap = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cf[i] == 1) {
            if (nnz + 1 > cap) {
                cap *= 2;
                pc = (int32_t *)realloc(pc, sizeof(int32_t) * (size_t)cap);
                pv = (double *)realloc(pv, sizeof(double) * (size_t)cap);
            }
            pc[nnz] = ci[i];
            pv[nnz] = 1.0;
            ++nnz;
            pp[i + 1] = nnz;
            continue;
        }
        /* collect Chat_i */
        int64_t need = 0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t k = a->col[e];
            need += 1;
            if (cf[k] == -1) need += a->ptr[k + 1] - a->ptr[k];
        }
        if (need > hcap) {
            free(hat);
            free(w);
            hcap = need;
            hat = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)hcap);
            w = (double *)xmalloc(sizeof(double) * (size_t)hcap);
        }
        int64_t nh = 0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t k = a->col[e];
            if (cf[k] == 1) hat[nh++] = (int32_t)k;
            else if (!cc || !shares_strong_c(a, strong, cf, i, k))
                for (int64_t f = a->ptr[k]; f < a->ptr[k + 1]; ++f)
                    if (strong[f] && cf[a->col[f]] == 1) hat[nh++] = a->col[f];
        }
        qsort(hat, (size_t)nh, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t q = 0; q < nh; ++q)
            if (q == 0 || hat[q] != hat[q - 1]) hat[u++] = hat[q];
        nh = u;
        if (nh == 0) {
            pp[i + 1] = nnz;
            continue;
        }
        double aii = 0.0;
        for (int64_t q = 0; q < nh; ++q) w[q] = 0.0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            int32_t j = a->col[e];
            if (j == i) aii = a->val[e];
        }
        double diag = aii;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            int32_t j = a->col[e];
            if (j == i) continue;
            if (in_sorted(hat, nh, j)) {
                for (int64_t q = 0; q < nh; ++q)
                    if (hat[q] == j) w[q] = a->val[e];
            } else if (!strong[e]) {
                diag += a->val[e];
            }
        }
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            if (!strong[e]) continue;
            int64_t k = a->col[e];
            if (cf[k] != -1) continue;
            double aik = a->val[e], akk = 0.0;
            for (int64_t f = a->ptr[k]; f < a->ptr[k + 1]; ++f)
                if (a->col[f] == k) akk = a->val[f];
            double d = 0.0;
            for (int64_t f = a->ptr[k]; f < a->ptr[k + 1]; ++f) {
                int32_t l = a->col[f];
                if (l == k) continue;
                if (l == i || in_sorted(hat, nh, l)) d += abar(a->val[f], akk);
            }
            if (d == 0.0) {
                diag += aik;
                continue;
            }
            for (int64_t f = a->ptr[k]; f < a->ptr[k + 1]; ++f) {
                int32_t l = a->col[f];
                if (l == k) continue;
                double ab = abar(a->val[f], akk);
                if (l == i) diag += aik * ab / d;
                else
                    for (int64_t q = 0; q < nh; ++q)
                        if (hat[q] == l) w[q] += aik * ab / d;
            }
        }
        if (nnz + nh > cap) {
            while (nnz + nh > cap) cap *= 2;
            pc = (int32_t *)realloc(pc, sizeof(int32_t) * (size_t)cap);
            pv = (double *)realloc(pv, sizeof(double) * (size_t)cap);
        }
        for (int64_t q = 0; q < nh; ++q) {
            pc[nnz] = ci[hat[q]];
            pv[nnz] = -w[q] / diag;
            ++nnz;
        }
        pp[i + 1] = nnz;
    }
    free(hat);
    free(w);
    free(ci);
    ocsr *P = (ocsr *)xmalloc(sizeof(ocsr));
    P->nrows = n;
    P->ncols = nc;
    P->nnz = nnz;
    P->ptr = pp;
    P->col = pc;
    P->val = pv;
    return P;
}

ocsr *orc_transpose(const ocsr *a) {
    ocsr *t = csr_alloc(a->ncols, a->nrows, a->nnz);
    for (int64_t e = 0; e < a->nnz; ++e) t->ptr[a->col[e] + 1]++;
    for (int64_t j = 0; j < a->ncols; ++j) t->ptr[j + 1] += t->ptr[j];
    int64_t *fl = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(a->ncols ? a->ncols : 1));
    for (int64_t j = 0; j < a->ncols; ++j) fl[j] = t->ptr[j];
    for (int64_t i = 0; i < a->nrows; ++i)
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            int64_t q = fl[a->col[e]]++;
            t->col[q] = (int32_t)i;
            t->val[q] = a->val[e];
        }
    free(fl);
    return t;
}

/* C = A B, each entry summed in the order of A's row then B's row */
ocsr *orc_spgemm(const ocsr *a, const ocsr *b) {
    int64_t n = a->nrows, m = b->ncols;
    double *acc = (double *)xcalloc((size_t)(m ? m : 1), sizeof(double));
    int64_t *mark = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(m ? m : 1));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
    int32_t *rowc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int64_t cap = 1024, nnz = 0;
    int32_t *cc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)cap);
    double *cv = (double *)xmalloc(sizeof(double) * (size_t)cap);
    int64_t *cp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t nr = 0;
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) {
            int64_t k = a->col[e];
            for (int64_t f = b->ptr[k]; f < b->ptr[k + 1]; ++f) {
                int32_t j = b->col[f];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    rowc[nr++] = j;
                }
                acc[j] += a->val[e] * b->val[f];
            }
        }
        qsort(rowc, (size_t)nr, sizeof(int32_t), cmp_i32);
        if (nnz + nr > cap) {
            while (nnz + nr > cap) cap *= 2;
            cc = (int32_t *)realloc(cc, sizeof(int32_t) * (size_t)cap);
            cv = (double *)realloc(cv, sizeof(double) * (size_t)cap);
        }
        for (int64_t q = 0; q < nr; ++q) {
            cc[nnz] = rowc[q];
            cv[nnz] = acc[rowc[q]];
            ++nnz;
        }
        cp[i + 1] = nnz;
    }
    free(acc);
    free(mark);
    free(rowc);
    ocsr *c = (ocsr *)xmalloc(sizeof(ocsr));
    c->nrows = n;
    c->ncols = m;
    c->nnz = nnz;
    c->ptr = cp;
    c->col = cc;
    c->val = cv;
    return c;
}

/* Galerkin coarse matrix P^T A P (the relation A_H = I_R A_h I_P of Sec. 2, applied on
 * every AMG level) */
ocsr *orc_rap(const ocsr *a, const ocsr *p) {
    ocsr *ap = orc_spgemm(a, p);
    ocsr *r = orc_transpose(p);
    ocsr *c = orc_spgemm(r, ap);
    orc_csr_free(ap);
    orc_csr_free(r);
    return c;
}

/* dense Cholesky factor of the coarsest matrix (plain loops) */
static int cholesky(const ocsr *a, double **out) {
    int64_t n = a->nrows;
    double *L = (double *)xcalloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = a->ptr[i]; e < a->ptr[i + 1]; ++e) L[i * n + a->col[e]] = a->val[e];
    for (int64_t j = 0; j < n; ++j) {
        double s = L[j * n + j];
        for (int64_t q = 0; q < j; ++q) s -= L[j * n + q] * L[j * n + q];
        if (!(s > 0.0)) {
            free(L);
            return -1;
        }
        double d = sqrt(s);
        L[j * n + j] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = L[i * n + j];
            for (int64_t q = 0; q < j; ++q) t -= L[i * n + q] * L[j * n + q];
            L[i * n + j] = t / d;
        }
        for (int64_t i = 0; i < j; ++i) L[i * n + j] = 0.0;
    }
    *out = L;
    return 0;
}

static void chol_solve(const double *L, int64_t n, const double *b, double *x) {
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t q = 0; q < i; ++q) s -= L[i * n + q] * x[q];
        x[i] = s / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t q = i + 1; q < n; ++q) s -= L[q * n + i] * x[q];
        x[i] = s / L[i * n + i];
    }
}

/* ------------------------------------------------------------------------------------
 * 10. Setup: colouring of A_h, then the P1 hierarchy on A_H (Step 1 of Algorithm 2.1
 *     solved approximately by one AMG cycle, Remark 2.1). Coarsening stops at
 *     coarse_size rows, at max_levels, or when PMIS keeps no or all points.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Interpolation truncation (optional; the paper's BoomerAMG settings are not stated):
 * in every row of P, drop the weights with |w| < tf * max|w|, then keep the pmax
 * largest |w| (ties: the lower column first), then scale the kept weights so that the
 * row sum equals the row sum before truncation. tf = 0 and pmax = 0 leave P as it is.
 * Rows of coarse points (one weight 1) are unchanged by construction.
 * ---------------------------------------------------------------------------------- */
ocsr *orc_truncate(const ocsr *p, double tf, int pmax) {
    const int64_t n = p->nrows;
    int64_t *pp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
    int32_t *pc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(p->nnz ? p->nnz : 1));
    double *pv = (double *)xmalloc(sizeof(double) * (size_t)(p->nnz ? p->nnz : 1));
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t lo = p->ptr[i], hi = p->ptr[i + 1];
        double mx = 0.0, sum = 0.0;
        for (int64_t e = lo; e < hi; ++e) {
            mx = fmax(mx, fabs(p->val[e]));
            sum += p->val[e];
        }
        const int64_t start = nnz;
        for (int64_t e = lo; e < hi; ++e) {
            if (tf > 0.0 && fabs(p->val[e]) < tf * mx) continue;
            pc[nnz] = p->col[e];
            pv[nnz] = p->val[e];
            ++nnz;
        }
        if (pmax > 0 && nnz - start > pmax) {
            /* keep the pmax largest |w|: repeated selection, ties to the lower column */
            int64_t cnt = nnz - start;
            int32_t *kc = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)cnt);
            double *kv = (double *)xmalloc(sizeof(double) * (size_t)cnt);
            char *taken = (char *)xcalloc((size_t)cnt, 1);
            for (int q = 0; q < pmax; ++q) {
                int64_t best = -1;
                for (int64_t e = 0; e < cnt; ++e) {
                    if (taken[e]) continue;
                    const double a = fabs(pv[start + e]);
                    if (best < 0 || a > fabs(pv[start + best]) ||
                        (a == fabs(pv[start + best]) && pc[start + e] < pc[start + best]))
                        best = e;
                }
                taken[best] = 1;
            }
            int64_t m = 0;
            for (int64_t e = 0; e < cnt; ++e)
                if (taken[e]) {
                    kc[m] = pc[start + e];
                    kv[m] = pv[start + e];
                    ++m;
                }
            for (int64_t e = 0; e < m; ++e) {
                pc[start + e] = kc[e];
                pv[start + e] = kv[e];
            }
            nnz = start + m;
            free(kc);
            free(kv);
            free(taken);
        }
        double kept = 0.0;
        for (int64_t e = start; e < nnz; ++e) kept += pv[e];
        if (nnz - start < hi - lo && kept != 0.0) {
            const double scale = sum / kept;
            for (int64_t e = start; e < nnz; ++e) pv[e] *= scale;
        }
        pp[i + 1] = nnz;
    }
    ocsr *t = orc_csr_new(n, p->ncols, nnz, pp, pc, pv);
    free(pp);
    free(pc);
    free(pv);
    return t;
}

/* Changes the iteration cap of the solve without rebuilding the preconditioner (a solve
 * from x0 stopped after j iterations leaves the iterate x_j of Algorithm 2.1's outer
 * iteration, used to compare iterates one by one). */
int orc_set_max_iter(oproblem *P, int max_iter) {
    if (!P->have_setup || max_iter < 1) return 1;
    P->o.max_iter = max_iter;
    return 0;
}

int orc_setup(oproblem *P, const oopts *o) {
    free_levels(P);
    P->o = *o;
    P->colour_h = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(P->nh ? P->nh : 1));
    P->ncolour_h = orc_colour_jp(P->nh, P->Ah->ptr, P->Ah->col, stream_colour(o->seed, 0),
                                 P->colour_h);
    P->l1_h = l1_norms(P->Ah);
    int maxl = o->max_levels < 1 ? 1 : (o->max_levels > MAXLEV ? MAXLEV : o->max_levels);
    /* mode 2: plain AMG, the hierarchy starts from A_h itself (the comparison method of
       Sec. 1 and Sec. 6.2); otherwise from the P1 matrix A_H of the auxiliary space */
    ocsr *A = o->mode == 2 ? P->Ah : P->AH;
    int l = 0;
    for (;;) {
        olevel *L = &P->lev[l];
        L->A = A;
        L->colour = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(A->nrows ? A->nrows : 1));
        L->ncolour = orc_colour_jp(A->nrows, A->ptr, A->col, stream_colour(o->seed, 1 + l),
                                   L->colour);
        L->l1 = l1_norms(A);
        P->nlev = l + 1;
        if (A->nrows <= o->coarse_size || l + 1 >= maxl) break;
        L->strong = (uint8_t *)xmalloc((size_t)(A->nnz ? A->nnz : 1));
        orc_strength(A, o->theta, L->strong);
        L->cf = (int8_t *)xmalloc((size_t)(A->nrows ? A->nrows : 1));
        orc_pmis(A, L->strong, stream_pmis(o->seed, l), L->cf);
        int64_t nc = 0;
        for (int64_t i = 0; i < A->nrows; ++i) nc += (L->cf[i] == 1);
        if (nc == 0 || nc == A->nrows) break;
        L->P = orc_extpi(A, L->strong, L->cf, o->interp_cc);
        if (o->interp_trunc > 0 || o->interp_pmax > 0) {
            ocsr *Pt = orc_truncate(L->P, o->interp_trunc / 1000.0, o->interp_pmax);
            orc_csr_free(L->P);
            L->P = Pt;
        }
        L->R = orc_transpose(L->P);
        A = orc_rap(A, L->P);
        ++l;
    }
    olevel *Lc = &P->lev[P->nlev - 1];
    P->nc = Lc->A->nrows;
    if (P->nc > 8192) return -2;
    if (cholesky(Lc->A, &P->chol) != 0) return -3;
    P->have_setup = 1;
    return 0;
}

int orc_levels(const oproblem *P) { return P->nlev; }
const ocsr *orc_level_matrix(const oproblem *P, int l, int which) {
    return which == 0 ? P->lev[l].A : P->lev[l].P;
}
void orc_level_info(const oproblem *P, int l, int64_t *o) {
    const olevel *L = &P->lev[l];
    o[0] = L->A->nrows;
    o[1] = L->A->nnz;
    o[2] = L->ncolour;
    o[3] = L->P ? L->P->ncols : -1;
}
void orc_level_cf(const oproblem *P, int l, int8_t *cf) {
    memcpy(cf, P->lev[l].cf, (size_t)P->lev[l].A->nrows);
}
void orc_level_strong(const oproblem *P, int l, uint8_t *s) {
    memcpy(s, P->lev[l].strong, (size_t)P->lev[l].A->nnz);
}
void orc_level_colour(const oproblem *P, int l, int32_t *c) {
    memcpy(c, P->lev[l].colour, sizeof(int32_t) * (size_t)P->lev[l].A->nrows);
}
void orc_fine_colour(const oproblem *P, int32_t *c) {
    memcpy(c, P->colour_h, sizeof(int32_t) * (size_t)P->nh);
}

/* One V(1,1)-cycle on level l: forward GS from zero (or an l1-Jacobi step), residual,
 * restriction by P^T, recursion, prolongation, backward GS (or l1-Jacobi); the
 * coarsest level is solved by the Cholesky factor. */
static void vcycle_level(oproblem *P, int l, const double *b, double *x) {
    olevel *L = &P->lev[l];
    int64_t n = L->A->nrows;
    if (l == P->nlev - 1) {
        chol_solve(P->chol, n, b, x);
        return;
    }
    int jac = P->o.level_smoother == 1;
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    if (jac) l1_step(L->A, L->l1, b, x, 1);
    else gs_sweep(L->A, L->colour, L->ncolour, 1, b, x);
    double *r = (double *)xmalloc(sizeof(double) * (size_t)n);
    orc_spmv(L->A, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    int64_t nc = L->P->ncols;
    double *bc = (double *)xmalloc(sizeof(double) * (size_t)(nc ? nc : 1));
    double *xc = (double *)xmalloc(sizeof(double) * (size_t)(nc ? nc : 1));
    orc_spmv(L->R, r, bc);
    vcycle_level(P, l + 1, bc, xc);
    double *px = r; /* reuse */
    orc_spmv(L->P, xc, px);
    for (int64_t i = 0; i < n; ++i) x[i] += px[i];
    if (jac) l1_step(L->A, L->l1, b, x, 0);
    else gs_sweep(L->A, L->colour, L->ncolour, 0, b, x);
    free(bc);
    free(xc);
    free(r);
}

void orc_vcycle(oproblem *P, const double *b, double *x) { vcycle_level(P, 0, b, x); }

/* the P_k smoother S_k applied to r from a zero guess */
void orc_smoother(oproblem *P, const double *r, double *z) {
    if (P->o.smoother == 1) {
        l1_step(P->Ah, P->l1_h, r, z, 1);
    } else {
        orc_sgs(P->Ah, P->colour_h, P->ncolour_h, r, z);
    }
}

/* ------------------------------------------------------------------------------------
 * 11. The preconditioner.
 *   additive (Xu's auxiliary space form):  z = S_k r + I_P V(I_R r)
 *   multiplicative (Algorithm 2.1 with pre-smoothing, Remark 2.1):
 *       z1 = forward GS on A_h z = r from 0;  z2 = z1 + I_P V(I_R (r - A_h z1));
 *       z  = backward GS sweep on A_h z = r from z2
 *   (with the l1-Jacobi smoother the two GS sweeps become l1-Jacobi steps).
 * ---------------------------------------------------------------------------------- */
void orc_apply_prec(oproblem *P, const double *r, double *z) {
    int64_t nh = P->nh, nH = P->nH;
    double *rH = (double *)xmalloc(sizeof(double) * (size_t)(nH ? nH : 1));
    double *wH = (double *)xmalloc(sizeof(double) * (size_t)(nH ? nH : 1));
    double *t = (double *)xmalloc(sizeof(double) * (size_t)(nh ? nh : 1));
    if (P->o.mode == 2) {
        /* plain AMG: one V-cycle on the hierarchy of A_h */
        orc_vcycle(P, r, z);
    } else if (P->o.mode == 0) {
        orc_smoother(P, r, z);
        orc_spmv(P->PiT, r, rH);
        orc_vcycle(P, rH, wH);
        orc_spmv(P->Pi, wH, t);
        for (int64_t i = 0; i < nh; ++i) z[i] += t[i];
    } else {
        int jac = P->o.smoother == 1;
        for (int64_t i = 0; i < nh; ++i) z[i] = 0.0;
        if (jac) l1_step(P->Ah, P->l1_h, r, z, 1);
        else gs_sweep(P->Ah, P->colour_h, P->ncolour_h, 1, r, z);
        orc_spmv(P->Ah, z, t);
        for (int64_t i = 0; i < nh; ++i) t[i] = r[i] - t[i];
        orc_spmv(P->PiT, t, rH);
        orc_vcycle(P, rH, wH);
        orc_spmv(P->Pi, wH, t);
        for (int64_t i = 0; i < nh; ++i) z[i] += t[i];
        if (jac) l1_step(P->Ah, P->l1_h, r, z, 0);
        else gs_sweep(P->Ah, P->colour_h, P->ncolour_h, 0, r, z);
    }
    free(t);
    free(wH);
    free(rH);
}

/* ------------------------------------------------------------------------------------
 * 12. Preconditioned conjugate gradients on Eq. (7) with the preconditioner above
 *     (the paper uses FGMRES, Sec. 6.2). Stops when ||r_k||_2 <= tol ||r_0||_2 on the
 *     recurrence residual; then checks the true residual ||b - A x|| / ||r_0|| and, if
 *     it is above tol, restarts once from the current x. Flexible CG (Notay's FCG(1))
 *     uses beta = (z_new, r_new - r_old) / (z_old, r_old).
 *     Returns 0 converged, 1 not converged in max_iter, 2 breakdown (p^T A p <= 0).
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * 12b. FGMRES(m): the outer iteration of the paper's experiments (Sec. 6.2), Saad's
 *      flexible GMRES with right preconditioning.
 *        r0 = b - A x0, beta = ||r0||, v_1 = r0 / beta, g = beta e_1
 *        for j = 1..m:  z_j = B v_j;  w = A z_j;
 *                       h_ij = (w, v_i) and w -= sum_i h_ij v_i for i <= j, twice
 *                       (classical Gram-Schmidt with one reorthogonalisation; the
 *                       second pass's coefficients are added to h_ij);
 *                       h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j};
 *                       rotate column j of H by the earlier Givens rotations, choose
 *                       the rotation that zeroes h_{j+1,j}, apply it to g;
 *                       |g_{j+1}| = ||b - A x_j|| (in exact arithmetic); stop when it is
 *                       <= tol ||b - A x_initial|| or at max_iter total steps
 *        y = H(1:k,1:k)^{-1} g(1:k) (upper triangular), x += sum_j y_j z_j
 *      then restart from the true residual until converged. A zero h_{j+1,j} ends the
 *      cycle (the Krylov space holds the solution).
 * ---------------------------------------------------------------------------------- */
typedef void (*orc_apply_fn)(void *ctx, const double *x, double *y);

static int fgmres_core(int64_t n, orc_apply_fn op, orc_apply_fn prec, void *ctx, int restart, double tol,
                       int max_iter, const double *b, double *x, double *hist, int hist_cap, int *iters_out,
                       double *true_rel_out) {
    const int m = restart > 0 ? restart : 30;
    double *V = (double *)xmalloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
    double *Z = (double *)xmalloc(sizeof(double) * (size_t)n * (size_t)m);
    double *w = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *H = (double *)xmalloc(sizeof(double) * (size_t)(m + 1) * (size_t)m); /* H[i*m + j] */
    double *cs = (double *)xmalloc(sizeof(double) * (size_t)m);
    double *sn = (double *)xmalloc(sizeof(double) * (size_t)m);
    double *g = (double *)xmalloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)xmalloc(sizeof(double) * (size_t)m);
    double *hc = (double *)xmalloc(sizeof(double) * (size_t)(m + 1));
    int it = 0, status = 1;
    op(ctx, x, w);
    for (int64_t i = 0; i < n; ++i) V[i] = b[i] - w[i];
    const double r0 = sqrt(dot(n, V, V));
    if (hist && hist_cap > 0) hist[0] = r0;
    double beta = r0;
    if (r0 == 0.0) status = 0;
    while (status == 1) {
        for (int64_t i = 0; i < n; ++i) V[i] /= beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0; /* Arnoldi steps of this cycle */
        int converged = 0;
        for (int j = 0; j < m && it < max_iter; ++j) {
            double *vj = V + (size_t)j * (size_t)n, *zj = Z + (size_t)j * (size_t)n;
            prec(ctx, vj, zj);
            op(ctx, zj, w);
            for (int i = 0; i <= j; ++i) H[i * m + j] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = 0; i <= j; ++i) hc[i] = dot(n, w, V + (size_t)i * (size_t)n);
                for (int i = 0; i <= j; ++i) {
                    const double *vi = V + (size_t)i * (size_t)n;
                    for (int64_t q = 0; q < n; ++q) w[q] -= hc[i] * vi[q];
                    H[i * m + j] += hc[i];
                }
            }
            const double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            double *vn = V + (size_t)(j + 1) * (size_t)n;
            if (hn > 0.0)
                for (int64_t q = 0; q < n; ++q) vn[q] = w[q] / hn;
            /* earlier rotations on column j, then the new one */
            for (int i = 0; i < j; ++i) {
                const double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            const double a = H[j * m + j], c = H[(j + 1) * m + j];
            const double d = sqrt(a * a + c * c);
            cs[j] = d > 0.0 ? a / d : 1.0;
            sn[j] = d > 0.0 ? c / d : 0.0;
            H[j * m + j] = d;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            const double est = fabs(g[j + 1]);
            if (hist && it < hist_cap) hist[it] = est;
            if (est <= tol * r0 || hn == 0.0) {
                converged = 1;
                break;
            }
        }
        /* x += Z y with H(1:k,1:k) y = g(1:k) */
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        for (int l = 0; l < k; ++l) {
            const double *zl = Z + (size_t)l * (size_t)n;
            for (int64_t q = 0; q < n; ++q) x[q] += y[l] * zl[q];
        }
        /* restart from the true residual */
        op(ctx, x, w);
        for (int64_t i = 0; i < n; ++i) V[i] = b[i] - w[i];
        beta = sqrt(dot(n, V, V));
        if (beta <= tol * r0) {
            status = 0;
            break;
        }
        if (it >= max_iter) break;
        (void)converged;
    }
    if (true_rel_out) *true_rel_out = r0 > 0.0 ? beta / r0 : 0.0;
    if (iters_out) *iters_out = it;
    free(V);
    free(Z);
    free(w);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(hc);
    return status;
}

static void poisson_op(void *ctx, const double *x, double *y) { orc_spmv(((oproblem *)ctx)->Ah, x, y); }
static void poisson_prec(void *ctx, const double *r, double *z) { orc_apply_prec((oproblem *)ctx, r, z); }

int orc_fgmres(oproblem *P, const double *b, double *x, double *hist, int hist_cap, int *iters_out,
               double *true_rel_out) {
    return fgmres_core(P->nh, poisson_op, poisson_prec, P, P->o.restart, P->o.tol, P->o.max_iter, b, x, hist,
                       hist_cap, iters_out, true_rel_out);
}

int orc_solve(oproblem *P, const double *b, double *x, double *hist, int hist_cap,
              int *iters_out, double *true_rel_out) {
    if (P->o.krylov == 1) return orc_fgmres(P, b, x, hist, hist_cap, iters_out, true_rel_out);
    int64_t n = P->nh;
    double *r = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *z = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *p = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *q = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *rold = (double *)xmalloc(sizeof(double) * (size_t)n);
    int it = 0, status = 1, restarts = 0;
    orc_spmv(P->Ah, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double r0 = sqrt(dot(n, r, r));
    if (hist && hist_cap > 0) hist[0] = r0;
    double rn = r0;
    if (r0 == 0.0) status = 0;
    while (status == 1) {
        orc_apply_prec(P, r, z);
        for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        double rho = dot(n, r, z);
        while (it < P->o.max_iter) {
            orc_spmv(P->Ah, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0)) {
                status = 2;
                break;
            }
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) {
                rold[i] = r[i];
                x[i] += alpha * p[i];
                r[i] -= alpha * q[i];
            }
            ++it;
            rn = sqrt(dot(n, r, r));
            if (hist && it < hist_cap) hist[it] = rn;
            if (rn <= P->o.tol * r0) {
                status = 0;
                break;
            }
            orc_apply_prec(P, r, z);
            double rho_new = dot(n, r, z), beta;
            if (P->o.flexible) {
                double s = 0.0;
                for (int64_t i = 0; i < n; ++i) s += z[i] * (r[i] - rold[i]);
                beta = s / rho;
            } else {
                beta = rho_new / rho;
            }
            rho = rho_new;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        if (status != 0) break;
        /* true residual check, one restart */
        orc_spmv(P->Ah, x, q);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        double tr = sqrt(dot(n, r, r));
        if (tr <= P->o.tol * r0 || restarts >= 1 || it >= P->o.max_iter) break;
        ++restarts;
        status = 1;
    }
    orc_spmv(P->Ah, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    if (true_rel_out) *true_rel_out = r0 > 0.0 ? sqrt(dot(n, r, r)) / r0 : 0.0;
    if (iters_out) *iters_out = it;
    free(r);
    free(z);
    free(p);
    free(q);
    free(rold);
    return status;
}

/* ------------------------------------------------------------------------------------
 * 14. Stokes with Taylor-Hood P_k - P_{k-1} elements (Sec. 5): F = [A B^T; B 0] with A
 *     the block diagonal of three copies of the Dirichlet P_k Laplacian A_h (velocity
 *     unknowns component-major: component c, unknown j -> c n_h + j), B the discrete
 *     divergence -div_h: B_{q,(c,j)} = -int psi_q d_c phi_j (pressure on all P_{k-1}
 *     nodes), M_p the pressure mass matrix. The block upper-triangular preconditioner
 *     Q_t = [A B^T; 0 -S]^{-1} (Eq. 5.4) with A^{-1} ~ the auxiliary-space preconditioner
 *     per component and S ~ M_p, solved by mp_iters steps of CG with the diagonal of M_p
 *     as preconditioner:  z_p = -M_p^{-1} r_p,  z_u = B_aux (r_u - B^T z_p).
 *     Element integrals exactly by monomial integration on the reference tetrahedron.
 * ---------------------------------------------------------------------------------- */
struct ostokes {
    oproblem *U, *P;  /* velocity space (degree k, Dirichlet), pressure space (k-1, all nodes) */
    int64_t nh, np, n;
    ocsr *B, *BT, *M;
    double *mdiag;
    int mp_iters;
};

/* psi_m of degree k as monomials in lambda: coefficient prod_a c_a(e_a) */
static void phi_terms(int k, const int32_t *m, dterms *t) {
    double cf[4][8];
    for (int b = 0; b < 4; ++b) lag_factor(k, m[b], cf[b]);
    t->n = 0;
    for (int e0 = 0; e0 <= m[0]; ++e0)
        for (int e1 = 0; e1 <= m[1]; ++e1)
            for (int e2 = 0; e2 <= m[2]; ++e2)
                for (int e3 = 0; e3 <= m[3]; ++e3) {
                    int ee[4] = {e0, e1, e2, e3};
                    double c = 1.0;
                    for (int b = 0; b < 4; ++b) c *= cf[b][ee[b]];
                    if (c == 0.0) continue;
                    int q = t->n++;
                    for (int b = 0; b < 4; ++b) t->e[q][b] = ee[b];
                    t->c[q] = c;
                }
}

static double term_product_integral(const dterms *a, const dterms *b) {
    double s = 0.0;
    for (int p = 0; p < a->n; ++p)
        for (int q = 0; q < b->n; ++q) {
            int g[4];
            for (int c = 0; c < 4; ++c) g[c] = a->e[p][c] + b->e[q][c];
            s += a->c[p] * b->c[q] * mono_int(g);
        }
    return s;
}

/* gradients of the barycentric coordinates (rows) and |T| */
static double tet_grads(const double *x, double gl[4][3]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int c = 0; c < 3; ++c) {
        gl[1][c] = inv[0][c];
        gl[2][c] = inv[1][c];
        gl[3][c] = inv[2][c];
        gl[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
    }
    return det / 6.0;
}

typedef struct {
    int64_t r, c, seq;
    double v;
} otrip;

static int cmp_trip(const void *a, const void *b) {
    const otrip *x = (const otrip *)a, *y = (const otrip *)b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

/* CSR from triplets; duplicates summed in the order they were added */
static ocsr *csr_from_trips(otrip *t, int64_t nt, int64_t nrows, int64_t ncols) {
    qsort(t, (size_t)nt, sizeof(otrip), cmp_trip);
    int64_t *ptr = (int64_t *)xcalloc((size_t)nrows + 1, sizeof(int64_t));
    int32_t *col = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(nt ? nt : 1));
    double *val = (double *)xmalloc(sizeof(double) * (size_t)(nt ? nt : 1));
    int64_t nnz = 0;
    for (int64_t i = 0; i < nt;) {
        int64_t j = i;
        double s = 0.0;
        while (j < nt && t[j].r == t[i].r && t[j].c == t[i].c) s += t[j++].v;
        col[nnz] = (int32_t)t[i].c;
        val[nnz] = s;
        ++nnz;
        ptr[t[i].r + 1]++;
        i = j;
    }
    for (int64_t r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
    ocsr *a = orc_csr_new(nrows, ncols, nnz, ptr, col, val);
    free(ptr);
    free(col);
    free(val);
    return a;
}

ostokes *orc_stokes_create(oproblem *U, oproblem *Pp, int mp_iters) {
    if (!U || !Pp || U->k < 2 || Pp->k != U->k - 1 || Pp->dirichlet || U->nt != Pp->nt) return NULL;
    ostokes *S = (ostokes *)xcalloc(1, sizeof(ostokes));
    S->U = U;
    S->P = Pp;
    S->nh = U->nh;
    S->np = Pp->nh;
    S->n = 3 * S->nh + S->np;
    S->mp_iters = mp_iters;
    const int nu = U->nloc, npl = Pp->nloc;
    /* reference tensors: R[a][m][n] = (1/|T|) int psi_m dphi_n/dlambda_a,
       Mr[m][m'] = (1/|T|) int psi_m psi_m' */
    dterms *tp = (dterms *)xmalloc(sizeof(dterms) * (size_t)npl);
    dterms *tu = (dterms *)xmalloc(sizeof(dterms) * 4 * (size_t)nu);
    for (int m = 0; m < npl; ++m) phi_terms(Pp->k, Pp->mi[m], &tp[m]);
    for (int n = 0; n < nu; ++n)
        for (int a = 0; a < 4; ++a) dphi_terms(U->k, U->mi[n], a, &tu[n * 4 + a]);
    double *R = (double *)xmalloc(sizeof(double) * 4 * (size_t)npl * (size_t)nu);
    double *Mr = (double *)xmalloc(sizeof(double) * (size_t)npl * (size_t)npl);
    for (int a = 0; a < 4; ++a)
        for (int m = 0; m < npl; ++m)
            for (int n = 0; n < nu; ++n) R[(a * npl + m) * nu + n] = term_product_integral(&tp[m], &tu[n * 4 + a]);
    for (int m = 0; m < npl; ++m)
        for (int q = 0; q < npl; ++q) Mr[m * npl + q] = term_product_integral(&tp[m], &tp[q]);
    int64_t capB = U->nt * (int64_t)npl * 3 * nu, capM = U->nt * (int64_t)npl * npl;
    otrip *tb = (otrip *)xmalloc(sizeof(otrip) * (size_t)capB);
    otrip *tm = (otrip *)xmalloc(sizeof(otrip) * (size_t)capM);
    int64_t nb = 0, nm = 0;
    for (int64_t t = 0; t < U->nt; ++t) {
        double x[12], gl[4][3];
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) x[3 * v + c] = U->xyz[3 * (int64_t)U->tets[4 * t + v] + c];
        const double vol = tet_grads(x, gl);
        for (int m = 0; m < npl; ++m) {
            const int64_t q = Pp->elem_dof[t * npl + m];
            for (int n = 0; n < nu; ++n) {
                const int64_t j = U->elem_dof[t * nu + n];
                if (j < 0) continue;
                for (int c = 0; c < 3; ++c) {
                    double s = 0.0;
                    for (int a = 0; a < 4; ++a) s += gl[a][c] * R[(a * npl + m) * nu + n];
                    tb[nb] = (otrip){q, c * S->nh + j, nb, -vol * s};
                    ++nb;
                }
            }
            for (int m2 = 0; m2 < npl; ++m2) {
                tm[nm] = (otrip){q, Pp->elem_dof[t * npl + m2], nm, vol * Mr[m * npl + m2]};
                ++nm;
            }
        }
    }
    S->B = csr_from_trips(tb, nb, S->np, 3 * S->nh);
    S->M = csr_from_trips(tm, nm, S->np, S->np);
    S->BT = orc_transpose(S->B);
    S->mdiag = (double *)xmalloc(sizeof(double) * (size_t)S->np);
    for (int64_t i = 0; i < S->np; ++i)
        for (int64_t e = S->M->ptr[i]; e < S->M->ptr[i + 1]; ++e)
            if (S->M->col[e] == i) S->mdiag[i] = S->M->val[e];
    free(tb);
    free(tm);
    free(R);
    free(Mr);
    free(tp);
    free(tu);
    return S;
}

void orc_stokes_free(ostokes *S) {
    if (!S) return;
    orc_csr_free(S->B);
    orc_csr_free(S->BT);
    orc_csr_free(S->M);
    free(S->mdiag);
    free(S);
}

void orc_stokes_sizes(const ostokes *S, int64_t *out3) {
    out3[0] = S->nh;
    out3[1] = S->np;
    out3[2] = S->n;
}

const ocsr *orc_stokes_matrix(const ostokes *S, int which) {
    return which == 0 ? S->B : which == 1 ? S->BT : S->M;
}

/* y = F x */
void orc_stokes_apply(ostokes *S, const double *x, double *y) {
    const int64_t nh = S->nh, nu = 3 * nh;
    double *t = (double *)xmalloc(sizeof(double) * (size_t)(nu ? nu : 1));
    for (int c = 0; c < 3; ++c) orc_spmv(S->U->Ah, x + c * nh, y + c * nh);
    orc_spmv(S->BT, x + nu, t);
    for (int64_t i = 0; i < nu; ++i) y[i] += t[i];
    orc_spmv(S->B, x, y + nu);
    free(t);
}

/* z = Q_t r */
void orc_stokes_prec(ostokes *S, const double *r, double *z) {
    const int64_t nh = S->nh, nu = 3 * nh, np = S->np;
    double *xp = (double *)xcalloc((size_t)(np ? np : 1), sizeof(double));
    double *rr = (double *)xmalloc(sizeof(double) * (size_t)(np ? np : 1));
    double *zz = (double *)xmalloc(sizeof(double) * (size_t)(np ? np : 1));
    double *pp = (double *)xmalloc(sizeof(double) * (size_t)(np ? np : 1));
    double *qq = (double *)xmalloc(sizeof(double) * (size_t)(np ? np : 1));
    /* M_p x = r_p by CG with the diagonal of M_p, mp_iters steps from zero */
    for (int64_t i = 0; i < np; ++i) {
        rr[i] = r[nu + i];
        zz[i] = rr[i] / S->mdiag[i];
        pp[i] = zz[i];
    }
    double rho = dot(np, rr, zz);
    for (int it = 0; it < S->mp_iters && rho != 0.0; ++it) {
        orc_spmv(S->M, pp, qq);
        const double alpha = rho / dot(np, pp, qq);
        for (int64_t i = 0; i < np; ++i) {
            xp[i] += alpha * pp[i];
            rr[i] -= alpha * qq[i];
            zz[i] = rr[i] / S->mdiag[i];
        }
        const double rho2 = dot(np, rr, zz);
        const double beta = rho2 / rho;
        rho = rho2;
        for (int64_t i = 0; i < np; ++i) pp[i] = zz[i] + beta * pp[i];
    }
    for (int64_t i = 0; i < np; ++i) z[nu + i] = -xp[i];
    /* z_u = B_aux (r_u - B^T z_p), component by component */
    double *t = (double *)xmalloc(sizeof(double) * (size_t)(nu ? nu : 1));
    orc_spmv(S->BT, z + nu, t);
    for (int64_t i = 0; i < nu; ++i) t[i] = r[i] - t[i];
    for (int c = 0; c < 3; ++c) orc_apply_prec(S->U, t + c * nh, z + c * nh);
    free(t);
    free(xp);
    free(rr);
    free(zz);
    free(pp);
    free(qq);
}

static void stokes_op(void *ctx, const double *x, double *y) { orc_stokes_apply((ostokes *)ctx, x, y); }
static void stokes_pc(void *ctx, const double *r, double *z) { orc_stokes_prec((ostokes *)ctx, r, z); }

/* FGMRES(restart) on F x = b with Q_t (the velocity preconditioner needs orc_setup on U) */
int orc_stokes_solve(ostokes *S, const double *b, double *x, int restart, double tol, int max_iter, double *hist,
                     int hist_cap, int *iters_out, double *true_rel_out) {
    return fgmres_core(S->n, stokes_op, stokes_pc, S, restart, tol, max_iter, b, x, hist, hist_cap, iters_out,
                       true_rel_out);
}

/* ------------------------------------------------------------------------------------
 * 13. Adjoint gradient: with A(kappa) u = b and L(u), dL/dkappa_e = -lambda_e^T Khat_e u_e
 *     where A lambda = dL/du and Khat_e is the element stiffness with kappa = 1 (the
 *     element matrix of Eq. (7) is linear in kappa_e). Boundary values are zero.
 * ---------------------------------------------------------------------------------- */
void orc_grad_kappa(const oproblem *P, const double *u, const double *lam, double *g) {
    int nl = P->nloc;
    double *K = (double *)xmalloc(sizeof(double) * (size_t)nl * (size_t)nl);
    for (int64_t t = 0; t < P->nt; ++t) {
        double x12[12], G[4][4];
        tet_coords(P, t, x12);
        double vol = tet_geom(x12, G);
        element_matrix(nl, P->S, 1.0, vol, G, K);
        double s = 0.0;
        for (int m = 0; m < nl; ++m) {
            int32_t i = P->elem_dof[t * nl + m];
            if (i < 0) continue;
            double km = 0.0;
            for (int n = 0; n < nl; ++n) {
                int32_t j = P->elem_dof[t * nl + n];
                if (j < 0) continue;
                km += K[m * nl + n] * u[j];
            }
            s += lam[i] * km;
        }
        g[t] = -s;
    }
    free(K);
}

/* ||u_exact - u_h||_{L2} for the manufactured sine solution, degree 2k+5 quadrature */
double orc_l2_error_sine(const oproblem *P, const double *u) {
    int nl = P->nloc;
    double lam[4 * 1024], w[1024];
    int nq = orc_gm_rule(P->k + 2, lam, w, 1024);
    double *phiq = (double *)xmalloc(sizeof(double) * (size_t)(nq * nl));
    for (int q = 0; q < nq; ++q) orc_basis_eval(P->k, &lam[4 * q], &phiq[q * nl]);
    double err = 0.0;
    for (int64_t t = 0; t < P->nt; ++t) {
        double x12[12], G[4][4];
        tet_coords(P, t, x12);
        double vol = tet_geom(x12, G);
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) {
            double x[3];
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int a = 0; a < 4; ++a) v += lam[4 * q + a] * x12[3 * a + c];
                x[c] = v;
            }
            double uh = 0.0;
            for (int m = 0; m < nl; ++m) {
                int32_t i = P->elem_dof[t * nl + m];
                if (i >= 0) uh += u[i] * phiq[q * nl + m];
            }
            double d = exact_sine(x) - uh;
            acc += w[q] * d * d;
        }
        err += 6.0 * vol * acc;
    }
    free(phiq);
    return sqrt(err);
}
