// mesh.cpp -- host side of assembly: the P_k node numbering, element-to-unknown maps,
// sparsity patterns of A_h and A_H, and I_P (Eq. 10), plus the reference-element
// tables (Lagrange basis on evenly spaced nodes, Sec. 2) that the device kernels use.
//
// Numbering convention (the paper's Fig. 1 is not part of its text): all vertices by
// id, then edges in (low, high) vertex order with their k-1 nodes running away from the
// low vertex, then faces in sorted-triple order with their nodes in ascending
// multi-index order over the sorted vertices, then element interiors by element id.
// Nodes on boundary faces are Dirichlet nodes (Eq. 1) and are dropped; the remaining
// unknowns keep the order above.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

#include "internal.h"

namespace pk {

int nloc_of(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }

void ref_nodes(int k, std::vector<int> &m4) {
    m4.clear();
    for (int a = 0; a <= k; ++a)
        for (int b = 0; a + b <= k; ++b)
            for (int c = 0; a + b + c <= k; ++c) {
                m4.push_back(a);
                m4.push_back(b);
                m4.push_back(c);
                m4.push_back(k - a - b - c);
            }
}

namespace {

template <class F>
void parallel_for(int64_t n, F fn) {
    unsigned hw = std::thread::hardware_concurrency();
    int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
    if (n < 4096) nth = 1;
    if (nth == 1) {
        fn(0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nth - 1) / nth;
    for (int t = 0; t < nth; ++t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        th.emplace_back([=] { fn(b, e, t); });
    }
    for (auto &x : th) x.join();
}

// value and derivative of p_j(t) = prod_{i<j} (k t - i)/(i+1)
void lag1d(int k, int j, double t, double &v, double &dv) {
    v = 1.0;
    dv = 0.0;
    for (int i = 0; i < j; ++i) {
        double f = ((double)k * t - (double)i) / (double)(i + 1);
        double df = (double)k / (double)(i + 1);
        dv = dv * f + v * df;
        v = v * f;
    }
}

// rank of a composition of k (all parts >= 1) among all such, ascending lexicographic
int composition_rank(int k, const int *p, int parts) {
    std::vector<int> cur(parts);
    int rank = 0;
    // enumerate lexicographically with a simple odometer
    std::function<bool(int, int)> rec;
    bool found = false;
    rec = [&](int idx, int left) -> bool {
        if (idx == parts - 1) {
            if (left < 1) return false;
            cur[idx] = left;
            bool eq = true;
            for (int q = 0; q < parts; ++q) eq = eq && (cur[q] == p[q]);
            if (eq) {
                found = true;
                return true;
            }
            ++rank;
            return false;
        }
        for (int v = 1; v <= left - (parts - 1 - idx); ++v) {
            cur[idx] = v;
            if (rec(idx + 1, left - v)) return true;
        }
        return false;
    };
    rec(0, k);
    return found ? rank : -1;
}

}  // namespace

void basis_values(int k, const double *lam, double *phi) {
    std::vector<int> m4;
    ref_nodes(k, m4);
    int nl = nloc_of(k);
    for (int m = 0; m < nl; ++m) {
        double v = 1.0;
        for (int a = 0; a < 4; ++a) {
            double va, da;
            lag1d(k, m4[4 * m + a], lam[a], va, da);
            v *= va;
        }
        phi[m] = v;
    }
}

// Grundmann & Moeller (1978) rule of degree 2s+1 on the reference simplex (volume 1/6):
// weight (-1)^i 2^{-2s} (d+3-2i)^d / (i! (d+3-i)!) at the points (2 beta + 1)/(d+3-2i),
// |beta| = s - i, i = 0..s.
void gm_rule(int s, std::vector<double> &lam, std::vector<double> &w) {
    lam.clear();
    w.clear();
    const int d = 2 * s + 1;
    auto fac = [](int n) {
        double f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        return f;
    };
    for (int i = 0; i <= s; ++i) {
        double wi = std::ldexp(1.0, -2 * s) * std::pow((double)(d + 3 - 2 * i), d) /
                    (fac(i) * fac(d + 3 - i));
        if (i & 1) wi = -wi;
        const int r = s - i;
        const double den = (double)(d + 3 - 2 * i);
        for (int b0 = 0; b0 <= r; ++b0)
            for (int b1 = 0; b0 + b1 <= r; ++b1)
                for (int b2 = 0; b0 + b1 + b2 <= r; ++b2) {
                    int b3 = r - b0 - b1 - b2;
                    lam.push_back((2 * b0 + 1) / den);
                    lam.push_back((2 * b1 + 1) / den);
                    lam.push_back((2 * b2 + 1) / den);
                    lam.push_back((2 * b3 + 1) / den);
                    w.push_back(wi);
                }
    }
}

// S[a][b][m][n] = (1/|T|) int_T (d phi_m / d lambda_a)(d phi_n / d lambda_b): the
// integrand has degree 2k-2 in the barycentric coordinates, so a Grundmann-Moeller rule
// of degree >= 2k-1 integrates it exactly (up to rounding).
void reference_tensors(int k, std::vector<double> &S) {
    const int nl = nloc_of(k);
    std::vector<int> m4;
    ref_nodes(k, m4);
    std::vector<double> lam, w;
    gm_rule(std::max(k, 1), lam, w);  // degree 2k+1 >= 2k-2
    const int nq = (int)w.size();
    // dphi[q][a][m]
    std::vector<double> dphi((size_t)nq * 4 * nl);
    for (int q = 0; q < nq; ++q)
        for (int m = 0; m < nl; ++m) {
            double v[4], d[4];
            for (int a = 0; a < 4; ++a) lag1d(k, m4[4 * m + a], lam[4 * q + a], v[a], d[a]);
            for (int a = 0; a < 4; ++a) {
                double prod = d[a];
                for (int b = 0; b < 4; ++b)
                    if (b != a) prod *= v[b];
                dphi[((size_t)q * 4 + a) * nl + m] = prod;
            }
        }
    S.assign((size_t)16 * nl * nl, 0.0);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int m = 0; m < nl; ++m)
                for (int n = 0; n < nl; ++n) {
                    double acc = 0.0;
                    for (int q = 0; q < nq; ++q)
                        acc += w[q] * dphi[((size_t)q * 4 + a) * nl + m] *
                               dphi[((size_t)q * 4 + b) * nl + n];
                    S[((size_t)(a * 4 + b) * nl + m) * nl + n] = 6.0 * acc;
                }
}

namespace {

const int kEdgeA[6] = {0, 0, 0, 1, 1, 2};
const int kEdgeB[6] = {1, 2, 3, 2, 3, 3};

int local_edge(int a, int b) {
    if (a > b) std::swap(a, b);
    for (int e = 0; e < 6; ++e)
        if (kEdgeA[e] == a && kEdgeB[e] == b) return e;
    return -1;
}

struct FaceRec {
    int32_t v[3];
    int64_t slot;  // tet*4 + opposite vertex
    bool operator<(const FaceRec &o) const {
        if (v[0] != o.v[0]) return v[0] < o.v[0];
        if (v[1] != o.v[1]) return v[1] < o.v[1];
        if (v[2] != o.v[2]) return v[2] < o.v[2];
        return slot < o.slot;
    }
};

// Sparsity pattern of the matrix with element map `ed` (nloc entries per element, -1 =
// Dirichlet) from the unknown -> element incidence (sorted by element).
void build_pattern(int64_t n, int nl, const std::vector<int32_t> &ed,
                   const std::vector<int64_t> &iptr, const std::vector<int32_t> &inc, HCSR &A) {
    A.n = A.m = n;
    A.ptr.assign(n + 1, 0);
    unsigned hw = std::thread::hardware_concurrency();
    int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
    if (n < 4096) nth = 1;
    std::vector<std::vector<int32_t>> parts(nth);
    int64_t chunk = (n + nth - 1) / nth;
    std::vector<std::thread> th;
    auto work = [&](int t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        std::vector<int32_t> buf;
        auto &out = parts[t];
        for (int64_t i = b; i < e; ++i) {
            buf.clear();
            for (int64_t q = iptr[i]; q < iptr[i + 1]; ++q) {
                int64_t tet = inc[q] >> 6;
                for (int m = 0; m < nl; ++m) {
                    int32_t j = ed[tet * nl + m];
                    if (j >= 0) buf.push_back(j);
                }
            }
            std::sort(buf.begin(), buf.end());
            buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
            A.ptr[i + 1] = (int64_t)buf.size();
            out.insert(out.end(), buf.begin(), buf.end());
        }
    };
    if (nth == 1) work(0);
    else {
        for (int t = 0; t < nth; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    for (int64_t i = 0; i < n; ++i) A.ptr[i + 1] += A.ptr[i];
    A.col.resize(A.ptr[n]);
    int64_t o = 0;
    for (auto &p : parts) {
        std::copy(p.begin(), p.end(), A.col.begin() + o);
        o += (int64_t)p.size();
    }
    A.val.clear();
}

void incidence(int64_t n, int64_t nt, int nl, const std::vector<int32_t> &ed,
               std::vector<int64_t> &iptr, std::vector<int32_t> &inc) {
    iptr.assign(n + 1, 0);
    for (int64_t i = 0; i < nt * nl; ++i)
        if (ed[i] >= 0) iptr[ed[i] + 1]++;
    for (int64_t i = 0; i < n; ++i) iptr[i + 1] += iptr[i];
    inc.resize(iptr[n]);
    std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            int32_t i = ed[t * nl + m];
            if (i >= 0) inc[fill[i]++] = (int32_t)(t * 64 + m);
        }
}

}  // namespace

void build_dofmap(const HostMesh &M, DofMap &D) {
    const int k = M.k, nl = nloc_of(k);
    const int64_t nv = M.nv, nt = M.nt;
    if (nt > (int64_t)INT32_MAX / 64) fail(PKASP_EINVAL, "too many elements for the packed incidence");
    std::vector<int> m4;
    ref_nodes(k, m4);
    // ---- edges: sort (low, high) keys, one id per unique pair
    std::vector<std::pair<int64_t, int64_t>> ek((size_t)nt * 6);
    for (int64_t t = 0; t < nt; ++t)
        for (int e = 0; e < 6; ++e) {
            int64_t u = M.tets[4 * t + kEdgeA[e]], v = M.tets[4 * t + kEdgeB[e]];
            if (u > v) std::swap(u, v);
            ek[t * 6 + e] = {u * nv + v, t * 6 + e};
        }
    std::sort(ek.begin(), ek.end());
    std::vector<int64_t> edge_id((size_t)nt * 6);
    std::vector<int64_t> edge_key;
    for (size_t i = 0; i < ek.size(); ++i) {
        if (i == 0 || ek[i].first != ek[i - 1].first) edge_key.push_back(ek[i].first);
        edge_id[ek[i].second] = (int64_t)edge_key.size() - 1;
    }
    const int64_t ne = (int64_t)edge_key.size();
    ek.clear();
    ek.shrink_to_fit();
    // ---- faces: sorted triples; a face seen once is a boundary face
    std::vector<FaceRec> fr((size_t)nt * 4);
    for (int64_t t = 0; t < nt; ++t)
        for (int o = 0; o < 4; ++o) {
            FaceRec &f = fr[t * 4 + o];
            int c = 0;
            for (int a = 0; a < 4; ++a)
                if (a != o) f.v[c++] = M.tets[4 * t + a];
            std::sort(f.v, f.v + 3);
            f.slot = t * 4 + o;
        }
    std::sort(fr.begin(), fr.end());
    std::vector<int64_t> face_id((size_t)nt * 4);
    std::vector<uint8_t> face_bnd;
    std::vector<int32_t> face_v;
    for (size_t i = 0; i < fr.size();) {
        size_t j = i;
        while (j < fr.size() && fr[j].v[0] == fr[i].v[0] && fr[j].v[1] == fr[i].v[1] &&
               fr[j].v[2] == fr[i].v[2])
            ++j;
        if (j - i > 2) fail(PKASP_EMESH, "a face is shared by more than two elements");
        int64_t id = (int64_t)face_bnd.size();
        face_bnd.push_back(j - i == 1);
        face_v.insert(face_v.end(), fr[i].v, fr[i].v + 3);
        for (size_t q = i; q < j; ++q) face_id[fr[q].slot] = id;
        i = j;
    }
    const int64_t nf = (int64_t)face_bnd.size();
    fr.clear();
    fr.shrink_to_fit();
    const int ned = k - 1, nfd = (k - 1) * (k - 2) / 2, nid = (k - 1) * (k - 2) * (k - 3) / 6;
    const int64_t off_e = nv, off_f = nv + ne * ned, off_i = off_f + nf * nfd;
    D.n_all = off_i + nt * nid;
    // ---- boundary closure
    std::vector<uint8_t> vb(nv, 0), eb(ne, 0);
    for (int64_t t = 0; t < nt; ++t)
        for (int o = 0; o < 4; ++o) {
            if (!face_bnd[face_id[t * 4 + o]]) continue;
            for (int a = 0; a < 4; ++a)
                if (a != o) vb[M.tets[4 * t + a]] = 1;
            for (int e = 0; e < 6; ++e)
                if (kEdgeA[e] != o && kEdgeB[e] != o) eb[edge_id[t * 6 + e]] = 1;
        }
    // ---- element -> all-node index
    std::vector<int64_t> elem_all((size_t)nt * nl);
    parallel_for(nt, [&](int64_t b, int64_t e, int) {
        for (int64_t t = b; t < e; ++t) {
            const int32_t *g = &M.tets[4 * t];
            for (int m = 0; m < nl; ++m) {
                const int *mm = &m4[4 * m];
                int sup[4], ns = 0;
                for (int a = 0; a < 4; ++a)
                    if (mm[a] > 0) sup[ns++] = a;
                int64_t d;
                if (ns == 1) {
                    d = g[sup[0]];
                } else if (ns == 2) {
                    int a = sup[0], c = sup[1];
                    int hi = g[a] > g[c] ? a : c;
                    d = off_e + edge_id[t * 6 + local_edge(a, c)] * ned + (mm[hi] - 1);
                } else if (ns == 3) {
                    int opp = 0;
                    while (mm[opp] > 0) ++opp;
                    int idx[3] = {sup[0], sup[1], sup[2]};
                    std::sort(idx, idx + 3, [&](int x, int y) { return g[x] < g[y]; });
                    int p[3] = {mm[idx[0]], mm[idx[1]], mm[idx[2]]};
                    d = off_f + face_id[t * 4 + opp] * nfd + composition_rank(k, p, 3);
                } else {
                    int idx[4] = {0, 1, 2, 3};
                    std::sort(idx, idx + 4, [&](int x, int y) { return g[x] < g[y]; });
                    int p[4] = {mm[idx[0]], mm[idx[1]], mm[idx[2]], mm[idx[3]]};
                    d = off_i + t * nid + composition_rank(k, p, 4);
                }
                elem_all[t * nl + m] = d;
            }
        }
    });
    // ---- Dirichlet flags per all-node index, then compact numbering
    std::vector<uint8_t> bnd(D.n_all, 0);
    for (int64_t v = 0; v < nv; ++v) bnd[v] = vb[v];
    for (int64_t e = 0; e < ne; ++e)
        if (eb[e])
            for (int q = 0; q < ned; ++q) bnd[off_e + e * ned + q] = 1;
    for (int64_t f = 0; f < nf; ++f)
        if (face_bnd[f])
            for (int q = 0; q < nfd; ++q) bnd[off_f + f * nfd + q] = 1;
    std::vector<int64_t> cmap(D.n_all);
    int64_t nh = 0;
    for (int64_t d = 0; d < D.n_all; ++d) cmap[d] = bnd[d] ? -1 : nh++;
    D.nh = nh;
    if (nh > INT32_MAX) fail(PKASP_EINVAL, "more than 2^31 unknowns");
    D.dof_all.resize(nh);
    for (int64_t d = 0; d < D.n_all; ++d)
        if (cmap[d] >= 0) D.dof_all[cmap[d]] = d;
    D.elem_dof.resize((size_t)nt * nl);
    for (size_t i = 0; i < elem_all.size(); ++i) D.elem_dof[i] = (int32_t)cmap[elem_all[i]];
    if (D.n_all > INT32_MAX) fail(PKASP_EINVAL, "more than 2^31 nodes");
    D.elem_all.resize(elem_all.size());
    for (size_t i = 0; i < elem_all.size(); ++i) D.elem_all[i] = (int32_t)elem_all[i];
    std::vector<int64_t> vmap(nv);
    int64_t nH = 0;
    for (int64_t v = 0; v < nv; ++v) vmap[v] = vb[v] ? -1 : nH++;
    D.nH = nH;
    D.elem_vdof.resize((size_t)nt * 4);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a) D.elem_vdof[t * 4 + a] = (int32_t)vmap[M.tets[4 * t + a]];
    // ---- node coordinates
    D.dof_xyz.assign((size_t)nh * 3, 0.0);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            int32_t i = D.elem_dof[t * nl + m];
            if (i < 0) continue;
            for (int c = 0; c < 3; ++c) {
                double s = 0;
                for (int a = 0; a < 4; ++a) s += m4[4 * m + a] * M.xyz[3 * M.tets[4 * t + a] + c];
                D.dof_xyz[3 * (size_t)i + c] = s / k;
            }
        }
    // ---- incidence and patterns
    incidence(nh, nt, nl, D.elem_dof, D.inc_ptr, D.inc);
    incidence(nH, nt, 4, D.elem_vdof, D.vinc_ptr, D.vinc);
    build_pattern(nh, nl, D.elem_dof, D.inc_ptr, D.inc, D.Ah_pattern);
    build_pattern(nH, 4, D.elem_vdof, D.vinc_ptr, D.vinc, D.AH_pattern);
    // ---- I_P (Eq. 10): psi_j(x_i) = m_a / k at the first element holding node i
    HCSR &P = D.Pi;
    P.n = nh;
    P.m = nH;
    P.ptr.assign(nh + 1, 0);
    P.col.clear();
    P.val.clear();
    for (int64_t i = 0; i < nh; ++i) {
        int32_t pk = D.inc[D.inc_ptr[i]];
        int64_t t = pk >> 6;
        int m = pk & 63;
        std::pair<int32_t, double> ent[4];
        int c = 0;
        for (int a = 0; a < 4; ++a) {
            int32_t j = D.elem_vdof[t * 4 + a];
            if (m4[4 * m + a] > 0 && j >= 0) ent[c++] = {j, (double)m4[4 * m + a] / k};
        }
        for (int q = 1; q < c; ++q)  // at most 4 entries: insertion sort by column
            for (int r = q; r > 0 && ent[r].first < ent[r - 1].first; --r) std::swap(ent[r], ent[r - 1]);
        for (int q = 0; q < c; ++q) {
            P.col.push_back(ent[q].first);
            P.val.push_back(ent[q].second);
        }
        P.ptr[i + 1] = (int64_t)P.col.size();
    }
    // transpose (rows of I_R ascending)
    HCSR &T = D.PiT;
    T.n = nH;
    T.m = nh;
    T.ptr.assign(nH + 1, 0);
    for (int32_t j : P.col) T.ptr[j + 1]++;
    for (int64_t j = 0; j < nH; ++j) T.ptr[j + 1] += T.ptr[j];
    T.col.resize(P.col.size());
    T.val.resize(P.col.size());
    std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t i = 0; i < nh; ++i)
        for (int64_t e = P.ptr[i]; e < P.ptr[i + 1]; ++e) {
            int64_t q = fill[P.col[e]]++;
            T.col[q] = (int32_t)i;
            T.val[q] = P.val[e];
        }
}

}  // namespace pk
