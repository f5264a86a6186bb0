// stokes.cpp -- host part of the Taylor-Hood P_k - P_{k-1} Stokes blocks (Sec. 5):
// B = -div_h (rows: the P_{k-1} pressure nodes, all of them; columns: the velocity
// unknowns, component-major c n_h + j), its transpose and the pressure mass matrix M_p.
// Like the DOF map and the A_h pattern, the patterns and the reference tensors are built
// here (one-off setup work); pkasp_stokes_setup assembles the values on the device
// (stokes.cu). The host values below serve the host-only entry point. Every row sums its
// elements in ascending element order.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace pk {

namespace {

template <class F>
void rows_parallel(int64_t n, F fn) {
    unsigned hw = std::thread::hardware_concurrency();
    int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
    if (n < 2048) nth = 1;
    std::vector<std::thread> th;
    const int64_t chunk = (n + nth - 1) / nth;
    for (int t = 0; t < nth; ++t) {
        const int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        if (nth == 1) {
            fn(b, e);
            return;
        }
        th.emplace_back([=] { fn(b, e); });
    }
    for (auto &x : th) x.join();
}

// value and derivative in t of prod_{i<j} (k t - i) / (i + 1)
void lag_1d(int k, int j, double t, double &v, double &dv) {
    v = 1.0;
    dv = 0.0;
    for (int i = 0; i < j; ++i) {
        const double f = ((double)k * t - (double)i) / (double)(i + 1);
        dv = dv * f + v * (double)k / (double)(i + 1);
        v *= f;
    }
}

// grad lambda_a (rows) of a tetrahedron and its volume
double tet_gradients(const double *X, double g[4][3]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = X[3 * (c + 1) + r] - X[r];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    // rows of J^{-1} = gradients of lambda_1..3
    const double inv[3][3] = {{c00 / det, (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det,
                               (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det},
                              {c01 / det, (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det,
                               (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det},
                              {c02 / det, (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det,
                               (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det}};
    for (int c = 0; c < 3; ++c) {
        g[1][c] = inv[0][c];
        g[2][c] = inv[1][c];
        g[3][c] = inv[2][c];
        g[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
    }
    return det / 6.0;
}

// incidence node -> (element, local) with elements ascending
void node_incidence(int64_t nnodes, int64_t nt, int nl, const std::vector<int32_t> &emap,
                    std::vector<int64_t> &ptr, std::vector<int64_t> &ent) {
    ptr.assign(nnodes + 1, 0);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            const int32_t q = emap[t * nl + m];
            if (q >= 0) ptr[q + 1]++;
        }
    for (int64_t i = 0; i < nnodes; ++i) ptr[i + 1] += ptr[i];
    ent.assign(ptr[nnodes], 0);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int m = 0; m < nl; ++m) {
            const int32_t q = emap[t * nl + m];
            if (q >= 0) ent[fill[q]++] = t * 64 + m;
        }
}

}  // namespace

// Patterns and reference data of the Taylor-Hood blocks: the pressure DOF map (degree
// k-1, no Dirichlet removal), the reference tensors R[a][m][n] = (1/|T|) int psi_m
// dphi_n/dlambda_a and Mr[m][r] = (1/|T|) int psi_m psi_r by Grundmann-Moeller quadrature
// (exact to degree 2(k-1)+1), the incidence pressure node -> (element, local) with
// elements ascending, the sorted column patterns of B and M_p per pressure row, and the
// pattern of B^T with the B entry each of its entries copies (bt_src).
void stokes_patterns(int k, int64_t nv, int64_t nt, const double *xyz, const int32_t *tets, int64_t nh,
                     const int32_t *elem_dof, StokesPattern &P) {
    const int kp = k - 1;
    const int nu = nloc_of(k), npl = nloc_of(kp);
    P.nu = nu;
    P.npl = npl;
    HostMesh hm{kp, nv, nt, xyz, tets};
    DofMap Dp;
    build_dofmap(hm, Dp);
    const int64_t np = Dp.n_all;
    P.np = np;
    P.elem_p = Dp.elem_all;
    std::vector<double> lam, w;
    gm_rule(std::max(kp, 1), lam, w);
    const int nq = (int)w.size();
    std::vector<int> mu, mp;
    ref_nodes(k, mu);
    ref_nodes(kp, mp);
    P.R.assign((size_t)4 * npl * nu, 0.0);
    P.Mr.assign((size_t)npl * npl, 0.0);
    std::vector<double> psi(npl), dphi((size_t)4 * nu);
    for (int q = 0; q < nq; ++q) {
        const double *l = &lam[4 * q];
        basis_values(kp, l, psi.data());
        for (int n = 0; n < nu; ++n) {
            double v[4], d[4];
            for (int a = 0; a < 4; ++a) lag_1d(k, mu[4 * n + a], l[a], v[a], d[a]);
            for (int a = 0; a < 4; ++a) {
                double prod = d[a];
                for (int b = 0; b < 4; ++b)
                    if (b != a) prod *= v[b];
                dphi[a * nu + n] = prod;
            }
        }
        for (int a = 0; a < 4; ++a)
            for (int m = 0; m < npl; ++m)
                for (int n = 0; n < nu; ++n) P.R[((size_t)a * npl + m) * nu + n] += 6.0 * w[q] * psi[m] * dphi[a * nu + n];
        for (int m = 0; m < npl; ++m)
            for (int r = 0; r < npl; ++r) P.Mr[(size_t)m * npl + r] += 6.0 * w[q] * psi[m] * psi[r];
    }
    node_incidence(np, nt, npl, Dp.elem_all, P.iptr, P.ient);
    HCSR &B = P.B, &M = P.M, &BT = P.BT;
    B.n = np;
    B.m = 3 * nh;
    M.n = np;
    M.m = np;
    B.ptr.assign(np + 1, 0);
    M.ptr.assign(np + 1, 0);
    std::vector<std::vector<int32_t>> bcols(np), mcols(np);
    rows_parallel(np, [&](int64_t b, int64_t e) {
        std::vector<int32_t> bc, mc;
        for (int64_t q = b; q < e; ++q) {
            bc.clear();
            mc.clear();
            for (int64_t x = P.iptr[q]; x < P.iptr[q + 1]; ++x) {
                const int64_t t = P.ient[x] / 64;
                for (int n = 0; n < nu; ++n) {
                    const int32_t j = elem_dof[t * nu + n];
                    if (j < 0) continue;
                    for (int c = 0; c < 3; ++c) bc.push_back((int32_t)(c * nh + j));
                }
                for (int r = 0; r < npl; ++r) mc.push_back(Dp.elem_all[t * npl + r]);
            }
            std::sort(bc.begin(), bc.end());
            bc.erase(std::unique(bc.begin(), bc.end()), bc.end());
            std::sort(mc.begin(), mc.end());
            mc.erase(std::unique(mc.begin(), mc.end()), mc.end());
            bcols[q] = bc;
            mcols[q] = mc;
        }
    });
    for (int64_t q = 0; q < np; ++q) {
        B.ptr[q + 1] = B.ptr[q] + (int64_t)bcols[q].size();
        M.ptr[q + 1] = M.ptr[q] + (int64_t)mcols[q].size();
    }
    B.col.resize(B.ptr[np]);
    M.col.resize(M.ptr[np]);
    rows_parallel(np, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) {
            std::copy(bcols[q].begin(), bcols[q].end(), B.col.begin() + B.ptr[q]);
            std::copy(mcols[q].begin(), mcols[q].end(), M.col.begin() + M.ptr[q]);
        }
    });
    // B^T: columns of B become rows, entries in ascending pressure row
    BT.n = 3 * nh;
    BT.m = np;
    BT.ptr.assign(BT.n + 1, 0);
    for (int64_t x = 0; x < B.ptr[np]; ++x) BT.ptr[B.col[x] + 1]++;
    for (int64_t i = 0; i < BT.n; ++i) BT.ptr[i + 1] += BT.ptr[i];
    BT.col.resize(B.ptr[np]);
    P.bt_src.resize(B.ptr[np]);
    std::vector<int64_t> fill(BT.ptr.begin(), BT.ptr.end() - 1);
    for (int64_t q = 0; q < np; ++q)
        for (int64_t x = B.ptr[q]; x < B.ptr[q + 1]; ++x) {
            const int64_t o = fill[B.col[x]]++;
            BT.col[o] = (int32_t)q;
            P.bt_src[o] = x;
        }
}

// Host values of the blocks (the host-only entry point; pkasp_stokes_setup assembles the
// same values on the device): every pressure row sums its elements in ascending order.
void stokes_blocks(int k, int64_t nv, int64_t nt, const double *xyz, const int32_t *tets, int64_t nh,
                   const int32_t *elem_dof, HCSR &B, HCSR &BT, HCSR &M, int64_t &np) {
    StokesPattern P;
    stokes_patterns(k, nv, nt, xyz, tets, nh, elem_dof, P);
    np = P.np;
    const int nu = P.nu, npl = P.npl;
    std::vector<double> grads((size_t)nt * 12), vols(nt);
    for (int64_t t = 0; t < nt; ++t) {
        double X[12], g[4][3];
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) X[3 * v + c] = xyz[3 * (int64_t)tets[4 * t + v] + c];
        vols[t] = tet_gradients(X, g);
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) grads[t * 12 + a * 3 + c] = g[a][c];
    }
    B = std::move(P.B);
    M = std::move(P.M);
    BT = std::move(P.BT);
    B.val.assign(B.col.size(), 0.0);
    M.val.assign(M.col.size(), 0.0);
    rows_parallel(np, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) {
            const int32_t *bcb = &B.col[B.ptr[q]], *bce = bcb + (B.ptr[q + 1] - B.ptr[q]);
            const int32_t *mcb = &M.col[M.ptr[q]], *mce = mcb + (M.ptr[q + 1] - M.ptr[q]);
            for (int64_t x = P.iptr[q]; x < P.iptr[q + 1]; ++x) {
                const int64_t t = P.ient[x] / 64;
                const int m = (int)(P.ient[x] % 64);
                const double vol = vols[t];
                const double *g = &grads[t * 12];
                for (int n = 0; n < nu; ++n) {
                    const int32_t j = elem_dof[t * nu + n];
                    if (j < 0) continue;
                    for (int c = 0; c < 3; ++c) {
                        double s = 0.0;
                        for (int a = 0; a < 4; ++a) s += g[a * 3 + c] * P.R[((size_t)a * npl + m) * nu + n];
                        const int32_t col = (int32_t)(c * nh + j);
                        const int64_t pos = std::lower_bound(bcb, bce, col) - bcb;
                        B.val[B.ptr[q] + pos] += -vol * s;
                    }
                }
                for (int r = 0; r < npl; ++r) {
                    const int32_t col = P.elem_p[t * npl + r];
                    const int64_t pos = std::lower_bound(mcb, mce, col) - mcb;
                    M.val[M.ptr[q] + pos] += vol * P.Mr[(size_t)m * npl + r];
                }
            }
        }
    });
    BT.val.resize(BT.col.size());
    for (size_t o = 0; o < BT.val.size(); ++o) BT.val[o] = B.val[P.bt_src[o]];
}



}  // namespace pk
