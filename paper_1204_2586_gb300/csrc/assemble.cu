// assemble.cu -- device assembly of the P_k stiffness A_h and load f_h (Eq. 7), the P1
// stiffness A_H of the auxiliary space V_H (Sec. 2) and the adjoint element gradient.
//
// Every matrix row is owned by one warp that walks the row's incident elements in
// ascending element order, so each entry sums its element contributions in a fixed
// order (bitwise reproducible, no floating-point atomics).
#include "internal.h"

namespace pk {
namespace {

constexpr int kGF = 17;  // per element: G_ab (16) and |T|

// G_ab = grad lambda_a . grad lambda_b and |T| = det J / 6 with J = [x1-x0, x2-x0, x3-x0];
// grad lambda_1..3 are the rows of J^{-1} and grad lambda_0 = -(their sum).
__global__ void k_geometry(int64_t nt, const double *__restrict__ xyz, const int32_t *__restrict__ tets,
                           int64_t nv, double *__restrict__ gf, int *__restrict__ bad) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double x[4][3];
    for (int a = 0; a < 4; ++a) {
        int32_t v = tets[4 * t + a];
        if (v < 0 || v >= nv) {
            atomicExch(bad, 2);
            return;
        }
        for (int c = 0; c < 3; ++c) x[a][c] = xyz[3 * (int64_t)v + c];
    }
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = __dsub_rn(x[c + 1][r], x[0][r]);
    // cofactors (products rounded separately, no contraction)
    auto mul = [](double a, double b) { return __dmul_rn(a, b); };
    auto sub = [](double a, double b) { return __dsub_rn(a, b); };
    double c00 = sub(mul(J[1][1], J[2][2]), mul(J[1][2], J[2][1]));
    double c01 = sub(mul(J[1][0], J[2][2]), mul(J[1][2], J[2][0]));
    double c02 = sub(mul(J[1][0], J[2][1]), mul(J[1][1], J[2][0]));
    double det = __dadd_rn(sub(mul(J[0][0], c00), mul(J[0][1], c01)), mul(J[0][2], c02));
    if (!(det > 0.0)) {
        atomicExch(bad, 1);
        return;
    }
    double inv[3][3];
    inv[0][0] = __ddiv_rn(c00, det);
    inv[0][1] = __ddiv_rn(sub(mul(J[0][2], J[2][1]), mul(J[0][1], J[2][2])), det);
    inv[0][2] = __ddiv_rn(sub(mul(J[0][1], J[1][2]), mul(J[0][2], J[1][1])), det);
    inv[1][0] = __ddiv_rn(sub(mul(J[1][2], J[2][0]), mul(J[1][0], J[2][2])), det);
    inv[1][1] = __ddiv_rn(sub(mul(J[0][0], J[2][2]), mul(J[0][2], J[2][0])), det);
    inv[1][2] = __ddiv_rn(sub(mul(J[0][2], J[1][0]), mul(J[0][0], J[1][2])), det);
    inv[2][0] = __ddiv_rn(c02, det);
    inv[2][1] = __ddiv_rn(sub(mul(J[0][1], J[2][0]), mul(J[0][0], J[2][1])), det);
    inv[2][2] = __ddiv_rn(sub(mul(J[0][0], J[1][1]), mul(J[0][1], J[1][0])), det);
    double g[4][3];
    for (int c = 0; c < 3; ++c) {
        g[1][c] = inv[0][c];
        g[2][c] = inv[1][c];
        g[3][c] = inv[2][c];
        g[0][c] = -__dadd_rn(__dadd_rn(inv[0][c], inv[1][c]), inv[2][c]);
    }
    double *o = gf + t * kGF;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            o[a * 4 + b] = __dadd_rn(__dadd_rn(mul(g[a][0], g[b][0]), mul(g[a][1], g[b][1])),
                                     mul(g[a][2], g[b][2]));
    o[16] = __ddiv_rn(det, 6.0);
}

__device__ __forceinline__ int64_t find_col(const int32_t *__restrict__ col, int64_t lo, int64_t hi,
                                            int32_t j) {
    // first position in [lo, hi) with col == j (the pattern contains every pair)
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// (K_e)_mn = kappa |T| sum_ab G_ab S[a][b][m][n]
__device__ __forceinline__ double elem_entry(const double *__restrict__ gf, double kv,
                                             const double *__restrict__ S, int nl, int m, int n) {
    double s = 0.0;
#pragma unroll
    for (int ab = 0; ab < 16; ++ab)
        s = __dadd_rn(s, __dmul_rn(gf[ab], __ldg(&S[((int64_t)ab * nl + m) * nl + n])));
    return __dmul_rn(__dmul_rn(kv, gf[16]), s);
}

// One warp per row of A_h: zero the row, then add the element matrices of the incident
// elements in ascending element order (lanes own distinct columns of one element).
__global__ void k_assemble_pk(int64_t nrows, int nl, const int64_t *__restrict__ inc_ptr,
                              const int32_t *__restrict__ inc, const int32_t *__restrict__ elem_dof,
                              const double *__restrict__ gf, const double *__restrict__ kappa,
                              const double *__restrict__ S, const int64_t *__restrict__ ptr,
                              const int32_t *__restrict__ col, double *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < nrows; i += nwarps) {
        const int64_t lo = ptr[i], hi = ptr[i + 1];
        for (int64_t e = lo + lane; e < hi; e += 32) val[e] = 0.0;
        __syncwarp();
        for (int64_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
            const int32_t pk = inc[q];
            const int64_t t = pk >> 6;
            const int m = pk & 63;
            const double *g = gf + t * kGF;
            const double kv = kappa[t];
            for (int n = lane; n < nl; n += 32) {
                int32_t j = elem_dof[t * nl + n];
                if (j < 0) continue;
                double kmn = elem_entry(g, kv, S, nl, m, n);
                int64_t pos = find_col(col, lo, hi, j);
                if (pos < hi && col[pos] == j) val[pos] = __dadd_rn(val[pos], kmn);
            }
            __syncwarp();
        }
    }
}

// One thread per row of A_H: (K1_e)_ab = kappa |T| G_ab.
__global__ void k_assemble_p1(int64_t nrows, const int64_t *__restrict__ inc_ptr,
                              const int32_t *__restrict__ inc, const int32_t *__restrict__ elem_vdof,
                              const double *__restrict__ gf, const double *__restrict__ kappa,
                              const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              double *__restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    const int64_t lo = ptr[i], hi = ptr[i + 1];
    for (int64_t e = lo; e < hi; ++e) val[e] = 0.0;
    for (int64_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
        const int32_t pk = inc[q];
        const int64_t t = pk >> 6;
        const int a = pk & 63;
        const double *g = gf + t * kGF;
        const double kv = __dmul_rn(kappa[t], g[16]);
        for (int b = 0; b < 4; ++b) {
            int32_t j = elem_vdof[t * 4 + b];
            if (j < 0) continue;
            int64_t pos = find_col(col, lo, hi, j);
            if (pos < hi && col[pos] == j) val[pos] = __dadd_rn(val[pos], __dmul_rn(kv, g[a * 4 + b]));
        }
    }
}

// Element load vectors be[t][m] = 6|T| sum_q w_q f(x_q) phi_m(lambda_q) for the source
// f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z); one warp per element.
__global__ void k_element_load(int64_t nt, int nl, int nq, const double *__restrict__ xyz,
                               const int32_t *__restrict__ tets, const double *__restrict__ gf,
                               const double *__restrict__ lamq, const double *__restrict__ wq,
                               const double *__restrict__ phiq, double *__restrict__ be) {
    extern __shared__ double fsh[];  // [warps][nq]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *fq = fsh + (int64_t)wid * nq;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double pi = 3.141592653589793238462643383279502884;
    for (int64_t t = warp; t < nt; t += nwarps) {
        double x[4][3];
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) x[a][c] = xyz[3 * (int64_t)tets[4 * t + a] + c];
        for (int q = lane; q < nq; q += 32) {
            double p[3];
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int a = 0; a < 4; ++a) v = __dadd_rn(v, __dmul_rn(lamq[4 * q + a], x[a][c]));
                p[c] = v;
            }
            double f = __dmul_rn(3.0 * pi, pi);
            f = __dmul_rn(f, sin(__dmul_rn(pi, p[0])));
            f = __dmul_rn(f, sin(__dmul_rn(pi, p[1])));
            f = __dmul_rn(f, sin(__dmul_rn(pi, p[2])));
            fq[q] = f;
        }
        __syncwarp();
        const double vol = gf[t * kGF + 16];
        for (int m = lane; m < nl; m += 32) {
            double acc = 0.0;
            for (int q = 0; q < nq; ++q)
                acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(wq[q], fq[q]), phiq[(int64_t)q * nl + m]));
            be[t * nl + m] = __dmul_rn(__dmul_rn(6.0, vol), acc);
        }
        __syncwarp();
    }
}

// Element load vectors for a caller's f given at the P_k nodes (PKASP_SOURCE_NODAL):
// f_h = sum_n f_n phi_n is evaluated at each quadrature point through the basis, then
// be[t][m] = 6|T| sum_q w_q f_h(x_q) phi_m(lambda_q); one warp per element.
__global__ void k_element_load_nodal(int64_t nt, int nl, int nq, const int32_t *__restrict__ elem_all,
                                     const double *__restrict__ fall, const double *__restrict__ gf,
                                     const double *__restrict__ wq, const double *__restrict__ phiq,
                                     double *__restrict__ be) {
    extern __shared__ double fsh[];  // [warps][nq]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *fq = fsh + (int64_t)wid * nq;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < nt; t += nwarps) {
        const int32_t *ea = elem_all + t * nl;
        for (int q = lane; q < nq; q += 32) {
            double v = 0.0;
            for (int n = 0; n < nl; ++n) v = __dadd_rn(v, __dmul_rn(fall[ea[n]], phiq[(int64_t)q * nl + n]));
            fq[q] = v;
        }
        __syncwarp();
        const double vol = gf[t * kGF + 16];
        for (int m = lane; m < nl; m += 32) {
            double acc = 0.0;
            for (int q = 0; q < nq; ++q)
                acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(wq[q], fq[q]), phiq[(int64_t)q * nl + m]));
            be[t * nl + m] = __dmul_rn(__dmul_rn(6.0, vol), acc);
        }
        __syncwarp();
    }
}

__global__ void k_gather_load(int64_t nrows, int nl, const int64_t *__restrict__ inc_ptr,
                              const int32_t *__restrict__ inc, const double *__restrict__ be,
                              double *__restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    double s = 0.0;
    for (int64_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
        const int32_t pk = inc[q];
        s = __dadd_rn(s, be[(int64_t)(pk >> 6) * nl + (pk & 63)]);
    }
    b[i] = s;
}

// dL/dkappa_e = -sum_c lambda_{c,e}^T Khat_e u_{c,e} over the ncols columns of u and
// lambda ([n][ld], column c at offset c), one warp per element (lanes over rows m). Each
// column's term is formed as for one column and the terms are added in column order.
__global__ void k_grad_kappa(int64_t nt, int nl, const int32_t *__restrict__ elem_dof,
                             const double *__restrict__ gf, const double *__restrict__ S,
                             const double *__restrict__ u, const double *__restrict__ lam, int ncols,
                             int64_t ld, double *__restrict__ g) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < nt; t += nwarps) {
        const double *gt = gf + t * kGF;
        const int32_t *ed = elem_dof + t * nl;
        double tot = 0.0;
        for (int c = 0; c < ncols; ++c) {
            double part = 0.0;
            for (int m = lane; m < nl; m += 32) {
                int32_t i = ed[m];
                if (i < 0) continue;
                double km = 0.0;
                for (int n = 0; n < nl; ++n) {
                    int32_t j = ed[n];
                    if (j < 0) continue;
                    km += elem_entry(gt, 1.0, S, nl, m, n) * u[(int64_t)j * ld + c];
                }
                part += lam[(int64_t)i * ld + c] * km;
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            tot += part;
        }
        if (lane == 0) g[t] = -tot;
    }
}

unsigned grid_for(int64_t work_items, int per_block, int64_t cap) {
    int64_t b = (work_items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

// Geometry, A_h, A_H and (optionally) f_h for the current kappa.
void assemble_values(pkasp_problem *p, cudaStream_t s) {
    int *bad = p->d_flag;
    PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_geometry<<<grid_for(p->nt, 256, INT32_MAX), 256, 0, s>>>(p->nt, p->d_xyz, p->d_tets, p->nv,
                                                                p->d_gfac, bad);
    PK_LAUNCH();
    int hbad = 0;
    PK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (hbad == 1) fail(PKASP_EMESH, "a tetrahedron has non-positive volume (det J <= 0)");
    if (hbad == 2) fail(PKASP_EMESH, "a tetrahedron references a vertex index out of range");
    const unsigned big = 152 * 64;
    k_assemble_pk<<<grid_for(p->nh * 32, 256, big), 256, 0, s>>>(
        p->nh, p->nloc, p->d_inc_ptr, p->d_inc, p->d_elem_dof, p->d_gfac, p->d_kappa, p->d_S,
        p->Ah.ptr, p->Ah.col, p->Ah.val);
    PK_LAUNCH();
    k_assemble_p1<<<grid_for(p->nH, 128, INT32_MAX), 128, 0, s>>>(
        p->nH, p->d_vinc_ptr, p->d_vinc, p->d_elem_vdof, p->d_gfac, p->d_kappa, p->AH.ptr,
        p->AH.col, p->AH.val);
    PK_LAUNCH();
    if (p->source == PKASP_SOURCE_SINE || p->source == PKASP_SOURCE_NODAL) {
        double *be = nullptr;
        PK_CUDA(cudaMallocAsync((void **)&be, sizeof(double) * p->nt * p->nloc, s));
        size_t shm = sizeof(double) * (size_t)p->nq * 8;
        if (p->source == PKASP_SOURCE_SINE)
            k_element_load<<<grid_for(p->nt * 32, 256, big), 256, shm, s>>>(
                p->nt, p->nloc, p->nq, p->d_xyz, p->d_tets, p->d_gfac, p->d_lamq, p->d_wq, p->d_phiq, be);
        else
            k_element_load_nodal<<<grid_for(p->nt * 32, 256, big), 256, shm, s>>>(
                p->nt, p->nloc, p->nq, p->d_elem_all, p->d_fall, p->d_gfac, p->d_wq, p->d_phiq, be);
        PK_LAUNCH();
        k_gather_load<<<grid_for(p->nh, 256, INT32_MAX), 256, 0, s>>>(p->nh, p->nloc, p->d_inc_ptr,
                                                                       p->d_inc, be, p->d_b);
        PK_LAUNCH();
        PK_CUDA(cudaFreeAsync(be, s));
    } else {
        PK_CUDA(cudaMemsetAsync(p->d_b, 0, sizeof(double) * p->nh, s));
    }
    PK_CUDA(cudaStreamSynchronize(s));
}

void assemble_device(pkasp_problem *p, cudaStream_t s) {
    // reference tables
    std::vector<double> S, lam, w, phi;
    reference_tensors(p->k, S);
    gm_rule(p->k + 1, lam, w);
    p->nq = (int)w.size();
    phi.resize((size_t)p->nq * p->nloc);
    for (int q = 0; q < p->nq; ++q) basis_values(p->k, &lam[4 * q], &phi[(size_t)q * p->nloc]);
    p->d_S = p->pool.get<double>(S.size());
    p->d_lamq = p->pool.get<double>(lam.size());
    p->d_wq = p->pool.get<double>(w.size());
    p->d_phiq = p->pool.get<double>(phi.size());
    PK_CUDA(cudaMemcpyAsync(p->d_S, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(p->d_lamq, lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(p->d_wq, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(p->d_phiq, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice, s));
    p->d_gfac = p->pool.get<double>((size_t)p->nt * kGF);
    PK_CUDA(cudaStreamSynchronize(s));
    assemble_values(p, s);
}

void grad_kappa_device(const pkasp_problem *p, const double *u, const double *lam, int ncols, int64_t ld,
                       double *g, cudaStream_t s) {
    k_grad_kappa<<<grid_for(p->nt * 32, 256, 152 * 64), 256, 0, s>>>(
        p->nt, p->nloc, p->d_elem_dof, p->d_gfac, p->d_S, u, lam, ncols, ld, g);
    PK_LAUNCH();
}

}  // namespace pk
