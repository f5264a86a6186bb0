// api.cu -- the C ABI declared in include/pkasp.h. Converts internal exceptions into
// status codes plus a per-thread message, validates arguments, and stages host arrays.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

template <class F>
int guarded(F fn) {
    try {
        return fn();
    } catch (const pk::Error &e) {
        return set_error(e.code, e.msg);
    } catch (const std::bad_alloc &) {
        return set_error(PKASP_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return set_error(PKASP_EINVAL, e.what());
    }
}

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// A device view of a caller array: the array itself if it lives on the device, else a
// staged copy in `pool` (from host memory).
template <class T>
const T *device_view(pk::DevPool &pool, const T *arr, int64_t n, cudaStream_t s) {
    if (is_device_ptr(arr)) return arr;
    T *d = pool.get<T>(n > 0 ? n : 1);
    PK_CUDA(cudaMemcpyAsync(d, arr, sizeof(T) * n, cudaMemcpyHostToDevice, s));
    return d;
}

}  // namespace

extern "C" {

void pkasp_default_options(pkasp_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->theta = 0.25;
    o->mode = PKASP_MODE_ADDITIVE;
    o->smoother = PKASP_SMOOTHER_SGS;
    o->level_smoother = PKASP_SMOOTHER_SGS;
    o->coarse_size = 256;
    o->max_levels = 25;
    o->seed = 0;
    o->tol = 1e-8;
    o->max_iter = 500;
    o->flexible = 0;
    o->precond_precision = PKASP_PREC_FP64;
    o->use_graph = 1;
    o->spmv_threads = 0;
    o->smoother_layout = 0;
    o->krylov = PKASP_KRYLOV_CG;
    o->restart = 30;
    o->interp_pmax = 0;
    o->interp_trunc = 0;
    o->interp_cc = 0;
    o->l2_persist = 1;
}

int pkasp_last_error(char *buf, size_t n) {
    if (!buf || n == 0) return PKASP_EINVAL;
    snprintf(buf, n, "%s", g_last_error.c_str());
    return PKASP_OK;
}

int pkasp_assemble(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                   const double *kappa, int source, const double *f_nodal, pkasp_problem **out) {
    if (!out) return set_error(PKASP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!xyz_host || !tets_host || !kappa) return set_error(PKASP_EINVAL, "NULL mesh or kappa array");
    if (nv <= 0 || nt <= 0) return set_error(PKASP_EINVAL, "empty mesh");
    if (k < 1 || k > 4) return set_error(PKASP_EINVAL, "degree k must be 1..4");
    if (source != PKASP_SOURCE_NONE && source != PKASP_SOURCE_SINE && source != PKASP_SOURCE_NODAL)
        return set_error(PKASP_EINVAL, "unknown source");
    if ((source == PKASP_SOURCE_NODAL) != (f_nodal != nullptr))
        return set_error(PKASP_EINVAL, "f_nodal must be given exactly when source is PKASP_SOURCE_NODAL");
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (tets_host[i] < 0 || tets_host[i] >= nv)
            return set_error(PKASP_EMESH, "tetrahedron vertex index out of range");
    pkasp_problem *p = new pkasp_problem();
    int rc = guarded([&]() -> int {
        auto t0 = std::chrono::steady_clock::now();
        PK_CUDA(cudaGetDevice(&p->device));
        cudaStream_t s = nullptr;
        p->k = k;
        p->nloc = pk::nloc_of(k);
        p->nv = nv;
        p->nt = nt;
        p->source = source;
        p->xyz.assign(xyz_host, xyz_host + 3 * nv);
        p->tets.assign(tets_host, tets_host + 4 * nt);
        pk::DofMap D;
        pk::HostMesh M{k, nv, nt, p->xyz.data(), p->tets.data()};
        pk::build_dofmap(M, D);
        if (D.nh == 0 || D.nH == 0) pk::fail(PKASP_EINVAL, "the mesh has no interior unknowns");
        p->n_all = D.n_all;
        p->nh = D.nh;
        p->nH = D.nH;
        p->dof_all = std::move(D.dof_all);
        p->dof_xyz = std::move(D.dof_xyz);
        p->elem_dof = D.elem_dof;
        p->elem_vdof = D.elem_vdof;
        pk::DevPool &pool = p->pool;
        auto up = [&](auto *dst, const auto &vec) {
            PK_CUDA(cudaMemcpyAsync(dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice, s));
        };
        p->d_xyz = pool.get<double>(3 * nv);
        up(p->d_xyz, p->xyz);
        p->d_tets = pool.get<int32_t>(4 * nt);
        up(p->d_tets, p->tets);
        p->d_kappa = pool.get<double>(nt);
        if (is_device_ptr(kappa))
            PK_CUDA(cudaMemcpyAsync(p->d_kappa, kappa, sizeof(double) * nt, cudaMemcpyDeviceToDevice, s));
        else
            PK_CUDA(cudaMemcpyAsync(p->d_kappa, kappa, sizeof(double) * nt, cudaMemcpyHostToDevice, s));
        p->d_elem_dof = pool.get<int32_t>(D.elem_dof.size());
        up(p->d_elem_dof, D.elem_dof);
        p->d_elem_vdof = pool.get<int32_t>(D.elem_vdof.size());
        up(p->d_elem_vdof, D.elem_vdof);
        p->d_inc_ptr = pool.get<int64_t>(D.inc_ptr.size());
        up(p->d_inc_ptr, D.inc_ptr);
        p->d_inc = pool.get<int32_t>(std::max<size_t>(D.inc.size(), 1));
        up(p->d_inc, D.inc);
        p->d_vinc_ptr = pool.get<int64_t>(D.vinc_ptr.size());
        up(p->d_vinc_ptr, D.vinc_ptr);
        p->d_vinc = pool.get<int32_t>(std::max<size_t>(D.vinc.size(), 1));
        up(p->d_vinc, D.vinc);
        if (source == PKASP_SOURCE_NODAL) {
            p->d_elem_all = pool.get<int32_t>(D.elem_all.size());
            up(p->d_elem_all, D.elem_all);
            p->d_fall = pool.get<double>(D.n_all);
            PK_CUDA(cudaMemcpyAsync(p->d_fall, f_nodal, sizeof(double) * D.n_all,
                                    is_device_ptr(f_nodal) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        }
        pk::dcsr_upload(pool, p->Ah, D.Ah_pattern, s);
        pk::dcsr_upload(pool, p->AH, D.AH_pattern, s);
        pk::dcsr_upload(pool, p->Pi, D.Pi, s);
        pk::dcsr_upload(pool, p->PiT, D.PiT, s);
        pk::pi_codes_upload(pool, D.Pi, D.PiT, k, p->pic, s);
        p->d_b = pool.get<double>(p->nh);
        p->d_flag = pool.get<int>(4);
        PK_CUDA(cudaStreamSynchronize(s));
        pk::assemble_device(p, s);
        p->assemble_ms = ms_since(t0);
        return PKASP_OK;
    });
    if (rc != PKASP_OK) {
        cudaDeviceSynchronize();
        p->pool.free_all();
        delete p;
        return rc;
    }
    *out = p;
    return PKASP_OK;
}

int pkasp_problem_info(const pkasp_problem *p, pkasp_info *info) {
    if (!p || !info) return set_error(PKASP_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_h = p->nh;
    info->n_H = p->nH;
    info->nnz_h = p->Ah.nnz;
    info->nnz_H = p->AH.nnz;
    info->nnz_pi = p->Pi.nnz;
    info->n_all = p->n_all;
    info->n_tets = p->nt;
    info->n_verts = p->nv;
    info->k = p->k;
    info->assemble_ms = p->assemble_ms;
    if (p->have_setup) {
        info->levels = (int)p->lev.size();
        info->fine_colours = p->fine.ncol;
        info->coarse_rows = (int)p->nc;
        double tot = 0;
        for (size_t l = 0; l < p->lev.size() && l < PKASP_MAX_LEVELS; ++l) {
            info->level_rows[l] = p->lev[l].A.n;
            info->level_nnz[l] = p->lev[l].A.nnz;
            info->level_colours[l] = p->lev[l].sp.ncol;
            tot += (double)p->lev[l].A.nnz;
        }
        // relative to level 0: A_H, or A_h in plain AMG mode
        const int64_t nnz0 = p->lev.empty() ? 0 : p->lev[0].A.nnz;
        info->op_complexity = nnz0 > 0 ? tot / (double)nnz0 : 0;
        info->setup_ms = p->setup_ms;
        info->spmv_layout = p->spmv_tpr;
        info->smoother_layout = p->fine_tpr;
        info->block_width = p->bwork_nc > 0 ? p->bwork_nc : 0;
        info->block_group = p->bgroup_cols;
        info->block_lanes = p->blanes;
        info->l2_persist_bytes = (int64_t)p->l2_win_bytes;
    }
    return PKASP_OK;
}

int pkasp_get_dofmap(const pkasp_problem *p, int64_t *dof_all_host, double *dof_xyz_host) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    if (dof_all_host) memcpy(dof_all_host, p->dof_all.data(), sizeof(int64_t) * p->nh);
    if (dof_xyz_host) memcpy(dof_xyz_host, p->dof_xyz.data(), sizeof(double) * 3 * p->nh);
    return PKASP_OK;
}

int pkasp_get_rhs(const pkasp_problem *p, double *b, pkasp_stream_t stream) {
    if (!p || !b) return set_error(PKASP_EINVAL, "NULL argument");
    return guarded([&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        PK_CUDA(cudaMemcpyAsync(b, p->d_b, sizeof(double) * p->nh, cudaMemcpyDefault, s));
        PK_CUDA(cudaStreamSynchronize(s));
        return PKASP_OK;
    });
}

int pkasp_set_kappa(pkasp_problem *p, const double *kappa, pkasp_stream_t stream) {
    if (!p || !kappa) return set_error(PKASP_EINVAL, "NULL argument");
    return guarded([&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        PK_CUDA(cudaMemcpyAsync(p->d_kappa, kappa, sizeof(double) * p->nt, cudaMemcpyDefault, s));
        pk::free_setup(p);  // the preconditioner belongs to the old kappa
        pk::assemble_values(p, s);
        return PKASP_OK;
    });
}

int pkasp_setup(pkasp_problem *p, const pkasp_options *opt, pkasp_stream_t stream) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    pkasp_options o;
    if (opt) o = *opt;
    else pkasp_default_options(&o);
    if (!(o.theta >= 0.0 && o.theta < 1.0)) return set_error(PKASP_EINVAL, "theta must be in [0, 1)");
    if (o.mode != 0 && o.mode != 1 && o.mode != 2) return set_error(PKASP_EINVAL, "unknown mode");
    if (o.smoother != 0 && o.smoother != 1) return set_error(PKASP_EINVAL, "unknown smoother");
    if (o.level_smoother != 0 && o.level_smoother != 1) return set_error(PKASP_EINVAL, "unknown level smoother");
    if (o.max_levels < 1 || o.max_levels > PKASP_MAX_LEVELS) return set_error(PKASP_EINVAL, "max_levels out of range");
    if (o.coarse_size < 1) return set_error(PKASP_EINVAL, "coarse_size must be positive");
    if (!(o.tol > 0.0) || o.max_iter < 1) return set_error(PKASP_EINVAL, "tol and max_iter must be positive");
    if (o.precond_precision != 0 && o.precond_precision != 1) return set_error(PKASP_EINVAL, "unknown precision");
    if (o.spmv_threads != 0 && o.spmv_threads != 4 && o.spmv_threads != 8 && o.spmv_threads != 16 &&
        o.spmv_threads != 32)
        return set_error(PKASP_EINVAL, "spmv_threads must be 0, 4, 8, 16 or 32");
    if (o.interp_pmax < 0 || o.interp_trunc < 0 || o.interp_trunc > 999)
        return set_error(PKASP_EINVAL, "interp_pmax must be >= 0 and interp_trunc 0..999");
    if (o.interp_cc != 0 && o.interp_cc != 1) return set_error(PKASP_EINVAL, "interp_cc must be 0 or 1");
    if (o.l2_persist != 0 && o.l2_persist != 1) return set_error(PKASP_EINVAL, "l2_persist must be 0 or 1");
    if (o.krylov != PKASP_KRYLOV_CG && o.krylov != PKASP_KRYLOV_FGMRES)
        return set_error(PKASP_EINVAL, "krylov must be PKASP_KRYLOV_CG or PKASP_KRYLOV_FGMRES");
    if (o.krylov == PKASP_KRYLOV_FGMRES && (o.restart < 1 || o.restart > 256))
        return set_error(PKASP_EINVAL, "restart must be 1..256");
    {
        const int l = o.smoother_layout;
        if (!(l == 0 || l == 1 || l == 2 || l == 3 || l == 4 || l == 8 || l == 16 || l == -4 || l == -8 ||
              l == -16 || l == 102 || l == 104 || l == 108 || l == 116 || l == 404 || l == 408 ||
              l == 416))
            return set_error(PKASP_EINVAL, "smoother_layout must be 0, 1, 2, 3, 4, 8, 16, -4, -8, -16, 102, 104, "
                                           "108, 116, 404, 408 or 416");
    }
    return guarded([&]() -> int {
        auto t0 = std::chrono::steady_clock::now();
        p->opt = o;
        pk::setup_device(p, (cudaStream_t)stream);
        p->setup_ms = ms_since(t0);
        return PKASP_OK;
    });
}

static int solve_common(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                        pkasp_stream_t stream, bool from_zero = false) {
    if (!p || !b || !x) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "pkasp_setup must precede pkasp_solve");
    if (ncols < 1 || ncols > PKASP_MAX_COLS) return set_error(PKASP_EINVAL, "ncols must be 1..64");
    if (ld < ncols) return set_error(PKASP_EINVAL, "ld must be >= ncols");
    return guarded([&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
        pk::ensure_work(p, 1);
        const int64_t n = p->nh * ld;
        if ((!bd || !xd) && p->stage_elems < n) {
            p->stage_pool.free_all();
            p->stage_b = p->stage_pool.get<double>(std::max<int64_t>(n, 1));
            p->stage_x = p->stage_pool.get<double>(std::max<int64_t>(n, 1));
            p->stage_elems = n;
        }
        const double *bb = b;
        double *xx = x;
        if (!bd) {
            PK_CUDA(cudaMemcpyAsync(p->stage_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            bb = p->stage_b;
        }
        // from zero: only the ncols columns are zeroed (and, for a host x, copied back),
        // so padding columns of an [n][ld] array and memory past a column-sliced view's
        // last row are never written
        auto zero_cols = [&](double *a) {
            if (ld == ncols) PK_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * n, s));
            else PK_CUDA(cudaMemset2DAsync(a, sizeof(double) * ld, 0, sizeof(double) * ncols, p->nh, s));
        };
        if (!xd) {
            xx = p->stage_x;
            if (from_zero) zero_cols(xx);
            else PK_CUDA(cudaMemcpyAsync(xx, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        } else if (from_zero) {
            zero_cols(xx);
        }
        int rc = pk::solve_device(p, bb, xx, ncols, ld, st, s);
        pk::l2_window_idle(p);  // the solve has synchronised its stream
        if (!xd) {
            if (from_zero && ld != ncols)
                PK_CUDA(cudaMemcpy2DAsync(x, sizeof(double) * ld, xx, sizeof(double) * ld, sizeof(double) * ncols,
                                          p->nh, cudaMemcpyDeviceToHost, s));
            else
                PK_CUDA(cudaMemcpyAsync(x, xx, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaStreamSynchronize(s));
        }
        if (rc != PKASP_OK) {
            return set_error(rc, rc == PKASP_ENOTCONV ? "PCG reached max_iter before the tolerance"
                                                      : "PCG breakdown: p^T A p <= 0 (system not SPD)");
        }
        return PKASP_OK;
    });
}

int pkasp_solve(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                pkasp_stream_t stream) {
    return solve_common(p, b, x, ncols, ld, st, stream);
}

int pkasp_solve_from_zero(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld,
                          pkasp_stats *st, pkasp_stream_t stream) {
    return solve_common(p, b, x, ncols, ld, st, stream, true);
}

int pkasp_solve_adjoint(pkasp_problem *p, const double *g, double *lambda, int ncols, int64_t ld,
                        pkasp_stats *st, pkasp_stream_t stream) {
    // A_h is symmetric: the adjoint system uses the same operator and preconditioner
    return solve_common(p, g, lambda, ncols, ld, st, stream);
}

int pkasp_grad_kappa(const pkasp_problem *p, const double *u_dev, const double *lambda_dev, int ncols, int64_t ld,
                     double *dkappa_dev, pkasp_stream_t stream) {
    if (!p || !u_dev || !lambda_dev || !dkappa_dev) return set_error(PKASP_EINVAL, "NULL argument");
    if (ncols < 1 || ncols > PKASP_MAX_COLS) return set_error(PKASP_EINVAL, "ncols must be 1..64");
    if (ld < ncols) return set_error(PKASP_EINVAL, "ld must be >= ncols");
    return guarded([&]() -> int {
        pk::grad_kappa_device(p, u_dev, lambda_dev, ncols, ld, dkappa_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_destroy(pkasp_problem *p) {
    if (!p) return PKASP_OK;
    cudaDeviceSynchronize();
    pk::free_setup(p);
    pk::stokes_free(p);
    p->stage_pool.free_all();
    p->pool.free_all();
    pk::l2_window_release(p);
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    delete p;
    return PKASP_OK;
}

int pkasp_spmv(const pkasp_problem *p, const double *x_dev, double *y_dev, pkasp_stream_t stream) {
    if (!p || !x_dev || !y_dev) return set_error(PKASP_EINVAL, "NULL argument");
    return guarded([&]() -> int {
        pk::spmv_fine(const_cast<pkasp_problem *>(p), x_dev, y_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_apply_prec(pkasp_problem *p, const double *r_dev, double *z_dev, pkasp_stream_t stream) {
    if (!p || !r_dev || !z_dev) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    return guarded([&]() -> int {
        pk::apply_prec(p, r_dev, z_dev, (cudaStream_t)stream);
        if (p->fine_tpr < -1) pk::check_barrier(p, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_apply_smoother(pkasp_problem *p, const double *r_dev, double *z_dev, pkasp_stream_t stream) {
    if (!p || !r_dev || !z_dev) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    return guarded([&]() -> int {
        pk::apply_smoother(p, r_dev, z_dev, (cudaStream_t)stream);
        if (p->fine_tpr < -1) pk::check_barrier(p, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_apply_vcycle(pkasp_problem *p, const double *b_dev, double *x_dev, pkasp_stream_t stream) {
    if (!p || !b_dev || !x_dev) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    return guarded([&]() -> int {
        pk::apply_vcycle(p, b_dev, x_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_get_matrix(const pkasp_problem *p, int which, int64_t *rows_out, int64_t *cols_out, int64_t *nnz_out,
                     int64_t *ptr_host, int32_t *col_host, double *val_host) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    const pk::DCSR *A = nullptr;
    if (which < 0) {
        if (!p->st) return set_error(PKASP_ESTATE, "pkasp_stokes_setup first");
        A = pk::stokes_matrix(p, which);
        if (!A) return set_error(PKASP_EINVAL, "unknown matrix");
    } else if (which == 0) A = &p->Ah;
    else if (which == 1) A = &p->AH;
    else if (which == 2) A = &p->Pi;
    else if (which >= 3) {
        int l = (which - 3) / 2;
        bool interp = ((which - 3) % 2) == 1;
        if (!p->have_setup || l >= (int)p->lev.size()) return set_error(PKASP_EINVAL, "no such level");
        A = interp ? &p->lev[l].P : &p->lev[l].A;
        if (interp && A->n == 0) return set_error(PKASP_EINVAL, "the coarsest level has no interpolation");
    } else {
        return set_error(PKASP_EINVAL, "unknown matrix");
    }
    if (rows_out) *rows_out = A->n;
    if (cols_out) *cols_out = A->m;
    if (nnz_out) *nnz_out = A->nnz;
    return guarded([&]() -> int {
        if (ptr_host) PK_CUDA(cudaMemcpy(ptr_host, A->ptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyDeviceToHost));
        if (col_host && A->nnz) PK_CUDA(cudaMemcpy(col_host, A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost));
        if (val_host && A->nnz) PK_CUDA(cudaMemcpy(val_host, A->val, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost));
        return PKASP_OK;
    });
}

int pkasp_stokes_setup(pkasp_problem *p, int mp_iters, pkasp_stream_t stream) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    return guarded([&]() -> int {
        pk::stokes_setup(p, mp_iters, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_stokes_sizes(const pkasp_problem *p, int64_t *sizes_out) {
    if (!p || !sizes_out) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->st) return set_error(PKASP_ESTATE, "pkasp_stokes_setup first");
    pk::stokes_sizes(p, sizes_out);
    return PKASP_OK;
}

int pkasp_stokes_apply(pkasp_problem *p, const double *x_dev, double *y_dev, pkasp_stream_t stream) {
    if (!p || !x_dev || !y_dev) return set_error(PKASP_EINVAL, "NULL argument");
    return guarded([&]() -> int {
        pk::stokes_apply(p, x_dev, y_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_stokes_apply_prec(pkasp_problem *p, const double *r_dev, double *z_dev, pkasp_stream_t stream) {
    if (!p || !r_dev || !z_dev) return set_error(PKASP_EINVAL, "NULL argument");
    return guarded([&]() -> int {
        pk::stokes_prec(p, r_dev, z_dev, (cudaStream_t)stream);
        if (p->fine_tpr < -1) pk::check_barrier(p, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_stokes_solve(pkasp_problem *p, const double *b_dev, double *x_dev, pkasp_stats *st,
                       pkasp_stream_t stream) {
    if (!p || !b_dev || !x_dev) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->st) return set_error(PKASP_ESTATE, "pkasp_stokes_setup first");
    return guarded([&]() -> int {
        const int rc = pk::stokes_solve(p, b_dev, x_dev, st, (cudaStream_t)stream);
        pk::l2_window_idle(p);
        if (rc != PKASP_OK) return set_error(rc, "FGMRES on the Stokes system reached max_iter before the tolerance");
        return PKASP_OK;
    });
}

int pkasp_get_colours(const pkasp_problem *p, int level, int32_t *colour_host, int *ncolours) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    const pk::DSplit *sp = nullptr;
    int64_t n = 0;
    if (level < 0) {
        sp = &p->fine;
        n = p->nh;
    } else if (level < (int)p->lev.size()) {
        sp = &p->lev[level].sp;
        n = p->lev[level].A.n;
    } else {
        return set_error(PKASP_EINVAL, "no such level");
    }
    if (ncolours) *ncolours = sp->ncol;
    return guarded([&]() -> int {
        if (colour_host) PK_CUDA(cudaMemcpy(colour_host, sp->colour, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        return PKASP_OK;
    });
}

int pkasp_get_splitting(const pkasp_problem *p, int level, int8_t *cf_host, uint8_t *strong_host) {
    if (!p) return set_error(PKASP_EINVAL, "NULL problem");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    if (level < 0 || level >= (int)p->lev.size() || !p->lev[level].cf)
        return set_error(PKASP_EINVAL, "level has no splitting");
    const pk::Level &L = p->lev[level];
    return guarded([&]() -> int {
        if (cf_host) PK_CUDA(cudaMemcpy(cf_host, L.cf, L.A.n, cudaMemcpyDeviceToHost));
        if (strong_host && L.A.nnz) PK_CUDA(cudaMemcpy(strong_host, L.strong, L.A.nnz, cudaMemcpyDeviceToHost));
        return PKASP_OK;
    });
}

int pkasp_pmis(int64_t n, const int64_t *ptr_dev, const int32_t *col_dev, const uint8_t *strong_dev,
               uint64_t stream_id, int8_t *cf_dev, pkasp_stream_t stream) {
    if (n < 0 || !ptr_dev || !col_dev || !strong_dev || !cf_dev) return set_error(PKASP_EINVAL, "bad argument");
    return guarded([&]() -> int {
        pk::pmis_device(n, ptr_dev, col_dev, strong_dev, stream_id, cf_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_pmis_noalloc(int64_t n, const int64_t *ptr_dev, const int32_t *col_dev, const uint8_t *strong_dev,
                       uint64_t stream_id, int8_t *cf_dev, pkasp_stream_t stream) {
    if (n < 0 || !ptr_dev || !col_dev || !strong_dev || !cf_dev) return set_error(PKASP_EINVAL, "bad argument");
    return guarded([&]() -> int {
        pk::pmis_noalloc(n, ptr_dev, col_dev, strong_dev, stream_id, cf_dev, (cudaStream_t)stream);
        return PKASP_OK;
    });
}

int pkasp_dofmap_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                      int64_t *sizes_out, int64_t *dof_all_host, int32_t *elem_dof_host, int64_t *ah_ptr_host,
                      int32_t *ah_col_host, int64_t *pi_ptr_host, int32_t *pi_col_host, double *pi_val_host) {
    if (!xyz_host || !tets_host || !sizes_out) return set_error(PKASP_EINVAL, "NULL argument");
    if (nv <= 0 || nt <= 0 || k < 1 || k > 4) return set_error(PKASP_EINVAL, "bad sizes or degree");
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (tets_host[i] < 0 || tets_host[i] >= nv)
            return set_error(PKASP_EMESH, "tetrahedron vertex index out of range");
    return guarded([&]() -> int {
        pk::DofMap D;
        pk::HostMesh M{k, nv, nt, xyz_host, tets_host};
        pk::build_dofmap(M, D);
        sizes_out[0] = D.n_all;
        sizes_out[1] = D.nh;
        sizes_out[2] = D.nH;
        sizes_out[3] = D.Ah_pattern.ptr.back();
        sizes_out[4] = D.AH_pattern.ptr.back();
        sizes_out[5] = D.Pi.ptr.back();
        if (dof_all_host) memcpy(dof_all_host, D.dof_all.data(), sizeof(int64_t) * D.nh);
        if (elem_dof_host) memcpy(elem_dof_host, D.elem_dof.data(), sizeof(int32_t) * D.elem_dof.size());
        if (ah_ptr_host) memcpy(ah_ptr_host, D.Ah_pattern.ptr.data(), sizeof(int64_t) * (D.nh + 1));
        if (ah_col_host) memcpy(ah_col_host, D.Ah_pattern.col.data(), sizeof(int32_t) * D.Ah_pattern.col.size());
        if (pi_ptr_host) memcpy(pi_ptr_host, D.Pi.ptr.data(), sizeof(int64_t) * (D.nh + 1));
        if (pi_col_host) memcpy(pi_col_host, D.Pi.col.data(), sizeof(int32_t) * D.Pi.col.size());
        if (pi_val_host) memcpy(pi_val_host, D.Pi.val.data(), sizeof(double) * D.Pi.val.size());
        return PKASP_OK;
    });
}

int pkasp_nodes_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                     int64_t *n_all_out, double *node_xyz_host) {
    if (!xyz_host || !tets_host || !n_all_out) return set_error(PKASP_EINVAL, "NULL argument");
    if (nv <= 0 || nt <= 0 || k < 1 || k > 4) return set_error(PKASP_EINVAL, "bad sizes or degree");
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (tets_host[i] < 0 || tets_host[i] >= nv)
            return set_error(PKASP_EMESH, "tetrahedron vertex index out of range");
    return guarded([&]() -> int {
        pk::DofMap D;
        pk::HostMesh M{k, nv, nt, xyz_host, tets_host};
        pk::build_dofmap(M, D);
        *n_all_out = D.n_all;
        if (!node_xyz_host) return PKASP_OK;
        std::vector<int> m4;
        pk::ref_nodes(k, m4);
        const int nl = pk::nloc_of(k);
        for (int64_t t = 0; t < nt; ++t)
            for (int m = 0; m < nl; ++m) {
                const int64_t d = D.elem_all[t * nl + m];
                for (int c = 0; c < 3; ++c) {
                    double v = 0;
                    for (int a = 0; a < 4; ++a) v += m4[4 * m + a] * xyz_host[3 * (int64_t)tets_host[4 * t + a] + c];
                    node_xyz_host[3 * d + c] = v / k;
                }
            }
        return PKASP_OK;
    });
}

int pkasp_stokes_blocks_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                             int64_t *sizes_out, int64_t *b_ptr, int32_t *b_col, double *b_val,
                             int64_t *m_ptr, int32_t *m_col, double *m_val) {
    if (!xyz_host || !tets_host || !sizes_out) return set_error(PKASP_EINVAL, "NULL argument");
    if (nv <= 0 || nt <= 0 || k < 2 || k > 4) return set_error(PKASP_EINVAL, "bad sizes or degree (k = 2..4)");
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (tets_host[i] < 0 || tets_host[i] >= nv)
            return set_error(PKASP_EMESH, "tetrahedron vertex index out of range");
    return guarded([&]() -> int {
        pk::DofMap D;
        pk::HostMesh M{k, nv, nt, xyz_host, tets_host};
        pk::build_dofmap(M, D);
        pk::HCSR B, BT, Mp;
        int64_t np = 0;
        pk::stokes_blocks(k, nv, nt, xyz_host, tets_host, D.nh, D.elem_dof.data(), B, BT, Mp, np);
        sizes_out[0] = D.nh;
        sizes_out[1] = np;
        sizes_out[2] = B.ptr.back();
        sizes_out[3] = Mp.ptr.back();
        if (b_ptr) memcpy(b_ptr, B.ptr.data(), sizeof(int64_t) * B.ptr.size());
        if (b_col) memcpy(b_col, B.col.data(), sizeof(int32_t) * B.col.size());
        if (b_val) memcpy(b_val, B.val.data(), sizeof(double) * B.val.size());
        if (m_ptr) memcpy(m_ptr, Mp.ptr.data(), sizeof(int64_t) * Mp.ptr.size());
        if (m_col) memcpy(m_col, Mp.col.data(), sizeof(int32_t) * Mp.col.size());
        if (m_val) memcpy(m_val, Mp.val.data(), sizeof(double) * Mp.val.size());
        return PKASP_OK;
    });
}

int pkasp_reference_tensors(int k, double *S_out) {
    if (k < 1 || k > 4 || !S_out) return set_error(PKASP_EINVAL, "bad argument");
    return guarded([&]() -> int {
        std::vector<double> S;
        pk::reference_tensors(k, S);
        memcpy(S_out, S.data(), sizeof(double) * S.size());
        return PKASP_OK;
    });
}

int pkasp_time_kernel(pkasp_problem *p, int which, int reps, float *ms_out, pkasp_stream_t stream) {
    if (!p || !ms_out) return set_error(PKASP_EINVAL, "NULL argument");
    if (!p->have_setup) return set_error(PKASP_ESTATE, "setup first");
    return guarded([&]() -> int {
        *ms_out = pk::time_kernel(p, which, reps, (cudaStream_t)stream);
        pk::l2_window_idle(p);
        return PKASP_OK;
    });
}

}  // extern "C"
