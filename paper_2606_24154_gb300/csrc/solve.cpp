// solve.cpp -- solve orchestration on the context stream: influence-matrix fill,
// LU factorisation (FP64, or FP32 for mixed solves), right-hand side, substitution and
// FP64 iterative refinement; evaluation dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "geometry.h"

namespace nb {

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)

static int elapsed_ms(Ctx* c, double* ms) {
    CK(cudaEventRecord(c->ev1, c->stream));
    CK(cudaEventSynchronize(c->ev1));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, c->ev0, c->ev1));
    if (ms) *ms = f;
    return 0;
}

int ensure_fill_tables(Ctx* c) {
    if (c->fill_tables) return 0;
    std::vector<FillEl> fe;
    std::vector<float4> nodes, tau;
    build_fill_tables(c->h_el, c->img, fe, nodes, tau);
    std::vector<int32_t> cell_start, cell_items;
    std::string why;
    int rc = build_near_grid(c->h_el, c->img, kFillRatioC, c->fill_grid, cell_start, cell_items, why);
    if (rc) return fail(rc, why);
    CK(c->d_fill_el.ensure(sizeof(FillEl) * fe.size()));
    CK(c->d_fill_nodes.ensure(sizeof(float4) * nodes.size()));
    CK(c->d_fill_tau.ensure(sizeof(float4) * tau.size()));
    CK(c->d_fill_cell_start.ensure(sizeof(int32_t) * cell_start.size()));
    CK(c->d_fill_cell_items.ensure(sizeof(int32_t) * cell_items.size()));
    CK(cudaMemcpyAsync(c->d_fill_el.ptr, fe.data(), sizeof(FillEl) * fe.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fill_nodes.ptr, nodes.data(), sizeof(float4) * nodes.size(), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_fill_tau.ptr, tau.data(), sizeof(float4) * tau.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fill_cell_start.ptr, cell_start.data(), sizeof(int32_t) * cell_start.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fill_cell_items.ptr, cell_items.data(), sizeof(int32_t) * cell_items.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    c->fill_tables = true;
    return 0;
}

int ensure_fill(Ctx* c, int precision, double* ms) {
    if (c->K_valid && (c->K_prec == NEBEM_FP64 || c->K_prec == precision)) return 0;
    const int64_t n = c->n;
    if (precision == NEBEM_MIXED) {
        int rc = ensure_fill_tables(c);
        if (rc) return rc;
    }
    CK(c->d_K.ensure(sizeof(double) * n * n));
    CK(cudaEventRecord(c->ev0, c->stream));
    if (precision == NEBEM_MIXED)
        CK(launch_fill_mixed(c->d_el.as<Elem>(), c->d_fill_el.as<FillEl>(), c->d_fill_nodes.as<float4>(),
                             c->d_fill_tau.as<float4>(), c->d_cjk.as<float4>(), c->d_diag.as<double>(), n, c->img,
                             c->fill_grid, c->d_fill_cell_start.as<int32_t>(), c->d_fill_cell_items.as<int32_t>(),
                             c->d_K.as<double>(), c->stream));
    else
        CK(launch_fill_f64(c->d_el.as<Elem>(), c->d_diag.as<double>(), n, c->img, c->d_K.as<double>(), c->stream));
    int rc = elapsed_ms(c, ms);
    if (rc) return rc;
    c->K_valid = true;
    c->K_prec = precision;
    c->fac64_valid = c->fac32_valid = false;
    return 0;
}

int ensure_factors(Ctx* c, int precision, double* ms) {
    const int64_t n = c->n;
    const int nb = c->opt.lu_block;
    int h_info = 0;
    if (precision == NEBEM_FP64) {
        if (c->fac64_valid) return 0;
        CK(c->d_LU64.ensure(sizeof(double) * n * n));
        CK(c->d_piv64.ensure(sizeof(int32_t) * n));
        CK(c->d_work.ensure(sizeof(double) * lu_work_elems(n, nb)));
        CK(c->d_small.ensure(256));
        CK(cudaEventRecord(c->ev0, c->stream));
        CK(cudaMemcpyAsync(c->d_LU64.ptr, c->d_K.ptr, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream));
        CK(lu_factor_f64(c->d_LU64.as<double>(), n, c->d_piv64.as<int32_t>(), nb, c->d_work.as<double>(),
                         c->d_small.as<int>(), c->stream));
        int rc = elapsed_ms(c, ms);
        if (rc) return rc;
        CK(cudaMemcpy(&h_info, c->d_small.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        if (h_info) return fail(NEBEM_SINGULAR, "zero pivot at column " + std::to_string(h_info - 1));
        CK(c->d_perm64.ensure(sizeof(int32_t) * n));
        CK(lu_make_perm(c->d_piv64.as<int32_t>(), n, c->d_perm64.as<int32_t>(), c->stream));
        c->fac64_valid = true;
    } else {
        if (c->fac32_valid) return 0;
        CK(c->d_LU32.ensure(sizeof(float) * n * n));
        CK(c->d_piv32.ensure(sizeof(int32_t) * n));
        CK(c->d_work.ensure(std::max(sizeof(double) * lu_work_elems(n, nb), lu_work_bytes_f32(n, nb))));
        CK(c->d_small.ensure(256));
        CK(cudaEventRecord(c->ev0, c->stream));
        CK(copy_f64_to_f32(c->d_K.as<double>(), c->d_LU32.as<float>(), n * n, c->stream));
        CK(lu_factor_f32(c->d_LU32.as<float>(), n, c->d_piv32.as<int32_t>(), nb, c->d_work.as<float>(),
                         c->d_small.as<int>(), c->stream, c->opt.wait_polls));
        int rc = elapsed_ms(c, ms);
        if (rc) return rc;
        int h2[2] = {0, 0};
        CK(cudaMemcpy(h2, c->d_small.ptr, sizeof(h2), cudaMemcpyDeviceToHost));
        h_info = h2[0];
        if (h2[1]) return fail(NEBEM_TIMEOUT, "FP32 factorisation: a bounded wait gave up (panel barrier or tensor-core update)");
        if (h_info) return fail(NEBEM_SINGULAR, "zero pivot at column " + std::to_string(h_info - 1));
        CK(c->d_perm32.ensure(sizeof(int32_t) * n));
        CK(lu_make_perm(c->d_piv32.as<int32_t>(), n, c->d_perm32.as<int32_t>(), c->stream));
        c->fac32_valid = true;
    }
    return 0;
}

// b_i = V(conductor_i) on conductor rows, 0 on interface rows; minus the known-charge
// potential / normal field at the collocation points when a charge set is present.
int build_rhs(Ctx* c) {
    const int64_t n = c->n;
    std::vector<double> b((size_t)n);
    for (int64_t i = 0; i < n; ++i) b[i] = (c->h_bc[i] == NEBEM_CONDUCTOR) ? c->voltages[c->h_cond[i]] : 0.0;
    CK(c->d_b.ensure(sizeof(double) * n));
    CK(cudaMemcpyAsync(c->d_b.ptr, b.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (c->n_car > 0) {
        int rc = rhs_known_charge(c);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(c->stream));
    return 0;
}

int solve_with_factors(Ctx* c, int precision, nebem_solve_info* info) {
    const int64_t n = c->n;
    CK(c->d_x.ensure(sizeof(double) * n));
    CK(c->d_r.ensure(sizeof(double) * n));
    CK(c->d_small.ensure(256));
    double* x = c->d_sigma.as<double>();
    double* b = c->d_b.as<double>();
    double* r = c->d_r.as<double>();
    double* norms = reinterpret_cast<double*>(c->d_small.as<char>() + 64);
    CK(c->d_swork.ensure(std::max(lu_solve_work_bytes(n, sizeof(double)), residual_work_bytes(n))));
    void* work = c->d_swork.ptr;
    CK(cudaEventRecord(c->ev0, c->stream));
    int status = 0;
    int gave_up = 0;  // a block-flag wait of a triangular sweep ran out (its block is NaN)
    if (precision == NEBEM_FP64) {
        CK(cudaMemcpyAsync(x, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        CK(lu_solve_f64(c->d_LU64.as<double>(), n, c->d_perm64.as<int32_t>(), x, work, c->stream, c->opt.wait_polls));
        CK(cudaMemcpyAsync(&gave_up, lu_solve_err_flag(work, n, sizeof(double)), sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
    } else {
        CK(c->d_r32.ensure(sizeof(float) * n));
        float* d32 = c->d_r32.as<float>();
        CK(cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
        CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        double corr = 1.0;
        int it = 0;
        status = NEBEM_NOT_CONVERGED;
        for (it = 1; it <= c->opt.ir_max_iter; ++it) {
            CK(copy_f64_to_f32(r, d32, n, c->stream));
            CK(lu_solve_f32(c->d_LU32.as<float>(), n, c->d_perm32.as<int32_t>(), d32, work, c->stream,
                            c->opt.wait_polls));
            CK(cudaMemcpyAsync(&gave_up, lu_solve_err_flag(work, n, sizeof(float)), sizeof(int),
                               cudaMemcpyDeviceToHost, c->stream));
            CK(ir_update(x, d32, n, norms, c->stream));
            double h[2];
            CK(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (gave_up) {
                status = NEBEM_TIMEOUT;
                break;
            }
            corr = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
            if (!std::isfinite(corr)) break;
            CK(gemv_residual(c->d_K.as<double>(), n, x, b, r, work, c->stream));
            if (corr <= c->opt.ir_tol) {
                status = 0;
                break;
            }
        }
        if (info) {
            info->iterations = std::min(it, c->opt.ir_max_iter);
            info->correction = corr;
        }
    }
    double ms = 0.0;
    int rc = elapsed_ms(c, &ms);
    if (rc) return rc;
    if (info) info->ms_solve = ms;
    // residual diagnostic ||K x - b||_inf / (||K||_inf-ish ||x||_inf)
    CK(gemv_residual(c->d_K.as<double>(), n, x, b, r, work, c->stream));
    CK(vec_absmax(r, n, norms, c->stream));
    CK(vec_absmax(x, n, norms + 1, c->stream));
    double h[2];
    CK(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (info) info->residual = (h[1] > 0.0) ? h[0] / h[1] : 0.0;
    ++c->sigma_version;
    if (gave_up || status == NEBEM_TIMEOUT) {
        c->sigma_valid = false;  // NaN in the blocks whose wait ran out
        return fail(NEBEM_TIMEOUT, "triangular sweep: a bounded wait gave up (sigma is NaN there)");
    }
    c->sigma_valid = true;
    if (status) return fail(status, "iterative refinement did not reach the tolerance");
    return 0;
}

// Weighting fields (Sec. 2.1): K does not depend on the voltages, so the k unit-readout
// right-hand sides are solved with the factors already made, all columns in one pass of
// each triangular sweep.  FP64: one multi-column solve.  MIXED: FP32 solves of the
// residuals with FP64 iterative refinement, every column stepping exactly as a single
// solve of its own right-hand side would (it drops out when its correction meets ir_tol),
// so column j equals that solve bit for bit.
int weighting_solve(Ctx* c, const int32_t* readout, int k, int precision, nebem_solve_info* info) {
    const int64_t n = c->n;
    const size_t nk = (size_t)n * (size_t)k;
    std::vector<double> b(nk, 0.0);
    for (int j = 0; j < k; ++j)
        for (int64_t i = 0; i < n; ++i)
            if (c->h_bc[i] == NEBEM_CONDUCTOR && c->h_cond[i] == readout[j]) b[(size_t)j * n + i] = 1.0;
    CK(c->d_wB.ensure(sizeof(double) * nk));
    CK(c->d_wX.ensure(sizeof(double) * nk));
    CK(c->d_wR.ensure(sizeof(double) * nk));
    CK(c->d_small.ensure(256));
    CK(c->d_r.ensure(sizeof(double) * 2 * 64));  // per-column norms
    const size_t tsize = (precision == NEBEM_FP64) ? sizeof(double) : sizeof(float);
    CK(c->d_swork.ensure(std::max(lu_solve_multi_work_bytes(n, tsize), residual_multi_work_bytes(n))));
    void* work = c->d_swork.ptr;
    double* B = c->d_wB.as<double>();
    double* X = c->d_wX.as<double>();
    double* R = c->d_wR.as<double>();
    double* norms = c->d_r.as<double>();
    CK(cudaMemcpyAsync(B, b.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->ev0, c->stream));
    int gave_up = 0, status = 0, iters = 0;
    double corr_max = 0.0;
    if (precision == NEBEM_FP64) {
        CK(cudaMemcpyAsync(X, B, sizeof(double) * nk, cudaMemcpyDeviceToDevice, c->stream));
        CK(lu_solve_multi_f64(c->d_LU64.as<double>(), n, c->d_perm64.as<int32_t>(), X, k, work, c->stream,
                              c->opt.wait_polls));
        CK(cudaMemcpyAsync(&gave_up, lu_solve_multi_err_flag(work, n, tsize), sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        CK(c->d_wR32.ensure(sizeof(float) * nk));
        float* D = c->d_wR32.as<float>();
        CK(cudaMemsetAsync(X, 0, sizeof(double) * nk, c->stream));
        CK(cudaMemcpyAsync(R, B, sizeof(double) * nk, cudaMemcpyDeviceToDevice, c->stream));
        uint64_t active = (k == 64) ? ~0ull : ((1ull << k) - 1ull);
        uint64_t converged = 0;
        std::vector<double> h(2 * (size_t)k);
        std::vector<double> corr((size_t)k, 1.0);
        int it = 0;
        for (it = 1; it <= c->opt.ir_max_iter && active; ++it) {
            CK(copy_f64_to_f32(R, D, (int64_t)nk, c->stream));
            CK(lu_solve_multi_f32(c->d_LU32.as<float>(), n, c->d_perm32.as<int32_t>(), D, k, work, c->stream,
                                  c->opt.wait_polls));
            CK(cudaMemcpyAsync(&gave_up, lu_solve_multi_err_flag(work, n, tsize), sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
            CK(ir_update_multi(X, D, n, k, active, norms, c->stream));
            CK(cudaMemcpyAsync(h.data(), norms, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (gave_up) break;
            uint64_t next = active;
            for (int j = 0; j < k; ++j) {
                if (!((active >> j) & 1ull)) continue;
                corr[j] = (h[2 * j + 1] > 0.0) ? h[2 * j] / h[2 * j + 1] : 0.0;
                if (!std::isfinite(corr[j])) next &= ~(1ull << j);  // stops unconverged
            }
            CK(gemv_residual_multi(c->d_K.as<double>(), n, X, k, B, R, work, c->stream));
            for (int j = 0; j < k; ++j)
                if (((next >> j) & 1ull) && corr[j] <= c->opt.ir_tol) {
                    next &= ~(1ull << j);
                    converged |= 1ull << j;
                }
            iters = it;
            active = next;
        }
        const uint64_t all = (k == 64) ? ~0ull : ((1ull << k) - 1ull);
        if (converged != all) status = NEBEM_NOT_CONVERGED;
        for (int j = 0; j < k; ++j) corr_max = std::max(corr_max, corr[j]);
    }
    double ms = 0.0;
    int rc = elapsed_ms(c, &ms);
    if (rc) return rc;
    // residual diagnostic per column, the largest ||K x_j - b_j||_inf / ||x_j||_inf
    CK(gemv_residual_multi(c->d_K.as<double>(), n, X, k, B, R, work, c->stream));
    double res = 0.0;
    for (int j = 0; j < k; ++j) {
        CK(vec_absmax(R + (size_t)j * n, n, norms, c->stream));
        CK(vec_absmax(X + (size_t)j * n, n, norms + 1, c->stream));
        double hh[2];
        CK(cudaMemcpyAsync(hh, norms, sizeof(hh), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        res = std::max(res, hh[1] > 0.0 ? hh[0] / hh[1] : 0.0);
    }
    if (info) {
        info->iterations = iters;
        info->correction = corr_max;
        info->residual = res;
        info->ms_solve = ms;
    }
    if (gave_up) return fail(NEBEM_TIMEOUT, "triangular sweep: a bounded wait gave up (NaN in its blocks)");
    if (status) return fail(status, "iterative refinement did not reach the tolerance for every readout");
    return 0;
}

int eval_set(Ctx* c, const EvalSet& es, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
             cudaStream_t s) {
    if (precision == NEBEM_MIXED) {
        CK(c->d_scratch.ensure(eval_mixed_scratch_bytes(n)));
        CK(launch_eval_mixed(es.el, es.far, es.cjk.as<float4>(), es.sigma, es.n, es.img, es.grid,
                             es.cell_start.as<int32_t>(), es.cell_items.as<int32_t>(), d_pts, n, d_phi, d_E,
                             mixed_scratch(c->d_scratch.ptr, n), s));
    } else {
        CK(launch_eval_f64(es.el, es.sigma, es.n, es.img, d_pts, n, d_phi, d_E, s));
    }
    return 0;
}

int eval_elements(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision, cudaStream_t s,
                  double* err) {
    if (c->am_on) return eval_adaptive(c, d_pts, n, d_phi, d_E, precision, s);
    if (precision == NEBEM_MIXED) {
        const bool refine = c->opt.mixed_point_tol > 0.0 && n > 0;
        if (refine || err) {
            const int rc = ensure_fill_tables(c);
            if (rc) return rc;
        }
        const size_t ms_bytes = eval_mixed_scratch_bytes(n);  // a multiple of 256
        CK(c->d_scratch.ensure(ms_bytes + refine_part_bytes(n, c->props.multiProcessorCount, c->n)));
        const MixedScratch ms = mixed_scratch(c->d_scratch.ptr, n);
        c->eval_timed = false;
        CK(cudaEventRecord(c->ev_eval[0], s));
        CK(launch_eval_mixed(c->d_el.as<Elem>(), c->d_far.as<FarNodes>(), c->d_cjk.as<float4>(),
                             c->d_sigma.as<double>(), c->n, c->img, c->grid, c->d_cell_start.as<int32_t>(),
                             c->d_cell_items.as<int32_t>(), d_pts, n, d_phi, d_E, ms, s));
        CK(cudaEventRecord(c->ev_eval[1], s));
        if (refine || err) {
            AccView A;
            A.view = make_view(c->d_el.as<Elem>(), c->d_far.as<FarNodes>(), c->d_cjk.as<float4>(),
                               c->d_sigma.as<double>(), c->n, c->img, c->grid, c->d_cell_start.as<int32_t>(),
                               c->d_cell_items.as<int32_t>());
            A.far = c->d_far.as<FarNodes>();
            A.el = c->d_el.as<Elem>();
            A.fe = c->d_fill_el.as<FillEl>();
            A.nodes = c->d_fill_nodes.as<float4>();
            A.tau = c->d_fill_tau.as<float4>();
            A.cjk = c->d_cjk.as<float4>();
            A.sigma = c->d_sigma.as<double>();
            A.n_el = c->n;
            A.grid = c->fill_grid;
            A.cell_start = c->d_fill_cell_start.as<int32_t>();
            A.cell_items = c->d_fill_cell_items.as<int32_t>();
            CK(launch_eval_refine(A, c->img, d_pts, n, d_phi, d_E, err, c->opt.mixed_point_tol, c->err_model, ms, c->props.multiProcessorCount, s, &c->ev_eval[2],
                                  static_cast<char*>(c->d_scratch.ptr) + ms_bytes));
            c->refine_list = ms.n_list;
        } else {
            CK(cudaMemsetAsync(ms.n_list, 0, 4 * sizeof(int32_t), s));
            CK(cudaEventRecord(c->ev_eval[2], s));
            CK(cudaEventRecord(c->ev_eval[3], s));
            c->refine_list = ms.n_list;
        }
        c->eval_timed = true;
        c->eval_points_n = n;
    } else {
        CK(launch_eval_f64(c->d_el.as<Elem>(), c->d_sigma.as<double>(), c->n, c->img, d_pts, n, d_phi, d_E, s));
    }
    return 0;
}

int eval_points(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision, cudaStream_t s,
                double* err) {
    int rc = eval_elements(c, d_pts, n, d_phi, d_E, precision, s, err);
    if (rc) return rc;
    return add_known_charge(c, d_pts, n, d_phi, d_E, precision, s);
}


}  // namespace nb
