// api.cpp -- the C-ABI of libnebem (declared in include/nebem.h): context lifetime,
// geometry and boundary conditions, solve orchestration (fill -> LU -> substitution
// [-> FP64 refinement]), evaluation at points, known-charge set and dynamic steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "context.h"
#include "geometry.h"

namespace nb {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? NEBEM_OUT_OF_MEMORY : NEBEM_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

cudaError_t DevBuf::ensure(size_t nbytes) {
    if (bytes >= nbytes && ptr) return cudaSuccess;
    release();
    if (nbytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&ptr, nbytes);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        return e;
    }
    bytes = nbytes;
    return cudaSuccess;
}

int check_count(int64_t n, const char* what) {
    if (n > NEBEM_MAX_COUNT) return fail(NEBEM_TOO_LARGE, std::string(what) + " above 2^31 - 1");
    return 0;
}

Ctx::~Ctx() {
    // the device buffers free themselves after this body, on the device set here
    cudaSetDevice(device);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : ev_eval)
        if (e) cudaEventDestroy(e);
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace nb

using namespace nb;

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)

extern "C" {

const char* nebem_last_error(void) { return g_last_error.c_str(); }

const char* nebem_status_string(int s) {
    switch (s) {
        case NEBEM_OK: return "NEBEM_OK";
        case NEBEM_INVALID_ARG: return "NEBEM_INVALID_ARG";
        case NEBEM_BAD_STATE: return "NEBEM_BAD_STATE";
        case NEBEM_OUT_OF_MEMORY: return "NEBEM_OUT_OF_MEMORY";
        case NEBEM_CUDA: return "NEBEM_CUDA";
        case NEBEM_SINGULAR: return "NEBEM_SINGULAR";
        case NEBEM_NOT_CONVERGED: return "NEBEM_NOT_CONVERGED";
        case NEBEM_TIMEOUT: return "NEBEM_TIMEOUT";
        case NEBEM_DEGENERATE_ELEMENT: return "NEBEM_DEGENERATE_ELEMENT";
        case NEBEM_NO_DEVICE: return "NEBEM_NO_DEVICE";
        case NEBEM_TOO_LARGE: return "NEBEM_TOO_LARGE";
        default: return "NEBEM_UNKNOWN_STATUS";
    }
}

int nebem_default_options(nebem_options* opt) {
    if (!opt) return fail(NEBEM_INVALID_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->device = 0;
    opt->ir_max_iter = 30;
    opt->ir_tol = 1e-8;
    opt->ratio_0 = 64.0;
    opt->ratio_a = 24.0;
    opt->ratio_b = 8.0;
    opt->ratio_near = 3.0;
    opt->softening = 1e-6;
    opt->sc_near = 1e-4;
    opt->lu_block = 64;
    opt->mixed_point_tol = 1e-6;
    return NEBEM_OK;
}

int nebem_create(nebem_ctx** out, const nebem_options* opt) {
    if (!out) return fail(NEBEM_INVALID_ARG, "out is NULL");
    *out = nullptr;
    nebem_options o;
    nebem_default_options(&o);
    if (opt) o = *opt;
    if (o.lu_block < 32 || o.lu_block > 64 || o.lu_block % 32) return fail(NEBEM_INVALID_ARG, "lu_block must be 32 or 64");
    if (!(o.ir_tol > 0.0) || o.ir_max_iter < 1) return fail(NEBEM_INVALID_ARG, "bad refinement options");
    if (!(o.ratio_near >= 1.5) || !(o.ratio_b >= o.ratio_near) || !(o.ratio_a >= o.ratio_b) ||
        !(o.ratio_0 >= o.ratio_a) || !(o.ratio_0 < 1e6))
        return fail(NEBEM_INVALID_ARG, "need 1.5 <= ratio_near <= ratio_b <= ratio_a <= ratio_0");
    if (!(o.softening > 0.0)) return fail(NEBEM_INVALID_ARG, "softening must be > 0");
    if (!(o.mixed_point_tol >= 0.0) || !(o.mixed_point_tol < 1.0))
        return fail(NEBEM_INVALID_ARG, "mixed_point_tol must be in [0, 1)");
    if (o.wait_polls < 0) return fail(NEBEM_INVALID_ARG, "wait_polls must be >= 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(NEBEM_NO_DEVICE, "no CUDA device");
    }
    if (o.device < 0 || o.device >= ndev) return fail(NEBEM_INVALID_ARG, "device ordinal out of range");
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return fail(NEBEM_OUT_OF_MEMORY, "host allocation failed");
    c->opt = o;
    c->device = o.device;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev_eval[k]);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&c->props, c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "nebem_create");
    }
    *out = reinterpret_cast<nebem_ctx*>(c);
    return NEBEM_OK;
}

int nebem_destroy(nebem_ctx* ctx) {
    if (!ctx) return NEBEM_OK;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    delete c;
    return NEBEM_OK;
}

int nebem_set_geometry(nebem_ctx* ctx, const nebem_element* el, int64_t n, const double* lattice, int32_t img_lo,
                       int32_t img_hi) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n <= 0 || !el) return fail(NEBEM_INVALID_ARG, "need n > 0 elements");
    if (n > (int64_t)INT32_MAX) return fail(NEBEM_TOO_LARGE, "too many elements");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    CK(cudaSetDevice(c->device));
    std::string why;
    ImageTable img;
    int rc = build_images(lattice, img_lo, img_hi, img, why);
    if (rc) return fail(rc, why);
    std::vector<Elem> h_el((size_t)n);
    std::vector<FarNodes> h_far((size_t)n);
    std::vector<double> h_diag((size_t)n);
    std::vector<int32_t> h_bc((size_t)n), h_cond((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        if (el[i].reserved != 0) return fail(NEBEM_INVALID_ARG, "element " + std::to_string(i) + ": reserved != 0");
        rc = build_element(el[i], c->opt, h_el[i], h_diag[i], h_far[i], why);
        if (rc) return fail(rc, "element " + std::to_string(i) + ": " + why);
        h_bc[i] = el[i].bc;
        h_cond[i] = el[i].conductor;
    }
    NearGrid grid;
    std::vector<int32_t> cell_start, cell_items;
    rc = build_near_grid(h_el, img, c->opt.ratio_near, grid, cell_start, cell_items, why);
    if (rc) return fail(rc, why);
    CK(cudaStreamSynchronize(c->stream));
    // invalidate everything that depends on the geometry
    c->n = 0;
    c->K_valid = c->fac64_valid = c->fac32_valid = c->sigma_valid = false;
    c->fill_tables = false;
    ++c->sigma_version;
    c->bc_set = false;
    c->n_car = 0;
    c->sc_lines = false;
    c->am_on = false;
    c->am_prim_after = -1;
    c->am_near.release_all();
    c->am_far.release_all();
    CK(c->d_el.ensure(sizeof(Elem) * n));
    CK(c->d_far.ensure(sizeof(FarNodes) * n));
    CK(c->d_diag.ensure(sizeof(double) * n));
    CK(c->d_sigma.ensure(sizeof(double) * n));
    CK(cudaMemcpyAsync(c->d_el.ptr, h_el.data(), sizeof(Elem) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_far.ptr, h_far.data(), sizeof(FarNodes) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_diag.ptr, h_diag.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(c->d_cjk.ensure(sizeof(float4) * 2 * n * img.n));
    CK(launch_image_centroids(c->d_el.as<Elem>(), n, img, c->d_cjk.as<float4>(), c->stream));
    CK(c->d_cell_start.ensure(sizeof(int32_t) * cell_start.size()));
    CK(c->d_cell_items.ensure(sizeof(int32_t) * cell_items.size()));
    CK(cudaMemcpyAsync(c->d_cell_start.ptr, cell_start.data(), sizeof(int32_t) * cell_start.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_cell_items.ptr, cell_items.data(), sizeof(int32_t) * cell_items.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->grid = grid;
    c->img = img;
    c->img_lo = lattice ? img_lo : 0;
    c->img_hi = lattice ? img_hi : 0;
    c->h_bc = std::move(h_bc);
    c->h_cond = std::move(h_cond);
    c->h_el = std::move(h_el);
    c->n = n;
    return NEBEM_OK;
}

int nebem_set_bc(nebem_ctx* ctx, const double* voltages, int32_t n_conductors) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    if (n_conductors < 0 || (n_conductors > 0 && !voltages)) return fail(NEBEM_INVALID_ARG, "bad voltages");
    for (int64_t i = 0; i < c->n; ++i)
        if (c->h_bc[i] == NEBEM_CONDUCTOR && (c->h_cond[i] < 0 || c->h_cond[i] >= n_conductors))
            return fail(NEBEM_INVALID_ARG, "element " + std::to_string(i) + " has conductor index out of range");
    for (int32_t k = 0; k < n_conductors; ++k)
        if (!std::isfinite(voltages[k])) return fail(NEBEM_INVALID_ARG, "non-finite voltage");
    c->voltages.assign(voltages, voltages + n_conductors);
    c->bc_set = true;
    c->sigma_valid = false;
    return NEBEM_OK;
}

int nebem_image_table(nebem_ctx* ctx, double* t_out, int64_t* count) {
    if (!ctx || !count) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    *count = c->img.n;
    if (t_out) std::memcpy(t_out, c->img.t, sizeof(double) * 3 * c->img.n);
    return NEBEM_OK;
}

int nebem_fill(nebem_ctx* ctx, int32_t precision, double* K_out) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    CK(cudaSetDevice(c->device));
    int rc = ensure_fill(c, precision, nullptr);
    if (rc) return rc;
    if (K_out) {
        CK(cudaMemcpyAsync(K_out, c->d_K.ptr, sizeof(double) * c->n * c->n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return NEBEM_OK;
}

int nebem_matrix_entries(nebem_ctx* ctx, const int64_t* rows, const int64_t* cols, int64_t count, double* out) {
    if (!ctx || count < 0 || (count > 0 && (!rows || !cols || !out))) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(count, "entry count")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    for (int64_t e = 0; e < count; ++e)
        if (rows[e] < 0 || rows[e] >= c->n || cols[e] < 0 || cols[e] >= c->n)
            return fail(NEBEM_INVALID_ARG, "entry index out of range");
    if (count == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    int rc = ensure_fill(c, c->K_valid ? c->K_prec : NEBEM_FP64, nullptr);
    if (rc) return rc;
    DevBuf idx, val;
    CK(idx.ensure(sizeof(int64_t) * count));
    CK(val.ensure(sizeof(double) * count));
    std::vector<int64_t> lin((size_t)count);
    for (int64_t e = 0; e < count; ++e) lin[e] = rows[e] + cols[e] * c->n;
    CK(cudaMemcpyAsync(idx.ptr, lin.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, c->stream));
    CK(launch_gather(c->d_K.as<double>(), idx.as<int64_t>(), count, val.as<double>(), c->stream));
    CK(cudaMemcpyAsync(out, val.ptr, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    idx.release();
    val.release();
    return NEBEM_OK;
}

int nebem_solve(nebem_ctx* ctx, int32_t precision, double* sigma_out, nebem_solve_info* info) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    if (!c->bc_set) return fail(NEBEM_BAD_STATE, "set_bc first");
    CK(cudaSetDevice(c->device));
    nebem_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.precision = precision;
    int rc = ensure_fill(c, precision, &inf.ms_fill);
    if (rc) return rc;
    c->sc_precision = precision;
    rc = ensure_factors(c, precision, &inf.ms_factor);
    if (rc) return rc;
    rc = build_rhs(c);
    if (rc) return rc;
    rc = solve_with_factors(c, precision, &inf);
    // sigma is written on success, at the refinement limit, and after a sweep's wait gave up
    // (NaN in its blocks; a factorisation that gave up returned above)
    if (sigma_out && (rc == NEBEM_OK || rc == NEBEM_NOT_CONVERGED || rc == NEBEM_TIMEOUT)) {
        CK(cudaMemcpyAsync(sigma_out, c->d_sigma.ptr, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (info) *info = inf;
    return rc;
}

int nebem_weighting_fields(nebem_ctx* ctx, const int32_t* readout, int32_t k, int32_t precision, double* sigma_out,
                           nebem_solve_info* info) {
    if (!ctx || !readout) return fail(NEBEM_INVALID_ARG, "NULL argument");
    if (k < 1 || k > 64) return fail(NEBEM_INVALID_ARG, "k must be 1..64");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    for (int32_t j = 0; j < k; ++j) {
        bool found = false;
        for (int64_t i = 0; i < c->n && !found; ++i)
            found = c->h_bc[i] == NEBEM_CONDUCTOR && c->h_cond[i] == readout[j];
        if (!found)
            return fail(NEBEM_INVALID_ARG, "readout " + std::to_string(readout[j]) + " is no conductor of the geometry");
    }
    CK(cudaSetDevice(c->device));
    nebem_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.precision = precision;
    int rc = ensure_fill(c, precision, &inf.ms_fill);
    if (rc) return rc;
    rc = ensure_factors(c, precision, &inf.ms_factor);
    if (rc) return rc;
    rc = weighting_solve(c, readout, k, precision, &inf);
    if (sigma_out && (rc == NEBEM_OK || rc == NEBEM_NOT_CONVERGED || rc == NEBEM_TIMEOUT)) {
        CK(cudaMemcpyAsync(sigma_out, c->d_wX.ptr, sizeof(double) * (size_t)c->n * (size_t)k, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (info) *info = inf;
    return rc;
}

int nebem_set_sigma(nebem_ctx* ctx, const double* sigma, int64_t n) {
    if (!ctx || !sigma) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    if (n != c->n) return fail(NEBEM_INVALID_ARG, "sigma length must equal the element count");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(c->d_sigma.ptr, sigma, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->sigma_valid = true;
    ++c->sigma_version;
    return NEBEM_OK;
}

int nebem_get_sigma(nebem_ctx* ctx, double* sigma_out, int64_t n) {
    if (!ctx || !sigma_out) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities");
    if (n != c->n) return fail(NEBEM_INVALID_ARG, "length must equal the element count");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(sigma_out, c->d_sigma.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NEBEM_OK;
}

int nebem_eval_device(nebem_ctx* ctx, const double* d_pts, int64_t n, double* d_phi, double* d_E, int32_t precision,
                      void* stream) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !d_pts)) return fail(NEBEM_INVALID_ARG, "bad points");
    if (int rc = check_count(n, "point count")) return rc;
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return eval_points(c, d_pts, n, d_phi, d_E, precision, s);
}

int nebem_eval(nebem_ctx* ctx, const double* pts, int64_t n, double* phi, double* E, int32_t precision) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !pts)) return fail(NEBEM_INVALID_ARG, "bad points");
    if (int rc = check_count(n, "point count")) return rc;
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    CK(c->d_pts.ensure(sizeof(double) * 3 * n));
    CK(c->d_phi.ensure(sizeof(double) * n));
    CK(c->d_E.ensure(sizeof(double) * 3 * n));
    CK(cudaMemcpyAsync(c->d_pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    int rc = eval_points(c, (const double*)c->d_pts.ptr, n, phi ? (double*)c->d_phi.ptr : nullptr,
                         E ? (double*)c->d_E.ptr : nullptr, precision, c->stream);
    if (rc) return rc;
    if (phi) CK(cudaMemcpyAsync(phi, c->d_phi.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    if (E) CK(cudaMemcpyAsync(E, c->d_E.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NEBEM_OK;
}

int nebem_eval_device_err(nebem_ctx* ctx, const double* d_pts, int64_t n, double* d_phi, double* d_E, double* d_err,
                          void* stream) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !d_pts)) return fail(NEBEM_INVALID_ARG, "bad points");
    if (int rc = check_count(n, "point count")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    if (c->am_on) return fail(NEBEM_BAD_STATE, "error estimates are not made with Adaptive Modelling");
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    return eval_points(c, d_pts, n, d_phi, d_E, NEBEM_MIXED, s, d_err);
}

int nebem_eval_err(nebem_ctx* ctx, const double* pts, int64_t n, double* phi, double* E, double* err,
                   int64_t* n_refined) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !pts)) return fail(NEBEM_INVALID_ARG, "bad points");
    if (int rc = check_count(n, "point count")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    if (c->am_on) return fail(NEBEM_BAD_STATE, "error estimates are not made with Adaptive Modelling");
    if (n_refined) *n_refined = 0;
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    CK(c->d_pts.ensure(sizeof(double) * 3 * n));
    CK(c->d_phi.ensure(sizeof(double) * n));
    CK(c->d_E.ensure(sizeof(double) * 3 * n));
    CK(c->d_err.ensure(sizeof(double) * 2 * n));
    CK(cudaMemcpyAsync(c->d_pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    c->refine_list = nullptr;
    int rc = eval_points(c, (const double*)c->d_pts.ptr, n, phi ? (double*)c->d_phi.ptr : nullptr,
                         E ? (double*)c->d_E.ptr : nullptr, NEBEM_MIXED, c->stream, (double*)c->d_err.ptr);
    if (rc) return rc;
    int32_t h_ref[4] = {0, 0, 0, 0};  // level 1 (phi and E), level 2, level 1 phi only, level 1 E only
    if (c->refine_list) CK(cudaMemcpyAsync(h_ref, c->refine_list, sizeof(h_ref), cudaMemcpyDeviceToHost, c->stream));
    if (phi) CK(cudaMemcpyAsync(phi, c->d_phi.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    if (E) CK(cudaMemcpyAsync(E, c->d_E.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    if (err) CK(cudaMemcpyAsync(err, c->d_err.ptr, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_refined) *n_refined = (int64_t)h_ref[0] + h_ref[2] + h_ref[3];
    return NEBEM_OK;
}

int nebem_set_error_model(nebem_ctx* ctx, double gamma_r, double gamma_b, double gamma_s) {
    if (!ctx || !std::isfinite(gamma_r) || !std::isfinite(gamma_b) || !std::isfinite(gamma_s))
        return fail(NEBEM_INVALID_ARG, "bad argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    const ErrModel d = default_err_model();
    c->err_model.gamma_r = gamma_r < 0.0 ? d.gamma_r : gamma_r;
    c->err_model.gamma_b = gamma_b < 0.0 ? d.gamma_b : gamma_b;
    c->err_model.gamma_s = gamma_s < 0.0 ? d.gamma_s : gamma_s;
    return NEBEM_OK;
}

int nebem_set_wait_polls(nebem_ctx* ctx, int32_t polls) {
    if (!ctx || polls < 0) return fail(NEBEM_INVALID_ARG, "bad argument");
    reinterpret_cast<Ctx*>(ctx)->opt.wait_polls = polls;
    return NEBEM_OK;
}

int nebem_eval_stats(nebem_ctx* ctx, nebem_eval_stats_t* out) {
    if (!ctx || !out) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->eval_timed || !c->refine_list) return fail(NEBEM_BAD_STATE, "no plain mixed evaluation yet");
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(c->ev_eval[3]));
    float t[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3; ++k) CK(cudaEventElapsedTime(&t[k], c->ev_eval[k], c->ev_eval[k + 1]));
    int32_t n4[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(n4, c->refine_list, sizeof(n4), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->points = c->eval_points_n;
    out->refined_level1 = (int64_t)n4[0] + n4[2] + n4[3];
    out->refined_level2 = n4[1];
    out->refined_level1_phi_only = n4[2];
    out->refined_level1_E_only = n4[3];
    out->ms_fp32 = t[0];
    out->ms_level1 = t[1];
    out->ms_level2 = t[2];
    return NEBEM_OK;
}

int nebem_lu_factor_device(nebem_ctx* ctx, double* d_A, int64_t n, int32_t* d_piv, void* stream) {
    if (!ctx || n <= 0 || !d_A || !d_piv) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "matrix order")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const int nb = c->opt.lu_block;
    DevBuf work, info;
    CK(work.ensure(sizeof(double) * lu_work_elems(n, nb)));
    CK(info.ensure(2 * sizeof(int)));
    CK(lu_factor_f64(d_A, n, d_piv, nb, work.as<double>(), info.as<int>(), s));
    int h_info = 0;
    CK(cudaMemcpyAsync(&h_info, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    work.release();
    info.release();
    if (h_info) return fail(NEBEM_SINGULAR, "zero pivot at column " + std::to_string(h_info - 1));
    return NEBEM_OK;
}

int nebem_lu_factor_device_f32(nebem_ctx* ctx, float* d_A, int64_t n, int32_t* d_piv, void* stream) {
    if (!ctx || n <= 0 || !d_A || !d_piv) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "matrix order")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const int nb = c->opt.lu_block;
    DevBuf work, info;
    CK(work.ensure(lu_work_bytes_f32(n, nb)));
    CK(info.ensure(2 * sizeof(int)));
    CK(lu_factor_f32(d_A, n, d_piv, nb, work.as<float>(), info.as<int>(), s));
    int h2[2] = {0, 0};
    CK(cudaMemcpyAsync(h2, info.ptr, sizeof(h2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    work.release();
    info.release();
    if (h2[1]) return fail(NEBEM_TIMEOUT, "tensor-core trailing update: bounded wait gave up");
    if (h2[0]) return fail(NEBEM_SINGULAR, "zero pivot at column " + std::to_string(h2[0] - 1));
    return NEBEM_OK;
}

int nebem_lu_solve_device(nebem_ctx* ctx, const double* d_LU, int64_t n, const int32_t* d_piv, double* d_b,
                          void* stream) {
    if (!ctx || n <= 0 || !d_LU || !d_piv || !d_b) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "matrix order")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    // stream-ordered scratch: calls in flight on different streams never share it
    const size_t wbytes = lu_solve_work_bytes(n, sizeof(double));
    void* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, wbytes + sizeof(int32_t) * (size_t)n + 256, s));
    int32_t* perm = reinterpret_cast<int32_t*>(static_cast<char*>(scratch) + ((wbytes + 255) & ~(size_t)255));
    cudaError_t e = lu_make_perm(d_piv, n, perm, s);
    if (e == cudaSuccess) e = lu_solve_f64(d_LU, n, perm, d_b, scratch, s);
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "lu_solve_f64");
    CK(ef);
    return NEBEM_OK;
}

int nebem_pair_tiers(nebem_ctx* ctx, const double* pts, int64_t n, uint8_t* codes) {
    if (!ctx || n < 0 || (n > 0 && (!pts || !codes))) return fail(NEBEM_INVALID_ARG, "bad argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    if (n > 200000000LL) return fail(NEBEM_TOO_LARGE, "more than 2e8 pairs");
    const int64_t total = n * c->n * c->img.n;
    if (total > 200000000LL) return fail(NEBEM_TOO_LARGE, "more than 2e8 pairs");
    if (total == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    DevBuf bp, bc;
    CK(bp.ensure(sizeof(double) * 3 * n));
    CK(bc.ensure((size_t)total));
    CK(cudaMemcpyAsync(bp.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(launch_pair_tiers(c->d_far.as<FarNodes>(), c->d_cjk.as<float4>(), c->n, c->img.n, bp.as<double>(), n,
                         bc.as<uint8_t>(), c->stream));
    CK(cudaMemcpyAsync(codes, bc.ptr, (size_t)total, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    bp.release();
    bc.release();
    return NEBEM_OK;
}

int nebem_element_influence(nebem_ctx* ctx, const nebem_element* el, int64_t n_el, const double* pts, int64_t n_pts,
                            double* phi_out, double* E_out) {
    if (!ctx || !el || !pts || !phi_out || !E_out || n_el <= 0 || n_pts <= 0)
        return fail(NEBEM_INVALID_ARG, "bad argument");
    if (n_el > 100000000LL || n_pts > 100000000LL || n_el * n_pts > 100000000LL)
        return fail(NEBEM_TOO_LARGE, "more than 1e8 pairs");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    CK(cudaSetDevice(c->device));
    std::vector<Elem> h((size_t)n_el);
    std::string why;
    for (int64_t i = 0; i < n_el; ++i) {
        double dg;
        FarNodes fn;
        int rc = build_element(el[i], c->opt, h[i], dg, fn, why);
        if (rc) return fail(rc, "element " + std::to_string(i) + ": " + why);
    }
    const int64_t pairs = n_el * n_pts;
    DevBuf be, bp, bphi, bE;
    CK(be.ensure(sizeof(Elem) * n_el));
    CK(bp.ensure(sizeof(double) * 3 * n_pts));
    CK(bphi.ensure(sizeof(double) * pairs));
    CK(bE.ensure(sizeof(double) * 3 * pairs));
    CK(cudaMemcpyAsync(be.ptr, h.data(), sizeof(Elem) * n_el, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(bp.ptr, pts, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, c->stream));
    CK(launch_element_influence((const Elem*)be.ptr, n_el, (const double*)bp.ptr, n_pts, (double*)bphi.ptr,
                                (double*)bE.ptr, c->stream));
    CK(cudaMemcpyAsync(phi_out, bphi.ptr, sizeof(double) * pairs, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(E_out, bE.ptr, sizeof(double) * 3 * pairs, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    be.release();
    bp.release();
    bphi.release();
    bE.release();
    return NEBEM_OK;
}

}  // extern "C"
