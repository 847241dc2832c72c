// fastvol_api.cpp -- C-ABI of the FastVolume maps (declared in include/nebem.h).
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "context.h"

namespace nb {
#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)
}  // namespace nb

using namespace nb;

// Node axes of a map: at least 2 finite, strictly increasing coordinates per axis, at most
// 1e8 nodes in all.
static int check_axes(const double* x_nodes, int32_t nx, const double* y_nodes, int32_t ny, const double* z_nodes,
                      int32_t nz) {
    const double* ax[3] = {x_nodes, y_nodes, z_nodes};
    const int32_t nn[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (nn[a] < 2) return fail(NEBEM_INVALID_ARG, "each axis needs at least 2 nodes");
        for (int32_t i = 0; i < nn[a]; ++i) {
            if (!std::isfinite(ax[a][i])) return fail(NEBEM_INVALID_ARG, "non-finite node coordinate");
            if (i > 0 && !(ax[a][i] > ax[a][i - 1])) return fail(NEBEM_INVALID_ARG, "node coordinates must increase");
        }
    }
    if ((int64_t)nx * ny * nz > 100000000LL) return fail(NEBEM_TOO_LARGE, "more than 1e8 grid nodes");
    return NEBEM_OK;
}

extern "C" {

int nebem_fastvol_build(nebem_ctx* ctx, const double* x_nodes, int32_t nx, const double* y_nodes, int32_t ny,
                        const double* z_nodes, int32_t nz, int32_t precision) {
    if (!ctx || !x_nodes || !y_nodes || !z_nodes) return fail(NEBEM_INVALID_ARG, "NULL argument");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    if (int rc = check_axes(x_nodes, nx, y_nodes, ny, z_nodes, nz)) return rc;
    const int64_t total = (int64_t)nx * ny * nz;
    CK(cudaSetDevice(c->device));
    CK(c->d_fv_ax.ensure(sizeof(double) * nx));
    CK(c->d_fv_ay.ensure(sizeof(double) * ny));
    CK(c->d_fv_az.ensure(sizeof(double) * nz));
    CK(c->d_fv_phi.ensure(sizeof(double) * total));
    CK(c->d_fv_E.ensure(sizeof(double) * 3 * total));
    CK(cudaMemcpyAsync(c->d_fv_ax.ptr, x_nodes, sizeof(double) * nx, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fv_ay.ptr, y_nodes, sizeof(double) * ny, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_fv_az.ptr, z_nodes, sizeof(double) * nz, cudaMemcpyHostToDevice, c->stream));
    DevBuf nodes;
    CK(nodes.ensure(sizeof(double) * 3 * total));
    CK(launch_grid_nodes(c->d_fv_ax.as<double>(), c->d_fv_ay.as<double>(), c->d_fv_az.as<double>(), nx, ny, nz,
                         nodes.as<double>(), c->stream));
    int rc = eval_points(c, nodes.as<double>(), total, c->d_fv_phi.as<double>(), c->d_fv_E.as<double>(), precision,
                         c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    nodes.release();
    c->fv_dims[0] = nx;
    c->fv_dims[1] = ny;
    c->fv_dims[2] = nz;
    c->fv_version = c->sigma_version;
    return NEBEM_OK;
}

static int fastvol_check(Ctx* c) {
    if (c->fv_version < 0) return fail(NEBEM_BAD_STATE, "no FastVolume map (nebem_fastvol_build first)");
    if (c->fv_version != c->sigma_version)
        return fail(NEBEM_BAD_STATE, "the charge densities changed since the map was built: rebuild it");
    return NEBEM_OK;
}

int nebem_fastvol_eval_device(nebem_ctx* ctx, const double* d_pts, int64_t n, double* d_phi, double* d_E,
                              void* stream) {
    if (!ctx || n < 0 || (n > 0 && !d_pts)) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "point count")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = fastvol_check(c);
    if (rc) return rc;
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    CK(launch_fastvol_lookup(c->d_fv_ax.as<double>(), c->d_fv_ay.as<double>(), c->d_fv_az.as<double>(), c->fv_dims[0],
                             c->fv_dims[1], c->fv_dims[2], c->d_fv_phi.as<double>(), c->d_fv_E.as<double>(), d_pts, n,
                             d_phi, d_E, s));
    return NEBEM_OK;
}

int nebem_fastvol_eval(nebem_ctx* ctx, const double* pts, int64_t n, double* phi, double* E) {
    if (!ctx || n < 0 || (n > 0 && !pts)) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "point count")) return rc;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = fastvol_check(c);
    if (rc) return rc;
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    CK(c->d_pts.ensure(sizeof(double) * 3 * n));
    CK(c->d_phi.ensure(sizeof(double) * n));
    CK(c->d_E.ensure(sizeof(double) * 3 * n));
    CK(cudaMemcpyAsync(c->d_pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(launch_fastvol_lookup(c->d_fv_ax.as<double>(), c->d_fv_ay.as<double>(), c->d_fv_az.as<double>(), c->fv_dims[0],
                             c->fv_dims[1], c->fv_dims[2], c->d_fv_phi.as<double>(), c->d_fv_E.as<double>(),
                             c->d_pts.as<double>(), n, phi ? c->d_phi.as<double>() : nullptr,
                             E ? c->d_E.as<double>() : nullptr, c->stream));
    if (phi) CK(cudaMemcpyAsync(phi, c->d_phi.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    if (E) CK(cudaMemcpyAsync(E, c->d_E.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NEBEM_OK;
}

}  // extern "C"

// A FastVolume map of its own (a weighting-field map), outside any context.
struct nebem_fvmap {
    int device = 0;
    cudaStream_t stream = nullptr;
    nb::DevBuf ax, ay, az, phi, E, pts, ophi, oE;
    int32_t dims[3] = {0, 0, 0};
};

namespace {
// c->d_sigma replaced by another set of charge densities for the life of the object
struct SigmaSwap {
    Ctx* c;
    DevBuf& other;
    SigmaSwap(Ctx* c_, DevBuf& o) : c(c_), other(o) { swap(); }
    ~SigmaSwap() { swap(); }
    void swap() {
        std::swap(c->d_sigma.ptr, other.ptr);
        std::swap(c->d_sigma.bytes, other.bytes);
    }
};
void destroy_map(nebem_fvmap* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    m->ax.release(), m->ay.release(), m->az.release(), m->phi.release(), m->E.release();
    m->pts.release(), m->ophi.release(), m->oE.release();
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}
}  // namespace

extern "C" {

int nebem_weighting_fastvol_build(nebem_ctx* ctx, const int32_t* readout, int32_t k, const double* x_nodes,
                                  int32_t nx, const double* y_nodes, int32_t ny, const double* z_nodes, int32_t nz,
                                  int32_t precision, nebem_fvmap** maps_out, nebem_solve_info* info) {
    if (!ctx || !readout || !maps_out || !x_nodes || !y_nodes || !z_nodes)
        return fail(NEBEM_INVALID_ARG, "NULL argument");
    if (k < 1 || k > 64) return fail(NEBEM_INVALID_ARG, "k must be 1..64");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->am_on) return fail(NEBEM_BAD_STATE, "weighting maps are built without Adaptive Modelling");
    if (int rc = check_axes(x_nodes, nx, y_nodes, ny, z_nodes, nz)) return rc;
    for (int32_t j = 0; j < k; ++j) maps_out[j] = nullptr;
    // the k weighting fields (validates readout, precision and state)
    int rc = nebem_weighting_fields(ctx, readout, k, precision, nullptr, info);
    if (rc) return rc;
    const int64_t total = (int64_t)nx * ny * nz;
    const int64_t n = c->n;
    DevBuf nodes, sw;
    std::vector<nebem_fvmap*> made;
    auto bail = [&](int code) {
        for (nebem_fvmap* m : made) destroy_map(m);
        return code;
    };
#define CKM(call)                                                          \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call));          \
    } while (0)
    CKM(nodes.ensure(sizeof(double) * 3 * total));
    CKM(sw.ensure(sizeof(double) * n));
    for (int32_t j = 0; j < k; ++j) {
        nebem_fvmap* m = new nebem_fvmap();
        made.push_back(m);
        m->device = c->device;
        CKM(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
        CKM(m->ax.ensure(sizeof(double) * nx));
        CKM(m->ay.ensure(sizeof(double) * ny));
        CKM(m->az.ensure(sizeof(double) * nz));
        CKM(m->phi.ensure(sizeof(double) * total));
        CKM(m->E.ensure(sizeof(double) * 3 * total));
        CKM(cudaMemcpyAsync(m->ax.ptr, x_nodes, sizeof(double) * nx, cudaMemcpyHostToDevice, c->stream));
        CKM(cudaMemcpyAsync(m->ay.ptr, y_nodes, sizeof(double) * ny, cudaMemcpyHostToDevice, c->stream));
        CKM(cudaMemcpyAsync(m->az.ptr, z_nodes, sizeof(double) * nz, cudaMemcpyHostToDevice, c->stream));
        m->dims[0] = nx, m->dims[1] = ny, m->dims[2] = nz;
        if (j == 0)
            CKM(launch_grid_nodes(m->ax.as<double>(), m->ay.as<double>(), m->az.as<double>(), nx, ny, nz,
                                  nodes.as<double>(), c->stream));
        // readout j's densities in place of the context's for the node evaluation (elements
        // only: a weighting field has no known charges)
        CKM(cudaMemcpyAsync(sw.ptr, c->d_wX.as<double>() + (size_t)j * n, sizeof(double) * n,
                            cudaMemcpyDeviceToDevice, c->stream));
        {
            SigmaSwap guard(c, sw);
            rc = eval_elements(c, nodes.as<double>(), total, m->phi.as<double>(), m->E.as<double>(), precision,
                               c->stream);
            if (rc == 0) {
                const cudaError_t e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) rc = cuda_fail(e, "weighting map nodes");
            }
        }
        if (rc) return bail(rc);
    }
#undef CKM
    for (int32_t j = 0; j < k; ++j) maps_out[j] = made[j];
    return NEBEM_OK;
}

int nebem_fvmap_eval_device(nebem_fvmap* map, const double* d_pts, int64_t n, double* d_phi, double* d_E,
                            void* stream) {
    if (!map || n < 0 || (n > 0 && !d_pts)) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "point count")) return rc;
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(map->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : map->stream;
    CK(launch_fastvol_lookup(map->ax.as<double>(), map->ay.as<double>(), map->az.as<double>(), map->dims[0],
                             map->dims[1], map->dims[2], map->phi.as<double>(), map->E.as<double>(), d_pts, n, d_phi,
                             d_E, s));
    return NEBEM_OK;
}

int nebem_fvmap_eval(nebem_fvmap* map, const double* pts, int64_t n, double* phi, double* E) {
    if (!map || n < 0 || (n > 0 && !pts)) return fail(NEBEM_INVALID_ARG, "bad argument");
    if (int rc = check_count(n, "point count")) return rc;
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(map->device));
    CK(map->pts.ensure(sizeof(double) * 3 * n));
    CK(map->ophi.ensure(sizeof(double) * n));
    CK(map->oE.ensure(sizeof(double) * 3 * n));
    cudaStream_t s = map->stream;
    CK(cudaMemcpyAsync(map->pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    CK(launch_fastvol_lookup(map->ax.as<double>(), map->ay.as<double>(), map->az.as<double>(), map->dims[0],
                             map->dims[1], map->dims[2], map->phi.as<double>(), map->E.as<double>(),
                             map->pts.as<double>(), n, phi ? map->ophi.as<double>() : nullptr,
                             E ? map->oE.as<double>() : nullptr, s));
    if (phi) CK(cudaMemcpyAsync(phi, map->ophi.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (E) CK(cudaMemcpyAsync(E, map->oE.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NEBEM_OK;
}

int nebem_fvmap_destroy(nebem_fvmap* map) {
    destroy_map(map);
    return NEBEM_OK;
}

}  // extern "C"
