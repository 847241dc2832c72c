// fastvol_api.cpp -- C-ABI of the FastVolume maps (declared in include/nebem.h).
#include <cmath>
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

extern "C" {

int nebem_fastvol_build(nebem_ctx* ctx, const double* x_nodes, int32_t nx, const double* y_nodes, int32_t ny,
                        const double* z_nodes, int32_t nz, int32_t precision) {
    if (!ctx || !x_nodes || !y_nodes || !z_nodes) return fail(NEBEM_INVALID_ARG, "NULL argument");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "no charge densities (solve or set_sigma first)");
    const double* ax[3] = {x_nodes, y_nodes, z_nodes};
    const int32_t nn[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (nn[a] < 2) return fail(NEBEM_INVALID_ARG, "each axis needs at least 2 nodes");
        for (int32_t i = 0; i < nn[a]; ++i) {
            if (!std::isfinite(ax[a][i])) return fail(NEBEM_INVALID_ARG, "non-finite node coordinate");
            if (i > 0 && !(ax[a][i] > ax[a][i - 1])) return fail(NEBEM_INVALID_ARG, "node coordinates must increase");
        }
    }
    const int64_t total = (int64_t)nx * ny * nz;
    if (total > 100000000LL) return fail(NEBEM_TOO_LARGE, "more than 1e8 grid nodes");
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
