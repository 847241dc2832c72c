// spacecharge_api.cpp -- known-charge set (Sec. 4.2 OptKnCh / UpdateSpaceCharge), the
// known-charge right-hand side term (RHVector + ValueKnCh), direct sums at points and
// the dynamic update loop (Sec. 4.3, Alg. 4).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

namespace nb {

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)

// b -= known-charge potential (conductor rows) / normal field (interface rows) at the
// collocation centroids.  The charges are not imaged (the copies inherit the base-cell
// right-hand side).
int rhs_known_charge(Ctx* c) {
    const int64_t n = c->n;
    CK(c->d_sc_tgt.ensure(sizeof(double) * 3 * n));
    CK(c->d_sc_phi.ensure(sizeof(double) * n));
    CK(c->d_sc_E.ensure(sizeof(double) * 3 * n));
    CK(launch_centroids(c->d_el.as<Elem>(), n, c->d_sc_tgt.as<double>(), c->stream));
    CK(launch_sc_eval(c->sc_precision, c->d_car.as<double>(), c->d_q.as<double>(), c->d_car2.as<float4>(),
                      c->d_car2.as<float4>() + c->n_car, c->n_car, c->d_sc_tgt.as<double>(), n, 0, c->soft, 0,
                      c->d_sc_phi.as<double>(), c->d_sc_E.as<double>(), c->stream));
    CK(launch_rhs_sc(c->d_el.as<Elem>(), n, c->d_sc_phi.as<double>(), c->d_sc_E.as<double>(), c->d_b.as<double>(),
                     c->stream));
    return 0;
}

// Add the known-charge potential and field at device points (PFAtPoint's KnCh part).
int add_known_charge(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
                     cudaStream_t s) {
    if (c->n_car == 0) return 0;
    CK(launch_sc_eval(precision, c->d_car.as<double>(), c->d_q.as<double>(), c->d_car2.as<float4>(),
                      c->d_car2.as<float4>() + c->n_car, c->n_car, d_pts, n, 0, c->soft, 1, d_phi, d_E, s));
    return 0;
}

}  // namespace nb

using namespace nb;

extern "C" {

int nebem_space_charge(nebem_ctx* ctx, const double* pos, const double* q, int64_t n, double softening) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && (!pos || !q))) return fail(NEBEM_INVALID_ARG, "bad carriers");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(pos[3 * i]) || !std::isfinite(pos[3 * i + 1]) || !std::isfinite(pos[3 * i + 2]) ||
            !std::isfinite(q[i]))
            return fail(NEBEM_INVALID_ARG, "non-finite carrier " + std::to_string(i));
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    c->sigma_valid = false;
    ++c->sigma_version;
    c->n_car = 0;
    if (n == 0) return NEBEM_OK;
    CK(c->d_car.ensure(sizeof(double) * 3 * n));
    CK(c->d_q.ensure(sizeof(double) * n));
    CK(c->d_car2.ensure(sizeof(float4) * 2 * n));
    CK(cudaMemcpyAsync(c->d_car.ptr, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_q.ptr, q, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(launch_sc_split(c->d_car.as<double>(), c->d_q.as<double>(), n, c->d_car2.as<float4>(),
                       c->d_car2.as<float4>() + n, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_car = n;
    c->soft = (softening > 0.0) ? softening : c->opt.softening;
    return NEBEM_OK;
}

int nebem_space_charge_eval(nebem_ctx* ctx, const double* pts, int64_t n, double* phi, double* E, int32_t precision,
                            int32_t exclude_self) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && !pts)) return fail(NEBEM_INVALID_ARG, "bad points");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n_car == 0) return fail(NEBEM_BAD_STATE, "no known-charge set");
    if (exclude_self && n != c->n_car) return fail(NEBEM_INVALID_ARG, "exclude_self needs n == carrier count");
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    CK(c->d_pts.ensure(sizeof(double) * 3 * n));
    CK(c->d_phi.ensure(sizeof(double) * n));
    CK(c->d_E.ensure(sizeof(double) * 3 * n));
    CK(cudaMemcpyAsync(c->d_pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(launch_sc_eval(precision, c->d_car.as<double>(), c->d_q.as<double>(), c->d_car2.as<float4>(),
                      c->d_car2.as<float4>() + c->n_car, c->n_car, c->d_pts.as<double>(), n, exclude_self ? 1 : 0,
                      c->soft, 0, c->d_phi.as<double>(), c->d_E.as<double>(), c->stream));
    if (phi) CK(cudaMemcpyAsync(phi, c->d_phi.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    if (E) CK(cudaMemcpyAsync(E, c->d_E.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NEBEM_OK;
}

int nebem_step(nebem_ctx* ctx, int32_t steps, double mu, double dt, int32_t precision, double* pos_out) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (steps < 0 || !std::isfinite(mu) || !std::isfinite(dt)) return fail(NEBEM_INVALID_ARG, "bad step arguments");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0 || !c->bc_set) return fail(NEBEM_BAD_STATE, "geometry and voltages first");
    if (c->n_car == 0) return fail(NEBEM_BAD_STATE, "no known-charge set");
    CK(cudaSetDevice(c->device));
    const int64_t m = c->n_car;
    int rc = ensure_fill(c, nullptr);
    if (rc) return rc;
    rc = ensure_factors(c, precision, nullptr);
    if (rc) return rc;
    CK(c->d_sc_E.ensure(sizeof(double) * 3 * (m > c->n ? m : c->n)));
    DevBuf Ec;
    CK(Ec.ensure(sizeof(double) * 3 * m));
    c->sc_precision = precision;
    for (int32_t s = 0; s < steps; ++s) {
        rc = build_rhs(c);  // V - known-charge term at the collocation points
        if (rc) return rc;
        rc = solve_with_factors(c, precision, nullptr);
        if (rc) return rc;
        // E at every carrier: elements (with images) + all other carriers
        rc = eval_elements(c, c->d_car.as<double>(), m, nullptr, Ec.as<double>(), precision, c->stream);
        if (rc) return rc;
        CK(launch_sc_eval(precision, c->d_car.as<double>(), c->d_q.as<double>(), c->d_car2.as<float4>(),
                          c->d_car2.as<float4>() + m, m, c->d_car.as<double>(), m, 1, c->soft, 1, nullptr,
                          Ec.as<double>(), c->stream));
        CK(launch_drift(c->d_car.as<double>(), c->d_q.as<double>(), Ec.as<double>(), m, mu * dt, c->stream));
        CK(launch_sc_split(c->d_car.as<double>(), c->d_q.as<double>(), m, c->d_car2.as<float4>(),
                           c->d_car2.as<float4>() + m, c->stream));
    }
    c->sigma_valid = false;  // sigma belongs to the positions before the last move
    ++c->sigma_version;
    if (pos_out) CK(cudaMemcpyAsync(pos_out, c->d_car.ptr, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    Ec.release();
    return NEBEM_OK;
}

}  // extern "C"
