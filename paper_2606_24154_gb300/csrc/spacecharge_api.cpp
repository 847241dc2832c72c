// spacecharge_api.cpp -- known-charge set (Sec. 4.2 OptKnCh / UpdateSpaceCharge), the
// known-charge right-hand side term (RHVector + ValueKnCh), direct sums at points and
// the dynamic update loop (Sec. 4.3, Alg. 4).  The known charges are either the point
// charges themselves or the line charges of their voxel reduction (Alg. 3, LineCh).
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

VoxWork vox_work(Ctx* c) {
    VoxWork w;
    w.keys = c->d_vkeys.as<long long>();
    w.flags = c->d_vflags.as<int>();
    w.bsum = c->d_vbsum.as<int>();
    w.partial = c->d_vpartial.as<double>();
    w.grid = c->d_vgrid.as<VoxGrid>();
    w.lines = c->d_lines.as<LineRec>();
    w.linesf = c->d_linesf.as<LineF>();
    w.line_vox = c->d_line_vox.as<long long>();
    return w;
}

namespace {

int ensure_vox(Ctx* c, int64_t n) {
    CK(c->d_vkeys.ensure(sizeof(long long) * vox_pad_len(n)));
    CK(c->d_vflags.ensure(sizeof(int) * n));
    CK(c->d_vbsum.ensure(sizeof(int) * vox_scan_blocks(n)));
    CK(c->d_vpartial.ensure(sizeof(double) * 6 * 512));
    if (!c->d_vgrid.ptr) {
        CK(c->d_vgrid.ensure(sizeof(VoxGrid)));
        CK(cudaMemsetAsync(c->d_vgrid.ptr, 0, sizeof(VoxGrid), c->stream));
    }
    CK(c->d_lines.ensure(sizeof(LineRec) * n));
    CK(c->d_linesf.ensure(sizeof(LineF) * n));
    CK(c->d_line_vox.ensure(sizeof(long long) * n));
    return 0;
}

// phi/E of the known charges at device targets (accumulate: add to the outputs).
// perm (line mode only, may be NULL): target order for the threads, perm[t] % perm_div.
int known_charge_at(Ctx* c, const double* d_tgt, int64_t nt, int exclude_self, int accumulate, double* d_phi,
                    double* d_E, int precision, const long long* perm, int64_t perm_div, cudaStream_t s) {
    if (c->sc_lines) {
        CK(launch_line_eval(precision, vox_work(c), d_tgt, perm, perm_div, nt, c->soft, accumulate, d_phi, d_E, s));
    } else {
        CK(launch_sc_eval(precision, c->d_car.as<double>(), c->d_q.as<double>(), c->d_car2.as<float4>(),
                          c->d_car2.as<float4>() + c->n_car, c->n_car, d_tgt, nt, exclude_self, c->soft,
                          accumulate, d_phi, d_E, s));
    }
    return 0;
}

}  // namespace

// b -= known-charge potential (conductor rows) / normal field (interface rows) at the
// collocation centroids.  The charges are not imaged (the copies inherit the base-cell
// right-hand side).
int rhs_known_charge(Ctx* c) {
    const int64_t n = c->n;
    CK(c->d_sc_tgt.ensure(sizeof(double) * 3 * n));
    CK(c->d_sc_phi.ensure(sizeof(double) * n));
    CK(c->d_sc_E.ensure(sizeof(double) * 3 * n));
    CK(launch_centroids(c->d_el.as<Elem>(), n, c->d_sc_tgt.as<double>(), c->stream));
    int rc = known_charge_at(c, c->d_sc_tgt.as<double>(), n, 0, 0, c->d_sc_phi.as<double>(), c->d_sc_E.as<double>(),
                             c->sc_precision, nullptr, 0, c->stream);
    if (rc) return rc;
    CK(launch_rhs_sc(c->d_el.as<Elem>(), n, c->d_sc_phi.as<double>(), c->d_sc_E.as<double>(), c->d_b.as<double>(),
                     c->stream));
    return 0;
}

// Add the known-charge potential and field at device points (PFAtPoint's KnCh part).
int add_known_charge(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
                     cudaStream_t s) {
    if (c->n_car == 0) return 0;
    return known_charge_at(c, d_pts, n, 0, 1, d_phi, d_E, precision, nullptr, 0, s);
}

}  // namespace nb

using namespace nb;

extern "C" {

int nebem_space_charge(nebem_ctx* ctx, const double* pos, const double* q, int64_t n, double softening) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    if (n < 0 || (n > 0 && (!pos || !q))) return fail(NEBEM_INVALID_ARG, "bad carriers");
    if (int rc = check_count(n, "carrier count")) return rc;
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
    c->sc_lines = false;
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
    if (int rc = check_count(n, "point count")) return rc;
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n_car == 0) return fail(NEBEM_BAD_STATE, "no known-charge set");
    if (exclude_self && n != c->n_car) return fail(NEBEM_INVALID_ARG, "exclude_self needs n == carrier count");
    if (exclude_self && c->sc_lines) return fail(NEBEM_INVALID_ARG, "exclude_self applies to point charges only");
    if (n == 0) return NEBEM_OK;
    CK(cudaSetDevice(c->device));
    CK(c->d_pts.ensure(sizeof(double) * 3 * n));
    CK(c->d_phi.ensure(sizeof(double) * n));
    CK(c->d_E.ensure(sizeof(double) * 3 * n));
    CK(cudaMemcpyAsync(c->d_pts.ptr, pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    int rc = known_charge_at(c, c->d_pts.as<double>(), n, exclude_self ? 1 : 0, 0, c->d_phi.as<double>(),
                             c->d_E.as<double>(), precision, nullptr, 0, c->stream);
    if (rc) return rc;
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
    int rc = ensure_fill(c, precision, nullptr);
    if (rc) return rc;
    rc = ensure_factors(c, precision, nullptr);
    if (rc) return rc;
    CK(c->d_sc_E.ensure(sizeof(double) * 3 * (m > c->n ? m : c->n)));
    DevBuf Ec;
    CK(Ec.ensure(sizeof(double) * 3 * m));
    c->sc_precision = precision;
    if (c->sc_lines) CK(cudaMemsetAsync(&c->d_vgrid.as<VoxGrid>()->sticky, 0, sizeof(int), c->stream));
    for (int32_t s = 0; s < steps; ++s) {
        // Alg. 4, Type == Line: the reduction of Alg. 3 on the current positions
        if (c->sc_lines)
            CK(launch_voxelize(c->d_car.as<double>(), c->d_q.as<double>(), m, c->voxel, vox_work(c), c->stream));
        rc = build_rhs(c);  // V - known-charge term at the collocation points
        if (rc) return rc;
        rc = solve_with_factors(c, precision, nullptr);
        if (rc) return rc;
        // E at every carrier: elements (with images) + all other carriers (points, self
        // excluded) or all lines; with lines the threads take the carriers in voxel order
        rc = eval_elements(c, c->d_car.as<double>(), m, nullptr, Ec.as<double>(), precision, c->stream);
        if (rc) return rc;
        rc = known_charge_at(c, c->d_car.as<double>(), m, 1, 1, nullptr, Ec.as<double>(), precision,
                             c->sc_lines ? c->d_vkeys.as<long long>() : nullptr, m, c->stream);
        if (rc) return rc;
        CK(launch_drift(c->d_car.as<double>(), c->d_q.as<double>(), Ec.as<double>(), m, mu * dt, c->stream));
        CK(launch_sc_split(c->d_car.as<double>(), c->d_q.as<double>(), m, c->d_car2.as<float4>(),
                           c->d_car2.as<float4>() + m, c->stream));
    }
    c->sigma_valid = false;  // sigma belongs to the positions before the last move
    ++c->sigma_version;
    if (pos_out) CK(cudaMemcpyAsync(pos_out, c->d_car.ptr, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, c->stream));
    int sticky = 0;
    if (c->sc_lines)
        CK(cudaMemcpyAsync(&sticky, &c->d_vgrid.as<VoxGrid>()->sticky, sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    Ec.release();
    if (sticky) return fail(NEBEM_TOO_LARGE, "voxel grid of a step too large for 62-bit keys");
    return NEBEM_OK;
}

int nebem_space_charge_lines(nebem_ctx* ctx, const double* voxel, int64_t* n_lines) {
    if (!ctx || !voxel) return fail(NEBEM_INVALID_ARG, "ctx or voxel is NULL");
    for (int a = 0; a < 3; ++a)
        if (!(voxel[a] > 0.0) || !std::isfinite(voxel[a])) return fail(NEBEM_INVALID_ARG, "voxel edges must be > 0");
    // the near-line search of a target visits the voxels within 3 half lengths (1.5 dz):
    // about (3 dz/dx + 3) (3 dz/dy + 3) 5 of them; refuse shapes that make it huge
    {
        const double cand = (3.0 * voxel[2] / voxel[0] + 3.0) * (3.0 * voxel[2] / voxel[1] + 3.0) * 5.0;
        if (!(cand <= 2.0e5))
            return fail(NEBEM_INVALID_ARG, "voxel edges dx, dy too small relative to dz (near-line search)");
    }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n_car == 0) return fail(NEBEM_BAD_STATE, "no point charges to reduce");
    if (c->n_car > kVoxMaxPoints) return fail(NEBEM_TOO_LARGE, "more than 2^26 point charges");
    CK(cudaSetDevice(c->device));
    int rc = ensure_vox(c, c->n_car);
    if (rc) return rc;
    CK(launch_voxelize(c->d_car.as<double>(), c->d_q.as<double>(), c->n_car, voxel, vox_work(c), c->stream));
    VoxGrid g;
    CK(cudaMemcpyAsync(&g, c->d_vgrid.ptr, sizeof(VoxGrid), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (g.err) return fail(NEBEM_TOO_LARGE, "voxel grid too large for 62-bit keys");
    for (int a = 0; a < 3; ++a) c->voxel[a] = voxel[a];
    c->sc_lines = true;
    c->sigma_valid = false;
    ++c->sigma_version;
    if (n_lines) *n_lines = g.nl;
    return NEBEM_OK;
}

int nebem_get_lines(nebem_ctx* ctx, double* start, double* stop, double* lambda, int64_t capacity,
                    int64_t* n_lines) {
    if (!ctx || capacity < 0) return fail(NEBEM_INVALID_ARG, "bad arguments");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->sc_lines) return fail(NEBEM_BAD_STATE, "the known charges are not line charges");
    CK(cudaSetDevice(c->device));
    VoxGrid g;
    CK(cudaMemcpyAsync(&g, c->d_vgrid.ptr, sizeof(VoxGrid), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_lines) *n_lines = g.nl;
    if (capacity < g.nl) return capacity == 0 ? NEBEM_OK : fail(NEBEM_TOO_LARGE, "capacity below the line count");
    std::vector<LineRec> h((size_t)g.nl);
    if (g.nl) CK(cudaMemcpyAsync(h.data(), c->d_lines.ptr, sizeof(LineRec) * g.nl, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t l = 0; l < g.nl; ++l) {
        const LineRec& r = h[(size_t)l];
        for (int a = 0; a < 3; ++a) {
            if (start) start[3 * l + a] = r.a[a];
            if (stop) stop[3 * l + a] = r.a[a] + r.len * r.u[a];
        }
        if (lambda) lambda[l] = r.lam;
    }
    return NEBEM_OK;
}

}  // extern "C"
