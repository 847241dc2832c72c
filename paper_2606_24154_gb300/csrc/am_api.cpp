// am_api.cpp -- Adaptive Modelling (Sec. 3.3; the PrimAfter parameter of Sec. 5.3.1):
// distant periodic copies are represented by whole primitives carrying the average
// charge density of their elements, the near copies by the elements themselves.
//
// A copy k = (k1, k2) of the lattice is distant when its ring index max(|k1|, |k2|)
// exceeds prim_after.  The evaluation is then two passes of the ordinary kernels (FP64
// or mixed): the elements with the near image set, and the primitives (plus any element
// that belongs to no primitive) with the distant image set, added together.  The
// primitives' densities are recomputed on the device whenever sigma changes.
#include <cuda_runtime.h>

#include <cmath>
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

void EvalSet::release_all() {
    for (DevBuf* b : {&own_el, &own_far, &own_sigma, &cjk, &cell_start, &cell_items}) b->release();
    n = 0;
    el = nullptr;
    far = nullptr;
    sigma = nullptr;
}

namespace {

double elem_area(const Elem& e) { return (e.nv == 4) ? 0.5 * (e.twoA[0] + e.twoA[1]) : 0.5 * e.twoA[0]; }

// Image centroids and near-pair cell list of an element table (host copy h_el, device
// copy es.el) under the image set es.img.
int finish_set(Ctx* c, const std::vector<Elem>& h_el, EvalSet& es) {
    std::string why;
    std::vector<int32_t> cell_start, cell_items;
    int rc = build_near_grid(h_el, es.img, c->opt.ratio_near, es.grid, cell_start, cell_items, why);
    if (rc) return fail(rc, why);
    CK(es.cjk.ensure(sizeof(float4) * 2 * es.n * es.img.n));
    CK(launch_image_centroids(es.el, es.n, es.img, es.cjk.as<float4>(), c->stream));
    CK(es.cell_start.ensure(sizeof(int32_t) * cell_start.size()));
    CK(es.cell_items.ensure(sizeof(int32_t) * cell_items.size()));
    CK(cudaMemcpyAsync(es.cell_start.ptr, cell_start.data(), sizeof(int32_t) * cell_start.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(es.cell_items.ptr, cell_items.data(), sizeof(int32_t) * cell_items.size(),
                       cudaMemcpyHostToDevice, c->stream));
    return 0;
}

}  // namespace

int eval_adaptive(Ctx* c, const double* d_pts, int64_t n, double* d_phi, double* d_E, int precision,
                  cudaStream_t s) {
    if (c->am_sigma_version != c->sigma_version) {
        CK(launch_prim_sigma(c->d_am_start.as<int32_t>(), c->d_am_items.as<int32_t>(), c->d_am_elarea.as<double>(),
                             c->d_am_parea.as<double>(), c->d_sigma.as<double>(), c->am_far.n,
                             c->am_far.own_sigma.as<double>(), s));
        c->am_sigma_version = c->sigma_version;
    }
    int rc = eval_set(c, c->am_near, d_pts, n, d_phi, d_E, precision, s);
    if (rc) return rc;
    CK(c->d_am_tmp.ensure(sizeof(double) * 4 * n));
    double* tphi = d_phi ? c->d_am_tmp.as<double>() : nullptr;
    double* tE = d_E ? c->d_am_tmp.as<double>() + n : nullptr;
    rc = eval_set(c, c->am_far, d_pts, n, tphi, tE, precision, s);
    if (rc) return rc;
    CK(launch_add_fields(d_phi, d_E, tphi, tE, n, s));
    return 0;
}

}  // namespace nb

using namespace nb;

extern "C" {

int nebem_set_primitives(nebem_ctx* ctx, const nebem_element* prims, int32_t n_prim, const int32_t* prim_of,
                         int32_t prim_after) {
    if (!ctx) return fail(NEBEM_INVALID_ARG, "ctx is NULL");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->n == 0) return fail(NEBEM_BAD_STATE, "set_geometry first");
    if (n_prim < 0 || (n_prim > 0 && !prims) || !prim_of) return fail(NEBEM_INVALID_ARG, "bad primitives");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    c->am_on = false;
    c->am_prim_after = prim_after;
    c->am_near.release_all();
    c->am_far.release_all();
    if (prim_after < 0) return NEBEM_OK;
    const int64_t n = c->n;
    // primitives as element records (their boundary conditions play no part)
    std::vector<Elem> p_el((size_t)n_prim);
    std::vector<FarNodes> p_far((size_t)n_prim);
    std::string why;
    for (int32_t p = 0; p < n_prim; ++p) {
        nebem_element r = prims[p];
        if (r.reserved != 0) return fail(NEBEM_INVALID_ARG, "primitive " + std::to_string(p) + ": reserved != 0");
        r.bc = NEBEM_CONDUCTOR;
        r.conductor = 0;
        r.eps_a = r.eps_b = 1.0;
        double diag = 0.0;
        int rc = build_element(r, c->opt, p_el[p], diag, p_far[p], why);
        if (rc) return fail(rc, "primitive " + std::to_string(p) + ": " + why);
    }
    // every element's primitive; tiling (areas) and coplanarity checks
    std::vector<double> elarea((size_t)n), sum_area((size_t)n_prim, 0.0);
    std::vector<int32_t> count((size_t)n_prim, 0);
    int64_t n_free = 0;
    for (int64_t j = 0; j < n; ++j) {
        const int32_t p = prim_of[j];
        if (p < -1 || p >= n_prim) return fail(NEBEM_INVALID_ARG, "element " + std::to_string(j) + ": bad primitive");
        elarea[j] = elem_area(c->h_el[j]);
        if (p < 0) {
            ++n_free;
            continue;
        }
        const Elem& P = p_el[p];
        const double* cj = c->h_el[j].c;
        const double off = (cj[0] - P.o[0]) * P.ey[0] + (cj[1] - P.o[1]) * P.ey[1] + (cj[2] - P.o[2]) * P.ey[2];
        if (std::fabs(off) > 1e-9 * P.rho)
            return fail(NEBEM_INVALID_ARG, "element " + std::to_string(j) + " is not in its primitive's plane");
        sum_area[p] += elarea[j];
        ++count[p];
    }
    for (int32_t p = 0; p < n_prim; ++p) {
        const double ap = elem_area(p_el[p]);
        if (count[p] == 0 || std::fabs(sum_area[p] - ap) > 1e-9 * ap)
            return fail(NEBEM_INVALID_ARG, "the elements of primitive " + std::to_string(p) + " do not tile it");
    }
    // image split by ring index
    ImageTable near_img{}, far_img{};
    const int32_t m = c->img_hi - c->img_lo + 1;
    for (int32_t k = 0; k < c->img.n; ++k) {
        const int32_t k1 = (c->img.n > 1) ? k / m + c->img_lo : 0, k2 = (c->img.n > 1) ? k % m + c->img_lo : 0;
        const int32_t ring = std::abs(k1) > std::abs(k2) ? std::abs(k1) : std::abs(k2);
        ImageTable& dst = (ring > prim_after) ? far_img : near_img;
        for (int a = 0; a < 3; ++a) dst.t[dst.n][a] = c->img.t[k][a];
        if (k == c->img.k0) dst.k0 = dst.n;
        ++dst.n;
    }
    if (far_img.n == 0) return NEBEM_OK;  // no distant copy: the plain evaluation
    far_img.k0 = -1;
    // far entries: the primitives, then the elements that belong to none
    const int64_t nf = n_prim + n_free;
    std::vector<Elem> f_el(p_el);
    std::vector<FarNodes> f_far(p_far);
    std::vector<double> parea((size_t)nf);
    std::vector<int32_t> start((size_t)nf + 1, 0), items((size_t)n);
    for (int32_t p = 0; p < n_prim; ++p) {
        parea[p] = elem_area(p_el[p]);
        start[p + 1] = start[p] + count[p];
    }
    std::vector<int32_t> fill_pos(start.begin(), start.begin() + n_prim);
    int64_t f = n_prim;
    for (int64_t j = 0; j < n; ++j) {
        const int32_t p = prim_of[j];
        if (p >= 0) {
            items[fill_pos[p]++] = (int32_t)j;
            continue;
        }
        // the element stands for itself (its far nodes are copied on the device below)
        f_el.push_back(c->h_el[j]);
        f_far.push_back(FarNodes{});
        parea[f] = elarea[j];
        items[start[n_prim] + (f - n_prim)] = (int32_t)j;
        ++f;
    }
    for (int64_t g = n_prim; g < nf; ++g) start[g + 1] = start[g] + 1;
    // device data
    EvalSet& nr = c->am_near;
    nr.n = n;
    nr.img = near_img;
    nr.el = c->d_el.as<Elem>();
    nr.far = c->d_far.as<FarNodes>();
    nr.sigma = c->d_sigma.as<double>();
    int rc = finish_set(c, c->h_el, nr);
    if (rc) return rc;
    EvalSet& fr = c->am_far;
    fr.n = nf;
    fr.img = far_img;
    CK(fr.own_el.ensure(sizeof(Elem) * nf));
    CK(fr.own_far.ensure(sizeof(FarNodes) * nf));
    CK(fr.own_sigma.ensure(sizeof(double) * nf));
    CK(cudaMemcpyAsync(fr.own_el.ptr, f_el.data(), sizeof(Elem) * nf, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(fr.own_far.ptr, f_far.data(), sizeof(FarNodes) * n_prim, cudaMemcpyHostToDevice, c->stream));
    // far nodes of the free elements: copied from the context's table
    for (int64_t g = n_prim; g < nf; ++g)
        CK(cudaMemcpyAsync(fr.own_far.as<FarNodes>() + g, c->d_far.as<FarNodes>() + items[start[g]],
                           sizeof(FarNodes), cudaMemcpyDeviceToDevice, c->stream));
    fr.el = fr.own_el.as<Elem>();
    fr.far = fr.own_far.as<FarNodes>();
    fr.sigma = fr.own_sigma.as<double>();
    rc = finish_set(c, f_el, fr);
    if (rc) return rc;
    CK(c->d_am_start.ensure(sizeof(int32_t) * (nf + 1)));
    CK(c->d_am_items.ensure(sizeof(int32_t) * n));
    CK(c->d_am_elarea.ensure(sizeof(double) * n));
    CK(c->d_am_parea.ensure(sizeof(double) * nf));
    CK(cudaMemcpyAsync(c->d_am_start.ptr, start.data(), sizeof(int32_t) * (nf + 1), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_am_items.ptr, items.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_am_elarea.ptr, elarea.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_am_parea.ptr, parea.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->am_n_prim = n_prim;
    c->am_sigma_version = -1;
    c->am_on = true;
    return NEBEM_OK;
}

}  // extern "C"
