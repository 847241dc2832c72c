// eval_mixed.cu -- mixed-precision evaluation kernels (bodies in eval_blocks.cuh): the FP32
// far-field kernel over all (element, image) pairs, the FP64 near-pair kernel over the
// cell list, and the per-geometry two-float image-centroid table.
#include "eval_blocks.cuh"

namespace nb {

namespace {

__global__ void __launch_bounds__(kEvalThreads, 8) k_eval_far(const GeomView g, const double* __restrict__ pts,
                                                            int64_t npts, double* __restrict__ phi,
                                                            double* __restrict__ E) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int count = (int)min((int64_t)blockDim.x, npts - base);
    far_block(g, pts + 3 * base, count, phi ? phi + base : nullptr, E ? E + 3 * base : nullptr);
}

__global__ void __launch_bounds__(kEvalThreads) k_eval_near(const GeomView g, const ImageTable img,
                                                          const double* __restrict__ pts, int64_t npts,
                                                          double* __restrict__ phi, double* __restrict__ E) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    near_point(g, img, pts, p, phi, E);
}

// Two-float image centroids, entry (j, k) at 2 * (j * nimg + k): hi then lo.
__global__ void k_image_centroids(const Elem* __restrict__ el, int64_t n, const ImageTable img,
                                  float4* __restrict__ cjk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * img.n) return;
    const int64_t j = i / img.n;
    const int k = (int)(i - j * img.n);
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) split2f(el[j].c[a] + img.t[k][a], h[a], l[a]);
    cjk[2 * i] = make_float4(h[0], h[1], h[2], 0.f);
    cjk[2 * i + 1] = make_float4(l[0], l[1], l[2], 0.f);
}

}  // namespace

cudaError_t launch_image_centroids(const Elem* el, int64_t n, const ImageTable& img, float4* cjk, cudaStream_t s) {
    const int64_t total = n * img.n;
    if (total == 0) return cudaSuccess;
    k_image_centroids<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(el, n, img, cjk);
    return cudaGetLastError();
}

GeomView make_view(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma, int64_t n_el,
                   const ImageTable& img, const NearGrid& grid, const int32_t* cell_start, const int32_t* cell_items) {
    GeomView g;
    g.el = el;
    g.far = far;
    g.cjk = cjk;
    g.sigma = sigma;
    g.cell_start = cell_start;
    g.cell_items = cell_items;
    g.n_el = n_el;
    g.nimg = img.n;
    g.tile_el = max(1, min(kTileMax, kCjkMax / img.n));
    g.grid = grid;
    return g;
}

cudaError_t launch_eval_mixed(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma,
                              int64_t n_el, const ImageTable& img, const NearGrid& grid, const int32_t* cell_start,
                              const int32_t* cell_items, const double* pts, int64_t npts, double* phi, double* E,
                              cudaStream_t s) {
    if (npts == 0) return cudaSuccess;
    const GeomView g = make_view(el, far, cjk, sigma, n_el, img, grid, cell_start, cell_items);
    const unsigned blocks = (unsigned)((npts + kEvalThreads - 1) / kEvalThreads);
    k_eval_far<<<blocks, kEvalThreads, 0, s>>>(g, pts, npts, phi, E);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_eval_near<<<blocks, kEvalThreads, 0, s>>>(g, img, pts, npts, phi, E);
    return cudaGetLastError();
}

}  // namespace nb
