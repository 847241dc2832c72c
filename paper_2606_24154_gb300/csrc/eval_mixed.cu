// eval_mixed.cu -- mixed-precision evaluation kernels (bodies in eval_blocks.cuh): spatial
// binning of the targets, the FP32 far-field kernel over all (element, image) pairs, the
// FP64 near-pair kernel over the cell list, and the per-geometry two-float image-centroid
// table.
#include "eval_blocks.cuh"

namespace nb {

namespace {

__global__ void __launch_bounds__(kEvalThreads, 6) k_eval_far(const GeomView g, const double* __restrict__ pts,
                                                            const int32_t* __restrict__ order, int64_t npts,
                                                            double* __restrict__ phi, double* __restrict__ E,
                                                            float4* __restrict__ bound) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int count = (int)min((int64_t)blockDim.x, npts - base);
    far_block(g, pts, order, base, count, phi, E, bound);
}

__global__ void __launch_bounds__(kEvalThreads) k_eval_near(const GeomView g, const ImageTable img,
                                                          const double* __restrict__ pts,
                                                          const int32_t* __restrict__ order, int64_t npts,
                                                          double* __restrict__ phi, double* __restrict__ E) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    near_point(g, img, pts, order ? (int64_t)order[i] : i, phi, E);
}

// ---- spatial binning of the targets: counting sort by the Morton index of a 64^3 grid
// over the near-pair grid's box (points outside are clamped to the border cells).  Warps
// then hold nearby points, whose (element, image) pairs mostly fall in the same distance
// tier, so the tier branches stay converged.  The order only changes which lane evaluates
// a point, never the point's arithmetic; positions within a cell come from atomics and
// may differ between runs without changing any result.
constexpr int kBinBits = 6;
constexpr int kBins = 1 << (3 * kBinBits);

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 6 bits -> every third bit
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < kBinBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

__global__ void k_bin_keys(const double* __restrict__ pts, int64_t n, const NearGrid grid,
                           int32_t* __restrict__ key, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double span = (double)grid.dims[a] / grid.inv_h;
        double f = floor((pts[3 * i + a] - grid.origin[a]) / span * (double)(1 << kBinBits));
        f = fmin(fmax(f, 0.0), (double)((1 << kBinBits) - 1));
        c[a] = (uint32_t)f;
    }
    const int32_t k = (int32_t)(spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
    key[i] = k;
    atomicAdd(&count[k], 1);
}

// Exclusive scan of kBins counts by one block of 1024 threads (kBins / 1024 per thread):
// per-thread sums, a block scan of those, then each thread rewrites its range in place.
__global__ void __launch_bounds__(1024) k_bin_scan(int32_t* __restrict__ count) {
    constexpr int per = kBins / 1024;
    __shared__ int32_t part[1024];
    int32_t* mine = count + threadIdx.x * per;
    int32_t s = 0;
    for (int j = 0; j < per; ++j) s += mine[j];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = (threadIdx.x >= (unsigned)off) ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;  // exclusive prefix of this thread's range
    for (int j = 0; j < per; ++j) {
        const int32_t c = mine[j];
        mine[j] = run;
        run += c;
    }
}

__global__ void k_bin_scatter(const int32_t* __restrict__ key, int64_t n, int32_t* __restrict__ next,
                              int32_t* __restrict__ order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    order[atomicAdd(&next[key[i]], 1)] = (int32_t)i;
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

// Distance-tier code of every (point, element, image) pair, as the evaluation decides it:
// 0 tier 0, 1 tier a, 2 tier b, 3 tier c, 4 FP64 near pair.
__global__ void k_pair_tiers(const FarNodes* __restrict__ far, const float4* __restrict__ cjk, int64_t n_el, int nimg,
                             const double* __restrict__ pts, int64_t npts, uint8_t* __restrict__ codes) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts * n_el * nimg) return;
    const int64_t p = t / (n_el * nimg);
    const int64_t jk = t - p * (n_el * nimg);
    const int64_t j = jk / nimg;
    float phx, phy, phz, plx, ply, plz;
    split2f(pts[3 * p], phx, plx);
    split2f(pts[3 * p + 1], phy, ply);
    split2f(pts[3 * p + 2], phz, plz);
    float dx, dy, dz;
    const float d2 = pair_d2(phx, phy, phz, plx, ply, plz, cjk[2 * jk], cjk[2 * jk + 1], dx, dy, dz);
    const float4 h = far[j].hdr;
    codes[t] = (d2 >= h.x) ? 0 : (d2 >= h.y) ? 1 : (d2 >= h.z) ? 2 : (d2 >= h.w) ? 3 : 4;
}

}  // namespace

cudaError_t launch_pair_tiers(const FarNodes* far, const float4* cjk, int64_t n_el, int nimg, const double* pts,
                              int64_t npts, uint8_t* codes, cudaStream_t s) {
    const int64_t total = npts * n_el * nimg;
    if (total == 0) return cudaSuccess;
    k_pair_tiers<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(far, cjk, n_el, nimg, pts, npts, codes);
    return cudaGetLastError();
}

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
    // largest power of two <= min(kTileMax, kCjkMax / images): divides the chunk width
    int t = 1;
    while (t * 2 <= kTileMax && t * 2 <= kCjkMax / img.n) t *= 2;
    g.tile_el = t;
    g.grid = grid;
    return g;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

MixedScratch mixed_scratch(void* base, int64_t npts) {
    char* p = static_cast<char*>(base);
    MixedScratch m;
    const size_t n = (size_t)npts;
    m.count = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * kBins);
    m.key = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.order = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.bound = reinterpret_cast<float4*>(p);
    p += align256(sizeof(float4) * n);
    m.list = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.list2 = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.list_p = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.list_e = reinterpret_cast<int32_t*>(p);
    p += align256(sizeof(int32_t) * n);
    m.n_list = reinterpret_cast<int32_t*>(p);
    return m;
}

size_t eval_mixed_scratch_bytes(int64_t npts) {
    const size_t n = (size_t)npts;
    return align256(sizeof(int32_t) * kBins) + 6 * align256(sizeof(int32_t) * n) + align256(sizeof(float4) * n) +
           256;
}

cudaError_t launch_eval_mixed(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma,
                              int64_t n_el, const ImageTable& img, const NearGrid& grid, const int32_t* cell_start,
                              const int32_t* cell_items, const double* pts, int64_t npts, double* phi, double* E,
                              const MixedScratch& ms, cudaStream_t s) {
    if (npts == 0) return cudaSuccess;
    if (npts > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
    const GeomView g = make_view(el, far, cjk, sigma, n_el, img, grid, cell_start, cell_items);
    const unsigned pblocks = (unsigned)((npts + 255) / 256);
    cudaError_t e = cudaMemsetAsync(ms.count, 0, sizeof(int32_t) * kBins, s);
    if (e != cudaSuccess) return e;
    k_bin_keys<<<pblocks, 256, 0, s>>>(pts, npts, grid, ms.key, ms.count);
    k_bin_scan<<<1, 1024, 0, s>>>(ms.count);
    k_bin_scatter<<<pblocks, 256, 0, s>>>(ms.key, npts, ms.count, ms.order);
    const unsigned blocks = (unsigned)((npts + kEvalThreads - 1) / kEvalThreads);
    k_eval_far<<<blocks, kEvalThreads, 0, s>>>(g, pts, ms.order, npts, phi, E, ms.bound);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_eval_near<<<blocks, kEvalThreads, 0, s>>>(g, img, pts, ms.order, npts, phi, E);
    return cudaGetLastError();
}

}  // namespace nb
