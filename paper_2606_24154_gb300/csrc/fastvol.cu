// fastvol.cu -- FastVolume field maps (Sec. 3.3 FastVolume; ComputeProperties /
// CreateFastVolPF in Sec. 4.1): potential and field precomputed at the nodes of a 3-D
// rectilinear grid (node coordinates per axis, so nodes can be packed densely where the
// field varies fast), then estimated anywhere inside by trilinear interpolation of the
// eight surrounding nodes.  The node values come from the same evaluation kernels as
// nebem_eval (FP64 or mixed), so a map inherits their accuracy at the nodes.
#include "context.h"

namespace nb {

namespace {

// node (i, j, k) -> coordinates, x fastest
__global__ void k_grid_nodes(const double* __restrict__ ax, const double* __restrict__ ay,
                             const double* __restrict__ az, int nx, int ny, int nz, double* __restrict__ pts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nx * ny * nz;
    if (t >= total) return;
    const int i = (int)(t % nx);
    const int j = (int)((t / nx) % ny);
    const int k = (int)(t / ((int64_t)nx * ny));
    pts[3 * t] = ax[i];
    pts[3 * t + 1] = ay[j];
    pts[3 * t + 2] = az[k];
}

// largest index c in [0, n-2] with a[c] <= x (clamped), by bisection
__device__ __forceinline__ int find_cell(const double* __restrict__ a, int n, double x) {
    int lo = 0, hi = n - 1;
    if (x <= a[0]) return 0;
    if (x >= a[n - 1]) return n - 2;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Trilinear interpolation of (phi, Ex, Ey, Ez) node values; points outside the box take the
// values of the nearest face (coordinates clamped to the box).  A point with a non-finite
// coordinate gets NaN (clamping would otherwise map it to a face).
__global__ void k_fastvol_lookup(const double* __restrict__ ax, const double* __restrict__ ay,
                                 const double* __restrict__ az, int nx, int ny, int nz,
                                 const double* __restrict__ vphi, const double* __restrict__ vE,
                                 const double* __restrict__ pts, int64_t n, double* __restrict__ phi,
                                 double* __restrict__ E) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (!isfinite(pts[3 * p]) || !isfinite(pts[3 * p + 1]) || !isfinite(pts[3 * p + 2])) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (phi) phi[p] = nan;
        if (E) E[3 * p] = E[3 * p + 1] = E[3 * p + 2] = nan;
        return;
    }
    const double x = fmin(fmax(pts[3 * p], ax[0]), ax[nx - 1]);
    const double y = fmin(fmax(pts[3 * p + 1], ay[0]), ay[ny - 1]);
    const double z = fmin(fmax(pts[3 * p + 2], az[0]), az[nz - 1]);
    const int i = find_cell(ax, nx, x), j = find_cell(ay, ny, y), k = find_cell(az, nz, z);
    const double tx = (x - ax[i]) / (ax[i + 1] - ax[i]);
    const double ty = (y - ay[j]) / (ay[j + 1] - ay[j]);
    const double tz = (z - az[k]) / (az[k + 1] - az[k]);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        const double w = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty) * (dk ? tz : 1.0 - tz);
        const int64_t node = ((int64_t)(k + dk) * ny + (j + dj)) * nx + (i + di);
        s[0] = fma(w, vphi[node], s[0]);
        s[1] = fma(w, vE[3 * node], s[1]);
        s[2] = fma(w, vE[3 * node + 1], s[2]);
        s[3] = fma(w, vE[3 * node + 2], s[3]);
    }
    if (phi) phi[p] = s[0];
    if (E) {
        E[3 * p] = s[1];
        E[3 * p + 1] = s[2];
        E[3 * p + 2] = s[3];
    }
}

}  // namespace

cudaError_t launch_grid_nodes(const double* ax, const double* ay, const double* az, int nx, int ny, int nz,
                              double* pts, cudaStream_t s) {
    const int64_t total = (int64_t)nx * ny * nz;
    if (total == 0) return cudaSuccess;
    k_grid_nodes<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ax, ay, az, nx, ny, nz, pts);
    return cudaGetLastError();
}

cudaError_t launch_fastvol_lookup(const double* ax, const double* ay, const double* az, int nx, int ny, int nz,
                                  const double* vphi, const double* vE, const double* pts, int64_t n, double* phi,
                                  double* E, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_fastvol_lookup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ax, ay, az, nx, ny, nz, vphi, vE, pts, n, phi, E);
    return cudaGetLastError();
}

}  // namespace nb
