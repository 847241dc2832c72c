// eval_f64.cu -- FP64 evaluation and influence-matrix fill kernels.
//
// Evaluation (Eq. Potential / Eq. Field with element charge densities):
//   phi(x) = ke sum_j sigma_j sum_k Phi'(x - t_k; j),  E(x) likewise with E'.
// One thread per target (body f64_block in eval_blocks.cuh); element tiles are staged in
// shared memory (broadcast reads); the image sum of one element is accumulated in its
// local frame and rotated once.
//
// Fill (Eq. Matrix, collocation at centroids):
//   conductor row i:  K_ij = ke sum_k Phi'(c_i - t_k; j)
//   interface row i:  K_ij = ke sum_k n_i . E'(c_i - t_k; j) + delta_ij diag_i
// Thread per row i (coalesced column-major stores K[i + j n]), grid.y over column chunks.
#include "eval_blocks.cuh"

namespace nb {

namespace {

constexpr int kTile = 32;
constexpr int kThreads = 128;
constexpr int kFillCols = 64;

__device__ __forceinline__ void load_tile(Elem* s_el, const Elem* __restrict__ el, int64_t base, int cnt) {
    const double2* src = reinterpret_cast<const double2*>(el + base);
    double2* dst = reinterpret_cast<double2*>(s_el);
    for (int i = threadIdx.x; i < cnt * 16; i += blockDim.x) dst[i] = src[i];
}

__global__ void __launch_bounds__(kThreads) k_eval_f64(const Elem* __restrict__ el, const double* __restrict__ sigma,
                                                       int64_t n_el, const ImageTable img,
                                                       const double* __restrict__ pts, int64_t npts,
                                                       double* __restrict__ phi, double* __restrict__ E) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int count = (int)min((int64_t)blockDim.x, npts - base);
    f64_block(el, sigma, n_el, img, pts + 3 * base, count, phi ? phi + base : nullptr, E ? E + 3 * base : nullptr);
}

__global__ void __launch_bounds__(kThreads) k_fill_f64(const Elem* __restrict__ el, const double* __restrict__ diag_in,
                                                       int64_t n, const ImageTable img, double* __restrict__ K) {
    __shared__ Elem s_el[kTile];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    double cx = 0.0, cy = 0.0, cz = 0.0, nx = 0.0, ny = 0.0, nz = 0.0, diag = 0.0;
    int bc = 0;
    if (active) {
        const Elem& ei = el[i];
        cx = ei.c[0];
        cy = ei.c[1];
        cz = ei.c[2];
        nx = ei.ey[0];
        ny = ei.ey[1];
        nz = ei.ey[2];
        bc = ei.bc;
        diag = diag_in[i];  // (eps_a + eps_b) / (2 eps0 (eps_b - eps_a)) on interface rows, else 0
    }
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const int64_t j0 = (int64_t)blockIdx.y * kFillCols;
    const int64_t j1 = min(n, j0 + kFillCols);
    for (int64_t base = j0; base < j1; base += kTile) {
        const int cnt = (int)min((int64_t)kTile, j1 - base);
        __syncthreads();
        load_tile(s_el, el, base, cnt);
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const Elem& e = s_el[jj];
            const int64_t j = base + jj;
            double acc = 0.0;
            for (int k = 0; k < img.n; ++k) {
                double f, gx, gy, gz;
                const bool self = (i == j) && (k == img.k0);
                elem_local_f64(e, cx - img.t[k][0], cy - img.t[k][1], cz - img.t[k][2], self, f, gx, gy, gz);
                if (bc == NEBEM_CONDUCTOR) {
                    acc += f;
                } else {
                    // n_i . (gx ex + gy ey + gz ez)
                    const double Ex = fma(gx, e.ex[0], fma(gy, e.ey[0], gz * e.ez[0]));
                    const double Ey = fma(gx, e.ex[1], fma(gy, e.ey[1], gz * e.ez[1]));
                    const double Ez = fma(gx, e.ex[2], fma(gy, e.ey[2], gz * e.ez[2]));
                    acc += fma(nx, Ex, fma(ny, Ey, nz * Ez));
                }
            }
            if (active) K[i + j * n] = (i == j) ? fma(ke, acc, diag) : ke * acc;
        }
    }
}

__global__ void k_element_influence(const Elem* __restrict__ el, int64_t n_el, const double* __restrict__ pts,
                                    int64_t npts, double* __restrict__ phi, double* __restrict__ E) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_el * npts) return;
    const int64_t e = t / npts, p = t % npts;
    const Elem& el_e = el[e];
    double f, gx, gy, gz;
    elem_local_f64(el_e, pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], false, f, gx, gy, gz);
    phi[t] = f;
    E[3 * t] = fma(gx, el_e.ex[0], fma(gy, el_e.ey[0], gz * el_e.ez[0]));
    E[3 * t + 1] = fma(gx, el_e.ex[1], fma(gy, el_e.ey[1], gz * el_e.ez[1]));
    E[3 * t + 2] = fma(gx, el_e.ex[2], fma(gy, el_e.ey[2], gz * el_e.ez[2]));
}

}  // namespace

cudaError_t launch_eval_f64(const Elem* el, const double* sigma, int64_t n_el, const ImageTable& img,
                            const double* pts, int64_t npts, double* phi, double* E, cudaStream_t s) {
    if (npts == 0) return cudaSuccess;
    const int64_t blocks = (npts + kThreads - 1) / kThreads;
    k_eval_f64<<<(unsigned)blocks, kThreads, 0, s>>>(el, sigma, n_el, img, pts, npts, phi, E);
    return cudaGetLastError();
}

cudaError_t launch_fill_f64(const Elem* el, const double* diag, int64_t n, const ImageTable& img, double* K,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + kThreads - 1) / kThreads), (unsigned)((n + kFillCols - 1) / kFillCols));
    k_fill_f64<<<grid, kThreads, 0, s>>>(el, diag, n, img, K);
    return cudaGetLastError();
}

cudaError_t launch_element_influence(const Elem* el, int64_t n_el, const double* pts, int64_t npts,
                                     double* phi, double* E, cudaStream_t s) {
    const int64_t total = n_el * npts;
    if (total == 0) return cudaSuccess;
    k_element_influence<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(el, n_el, pts, npts, phi, E);
    return cudaGetLastError();
}

}  // namespace nb
