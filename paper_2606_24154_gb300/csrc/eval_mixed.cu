// eval_mixed.cu -- mixed-precision evaluation of potential and field at points.
//
// Same sums as the FP64 kernel (Eq. Potential / Eq. Field over elements and periodic
// images), but each (point, element, image) pair picks its arithmetic by its distance d
// to the image centroid, in units of the element's circumradius rho:
//   d >= ratio_a rho      FP32 Gauss rule, tier a (6 nodes triangle / 9 rectangle)
//   d >= ratio_b rho      FP32 Gauss rule, tier b (16 nodes)
//   d >= ratio_near rho   FP32 Gauss rule, tier c (36 nodes)
//   nearer                FP64 closed form (influence.cuh), where ln/atan cancel
// Quadrature per node: Phi += w / r, E += w (P - x_n) / r^3 with one rsqrt.
//
// The FP32 difference P - x_n must keep its relative accuracy even when P and the
// node are millimetres from the origin but only micrometres apart, so both sides are
// held as two floats (hi + lo): (P_hi - C_hi) + (P_lo - C_lo), where C = c_j + t_k is the
// image centroid formed in FP64 once per block tile and split.  Node offsets from the
// centroid are small, so the remaining FP32 operations carry ~1e-7 relative error.
//
// Accumulation: per element over its images in FP32, weighted by sigma_j, summed in FP32
// over groups of kGroup elements and flushed to FP64 accumulators.  The choice of
// arithmetic depends only on the pair itself, so a point's result does not depend on
// which other points share its launch (bit-identical alone or batched).
#include "influence.cuh"

namespace nb {

namespace {

constexpr int kMT = 128;        // threads per block (one target each)
constexpr int kTileMax = 32;    // elements per shared-memory tile
constexpr int kCjkMax = 1024;   // (element, image) centres per tile
constexpr int kGroup = 4;       // elements per FP32 partial sum

__device__ __forceinline__ void nodes_f32(const float4* __restrict__ nd, int m, float dx, float dy, float dz,
                                          float& ph, float& ex, float& ey, float& ez) {
#pragma unroll 3
    for (int i = 0; i < m; ++i) {
        const float4 q = nd[i];
        const float rx = dx - q.x, ry = dy - q.y, rz = dz - q.z;
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float ri = rsqrtf(r2);
        const float wr = q.w * ri;
        const float wr3 = wr * ri * ri;
        ph += wr;
        ex = fmaf(wr3, rx, ex);
        ey = fmaf(wr3, ry, ey);
        ez = fmaf(wr3, rz, ez);
    }
}

__global__ void __launch_bounds__(kMT) k_eval_mixed(const Elem* __restrict__ el, const FarNodes* __restrict__ far,
                                                    const double* __restrict__ sigma, int64_t n_el,
                                                    const ImageTable img, int tile_el,
                                                    const double* __restrict__ pts, int64_t npts,
                                                    double* __restrict__ phi, double* __restrict__ E) {
    __shared__ Elem s_el[kTileMax];
    __shared__ float4 s_a[kTileMax][kNodesA];
    __shared__ float4 s_hdr[kTileMax];
    __shared__ float s_sig[kTileMax];
    __shared__ float s_c[kCjkMax][6];  // image centroids: hi.xyz, lo.xyz

    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < npts;
    double Px = 0.0, Py = 0.0, Pz = 0.0;
    if (active) {
        Px = pts[3 * p];
        Py = pts[3 * p + 1];
        Pz = pts[3 * p + 2];
    }
    const float phx = (float)Px, phy = (float)Py, phz = (float)Pz;
    const float plx = (float)(Px - (double)phx), ply = (float)(Py - (double)phy), plz = (float)(Pz - (double)phz);
    const int nimg = img.n;

    double aphi = 0.0, aEx = 0.0, aEy = 0.0, aEz = 0.0;
    for (int64_t base = 0; base < n_el; base += tile_el) {
        const int cnt = (int)min((int64_t)tile_el, n_el - base);
        __syncthreads();
        {
            const double2* src = reinterpret_cast<const double2*>(el + base);
            double2* dst = reinterpret_cast<double2*>(s_el);
            for (int i = threadIdx.x; i < cnt * 16; i += blockDim.x) dst[i] = src[i];
            for (int i = threadIdx.x; i < cnt * kNodesA; i += blockDim.x)
                s_a[i / kNodesA][i % kNodesA] = far[base + i / kNodesA].a[i % kNodesA];
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                s_hdr[i] = far[base + i].hdr;
                s_sig[i] = (float)sigma[base + i];
            }
            for (int i = threadIdx.x; i < cnt * nimg; i += blockDim.x) {
                const int jj = i / nimg, k = i % nimg;
                const Elem& e = el[base + jj];
                const double cx = e.c[0] + img.t[k][0];
                const double cy = e.c[1] + img.t[k][1];
                const double cz = e.c[2] + img.t[k][2];
                const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
                s_c[i][0] = hx;
                s_c[i][1] = hy;
                s_c[i][2] = hz;
                s_c[i][3] = (float)(cx - (double)hx);
                s_c[i][4] = (float)(cy - (double)hy);
                s_c[i][5] = (float)(cz - (double)hz);
            }
        }
        __syncthreads();
        float gphi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 hdr = s_hdr[jj];
            const int n_a = (int)hdr.w;
            float lphi = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
            double nphi = 0.0, nlx = 0.0, nly = 0.0, nlz = 0.0;  // FP64 near pairs, local frame
            bool any_near = false;
            for (int k = 0; k < nimg; ++k) {
                const float* C = s_c[jj * nimg + k];
                const float dx = (phx - C[0]) + (plx - C[3]);
                const float dy = (phy - C[1]) + (ply - C[4]);
                const float dz = (phz - C[2]) + (plz - C[5]);
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 >= hdr.x) {
                    nodes_f32(s_a[jj], n_a, dx, dy, dz, lphi, lx, ly, lz);
                } else if (d2 >= hdr.y) {
                    nodes_f32(far[base + jj].b, kNodesB, dx, dy, dz, lphi, lx, ly, lz);
                } else if (d2 >= hdr.z) {
                    nodes_f32(far[base + jj].c, kNodesC, dx, dy, dz, lphi, lx, ly, lz);
                } else {
                    double f, ux, uy, uz;
                    elem_local_f64(s_el[jj], Px - img.t[k][0], Py - img.t[k][1], Pz - img.t[k][2], false, f, ux, uy,
                                   uz);
                    nphi += f;
                    nlx += ux;
                    nly += uy;
                    nlz += uz;
                    any_near = true;
                }
            }
            const float s = s_sig[jj];
            gphi = fmaf(s, lphi, gphi);
            gx = fmaf(s, lx, gx);
            gy = fmaf(s, ly, gy);
            gz = fmaf(s, lz, gz);
            if (any_near) {
                const Elem& e = s_el[jj];
                const double sd = sigma[base + jj];
                aphi = fma(sd, nphi, aphi);
                aEx = fma(sd, fma(nlx, e.ex[0], fma(nly, e.ey[0], nlz * e.ez[0])), aEx);
                aEy = fma(sd, fma(nlx, e.ex[1], fma(nly, e.ey[1], nlz * e.ez[1])), aEy);
                aEz = fma(sd, fma(nlx, e.ex[2], fma(nly, e.ey[2], nlz * e.ez[2])), aEz);
            }
            if ((jj % kGroup) == kGroup - 1 || jj == cnt - 1) {
                aphi += (double)gphi;
                aEx += (double)gx;
                aEy += (double)gy;
                aEz += (double)gz;
                gphi = gx = gy = gz = 0.f;
            }
        }
    }
    if (active) {
        const double ke = 1.0 / (4.0 * kPi * kEps0);
        if (phi) phi[p] = ke * aphi;
        if (E) {
            E[3 * p] = ke * aEx;
            E[3 * p + 1] = ke * aEy;
            E[3 * p + 2] = ke * aEz;
        }
    }
}

}  // namespace

cudaError_t launch_eval_mixed(const Elem* el, const FarNodes* far, const double* sigma, int64_t n_el,
                              const ImageTable& img, const double* pts, int64_t npts, double* phi, double* E,
                              cudaStream_t s) {
    if (npts == 0) return cudaSuccess;
    const int tile_el = max(1, min(kTileMax, kCjkMax / img.n));
    const int64_t blocks = (npts + kMT - 1) / kMT;
    k_eval_mixed<<<(unsigned)blocks, kMT, 0, s>>>(el, far, sigma, n_el, img, tile_el, pts, npts, phi, E);
    return cudaGetLastError();
}

}  // namespace nb
