// spacecharge.cu -- direct space-charge sums (Sec. 4.2, Alg. 2) and the carrier drift
// step of the dynamic update (Sec. 4.3, Alg. 4).
//
//   phi_t = ke sum_{c != self(t)} q_c / sqrt(r^2 + s^2)
//   E_t   = ke sum_{c != self(t)} q_c (x_t - x_c) / (r^2 + s^2)^{3/2}
//
// The paper launches one kernel per field point with a grid-stride loop over charges,
// a shared-memory tree and one atomicAdd per block.  Here all targets are evaluated in
// one launch as a tiled all-pairs sum: one thread per target, source tiles staged in
// shared memory, a fixed summation order (no atomics, bit-reproducible).
//
// Mixed precision: carriers are stored as two floats per coordinate (hi = fl(x),
// lo = fl(x - hi)).  x_t - x_c = (hi_t - hi_c) + (lo_t - lo_c): for nearby carriers
// hi_t - hi_c is exact (Sterbenz), so the difference keeps FP64 accuracy where it
// matters (near pairs) while every operation is FP32; the rest of the pair term is
// FP32 with rsqrt.  Runs of 32 sources are summed in FP32 and added to FP64 accumulators.
#include "nb_internal.h"

namespace nb {

namespace {

constexpr int kSCThreads = 256;
constexpr int kFlush = 32;

struct __align__(16) Src64 {
    double x, y, z, w;  // position and charge
};

__global__ void __launch_bounds__(kSCThreads) k_sc_f64(const double* __restrict__ src, const double* __restrict__ q,
                                                       int64_t nsrc, const double* __restrict__ tgt, int64_t ntgt,
                                                       int exclude_self, double s2, double ke, int accumulate,
                                                       double* __restrict__ phi, double* __restrict__ E) {
    __shared__ Src64 ss[kSCThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < ntgt;
    double x = 0, y = 0, z = 0;
    if (active) {
        x = tgt[3 * t];
        y = tgt[3 * t + 1];
        z = tgt[3 * t + 2];
    }
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int64_t base = 0; base < nsrc; base += kSCThreads) {
        __syncthreads();
        const int64_t c = base + threadIdx.x;
        if (c < nsrc) ss[threadIdx.x] = Src64{src[3 * c], src[3 * c + 1], src[3 * c + 2], q[c]};
        __syncthreads();
        const int cnt = (int)min((int64_t)kSCThreads, nsrc - base);
        for (int k = 0; k < cnt; ++k) {
            const Src64 s = ss[k];
            const double dx = x - s.x, dy = y - s.y, dz = z - s.z;
            const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, s2)));
            const double ri = 1.0 / sqrt(r2);
            double qq = s.w;
            if (exclude_self && base + k == t) qq = 0.0;
            const double qr = qq * ri;
            const double qr3 = qr * ri * ri;
            ph += qr;
            ex = fma(qr3, dx, ex);
            ey = fma(qr3, dy, ey);
            ez = fma(qr3, dz, ez);
        }
    }
    if (!active) return;
    if (accumulate) {
        if (phi) phi[t] += ke * ph;
        if (E) {
            E[3 * t] += ke * ex;
            E[3 * t + 1] += ke * ey;
            E[3 * t + 2] += ke * ez;
        }
    } else {
        if (phi) phi[t] = ke * ph;
        if (E) {
            E[3 * t] = ke * ex;
            E[3 * t + 1] = ke * ey;
            E[3 * t + 2] = ke * ez;
        }
    }
}

// Two-float split of carriers: hq = (hi.x, hi.y, hi.z, q), lo = (lo.x, lo.y, lo.z, 0).
__global__ void k_split2f(const double* __restrict__ pos, const double* __restrict__ q, int64_t n,
                          float4* __restrict__ hq, float4* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    hq[i] = make_float4(hx, hy, hz, (float)q[i]);
    lo[i] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
}

template <bool SELF>
__device__ __forceinline__ void sc_tile_f32(const float4* __restrict__ sh, const float4* __restrict__ sl, int cnt,
                                            float thx, float thy, float thz, float tlx, float tly, float tlz,
                                            float s2, int self_k, float& ph, float& ex, float& ey, float& ez) {
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const float4 h = sh[k];
        const float4 l = sl[k];
        const float dx = (thx - h.x) + (tlx - l.x);
        const float dy = (thy - h.y) + (tly - l.y);
        const float dz = (thz - h.z) + (tlz - l.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, s2)));
        const float ri = rsqrtf(r2);
        float qq = h.w;
        if (SELF && k == self_k) qq = 0.f;
        const float qr = qq * ri;
        const float qr3 = qr * ri * ri;
        ph += qr;
        ex = fmaf(qr3, dx, ex);
        ey = fmaf(qr3, dy, ey);
        ez = fmaf(qr3, dz, ez);
    }
}

// Targets given as FP64 (split in-kernel); sources as two-float tiles.
__global__ void __launch_bounds__(kSCThreads) k_sc_mixed(const float4* __restrict__ shq, const float4* __restrict__ slo,
                                                         int64_t nsrc, const double* __restrict__ tgt, int64_t ntgt,
                                                         int exclude_self, float s2, double ke, int accumulate,
                                                         double* __restrict__ phi, double* __restrict__ E) {
    __shared__ float4 sh[kSCThreads];
    __shared__ float4 sl[kSCThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < ntgt;
    double x = 0, y = 0, z = 0;
    if (active) {
        x = tgt[3 * t];
        y = tgt[3 * t + 1];
        z = tgt[3 * t + 2];
    }
    const float thx = (float)x, thy = (float)y, thz = (float)z;
    const float tlx = (float)(x - thx), tly = (float)(y - thy), tlz = (float)(z - thz);
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int64_t base = 0; base < nsrc; base += kSCThreads) {
        __syncthreads();
        const int64_t c = base + threadIdx.x;
        if (c < nsrc) {
            sh[threadIdx.x] = shq[c];
            sl[threadIdx.x] = slo[c];
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kSCThreads, nsrc - base);
        // the tile that holds this thread's own carrier (block-uniform when targets are the
        // sources in order: the tile index equals the block index)
        const bool self_tile = exclude_self && (base == (int64_t)blockIdx.x * blockDim.x);
        const int self_k = self_tile ? (int)(t - base) : -1;
        // FP32 partial sums over 32 sources at a time, flushed to FP64: the +/- charges
        // cancel, so longer FP32 runs would lose the result in the partial sums' rounding
        for (int sub = 0; sub < cnt; sub += kFlush) {
            const int m = min(kFlush, cnt - sub);
            float fph = 0.f, fex = 0.f, fey = 0.f, fez = 0.f;
            if (self_k >= sub && self_k < sub + m)
                sc_tile_f32<true>(sh + sub, sl + sub, m, thx, thy, thz, tlx, tly, tlz, s2, self_k - sub, fph, fex,
                                  fey, fez);
            else
                sc_tile_f32<false>(sh + sub, sl + sub, m, thx, thy, thz, tlx, tly, tlz, s2, -1, fph, fex, fey, fez);
            ph += fph;
            ex += fex;
            ey += fey;
            ez += fez;
        }
    }
    if (!active) return;
    if (accumulate) {
        if (phi) phi[t] += ke * ph;
        if (E) {
            E[3 * t] += ke * ex;
            E[3 * t + 1] += ke * ey;
            E[3 * t + 2] += ke * ez;
        }
    } else {
        if (phi) phi[t] = ke * ph;
        if (E) {
            E[3 * t] = ke * ex;
            E[3 * t + 1] = ke * ey;
            E[3 * t + 2] = ke * ez;
        }
    }
}

// b_i -= phi_sc(c_i) on conductor rows, b_i -= n_i . E_sc(c_i) on interface rows.
__global__ void k_rhs_sc(const Elem* __restrict__ el, int64_t n, const double* __restrict__ phi,
                         const double* __restrict__ E, double* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Elem& e = el[i];
    if (e.bc == NEBEM_CONDUCTOR)
        b[i] -= phi[i];
    else
        b[i] -= e.ey[0] * E[3 * i] + e.ey[1] * E[3 * i + 1] + e.ey[2] * E[3 * i + 2];
}

__global__ void k_centroids(const Elem* __restrict__ el, int64_t n, double* __restrict__ c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    c[3 * i] = el[i].c[0];
    c[3 * i + 1] = el[i].c[1];
    c[3 * i + 2] = el[i].c[2];
}

// x_c += sign(q_c) mu E_c dt
__global__ void k_drift(double* __restrict__ pos, const double* __restrict__ q, const double* __restrict__ E,
                        int64_t n, double mu_dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = (q[i] > 0.0) ? 1.0 : ((q[i] < 0.0) ? -1.0 : 0.0);
    const double f = s * mu_dt;
    pos[3 * i] += f * E[3 * i];
    pos[3 * i + 1] += f * E[3 * i + 1];
    pos[3 * i + 2] += f * E[3 * i + 2];
}

}  // namespace

cudaError_t launch_sc_split(const double* pos, const double* q, int64_t n, float4* hq, float4* lo, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_split2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, q, n, hq, lo);
    return cudaGetLastError();
}

cudaError_t launch_sc_eval(int precision, const double* src, const double* q, const float4* hq, const float4* lo,
                           int64_t nsrc, const double* tgt, int64_t ntgt, int exclude_self, double soft,
                           int accumulate, double* phi, double* E, cudaStream_t s) {
    if (ntgt == 0) return cudaSuccess;
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const unsigned blocks = (unsigned)((ntgt + kSCThreads - 1) / kSCThreads);
    if (precision == NEBEM_FP64)
        k_sc_f64<<<blocks, kSCThreads, 0, s>>>(src, q, nsrc, tgt, ntgt, exclude_self, soft * soft, ke, accumulate, phi,
                                               E);
    else
        k_sc_mixed<<<blocks, kSCThreads, 0, s>>>(hq, lo, nsrc, tgt, ntgt, exclude_self, (float)(soft * soft), ke,
                                                 accumulate, phi, E);
    return cudaGetLastError();
}

cudaError_t launch_rhs_sc(const Elem* el, int64_t n, const double* phi, const double* E, double* b, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_rhs_sc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(el, n, phi, E, b);
    return cudaGetLastError();
}

cudaError_t launch_centroids(const Elem* el, int64_t n, double* c, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_centroids<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(el, n, c);
    return cudaGetLastError();
}

cudaError_t launch_drift(double* pos, const double* q, const double* E, int64_t n, double mu_dt, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_drift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, q, E, n, mu_dt);
    return cudaGetLastError();
}

}  // namespace nb
