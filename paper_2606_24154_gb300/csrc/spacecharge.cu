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
// FP32 with rsqrt.  Runs of 32 sources are summed in FP32 and added to two-float
// (hi + lo) running totals with an error-free two-sum; each thread takes two targets in
// the lanes of the packed FP32x2 instructions.
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

// Mixed sum: each thread takes two targets, t and t + kSC2Threads of its block, held in
// the two lanes of the packed FP32x2 instructions; a source tile is staged in shared
// memory with every value negated and duplicated into both lanes, so that a pair
// (target, source) costs the same rounded operations as the scalar form
//   d = (t_hi - s_hi) + (t_lo - s_lo),  r^2 = d.d + s^2,  q / r,  q d / r^3
// at half the issue slots.  Partial sums over kFlush sources are added to running totals
// kept as two floats (hi + lo, error-free two-sum), so no FP64 instruction runs per
// source; the totals are converted to FP64 once per target.
constexpr int kSC2Threads = 128;
constexpr int kSC2Tile = 2 * kSC2Threads;  // targets per block = sources per tile

struct F2Acc {  // two-float running total per lane: value = hi + lo
    float2 hi, lo;
};

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ void acc_add(F2Acc& a, float2 x) {
    two_sum_add(a.hi.x, a.lo.x, x.x);
    two_sum_add(a.hi.y, a.lo.y, x.y);
}

template <bool SELF>
__device__ __forceinline__ void sc_tile_f32x2(const float4* __restrict__ A, const float4* __restrict__ B,
                                              const float4* __restrict__ C, const float2* __restrict__ D, int k0,
                                              int k1, float2 thx, float2 thy, float2 thz, float2 tlx, float2 tly,
                                              float2 tlz, float2 s2, int self0, int self1, float2& ph, float2& ex,
                                              float2& ey, float2& ez) {
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const float4 a = A[k], b = B[k], c = C[k];
        const float2 d = D[k];
        const float2 dx = __fadd2_rn(__fadd2_rn(thx, make_float2(a.x, a.y)), __fadd2_rn(tlx, make_float2(c.x, c.y)));
        const float2 dy = __fadd2_rn(__fadd2_rn(thy, make_float2(a.z, a.w)), __fadd2_rn(tly, make_float2(c.z, c.w)));
        const float2 dz = __fadd2_rn(__fadd2_rn(thz, make_float2(b.x, b.y)), __fadd2_rn(tlz, d));
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, s2)));
        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        float2 qq = make_float2(b.z, b.w);
        if (SELF) {
            if (k == self0) qq.x = 0.f;
            if (k == self1) qq.y = 0.f;
        }
        const float2 qr = __fmul2_rn(qq, ri);
        const float2 qr3 = __fmul2_rn(qr, __fmul2_rn(ri, ri));
        ph = __fadd2_rn(ph, qr);
        ex = __ffma2_rn(qr3, dx, ex);
        ey = __ffma2_rn(qr3, dy, ey);
        ez = __ffma2_rn(qr3, dz, ez);
    }
}

__device__ __forceinline__ void load_target_2f(const double* __restrict__ tgt, int64_t t, bool active, float& hx,
                                               float& hy, float& hz, float& lx, float& ly, float& lz) {
    double x = 0, y = 0, z = 0;
    if (active) {
        x = tgt[3 * t];
        y = tgt[3 * t + 1];
        z = tgt[3 * t + 2];
    }
    hx = (float)x;
    hy = (float)y;
    hz = (float)z;
    lx = (float)(x - hx);
    ly = (float)(y - hy);
    lz = (float)(z - hz);
}

__device__ __forceinline__ void store_target(int64_t t, int accumulate, double ke, double ph, double ex, double ey,
                                             double ez, double* __restrict__ phi, double* __restrict__ E) {
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

// Targets given as FP64 (split in-kernel); sources as two-float (hi, lo) arrays.
__global__ void __launch_bounds__(kSC2Threads) k_sc_mixed(const float4* __restrict__ shq,
                                                          const float4* __restrict__ slo, int64_t nsrc,
                                                          const double* __restrict__ tgt, int64_t ntgt,
                                                          int exclude_self, float s2, double ke, int accumulate,
                                                          double* __restrict__ phi, double* __restrict__ E) {
    __shared__ float4 sA[kSC2Tile], sB[kSC2Tile], sC[kSC2Tile];
    __shared__ float2 sD[kSC2Tile];
    const int64_t t0 = (int64_t)blockIdx.x * kSC2Tile + threadIdx.x;
    const int64_t t1 = t0 + kSC2Threads;
    float h0x, h0y, h0z, l0x, l0y, l0z, h1x, h1y, h1z, l1x, l1y, l1z;
    load_target_2f(tgt, t0, t0 < ntgt, h0x, h0y, h0z, l0x, l0y, l0z);
    load_target_2f(tgt, t1, t1 < ntgt, h1x, h1y, h1z, l1x, l1y, l1z);
    const float2 thx = make_float2(h0x, h1x), thy = make_float2(h0y, h1y), thz = make_float2(h0z, h1z);
    const float2 tlx = make_float2(l0x, l1x), tly = make_float2(l0y, l1y), tlz = make_float2(l0z, l1z);
    const float2 s22 = make_float2(s2, s2);
    const float2 zero = make_float2(0.f, 0.f);
    F2Acc aph{zero, zero}, aex{zero, zero}, aey{zero, zero}, aez{zero, zero};
    for (int64_t base = 0; base < nsrc; base += kSC2Tile) {
        __syncthreads();
        for (int i = threadIdx.x; i < kSC2Tile; i += kSC2Threads) {
            const int64_t c = base + i;
            if (c < nsrc) {
                const float4 h = shq[c], l = slo[c];
                sA[i] = make_float4(-h.x, -h.x, -h.y, -h.y);
                sB[i] = make_float4(-h.z, -h.z, h.w, h.w);
                sC[i] = make_float4(-l.x, -l.x, -l.y, -l.y);
                sD[i] = make_float2(-l.z, -l.z);
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kSC2Tile, nsrc - base);
        // the tile that holds this block's own carriers (targets are the sources in order)
        const bool self_tile = exclude_self && (base == (int64_t)blockIdx.x * kSC2Tile);
        const int self0 = self_tile ? (int)threadIdx.x : -1;
        const int self1 = self_tile ? (int)threadIdx.x + kSC2Threads : -1;
        // FP32 partial sums over kFlush sources: the +/- charges cancel, so longer FP32
        // runs would lose the result in the partial sums' rounding
        for (int sub = 0; sub < cnt; sub += kFlush) {
            const int m = min(kFlush, cnt - sub);
            float2 fph = zero, fex = zero, fey = zero, fez = zero;
            if (self_tile && ((self0 >= sub && self0 < sub + m) || (self1 >= sub && self1 < sub + m)))
                sc_tile_f32x2<true>(sA, sB, sC, sD, sub, sub + m, thx, thy, thz, tlx, tly, tlz, s22, self0, self1, fph,
                                    fex, fey, fez);
            else
                sc_tile_f32x2<false>(sA, sB, sC, sD, sub, sub + m, thx, thy, thz, tlx, tly, tlz, s22, -1, -1, fph,
                                     fex, fey, fez);
            acc_add(aph, fph);
            acc_add(aex, fex);
            acc_add(aey, fey);
            acc_add(aez, fez);
        }
    }
    if (t0 < ntgt)
        store_target(t0, accumulate, ke, (double)aph.hi.x + (double)aph.lo.x, (double)aex.hi.x + (double)aex.lo.x,
                     (double)aey.hi.x + (double)aey.lo.x, (double)aez.hi.x + (double)aez.lo.x, phi, E);
    if (t1 < ntgt)
        store_target(t1, accumulate, ke, (double)aph.hi.y + (double)aph.lo.y, (double)aex.hi.y + (double)aex.lo.y,
                     (double)aey.hi.y + (double)aey.lo.y, (double)aez.hi.y + (double)aez.lo.y, phi, E);
}

// Four targets per thread for large target sets: two pairs of FP32x2 lanes, (t, t + 128)
// and (t + 256, t + 384) of a 512-target block, share every source load from shared memory,
// and the two independent chains give the scheduler more to overlap.  Per target the
// operations, their order, the 32-source flush groups (tiles of 512 sources hold sixteen of
// them, aligned as in the 256-source tiles) and the running totals are those of
// k_sc_mixed, so the two kernels give the same bits.
constexpr int kSC4Threads = 128;
constexpr int kSC4Tile = 4 * kSC4Threads;

template <bool SELF>
__device__ __forceinline__ void sc_tile_f32x2x2(const float4* __restrict__ A, const float4* __restrict__ B,
                                                const float4* __restrict__ C, const float2* __restrict__ D, int k0,
                                                int k1, const float2 (&th)[2][3], const float2 (&tl)[2][3], float2 s2,
                                                const int (&self)[4], float2 (&ph)[2], float2 (&ex)[2],
                                                float2 (&ey)[2], float2 (&ez)[2]) {
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
        const float4 a = A[k], b = B[k], c = C[k];
        const float2 d = D[k];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 dx =
                __fadd2_rn(__fadd2_rn(th[h][0], make_float2(a.x, a.y)), __fadd2_rn(tl[h][0], make_float2(c.x, c.y)));
            const float2 dy =
                __fadd2_rn(__fadd2_rn(th[h][1], make_float2(a.z, a.w)), __fadd2_rn(tl[h][1], make_float2(c.z, c.w)));
            const float2 dz = __fadd2_rn(__fadd2_rn(th[h][2], make_float2(b.x, b.y)), __fadd2_rn(tl[h][2], d));
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, s2)));
            const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            float2 qq = make_float2(b.z, b.w);
            if (SELF) {
                if (k == self[2 * h]) qq.x = 0.f;
                if (k == self[2 * h + 1]) qq.y = 0.f;
            }
            const float2 qr = __fmul2_rn(qq, ri);
            const float2 qr3 = __fmul2_rn(qr, __fmul2_rn(ri, ri));
            ph[h] = __fadd2_rn(ph[h], qr);
            ex[h] = __ffma2_rn(qr3, dx, ex[h]);
            ey[h] = __ffma2_rn(qr3, dy, ey[h]);
            ez[h] = __ffma2_rn(qr3, dz, ez[h]);
        }
    }
}

__global__ void __launch_bounds__(kSC4Threads) k_sc_mixed4(const float4* __restrict__ shq,
                                                           const float4* __restrict__ slo, int64_t nsrc,
                                                           const double* __restrict__ tgt, int64_t ntgt,
                                                           int exclude_self, float s2, double ke, int accumulate,
                                                           double* __restrict__ phi, double* __restrict__ E) {
    __shared__ float4 sA[kSC4Tile], sB[kSC4Tile], sC[kSC4Tile];
    __shared__ float2 sD[kSC4Tile];
    int64_t tq[4];
    float2 th[2][3], tl[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float hx[2], hy[2], hz[2], lx[2], ly[2], lz[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            tq[2 * h + q] = (int64_t)blockIdx.x * kSC4Tile + threadIdx.x + (2 * h + q) * kSC4Threads;
            load_target_2f(tgt, tq[2 * h + q], tq[2 * h + q] < ntgt, hx[q], hy[q], hz[q], lx[q], ly[q], lz[q]);
        }
        th[h][0] = make_float2(hx[0], hx[1]), th[h][1] = make_float2(hy[0], hy[1]), th[h][2] = make_float2(hz[0], hz[1]);
        tl[h][0] = make_float2(lx[0], lx[1]), tl[h][1] = make_float2(ly[0], ly[1]), tl[h][2] = make_float2(lz[0], lz[1]);
    }
    const float2 s22 = make_float2(s2, s2);
    const float2 zero = make_float2(0.f, 0.f);
    F2Acc aph[2] = {{zero, zero}, {zero, zero}}, aex[2] = {{zero, zero}, {zero, zero}},
          aey[2] = {{zero, zero}, {zero, zero}}, aez[2] = {{zero, zero}, {zero, zero}};
    for (int64_t base = 0; base < nsrc; base += kSC4Tile) {
        __syncthreads();
        for (int i = threadIdx.x; i < kSC4Tile; i += kSC4Threads) {
            const int64_t c = base + i;
            if (c < nsrc) {
                const float4 h = shq[c], l = slo[c];
                sA[i] = make_float4(-h.x, -h.x, -h.y, -h.y);
                sB[i] = make_float4(-h.z, -h.z, h.w, h.w);
                sC[i] = make_float4(-l.x, -l.x, -l.y, -l.y);
                sD[i] = make_float2(-l.z, -l.z);
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kSC4Tile, nsrc - base);
        const bool self_tile = exclude_self && (base == (int64_t)blockIdx.x * kSC4Tile);
        int self[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) self[q] = self_tile ? (int)threadIdx.x + q * kSC4Threads : -1;
        for (int sub = 0; sub < cnt; sub += kFlush) {
            const int m = min(kFlush, cnt - sub);
            float2 fph[2] = {zero, zero}, fex[2] = {zero, zero}, fey[2] = {zero, zero}, fez[2] = {zero, zero};
            bool hit = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) hit |= self[q] >= sub && self[q] < sub + m;
            if (hit)
                sc_tile_f32x2x2<true>(sA, sB, sC, sD, sub, sub + m, th, tl, s22, self, fph, fex, fey, fez);
            else
                sc_tile_f32x2x2<false>(sA, sB, sC, sD, sub, sub + m, th, tl, s22, self, fph, fex, fey, fez);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                acc_add(aph[h], fph[h]);
                acc_add(aex[h], fex[h]);
                acc_add(aey[h], fey[h]);
                acc_add(aez[h], fez[h]);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (tq[2 * h] < ntgt)
            store_target(tq[2 * h], accumulate, ke, (double)aph[h].hi.x + (double)aph[h].lo.x,
                         (double)aex[h].hi.x + (double)aex[h].lo.x, (double)aey[h].hi.x + (double)aey[h].lo.x,
                         (double)aez[h].hi.x + (double)aez[h].lo.x, phi, E);
        if (tq[2 * h + 1] < ntgt)
            store_target(tq[2 * h + 1], accumulate, ke, (double)aph[h].hi.y + (double)aph[h].lo.y,
                         (double)aex[h].hi.y + (double)aex[h].lo.y, (double)aey[h].hi.y + (double)aey[h].lo.y,
                         (double)aez[h].hi.y + (double)aez[h].lo.y, phi, E);
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
    else if (ntgt >= (int64_t)152 * 4 * kSC4Tile)  // enough 512-target blocks for several waves
        k_sc_mixed4<<<(unsigned)((ntgt + kSC4Tile - 1) / kSC4Tile), kSC4Threads, 0, s>>>(
            hq, lo, nsrc, tgt, ntgt, exclude_self, (float)(soft * soft), ke, accumulate, phi, E);
    else
        k_sc_mixed<<<(unsigned)((ntgt + kSC2Tile - 1) / kSC2Tile), kSC2Threads, 0, s>>>(
            hq, lo, nsrc, tgt, ntgt, exclude_self, (float)(soft * soft), ke, accumulate, phi, E);
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
