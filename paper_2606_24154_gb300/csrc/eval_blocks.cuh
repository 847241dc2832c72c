// eval_blocks.cuh -- per-block evaluation bodies shared by the standalone evaluation
// kernels (eval_f64.cu, eval_mixed.cu) and the serving kernel (server.cu): one thread per
// target, `count` <= blockDim.x targets starting at `pts`.  Using the same functions in
// both places makes a point's result identical whichever launch evaluates it.
//
// Mixed precision.
//
// Same sums as the FP64 kernel (Eq. Potential / Eq. Field over elements and periodic
// images), but each (point, element, image) pair picks its arithmetic by its distance d
// to the image centroid, in units of the element's circumradius rho:
//   d >= ratio_0 rho      FP32 Gauss rule, tier 0 (4 nodes)
//   d >= ratio_a rho      FP32 Gauss rule, tier a (6 nodes triangle / 9 rectangle)
//   d >= ratio_b rho      FP32 Gauss rule, tier b (16 nodes)
//   d >= ratio_near rho   FP32 Gauss rule, tier c (36 nodes)
//   nearer                FP64 closed form (influence.cuh), where ln/atan cancel
// Quadrature per node: Phi += w / r, E += w (P - x_n) / r^3 with one rsqrt; two nodes at
// a time in the packed FP32x2 instructions (half the issue slots of scalar FP32).
//
// Two kernels: k_eval_far runs every FP32 tier over all (element, image) pairs and skips
// near pairs; k_eval_near visits only the image centroids in the 27 grid cells around
// each point (a cell list built per geometry, cell edge >= the largest near radius) and
// adds the near pairs' FP64 closed forms.  Keeping the FP64 code out of the far kernel
// keeps its register count (and so its occupancy) at the FP32 kernel's level.  Both
// kernels decide "near" with the same rounded FP32 operations (pair_d2) on the same
// inputs, so every pair is counted exactly once.
//
// The FP32 difference P - x_n keeps its relative accuracy even when P and the node are
// millimetres from the origin but micrometres apart: both sides are held as two floats
// (hi + lo) and (P_hi - C_hi) + (P_lo - C_lo) is formed first, C = c_j + t_k being the
// image centroid (FP64 sum split once per geometry).  Node offsets from the centroid are
// small, so the remaining FP32 operations carry ~1e-7 relative error.
//
// Accumulation: per element over its images in FP32, weighted by sigma_j, summed in FP32
// over groups of kGroup elements and flushed to FP64.  Every decision depends only on the
// pair, and each point's sums run in a fixed order, so a point's result is bit-identical
// whatever other points share its launch.
//
// Error scales.  Beside the sums, the far part accumulates per point the scales of its
// rounding and truncation errors from the per-element terms b_j = |sigma_j| |sum_k Phi'_jk|
// (for E: |sigma_j| |sum_k E'_jk|_1) over the FP32 pairs: their sum B = sum_j b_j and their
// root sum of squares S = sqrt(sum_j b_j^2).  Errors that keep their sign from element to
// element (the Gauss rules' truncation) grow with B; rounding errors, whose signs vary
// from element to element, add up like a random sum and grow with S, which is far smaller
// than B when many elements contribute alike.  eval_acc.cu turns the scales into a
// per-point error estimate and refines the points whose estimate exceeds the requested
// relative tolerance.  The scales do not enter the sums themselves.
#pragma once
#include "influence.cuh"

namespace nb {

constexpr int kEvalThreads = 128;  // threads per block (one target each)
constexpr int kTileMax = 16;       // elements per shared-memory tile (mixed)
constexpr int kCjkMax = 512;       // (element, image) centres per tile (mixed)
constexpr int kGroup = 8;          // elements per FP32 partial sum (mixed)
constexpr int kTile64 = 32;        // elements per shared-memory tile (FP64)
constexpr int kChunkEl = 1024;     // elements per chunk of the far sums (multiple of every tile width)

// Squared FP32 distance between a point (two floats per coordinate) and an image centroid;
// the operation sequence is pinned (no contraction) so both kernels agree bit for bit.
__device__ __forceinline__ float pair_d2(float phx, float phy, float phz, float plx, float ply, float plz,
                                         const float4& ch, const float4& cl, float& dx, float& dy, float& dz) {
    dx = __fadd_rn(__fsub_rn(phx, ch.x), __fsub_rn(plx, cl.x));
    dy = __fadd_rn(__fsub_rn(phy, ch.y), __fsub_rn(ply, cl.y));
    dz = __fadd_rn(__fsub_rn(phz, ch.z), __fsub_rn(plz, cl.z));
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ void split2f(double x, float& hi, float& lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// NP node pairs of one tier (layout in nb_internal.h: s = centroid - node, so the
// node-to-point vector is d + s) with the packed FP32x2 instructions: each instruction
// advances two nodes, lane x the first of a pair and lane y the second.
template <int NP>
__device__ __forceinline__ void node_pairs(const float4* __restrict__ nd, float2 dx, float2 dy, float2 dz,
                                           float2& ph, float2& ex, float2& ey, float2& ez) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float4 u = nd[2 * i], v = nd[2 * i + 1];
        const float2 rx = __fadd2_rn(dx, make_float2(u.x, u.y));
        const float2 ry = __fadd2_rn(dy, make_float2(u.z, u.w));
        const float2 rz = __fadd2_rn(dz, make_float2(v.x, v.y));
        const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 wr = __fmul2_rn(make_float2(v.z, v.w), ri);
        const float2 wr3 = __fmul2_rn(wr, __fmul2_rn(ri, ri));
        ph = __fadd2_rn(ph, wr);
        ex = __ffma2_rn(wr3, rx, ex);
        ey = __ffma2_rn(wr3, ry, ey);
        ez = __ffma2_rn(wr3, rz, ez);
    }
}

// Tier 0 with its two node pairs held in registers (loaded once per element).
__device__ __forceinline__ void pairs0_reg(const float4 (&q)[2 * kPairs0], float2 dx, float2 dy, float2 dz,
                                           float2& ph, float2& ex, float2& ey, float2& ez) {
    node_pairs<kPairs0>(q, dx, dy, dz, ph, ex, ey, ez);
}

// Raw FP64 sums (phi, E; before the factor ke) of the far pairs of one point over the
// elements [e0, e1).  Called by every thread of the block (shared-memory tiles); the
// inactive threads' sums are unused.
struct Sum4 {
    double phi, x, y, z;
};
// far sums plus the error scales B_phi, B_E (raw, before the factor ke)
struct Sum6 {
    double phi, x, y, z, bphi, bE;
};

// Per-thread error scales of the far pass, raw (before the factor ke): (B_phi, B_E, the
// sums of squares of the terms b_j of B_phi and B_E, each term scaled by kScaleSq first).
// Positive sums, FP32 is ample.  They live in a shared-memory slot (read and written once
// per element) rather than in registers across the element loop; bound_reset() before a
// point's first range.
// The squares are taken of b_j * 2^33 (2^33 ~ ke): a term of 1e-19 .. 1e19 volts then
// squares to a normal FP32 number.
constexpr float kScaleSq = 8589934592.0f;  // 2^33
__device__ __forceinline__ float4* bound_slot() {
    __shared__ float4 s_bnd[kEvalThreads];
    return &s_bnd[threadIdx.x];
}
__device__ __forceinline__ void bound_reset() { *bound_slot() = make_float4(0.f, 0.f, 0.f, 0.f); }
// the point's scales summed over its element chunks (in chunk order), also in shared memory
__device__ __forceinline__ float4* bound_total_slot() {
    __shared__ float4 s_btot[kEvalThreads];
    return &s_btot[threadIdx.x];
}

__device__ __forceinline__ Sum4 far_range(const GeomView& g, float phx, float phy, float phz, float plx, float ply,
                                          float plz, int64_t e0, int64_t e1) {
    const FarNodes* __restrict__ far = g.far;
    const float4* __restrict__ cjk = g.cjk;
    const double* __restrict__ sigma = g.sigma;
    const int nimg = g.nimg;
    const int tile_el = g.tile_el;
    __shared__ float4 s_f[kTileMax][2 * kPairs0];
    __shared__ float4 s_a[kTileMax][2 * kPairsA];
    __shared__ int s_na[kTileMax];
    __shared__ float4 s_hdr[kTileMax];
    __shared__ float2 s_sig[kTileMax];  // sigma_j (1 + wcorr_j) as hi + lo
    __shared__ float4 s_c[kCjkMax][2];  // image centroids: hi, lo

    float4* bslot = bound_slot();
    double aphi = 0.0, aEx = 0.0, aEy = 0.0, aEz = 0.0;
    for (int64_t base = e0; base < e1; base += tile_el) {
        const int cnt = (int)min((int64_t)tile_el, e1 - base);
        __syncthreads();
        constexpr int kA = 2 * kPairsA, kF = 2 * kPairs0;
        for (int i = threadIdx.x; i < cnt * kA; i += blockDim.x) s_a[i / kA][i % kA] = far[base + i / kA].a[i % kA];
        for (int i = threadIdx.x; i < cnt * kF; i += blockDim.x) s_f[i / kF][i % kF] = far[base + i / kF].f[i % kF];
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            s_hdr[i] = far[base + i].hdr;
            s_na[i] = far[base + i].n_a;
            const double sd = fma(sigma[base + i], (double)far[base + i].wcorr, sigma[base + i]);
            const float sh = __double2float_rn(sd);
            s_sig[i] = make_float2(sh, __double2float_rn(sd - (double)sh));
        }
        const float4* src = cjk + 2 * base * nimg;
        for (int i = threadIdx.x; i < 2 * cnt * nimg; i += blockDim.x) s_c[i >> 1][i & 1] = src[i];
        __syncthreads();
        float gphi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 hdr = s_hdr[jj];
            const bool rect = s_na[jj] == kPairsA;
            const FarNodes* fj = far + base + jj;
            float4 q[2 * kPairs0];
#pragma unroll
            for (int i = 0; i < 2 * kPairs0; ++i) q[i] = s_f[jj][i];
            float2 lphi = make_float2(0.f, 0.f), lx = lphi, ly = lphi, lz = lphi;
            for (int k = 0; k < nimg; ++k) {
                float dx, dy, dz;
                const float d2 = pair_d2(phx, phy, phz, plx, ply, plz, s_c[jj * nimg + k][0], s_c[jj * nimg + k][1],
                                         dx, dy, dz);
                const float2 DX = make_float2(dx, dx), DY = make_float2(dy, dy), DZ = make_float2(dz, dz);
                if (d2 >= hdr.x) {
                    pairs0_reg(q, DX, DY, DZ, lphi, lx, ly, lz);
                } else if (d2 >= hdr.y) {
                    if (rect)
                        node_pairs<kPairsA>(s_a[jj], DX, DY, DZ, lphi, lx, ly, lz);
                    else
                        node_pairs<3>(s_a[jj], DX, DY, DZ, lphi, lx, ly, lz);
                } else if (d2 >= hdr.z) {
                    node_pairs<kPairsB>(fj->b, DX, DY, DZ, lphi, lx, ly, lz);
                } else if (d2 >= hdr.w) {
                    node_pairs<kPairsC>(fj->c, DX, DY, DZ, lphi, lx, ly, lz);
                }
                // nearer pairs: k_eval_near
            }
            const float2 sg = s_sig[jj];
            const float s = sg.x;
            const float fphi = lphi.x + lphi.y, fx = lx.x + lx.y, fy = ly.x + ly.y, fz = lz.x + lz.y;
            // sigma in two floats: a density that is uniform over many elements (a plane far
            // from the structure) would otherwise carry one FP32 rounding error for all of them
            gphi = fmaf(s, fphi, fmaf(sg.y, fphi, gphi));
            gx = fmaf(s, fx, fmaf(sg.y, fx, gx));
            gy = fmaf(s, fy, fmaf(sg.y, fy, gy));
            gz = fmaf(s, fz, fmaf(sg.y, fz, gz));
            float4 b = *bslot;
            const float t0 = fabsf(s) * fabsf(fphi), t1 = fabsf(s) * (fabsf(fx) + fabsf(fy) + fabsf(fz));
            const float q0 = t0 * kScaleSq, q1 = t1 * kScaleSq;
            b.x += t0;
            b.y += t1;
            b.z = fmaf(q0, q0, b.z);
            b.w = fmaf(q1, q1, b.w);
            *bslot = b;
            if ((jj % kGroup) == kGroup - 1 || jj == cnt - 1) {
                aphi += (double)gphi;
                aEx += (double)gx;
                aEy += (double)gy;
                aEz += (double)gz;
                gphi = gx = gy = gz = 0.f;
            }
        }
    }
    return Sum4{aphi, aEx, aEy, aEz};
}

__device__ __forceinline__ void load_point_2f(const double* __restrict__ pts, int64_t p, bool active, float& phx,
                                              float& phy, float& phz, float& plx, float& ply, float& plz) {
    double Px = 0.0, Py = 0.0, Pz = 0.0;
    if (active) {
        Px = pts[3 * p];
        Py = pts[3 * p + 1];
        Pz = pts[3 * p + 2];
    }
    split2f(Px, phx, plx);
    split2f(Py, phy, ply);
    split2f(Pz, phz, plz);
}

// Stores ke * sum for point p.  A point with a non-finite coordinate has no field: it gets
// NaN in both precisions (the FP32 tiers would otherwise fail every distance test for it
// and leave zeros).  Its coordinates are read again here rather than kept in a register
// through the element loop.
template <class S>
__device__ __forceinline__ void store_far(const double* __restrict__ pts, double* __restrict__ phi,
                                          double* __restrict__ E, int64_t p, const S& s) {
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const bool finite = isfinite(pts[3 * p]) && isfinite(pts[3 * p + 1]) && isfinite(pts[3 * p + 2]);
    const double f = finite ? ke : __longlong_as_double(0x7ff8000000000000ll);
    if (phi) phi[p] = f * s.phi;
    if (E) {
        E[3 * p] = f * s.x;
        E[3 * p + 1] = f * s.y;
        E[3 * p + 2] = f * s.z;
    }
}

// ke * (B_phi, B_E, S_phi, S_E) of point p (the FP32 pass's error scales, V and V/m) from
// the raw sums of bound_slot()
__device__ __forceinline__ void store_bound(float4* __restrict__ bound, int64_t p, float4 b) {
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const double inv = 1.0 / (double)kScaleSq;
    if (bound)
        bound[p] = make_float4((float)(ke * b.x), (float)(ke * b.y), (float)(ke * inv * sqrt((double)b.z)),
                               (float)(ke * inv * sqrt((double)b.w)));
}
__device__ __forceinline__ void add4f(float4& t, const float4& c) {
    t.x += c.x;
    t.y += c.y;
    t.z += c.z;
    t.w += c.w;
}

// Far part (FP32 tiers) of `count` targets; writes ke * sum (overwrites phi / E).  Thread
// t takes point idx[base + t] (or base + t when idx is null) of pts / phi / E.  The
// elements are summed in chunks of kChunkEl whose FP64 sums are added in order, so that
// a launch split over element chunks (the server's small requests) gives the same bits.
// `bound` (may be null) receives ke * (B_phi, B_E, S_phi, S_E) per point.
__device__ __forceinline__ void add6(Sum6& t, const Sum6& c) {
    t.phi += c.phi;
    t.x += c.x;
    t.y += c.y;
    t.z += c.z;
    t.bphi += c.bphi;
    t.bE += c.bE;
}

__device__ __forceinline__ void far_block(const GeomView& g, const double* __restrict__ pts,
                                          const int32_t* __restrict__ idx, int64_t base, int count,
                                          double* __restrict__ phi, double* __restrict__ E,
                                          float4* __restrict__ bound) {
    const bool active = (int)threadIdx.x < count;
    const int64_t p = active ? (idx ? (int64_t)idx[base + threadIdx.x] : base + threadIdx.x) : 0;
    float phx, phy, phz, plx, ply, plz;
    load_point_2f(pts, p, active, phx, phy, phz, plx, ply, plz);
    Sum4 tot{0.0, 0.0, 0.0, 0.0};
    float4* btot = bound_total_slot();  // chunk scales added in chunk order (as the server does)
    *btot = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t e0 = 0; e0 < g.n_el; e0 += kChunkEl) {
        bound_reset();
        const Sum4 c = far_range(g, phx, phy, phz, plx, ply, plz, e0, min(e0 + (int64_t)kChunkEl, g.n_el));
        tot.phi += c.phi;
        tot.x += c.x;
        tot.y += c.y;
        tot.z += c.z;
        add4f(*btot, *bound_slot());
    }
    if (active) {
        store_far(pts, phi, E, p, tot);
        store_bound(bound, p, *btot);
    }
}

// Near part (FP64 closed forms) of one target; adds ke * sum to phi[p] / E[p].
__device__ __forceinline__ void near_point(const GeomView& g, const ImageTable& img, const double* __restrict__ pts,
                                           int64_t p, double* __restrict__ phi, double* __restrict__ E) {
    const Elem* __restrict__ el = g.el;
    const FarNodes* __restrict__ far = g.far;
    const float4* __restrict__ cjk = g.cjk;
    const double* __restrict__ sigma = g.sigma;
    const int32_t* __restrict__ cell_start = g.cell_start;
    const int32_t* __restrict__ cell_items = g.cell_items;
    const int nimg = g.nimg;
    const NearGrid& grid = g.grid;
    const double Px = pts[3 * p], Py = pts[3 * p + 1], Pz = pts[3 * p + 2];
    float phx, phy, phz, plx, ply, plz;
    split2f(Px, phx, plx);
    split2f(Py, phy, ply);
    split2f(Pz, phz, plz);
    // cell of the point, clamped (a point more than one cell outside has no near pair)
    int cc[3];
    const double P[3] = {Px, Py, Pz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = floor((P[a] - grid.origin[a]) * grid.inv_h);
        f = fmin(fmax(f, -2.0), (double)grid.dims[a] + 1.0);
        cc[a] = (int)f;
    }
    double aphi = 0.0, aEx = 0.0, aEy = 0.0, aEz = 0.0;
    bool any = false;
    for (int z = max(cc[2] - 1, 0); z <= min(cc[2] + 1, grid.dims[2] - 1); ++z)
        for (int y = max(cc[1] - 1, 0); y <= min(cc[1] + 1, grid.dims[1] - 1); ++y)
            for (int x = max(cc[0] - 1, 0); x <= min(cc[0] + 1, grid.dims[0] - 1); ++x) {
                const int64_t cell = ((int64_t)z * grid.dims[1] + y) * grid.dims[0] + x;
                for (int32_t it = cell_start[cell]; it < cell_start[cell + 1]; ++it) {
                    const int32_t jk = cell_items[it];
                    const int32_t j = jk / nimg, k = jk - j * nimg;
                    float dx, dy, dz;
                    const float d2 = pair_d2(phx, phy, phz, plx, ply, plz, cjk[2 * (int64_t)jk], cjk[2 * (int64_t)jk + 1],
                                             dx, dy, dz);
                    if (!(d2 < far[j].hdr.w)) continue;
                    const Elem& e = el[j];
                    double f, ux, uy, uz;
                    elem_local_f64(e, Px - img.t[k][0], Py - img.t[k][1], Pz - img.t[k][2], false, f, ux, uy, uz);
                    const double s = sigma[j];
                    aphi = fma(s, f, aphi);
                    aEx = fma(s, fma(ux, e.ex[0], fma(uy, e.ey[0], uz * e.ez[0])), aEx);
                    aEy = fma(s, fma(ux, e.ex[1], fma(uy, e.ey[1], uz * e.ez[1])), aEy);
                    aEz = fma(s, fma(ux, e.ex[2], fma(uy, e.ey[2], uz * e.ez[2])), aEz);
                    any = true;
                }
            }
    if (!any) return;
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    if (phi) phi[p] += ke * aphi;
    if (E) {
        E[3 * p] += ke * aEx;
        E[3 * p + 1] += ke * aEy;
        E[3 * p + 2] += ke * aEz;
    }
}

__device__ __forceinline__ void load_elem_tile(Elem* s_el, const Elem* __restrict__ el, int64_t base, int cnt) {
    const double2* src = reinterpret_cast<const double2*>(el + base);
    double2* dst = reinterpret_cast<double2*>(s_el);
    for (int i = threadIdx.x; i < cnt * 16; i += blockDim.x) dst[i] = src[i];
}

// Raw FP64 sums (before the factor ke) of the closed forms of one point over the elements
// [e0, e1) and all images.  Called by every thread of the block (shared-memory tiles).
__device__ __forceinline__ Sum4 f64_range(const Elem* __restrict__ el, const double* __restrict__ sigma, int64_t e0,
                                          int64_t e1, const ImageTable& img, double Px, double Py, double Pz) {
    __shared__ Elem s_el[kTile64];
    __shared__ double s_sig[kTile64];
    double aphi = 0.0, aEx = 0.0, aEy = 0.0, aEz = 0.0;
    for (int64_t base = e0; base < e1; base += kTile64) {
        const int cnt = (int)min((int64_t)kTile64, e1 - base);
        __syncthreads();
        load_elem_tile(s_el, el, base, cnt);
        if (threadIdx.x < cnt) s_sig[threadIdx.x] = sigma[base + threadIdx.x];
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const Elem& e = s_el[jj];
            double lphi = 0.0, lx = 0.0, ly = 0.0, lz = 0.0;
            for (int k = 0; k < img.n; ++k) {
                double f, gx, gy, gz;
                elem_local_f64(e, Px - img.t[k][0], Py - img.t[k][1], Pz - img.t[k][2], false, f, gx, gy, gz);
                lphi += f;
                lx += gx;
                ly += gy;
                lz += gz;
            }
            const double s = s_sig[jj];
            aphi = fma(s, lphi, aphi);
            aEx = fma(s, fma(lx, e.ex[0], fma(ly, e.ey[0], lz * e.ez[0])), aEx);
            aEy = fma(s, fma(lx, e.ex[1], fma(ly, e.ey[1], lz * e.ez[1])), aEy);
            aEz = fma(s, fma(lx, e.ex[2], fma(ly, e.ey[2], lz * e.ez[2])), aEz);
        }
    }
    return Sum4{aphi, aEx, aEy, aEz};
}

// FP64 closed forms for every pair of `count` targets (overwrites phi / E).  Sums over
// kChunkEl-element chunks are added in order, so that a launch split over element chunks
// (the server's small requests) gives the same bits.
__device__ __forceinline__ void f64_block(const Elem* __restrict__ el, const double* __restrict__ sigma, int64_t n_el,
                                          const ImageTable& img, const double* __restrict__ pts, int count,
                                          double* __restrict__ phi, double* __restrict__ E) {
    const int p = threadIdx.x;
    const bool active = p < count;
    double Px = 0.0, Py = 0.0, Pz = 0.0;
    if (active) {
        Px = pts[3 * p];
        Py = pts[3 * p + 1];
        Pz = pts[3 * p + 2];
    }
    Sum4 tot{0.0, 0.0, 0.0, 0.0};
    for (int64_t e0 = 0; e0 < n_el; e0 += kChunkEl) {
        const Sum4 c = f64_range(el, sigma, e0, min(e0 + (int64_t)kChunkEl, n_el), img, Px, Py, Pz);
        tot.phi += c.phi;
        tot.x += c.x;
        tot.y += c.y;
        tot.z += c.z;
    }
    if (active) store_far(pts, phi, E, p, tot);
}

}  // namespace nb
