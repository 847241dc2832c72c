// lines.cu -- line-charge representation of the known charges (Sec. 4.2, Alg. 3; the
// LineCh branch of Alg. 4): point -> line reduction on a voxel grid, and the potential
// and field of finite uniform line charges at targets.
//
// Reduction.  The paper scatters the points into voxels with atomicAdd and numbers the
// lines with an atomic counter, so the line order and each voxel's summation order vary
// from run to run.  Here the reduction is deterministic:
//   1. min / max of the cloud (exact) -> the grid's corner (the cloud's minimum corner)
//      and its dimensions, floor((max - min) / d) + 1 per axis;
//   2. one key per point, voxel * n + point: the keys are unique;
//   3. bitonic sort of the keys (a set of unique keys has one sorted order);
//   4. segment heads (the first key of every voxel), scanned into line indices;
//   5. one thread per occupied voxel sums its points' charges in point order and writes
//      the line: along z through the voxel's centre, from its lower to its upper z face,
//      lambda = total charge / dz.
// Lines come out in increasing voxel index, as a sequential reading of Alg. 3 lists
// them.  Index and centre arithmetic uses explicitly rounded operations (the plain IEEE
// sequence, never contracted).
//
// Line-charge sums (softened like the point charges, s = softening).  For a line from a
// along unit u of length len and a target P: w = P - a, x = w.u, p = w - x u,
// rho^2 = |p|^2 + s^2, s1 = -x, s2 = len - x, R1,2 = sqrt(s1,2^2 + rho^2),
//   phi = ke lam ln((s2 + R2) / (s1 + R1))     (written without cancellation per side),
//   E   = ke lam [ -len (s1 + s2) / (R1 R2 (R1 + R2)) u + c_perp p ],
//   c_perp = (s2/R2 - s1/R1) / rho^2 = (s2^2 - s1^2) / (R1 R2 (s2 R1 + s1 R2)) when s1 and
//   s2 have the same sign (target beyond either end: the second form avoids cancellation).
// FP64 mode evaluates every pair so.  Mixed mode evaluates far lines by Gauss-Legendre
// nodes along the line in FP32 on the two-float target-minus-midpoint difference, with a
// node count by the distance d in half lengths h (>= 96 h: 2 nodes, >= 16 h: 3, >= 8 h: 4,
// >= 3 h: 6; worst per-pair error about 1e-8), FP32 partial sums over 32 lines flushed to
// FP64 (k_line_far); lines nearer than 3 h take the FP64 closed form in a second kernel
// that visits only the voxel rows around the target (k_line_near).  Both kernels decide
// "near" with the same rounded FP32 operations, so every pair is counted once.
#include <algorithm>
#include <climits>
#include <cmath>

#include "geometry.h"
#include "nb_internal.h"

namespace nb {

namespace {

constexpr int kMM = 256;          // min/max: threads per block
constexpr int kMMBlocks = 512;    // min/max: most blocks
constexpr int kSortTile = 2048;   // keys sorted in shared memory by one block
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kLT = 128;          // line sums: targets per block = lines per shared tile
constexpr int kLFlush = 32;       // lines per FP32 partial sum

// ------------------------------------------------------------------ reduction

__global__ void __launch_bounds__(kMM) k_minmax_partial(const double* __restrict__ pos, int64_t n,
                                                        double* __restrict__ partial) {
    __shared__ double smn[3][kMM], smx[3][kMM];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * kMM + threadIdx.x; i < n; i += (int64_t)gridDim.x * kMM) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = pos[3 * i + a];
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        smn[a][threadIdx.x] = mn[a];
        smx[a][threadIdx.x] = mx[a];
    }
    for (int off = kMM / 2; off > 0; off >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < off) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                smn[a][threadIdx.x] = fmin(smn[a][threadIdx.x], smn[a][threadIdx.x + off]);
                smx[a][threadIdx.x] = fmax(smx[a][threadIdx.x], smx[a][threadIdx.x + off]);
            }
        }
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            partial[6 * blockIdx.x + a] = smn[a][0];
            partial[6 * blockIdx.x + 3 + a] = smx[a][0];
        }
    }
}

// Grid of the reduction: corner = minimum, dims = floor((max - min) / d) + 1.  A grid
// whose flat voxel index, or whose key voxel * n + point, would not fit in 62 bits is
// flagged (err, and sticky for a sequence of steps); so is a set with no finite extent
// (every position NaN leaves the bounds at +inf / -inf).
__global__ void __launch_bounds__(kMMBlocks) k_minmax_final(const double* __restrict__ partial, int nblk, int64_t n,
                                                            double d0, double d1, double d2, VoxGrid* __restrict__ g) {
    __shared__ double smn[3][kMMBlocks], smx[3][kMMBlocks];
    const int t = threadIdx.x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        smn[a][t] = t < nblk ? partial[6 * t + a] : INFINITY;
        smx[a][t] = t < nblk ? partial[6 * t + 3 + a] : -INFINITY;
    }
    for (int off = kMMBlocks / 2; off > 0; off >>= 1) {
        __syncthreads();
        if (t < off) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                smn[a][t] = fmin(smn[a][t], smn[a][t + off]);
                smx[a][t] = fmax(smx[a][t], smx[a][t + off]);
            }
        }
    }
    if (t != 0) return;
    const double d[3] = {d0, d1, d2};
    int err = 0;
    double total = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double na = floor(__ddiv_rn(__dsub_rn(smx[a][0], smn[a][0]), d[a])) + 1.0;
        if (!(na >= 1.0 && na < 4.0e18)) err = 1;
        total *= na;
        g->lo[a] = smn[a][0];
        g->d[a] = d[a];
        g->dims[a] = err ? 1 : (long long)na;
    }
    if (!(total < 4.0e18) || !(total * (double)n < 4.0e18)) err = 1;
    if (err) g->dims[0] = g->dims[1] = g->dims[2] = 1;
    g->nvox = g->dims[0] * g->dims[1] * g->dims[2];
    g->nl = 0;
    g->err = err;
    g->sticky |= err;
}

__global__ void k_vox_keys(const double* __restrict__ pos, int64_t n, int64_t P, const VoxGrid* __restrict__ g,
                           long long* __restrict__ keys) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P) return;
    if (t >= n) {
        keys[t] = LLONG_MAX;
        return;
    }
    if (g->err) {  // everything in voxel 0: sizes stay in range, the caller reports the error
        keys[t] = t;
        return;
    }
    long long c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long ca = (long long)floor(__ddiv_rn(__dsub_rn(pos[3 * t + a], g->lo[a]), g->d[a]));
        ca = ca < g->dims[a] - 1 ? ca : g->dims[a] - 1;
        c[a] = ca > 0 ? ca : 0;
    }
    const long long v = (c[2] * g->dims[1] + c[1]) * g->dims[0] + c[0];
    keys[t] = v * n + t;
}

__device__ __forceinline__ void cswap(long long* s, int i, int l, bool asc) {
    const long long a = s[i], b = s[l];
    if ((a > b) == asc) {
        s[i] = b;
        s[l] = a;
    }
}

// Sort each kSortTile chunk (stages k = 2 .. kSortTile of the bitonic network; the
// direction of a pair follows the global index, so later merges see bitonic runs).
__global__ void __launch_bounds__(kSortTile / 2) k_bitonic_presort(long long* __restrict__ keys) {
    __shared__ long long s[kSortTile];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int t = threadIdx.x;
    s[t] = keys[base + t];
    s[t + kSortTile / 2] = keys[base + t + kSortTile / 2];
    for (int k = 2; k <= kSortTile; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
            cswap(s, i, i + j, ((base + i) & k) == 0);
        }
    }
    __syncthreads();
    keys[base + t] = s[t];
    keys[base + t + kSortTile / 2] = s[t + kSortTile / 2];
}

// One stage (k, j) with j >= kSortTile, pairs across chunks.
__global__ void k_bitonic_global(long long* __restrict__ keys, int64_t half, int64_t k, int64_t j) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half) return;
    const int64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
    const int64_t l = i + j;
    const bool asc = (i & k) == 0;
    const long long a = keys[i], b = keys[l];
    if ((a > b) == asc) {
        keys[i] = b;
        keys[l] = a;
    }
}

// The stages j = kSortTile/2 .. 1 of merge k, inside each chunk.
__global__ void __launch_bounds__(kSortTile / 2) k_bitonic_merge(long long* __restrict__ keys, int64_t k) {
    __shared__ long long s[kSortTile];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int t = threadIdx.x;
    s[t] = keys[base + t];
    s[t + kSortTile / 2] = keys[base + t + kSortTile / 2];
    const bool asc = (base & k) == 0;  // one direction per chunk when k > kSortTile
    for (int j = kSortTile / 2; j > 0; j >>= 1) {
        __syncthreads();
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        cswap(s, i, i + j, asc);
    }
    __syncthreads();
    keys[base + t] = s[t];
    keys[base + t + kSortTile / 2] = s[t + kSortTile / 2];
}

__global__ void k_heads(const long long* __restrict__ keys, int64_t n, int* __restrict__ flags) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    flags[t] = (t == 0 || keys[t] / n != keys[t - 1] / n) ? 1 : 0;
}

// Exclusive scan of one value per thread over a block of kScanThreads threads.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
    __shared__ int ws[kScanThreads / 32];
    __shared__ int tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int w = ws[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        ws[lane] = wi - w;
        if (lane == 31) tot = wi;
    }
    __syncthreads();
    const int r = x - v + ws[warp];
    *total = tot;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_block(int* __restrict__ data, int64_t n,
                                                             int* __restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? data[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_excl_scan(sum, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int* __restrict__ bsum, int64_t nb,
                                                           VoxGrid* __restrict__ g) {
    const int64_t per = (nb + kScanThreads - 1) / kScanThreads;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    int sum = 0;
    for (int64_t b = b0; b < b0 + per && b < nb; ++b) sum += bsum[b];
    int total;
    int run = block_excl_scan(sum, &total);
    for (int64_t b = b0; b < b0 + per && b < nb; ++b) {
        const int v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    if (threadIdx.x == 0) g->nl = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int* __restrict__ data, int64_t n,
                                                           const int* __restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    const int off = bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) data[base + k] += off;
}

__global__ void k_make_lines(const long long* __restrict__ keys, int64_t n, const double* __restrict__ q,
                             const int* __restrict__ line_of, const VoxGrid* __restrict__ g,
                             LineRec* __restrict__ lines, LineF* __restrict__ linesf, long long* __restrict__ line_vox) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long v = keys[j] / n;
    if (j > 0 && keys[j - 1] / n == v) return;
    double Q = 0.0;
    for (int64_t t = j; t < n && keys[t] / n == v; ++t) Q = __dadd_rn(Q, q[keys[t] % n]);
    const long long i = v % g->dims[0], jj = (v / g->dims[0]) % g->dims[1], k = v / (g->dims[0] * g->dims[1]);
    const double ax = __dadd_rn(g->lo[0], __dmul_rn(__dadd_rn((double)i, 0.5), g->d[0]));
    const double ay = __dadd_rn(g->lo[1], __dmul_rn(__dadd_rn((double)jj, 0.5), g->d[1]));
    const double az = __dadd_rn(g->lo[2], __dmul_rn((double)k, g->d[2]));
    const double dz = g->d[2];
    const double lam = __ddiv_rn(Q, dz);
    const int L = line_of[j];
    LineRec r;
    r.a[0] = ax;
    r.a[1] = ay;
    r.a[2] = az;
    r.lam = lam;
    r.u[0] = 0.0;
    r.u[1] = 0.0;
    r.u[2] = 1.0;
    r.len = dz;
    lines[L] = r;
    line_vox[L] = v;
    const double mz = __dadd_rn(az, __dmul_rn(0.5, dz));
    const float hx = (float)ax, hy = (float)ay, hz = (float)mz;
    LineF f;
    f.mh = make_float4(hx, hy, hz, (float)(0.5 * dz));
    f.ml = make_float4((float)(ax - (double)hx), (float)(ay - (double)hy), (float)(mz - (double)hz), (float)lam);
    f.u = make_float4(0.f, 0.f, 1.f, 0.f);
    linesf[L] = f;
}

// ------------------------------------------------------------------ line-charge sums

__device__ __forceinline__ void line_pair_f64(const LineRec& L, double px, double py, double pz, double s2,
                                              double& ph, double& ex, double& ey, double& ez) {
    const double wx = px - L.a[0], wy = py - L.a[1], wz = pz - L.a[2];
    const double x = wx * L.u[0] + wy * L.u[1] + wz * L.u[2];
    const double qx = wx - x * L.u[0], qy = wy - x * L.u[1], qz = wz - x * L.u[2];
    const double rho2 = qx * qx + qy * qy + qz * qz + s2;
    const double s1 = -x, s2e = L.len - x;
    const double R1 = sqrt(s1 * s1 + rho2), R2 = sqrt(s2e * s2e + rho2);
    double I, cp;
    if (s1 >= 0.0 || s2e <= 0.0) {
        // the target lies beyond one end of the line's span
        I = (s1 >= 0.0) ? log((s2e + R2) / (s1 + R1)) : log((R1 - s1) / (R2 - s2e));
        cp = (s2e - s1) * (s2e + s1) / (R1 * R2 * (s2e * R1 + s1 * R2));
    } else {
        // beside the span: s1 + R1 = rho^2 / (R1 - s1)
        I = log((s2e + R2) * (R1 - s1) / rho2);
        cp = (s2e / R2 - s1 / R1) / rho2;
    }
    const double cu = -L.len * (s1 + s2e) / (R1 * R2 * (R1 + R2));
    ph += L.lam * I;
    ex += L.lam * (cu * L.u[0] + cp * qx);
    ey += L.lam * (cu * L.u[1] + cp * qy);
    ez += L.lam * (cu * L.u[2] + cp * qz);
}

__device__ __forceinline__ int64_t target_index(const long long* perm, int64_t perm_div, int64_t t) {
    return perm ? (int64_t)(perm[t] % perm_div) : t;
}

__device__ __forceinline__ void store_result(int64_t p, int accumulate, double ke, double ph, double ex, double ey,
                                             double ez, double* __restrict__ phi, double* __restrict__ E) {
    if (accumulate) {
        if (phi) phi[p] += ke * ph;
        if (E) {
            E[3 * p] += ke * ex;
            E[3 * p + 1] += ke * ey;
            E[3 * p + 2] += ke * ez;
        }
    } else {
        if (phi) phi[p] = ke * ph;
        if (E) {
            E[3 * p] = ke * ex;
            E[3 * p + 1] = ke * ey;
            E[3 * p + 2] = ke * ez;
        }
    }
}

__global__ void __launch_bounds__(kLT) k_line_f64(const LineRec* __restrict__ lines, const VoxGrid* __restrict__ g,
                                                  const double* __restrict__ tgt, const long long* __restrict__ perm,
                                                  int64_t perm_div, int64_t nt, double s2, double ke, int accumulate,
                                                  double* __restrict__ phi, double* __restrict__ E) {
    __shared__ LineRec sl[kLT];
    const int64_t nl = g->nl;
    const int64_t t = (int64_t)blockIdx.x * kLT + threadIdx.x;
    const bool active = t < nt;
    const int64_t p = active ? target_index(perm, perm_div, t) : 0;
    double px = 0, py = 0, pz = 0;
    if (active) {
        px = tgt[3 * p];
        py = tgt[3 * p + 1];
        pz = tgt[3 * p + 2];
    }
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int64_t base = 0; base < nl; base += kLT) {
        __syncthreads();
        if (base + threadIdx.x < nl) sl[threadIdx.x] = lines[base + threadIdx.x];
        __syncthreads();
        const int cnt = (int)min((int64_t)kLT, nl - base);
        for (int k = 0; k < cnt; ++k) line_pair_f64(sl[k], px, py, pz, s2, ph, ex, ey, ez);
    }
    if (active) store_result(p, accumulate, ke, ph, ex, ey, ez, phi, E);
}

// Gauss-Legendre nodes on [-1, 1] for the 2, 3, 4 and 6 node rules.
struct LineRules {
    float x[4][6], w[4][6];
};

template <int N>
__device__ __forceinline__ void line_nodes(const float* __restrict__ x, const float* __restrict__ w, float dx,
                                           float dy, float dz, const LineF& L, float s2, float& ph, float& ex,
                                           float& ey, float& ez) {
    const float h = L.mh.w, hl = h * L.ml.w;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float o = x[k] * h;
        const float rx = fmaf(-o, L.u.x, dx), ry = fmaf(-o, L.u.y, dy), rz = fmaf(-o, L.u.z, dz);
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, s2)));
        const float ri = rsqrtf(r2);
        const float wr = w[k] * hl * ri;
        const float wr3 = wr * ri * ri;
        ph += wr;
        ex = fmaf(wr3, rx, ex);
        ey = fmaf(wr3, ry, ey);
        ez = fmaf(wr3, rz, ez);
    }
}

// FP32 squared distance between a target (two floats per coordinate) and a line's
// midpoint, and the near threshold (3 half lengths)^2: pinned operation sequences, so the
// far and near kernels take the same decision for every pair.
__device__ __forceinline__ float line_d2(float thx, float thy, float thz, float tlx, float tly, float tlz,
                                         const LineF& L, float& dx, float& dy, float& dz) {
    dx = __fadd_rn(__fsub_rn(thx, L.mh.x), __fsub_rn(tlx, L.ml.x));
    dy = __fadd_rn(__fsub_rn(thy, L.mh.y), __fsub_rn(tly, L.ml.y));
    dz = __fadd_rn(__fsub_rn(thz, L.mh.z), __fsub_rn(tlz, L.ml.z));
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ float line_near2(const LineF& L) { return __fmul_rn(9.f, __fmul_rn(L.mh.w, L.mh.w)); }

__device__ __forceinline__ void split_target(double px, double py, double pz, float& thx, float& thy, float& thz,
                                             float& tlx, float& tly, float& tlz) {
    thx = (float)px;
    thy = (float)py;
    thz = (float)pz;
    tlx = (float)(px - thx);
    tly = (float)(py - thy);
    tlz = (float)(pz - thz);
}

// Far pairs (d >= 3 h): FP32 Gauss-Legendre nodes along the line.  Near pairs are left to
// k_line_near.
__global__ void __launch_bounds__(kLT) k_line_far(const LineF* __restrict__ linesf, const VoxGrid* __restrict__ g,
                                                  const double* __restrict__ tgt, const long long* __restrict__ perm,
                                                  int64_t perm_div, int64_t nt, float s2f, double ke, int accumulate,
                                                  LineRules rules, double* __restrict__ phi, double* __restrict__ E) {
    __shared__ LineF sf[kLT];
    __shared__ float rx[4][6], rw[4][6];
    if (threadIdx.x < 24) {
        const int r = threadIdx.x / 6, k = threadIdx.x % 6;
        rx[r][k] = rules.x[r][k];
        rw[r][k] = rules.w[r][k];
    }
    const int64_t nl = g->nl;
    const int64_t t = (int64_t)blockIdx.x * kLT + threadIdx.x;
    const bool active = t < nt;
    const int64_t p = active ? target_index(perm, perm_div, t) : 0;
    double px = 0, py = 0, pz = 0;
    if (active) {
        px = tgt[3 * p];
        py = tgt[3 * p + 1];
        pz = tgt[3 * p + 2];
    }
    float thx, thy, thz, tlx, tly, tlz;
    split_target(px, py, pz, thx, thy, thz, tlx, tly, tlz);
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int64_t base = 0; base < nl; base += kLT) {
        __syncthreads();
        if (base + threadIdx.x < nl) sf[threadIdx.x] = linesf[base + threadIdx.x];
        __syncthreads();
        const int cnt = (int)min((int64_t)kLT, nl - base);
        for (int sub = 0; sub < cnt; sub += kLFlush) {
            const int m = min(kLFlush, cnt - sub);
            float fph = 0.f, fex = 0.f, fey = 0.f, fez = 0.f;
            for (int k = sub; k < sub + m; ++k) {
                const LineF L = sf[k];
                float dx, dy, dz;
                const float d2 = line_d2(thx, thy, thz, tlx, tly, tlz, L, dx, dy, dz);
                const float h2 = L.mh.w * L.mh.w;
                if (!(d2 >= line_near2(L))) continue;  // k_line_near
                if (d2 >= 9216.f * h2)
                    line_nodes<2>(rx[0], rw[0], dx, dy, dz, L, s2f, fph, fex, fey, fez);
                else if (d2 >= 256.f * h2)
                    line_nodes<3>(rx[1], rw[1], dx, dy, dz, L, s2f, fph, fex, fey, fez);
                else if (d2 >= 64.f * h2)
                    line_nodes<4>(rx[2], rw[2], dx, dy, dz, L, s2f, fph, fex, fey, fez);
                else
                    line_nodes<6>(rx[3], rw[3], dx, dy, dz, L, s2f, fph, fex, fey, fez);
            }
            ph += fph;
            ex += fex;
            ey += fey;
            ez += fez;
        }
    }
    if (active) store_result(p, accumulate, ke, ph, ex, ey, ez, phi, E);
}

// First index in line_vox[lo, hi) (ascending) with line_vox >= v.
__device__ __forceinline__ int64_t lower_bound_vox(const long long* __restrict__ lv, int64_t lo, int64_t hi,
                                                   long long v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (lv[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Near pairs (d < 3 h) in FP64: the candidate lines of a target lie in the voxels whose
// centre is within 3 h (padded by 1e-3 relative and one voxel) of it; every candidate row
// (fixed j, k) is a contiguous range of voxel indices, found by binary search in the sorted
// line_vox.  The decision d < 3 h is the far kernel's FP32 test.  Adds to phi / E.
__global__ void __launch_bounds__(kLT) k_line_near(const LineF* __restrict__ linesf,
                                                   const LineRec* __restrict__ lines,
                                                   const long long* __restrict__ line_vox,
                                                   const VoxGrid* __restrict__ g, const double* __restrict__ tgt,
                                                   const long long* __restrict__ perm, int64_t perm_div, int64_t nt,
                                                   double s2, double ke, double* __restrict__ phi,
                                                   double* __restrict__ E) {
    const int64_t t = (int64_t)blockIdx.x * kLT + threadIdx.x;
    if (t >= nt) return;
    const int64_t nl = g->nl;
    if (nl == 0) return;
    const int64_t p = target_index(perm, perm_div, t);
    const double px = tgt[3 * p], py = tgt[3 * p + 1], pz = tgt[3 * p + 2];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) return;  // no near line (the far sum is NaN)
    float thx, thy, thz, tlx, tly, tlz;
    split_target(px, py, pz, thx, thy, thz, tlx, tly, tlz);
    const double reach = 1.5 * g->d[2] * (1.0 + 1e-3);  // 3 half lengths, padded
    const double P[3] = {px, py, pz};
    long long lo3[3], hi3[3];
    for (int a = 0; a < 3; ++a) {
        // voxel centres: lo + (i + 1/2) d per axis (x, y); midpoints lo + (k + 1/2) dz in z
        const double c0 = (P[a] - reach - g->lo[a]) / g->d[a] - 0.5;
        const double c1 = (P[a] + reach - g->lo[a]) / g->d[a] - 0.5;
        double f0 = floor(c0), f1 = ceil(c1);
        f0 = fmax(f0, 0.0);
        f1 = fmin(f1, (double)(g->dims[a] - 1));
        lo3[a] = (long long)f0;
        hi3[a] = (long long)f1;
        if (f1 < f0) return;
    }
    double ph = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (long long k = lo3[2]; k <= hi3[2]; ++k)
        for (long long j = lo3[1]; j <= hi3[1]; ++j) {
            const long long row = (k * g->dims[1] + j) * g->dims[0];
            int64_t l = lower_bound_vox(line_vox, 0, nl, row + lo3[0]);
            for (; l < nl && line_vox[l] <= row + hi3[0]; ++l) {
                const LineF L = linesf[l];
                float dx, dy, dz;
                const float d2 = line_d2(thx, thy, thz, tlx, tly, tlz, L, dx, dy, dz);
                if (d2 >= line_near2(L)) continue;  // k_line_far
                line_pair_f64(lines[l], px, py, pz, s2, ph, ex, ey, ez);
            }
        }
    if (phi) phi[p] += ke * ph;
    if (E) {
        E[3 * p] += ke * ex;
        E[3 * p + 1] += ke * ey;
        E[3 * p + 2] += ke * ez;
    }
}

LineRules make_rules() {
    LineRules r{};
    const int counts[4] = {2, 3, 4, 6};
    for (int t = 0; t < 4; ++t) {
        double x[6], w[6];
        gauss_legendre01(counts[t], x, w);
        for (int k = 0; k < counts[t]; ++k) {
            r.x[t][k] = (float)(2.0 * x[k] - 1.0);
            r.w[t][k] = (float)(2.0 * w[k]);
        }
    }
    return r;
}

}  // namespace

int64_t vox_pad_len(int64_t n) {
    int64_t P = kSortTile;
    while (P < n) P <<= 1;
    return P;
}

int64_t vox_scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t launch_voxelize(const double* pos, const double* q, int64_t n, const double d[3], const VoxWork& w,
                            cudaStream_t s) {
    if (n <= 0 || n > kVoxMaxPoints) return cudaErrorInvalidValue;
    const int64_t P = vox_pad_len(n);
    const int mmb = (int)std::min<int64_t>(kMMBlocks, (n + kMM - 1) / kMM);
    k_minmax_partial<<<mmb, kMM, 0, s>>>(pos, n, w.partial);
    k_minmax_final<<<1, kMMBlocks, 0, s>>>(w.partial, mmb, n, d[0], d[1], d[2], w.grid);
    k_vox_keys<<<(unsigned)(P / 256), 256, 0, s>>>(pos, n, P, w.grid, w.keys);
    k_bitonic_presort<<<(unsigned)(P / kSortTile), kSortTile / 2, 0, s>>>(w.keys);
    for (int64_t k = 2 * kSortTile; k <= P; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortTile; j >>= 1)
            k_bitonic_global<<<(unsigned)(P / 2 / 256), 256, 0, s>>>(w.keys, P / 2, k, j);
        k_bitonic_merge<<<(unsigned)(P / kSortTile), kSortTile / 2, 0, s>>>(w.keys, k);
    }
    const unsigned nb256 = (unsigned)((n + 255) / 256);
    k_heads<<<nb256, 256, 0, s>>>(w.keys, n, w.flags);
    const int64_t nb = vox_scan_blocks(n);
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, s>>>(w.flags, n, w.bsum);
    k_scan_top<<<1, kScanThreads, 0, s>>>(w.bsum, nb, w.grid);
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(w.flags, n, w.bsum);
    k_make_lines<<<nb256, 256, 0, s>>>(w.keys, n, q, w.flags, w.grid, w.lines, w.linesf, w.line_vox);
    return cudaGetLastError();
}

cudaError_t launch_line_eval(int precision, const VoxWork& w, const double* tgt, const long long* perm,
                             int64_t perm_div, int64_t nt, double soft, int accumulate, double* phi, double* E,
                             cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    const double ke = 1.0 / (4.0 * kPi * kEps0);
    const unsigned blocks = (unsigned)((nt + kLT - 1) / kLT);
    if (precision == NEBEM_FP64) {
        k_line_f64<<<blocks, kLT, 0, s>>>(w.lines, w.grid, tgt, perm, perm_div, nt, soft * soft, ke, accumulate, phi,
                                          E);
    } else {
        static const LineRules rules = make_rules();
        k_line_far<<<blocks, kLT, 0, s>>>(w.linesf, w.grid, tgt, perm, perm_div, nt, (float)(soft * soft), ke,
                                          accumulate, rules, phi, E);
        k_line_near<<<blocks, kLT, 0, s>>>(w.linesf, w.lines, w.line_vox, w.grid, tgt, perm, perm_div, nt,
                                           soft * soft, ke, phi, E);
    }
    return cudaGetLastError();
}

}  // namespace nb
