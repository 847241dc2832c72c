// lu.cu -- dense LU with partial pivoting, triangular solves, residual and refinement
// helpers (Sec. 4.1, Alg. 1: the paper inverts K with an LU factorisation; here the
// factors are kept and applied by forward/back substitution instead of forming K^-1).
//
// Right-looking blocked LU, column-major, lda = n, panel width nb:
//   for each panel [k0, k0+nb):
//     per column j: pivot search (max |a|, lowest row index on ties) -> row swap
//                   inside the panel -> scale the column -> rank-1 update of the panel;
//     apply the panel's swaps to the other columns;
//     U12 = L11^-1 A12  (explicit inverse of the unit-lower nb x nb block, then a GEMM);
//     A22 -= L21 U12    (GEMM).
// Templated on the element type: double (FP64 solves) and float (mixed solves, the
// FP64 iterative refinement lives in the caller).
#include <algorithm>
#include <climits>
#include <vector>

#include "nb_internal.h"

namespace nb {

namespace {

constexpr int kPivBlocks = 256;
constexpr int kPivThreads = 256;

template <typename T>
__global__ void k_pivot_partial(const T* __restrict__ A, int64_t n, int64_t j, double* __restrict__ pval,
                                int64_t* __restrict__ pidx) {
    double best = -1.0;
    int64_t bidx = INT64_MAX;
    for (int64_t i = j + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fabs((double)A[i + j * n]);
        if (v > best || (v == best && i < bidx)) {
            best = v;
            bidx = i;
        }
    }
    __shared__ double sv[kPivThreads];
    __shared__ int64_t si[kPivThreads];
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v = sv[threadIdx.x + s];
            const int64_t ix = si[threadIdx.x + s];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ix < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = ix;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pval[blockIdx.x] = sv[0];
        pidx[blockIdx.x] = si[0];
    }
}

// Final pivot reduction + row swap inside the panel columns [k0, k1).
template <typename T>
__global__ void k_pivot_swap(T* __restrict__ A, int64_t n, int64_t j, int64_t k0, int64_t k1,
                             const double* __restrict__ pval, const int64_t* __restrict__ pidx, int nparts,
                             int32_t* __restrict__ piv, int* __restrict__ info) {
    __shared__ double sv[kPivThreads];
    __shared__ int64_t si[kPivThreads];
    double best = -1.0;
    int64_t bidx = INT64_MAX;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const double v = pval[b];
        const int64_t ix = pidx[b];
        if (v > best || (v == best && ix < bidx)) {
            best = v;
            bidx = ix;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v = sv[threadIdx.x + s];
            const int64_t ix = si[threadIdx.x + s];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ix < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = ix;
            }
        }
        __syncthreads();
    }
    // a column without a valid maximum (all NaN) keeps its own row: the factorisation is
    // then reported singular through info and no out-of-range row is ever swapped
    const int64_t p = (si[0] >= j && si[0] < n) ? si[0] : j;
    if (threadIdx.x == 0) {
        piv[j] = (int32_t)p;
        if (!(sv[0] > 0.0) && *info == 0) *info = (int)(j + 1);
    }
    if (p != j) {
        for (int64_t c = k0 + threadIdx.x; c < k1; c += blockDim.x) {
            const T a = A[j + c * n];
            A[j + c * n] = A[p + c * n];
            A[p + c * n] = a;
        }
    }
}

// Scale column j below the diagonal and apply the rank-1 update to panel columns (j, k1).
template <typename T>
__global__ void k_scale_update(T* __restrict__ A, int64_t n, int64_t j, int64_t k1) {
    extern __shared__ unsigned char smem_raw[];
    T* urow = reinterpret_cast<T*>(smem_raw);
    const int w = (int)(k1 - j - 1);
    for (int c = threadIdx.x; c < w; c += blockDim.x) urow[c] = A[j + (j + 1 + c) * n];
    __syncthreads();
    const T d = A[j + j * n];
    if (d == (T)0) return;
    const T inv = (T)1 / d;
    for (int64_t i = j + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T l = A[i + j * n] * inv;
        A[i + j * n] = l;
        for (int c = 0; c < w; ++c) A[i + (j + 1 + c) * n] -= l * urow[c];
    }
}

// One launch per panel column j, fusing what would otherwise be three launches:
//   (a) for j > k0: scale column j-1 below its diagonal and apply its rank-1 update to
//       the panel columns (j-1, k1), each thread for its own rows i >= j;
//   (b) the partial pivot search of column j over the same rows (so a thread reads only
//       values it has just updated itself);
//   (c) the last block to finish (an atomic ticket, no waiting) reduces the partial maxima,
//       records the pivot and swaps rows j and p inside the panel columns.
// With do_pivot = 0 only (a) runs (the launch after the panel's last column).  The
// per-element arithmetic is that of the three separate steps, in the same order.
template <typename T>
__global__ void __launch_bounds__(kPivThreads, 2) k_panel_col(T* __restrict__ A, int64_t n, int64_t j, int64_t k0,
                                                            int64_t k1, int do_pivot, double* __restrict__ pval,
                                                            int64_t* __restrict__ pidx, int* __restrict__ ticket,
                                                            int32_t* __restrict__ piv, int* __restrict__ info) {
    __shared__ T urow[64];
    __shared__ double sv[kPivThreads];
    __shared__ int64_t si[kPivThreads];
    __shared__ bool last;
    const bool update = j > k0;
    const int64_t jm = j - 1;
    const int w = update ? (int)(k1 - j) : 0;  // columns (j-1, k1)
    T inv = (T)0;
    bool ok = true;
    if (update) {
        for (int c = threadIdx.x; c < w; c += blockDim.x) urow[c] = A[jm + (j + c) * n];
        const T d = A[jm + jm * n];
        ok = d != (T)0;
        inv = ok ? (T)1 / d : (T)0;
    }
    __syncthreads();
    double best = -1.0;
    int64_t bidx = INT64_MAX;
    for (int64_t i = j + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T aj;  // A[i, j] after the update
        if (update && ok) {
            const T l = A[i + jm * n] * inv;
            A[i + jm * n] = l;
            // the row's panel values in batches of 16 independent loads (one memory round
            // trip per batch instead of one per column), then the updates
            T* row = A + i + j * n;
            aj = (T)0;
            for (int c0 = 0; c0 < w; c0 += 16) {
                T v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < w) v[q] = row[(int64_t)(c0 + q) * n];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < w) {
                        v[q] -= l * urow[c0 + q];
                        row[(int64_t)(c0 + q) * n] = v[q];
                    }
                if (c0 == 0) aj = v[0];
            }
        } else {
            aj = A[i + j * n];
        }
        if (do_pivot) {
            const double v = fabs((double)aj);
            if (v > best || (v == best && i < bidx)) {
                best = v;
                bidx = i;
            }
        }
    }
    if (!do_pivot) return;
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double v = sv[threadIdx.x + st];
            const int64_t ix = si[threadIdx.x + st];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ix < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = ix;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pval[blockIdx.x] = sv[0];
        pidx[blockIdx.x] = si[0];
        __threadfence();
        last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // final reduction over the blocks' partial maxima (lowest row index on ties)
    best = -1.0;
    bidx = INT64_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double v = __ldcg(pval + b);
        const int64_t ix = __ldcg(pidx + b);
        if (v > best || (v == best && ix < bidx)) {
            best = v;
            bidx = ix;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const double v = sv[threadIdx.x + st];
            const int64_t ix = si[threadIdx.x + st];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ix < si[threadIdx.x])) {
                sv[threadIdx.x] = v;
                si[threadIdx.x] = ix;
            }
        }
        __syncthreads();
    }
    const int64_t p = (si[0] >= j && si[0] < n) ? si[0] : j;
    if (threadIdx.x == 0) {
        piv[j] = (int32_t)p;
        if (!(sv[0] > 0.0) && *info == 0) *info = (int)(j + 1);
        *ticket = 0;
    }
    if (p != j) {
        for (int64_t c = k0 + threadIdx.x; c < k1; c += blockDim.x) {
            const T a = __ldcg(A + j + c * n);
            A[j + c * n] = __ldcg(A + p + c * n);
            A[p + c * n] = a;
        }
    }
}

// The whole panel of the FP32 factorisation in one cooperative launch (all CTAs resident).
// CTA b holds rows [k0 + b R, k0 + (b+1) R) of the panel columns in shared memory
// (column-major, R rows); per column j of the panel:
//   (a) scale column j-1 by the previous pivot and apply its rank-1 update to the rows
//       below it (the same per-element arithmetic as k_panel_col);
//   (b) each CTA finds its largest |a_ij| (lowest row on ties) and publishes it with its
//       row (candidate slot of parity j & 1); the CTA holding row j publishes row j;
//   (c) one grid barrier; every CTA reduces the candidates to the pivot p, reads the
//       pivot row, and the holders of rows j and p swap them in shared memory.
// The candidate slots alternate between two parities: a CTA writes slot j+1 only after it
// has passed barrier j, by which time every CTA has finished reading slot j-1.  The grid
// barrier (a cumulative arrival counter) waits a bounded number of polls; on giving up a
// CTA records *err and leaves the panel (the host reports a timeout).
constexpr int kCoopThreads = 256;
constexpr int kCoopMaxG = 1024;
constexpr long long kCoopSpinLimit = 1ll << 22;

struct CoopScratch {
    float cval[2][kCoopMaxG];
    int cidx[2][kCoopMaxG];
    float cand[2][kCoopMaxG][64];
    float srow[2][64];
    unsigned int bar[4];  // bar[0]: grid-barrier arrivals of the factorisation
    int err;
};

__device__ __forceinline__ unsigned int ld_acquire_u(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_i(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// every CTA of the grid arrives; false if the wait gave up.  bar[0] counts all arrivals
// of the factorisation (never reset): each CTA adds 1 with acquire-release semantics and
// waits until the count reaches `target` (this barrier's total), so one atomic and one
// polled load make the barrier, and the last arrival publishes everyone's writes (the
// acquire load that sees the final count synchronises with every add before it).
__device__ bool coop_barrier(CoopScratch* cs, unsigned int target, bool* s_flag, long long limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int v;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(&cs->bar[0]) : "memory");
        bool ok = true;
        if (v + 1u < target) {
            long long spins = 0;
            while (ld_acquire_u(&cs->bar[0]) < target) {
                // give up after the poll limit, or at once when another CTA has given up
                if (++spins > limit || ((spins & 1023) == 0 && ld_acquire_i(&cs->err))) {
                    ok = false;
                    break;
                }
                __nanosleep(20);
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag;
}

__global__ void __launch_bounds__(kCoopThreads, 1)
    k_panel_coop(float* __restrict__ A, int64_t n, int64_t k0, int64_t k1, int R, int32_t* __restrict__ piv,
                 int* __restrict__ info, int* __restrict__ tmo, CoopScratch* cs, unsigned int bar_base,
                 long long limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (ld_acquire_i(&cs->err)) return;  // an earlier panel gave up: leave the matrix as it is
    const int w = (int)(k1 - k0);
    float* S = reinterpret_cast<float*>(smem_raw);  // R x w, column-major
    __shared__ float prow[64];
    __shared__ bool s_flag;
    const int G = gridDim.x, b = blockIdx.x;
    const int64_t rb0 = k0 + (int64_t)b * R;
    const int nr = (int)max((int64_t)0, min((int64_t)R, n - rb0));
    for (int idx = threadIdx.x; idx < nr * w; idx += kCoopThreads) {
        const int r = idx % nr, c = idx / nr;
        S[c * R + r] = A[(rb0 + r) + (k0 + c) * n];
    }
    __syncthreads();
    bool ok_piv = true;  // the previous pivot was nonzero
    __shared__ float wv[kCoopThreads / 32];
    __shared__ int wi[kCoopThreads / 32];
    // (best, index) of the block: warp shuffles, then every thread over the warps' results;
    // the largest value with the lowest index on ties, so the order of the reduction does
    // not matter.  Magnitudes of FP32 values compare exactly in FP32 (no FP64 pipe), row
    // indices fit in 32 bits (n < 2^31).  Every thread returns with the result in (v, ix).
    auto block_best = [&](float& v, int& ix) {
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, ix, o);
            if (v2 > v || (v2 == v && i2 < ix)) {
                v = v2;
                ix = i2;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            wv[threadIdx.x >> 5] = v;
            wi[threadIdx.x >> 5] = ix;
        }
        __syncthreads();
        v = wv[0];
        ix = wi[0];
        for (int q = 1; q < kCoopThreads / 32; ++q)
            if (wv[q] > v || (wv[q] == v && wi[q] < ix)) {
                v = wv[q];
                ix = wi[q];
            }
        __syncthreads();  // wv / wi are rewritten by the next reduction
    };
    for (int jj = 0; jj < w; ++jj) {
        const int64_t j = k0 + jj;
        const int par = jj & 1;
        // (a) + (b): column jj-1 scaled and its rank-1 update applied to this thread's rows
        // below it, then this thread's candidate for column jj from the same rows
        float best = -1.0f;
        int bidx = INT_MAX;
        const float inv = (jj > 0 && ok_piv) ? 1.0f / prow[jj - 1] : 0.f;
        for (int r = threadIdx.x; r < nr; r += kCoopThreads) {
            if (rb0 + r < j) continue;
            if (jj > 0 && ok_piv) {
                const float l = S[(jj - 1) * R + r] * inv;
                S[(jj - 1) * R + r] = l;
                for (int c = jj; c < w; ++c) S[c * R + r] -= l * prow[c];
            }
            const float v = fabsf(S[jj * R + r]);
            if (v > best || (v == best && (int)(rb0 + r) < bidx)) {
                best = v;
                bidx = (int)(rb0 + r);
            }
        }
        block_best(best, bidx);
        const int mine = bidx;
        if (threadIdx.x == 0) {
            cs->cval[par][b] = best;
            cs->cidx[par][b] = mine;
        }
        if (threadIdx.x < w) {
            cs->cand[par][b][threadIdx.x] = (mine != INT_MAX) ? S[threadIdx.x * R + (int)(mine - rb0)] : 0.f;
            if (j >= rb0 && j < rb0 + nr) cs->srow[par][threadIdx.x] = S[threadIdx.x * R + (int)(j - rb0)];
        }
        if (!coop_barrier(cs, bar_base + (unsigned)(jj + 1) * (unsigned)G, &s_flag, limit)) {
            if (threadIdx.x == 0) {
                atomicExch(&cs->err, 1);
                atomicExch(tmo, 1);
            }
            return;
        }
        // (c) the pivot: largest |a| over the candidates, lowest row on ties
        best = -1.0f;
        bidx = INT_MAX;
        for (int q = threadIdx.x; q < G; q += kCoopThreads) {
            const float v = __ldcg(&cs->cval[par][q]);
            const int ix = __ldcg(&cs->cidx[par][q]);
            if (v > best || (v == best && ix < bidx)) {
                best = v;
                bidx = ix;
            }
        }
        block_best(best, bidx);
        const int64_t p = ((int64_t)bidx >= j && (int64_t)bidx < n) ? (int64_t)bidx : j;
        const int owner = (int)((p - k0) / R);
        if (threadIdx.x < w) prow[threadIdx.x] = __ldcg(&cs->cand[par][owner][threadIdx.x]);
        if (b == 0 && threadIdx.x == 0) {
            piv[j] = (int32_t)p;
            if (!(best > 0.0f) && *info == 0) *info = (int)(j + 1);
        }
        __syncthreads();
        ok_piv = prow[jj] != 0.f;  // the scaling below is skipped for a zero pivot, as in k_panel_col
        if (threadIdx.x < w) {
            if (j >= rb0 && j < rb0 + nr) S[threadIdx.x * R + (int)(j - rb0)] = prow[threadIdx.x];
            if (p != j && p >= rb0 && p < rb0 + nr)
                S[threadIdx.x * R + (int)(p - rb0)] = __ldcg(&cs->srow[par][threadIdx.x]);
        }
        __syncthreads();
    }
    // scale the last panel column below the panel
    if (ok_piv) {
        const float inv = 1.0f / prow[w - 1];
        for (int r = threadIdx.x; r < nr; r += kCoopThreads)
            if (rb0 + r >= k1) S[(w - 1) * R + r] *= inv;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * w; idx += kCoopThreads) {
        const int r = idx % nr, c = idx / nr;
        A[(rb0 + r) + (k0 + c) * n] = S[c * R + r];
    }
}

// Apply the row swaps of panel rows [k0, k1) to columns outside the panel.
// The row swaps of panel rows [k0, k1) (LAPACK order: row r with piv[r]) composed into one
// permutation of the rows they touch (at most 2 (k1 - k0)): after it, row dst[i] holds what
// row src[i] held before; *cnt = number of moved rows.  One warp: the touched rows are the
// panel rows (slot r - k0) and the distinct pivot rows below the panel (found by a
// warp-wide search of the list so far).  A pivot outside [r, n) is a row no panel wrote (its
// panel gave up a bounded wait) and is skipped, as in the swaps themselves.
constexpr int kSwapMax = 128;

__global__ void __launch_bounds__(32) k_swap_perm(const int32_t* __restrict__ piv, int64_t n, int64_t k0, int64_t k1,
                                                  int32_t* __restrict__ perm) {
    __shared__ int64_t row_of[kSwapMax];  // slot -> row
    __shared__ int32_t content[kSwapMax]; // slot -> slot whose original row is there now
    __shared__ int32_t pv[kSwapMax / 2];  // the panel's pivots
    __shared__ int n_slots;
    const int lane = threadIdx.x;
    const int w = (int)(k1 - k0);
    for (int q = lane; q < w; q += 32) pv[q] = piv[k0 + q];
    for (int s = lane; s < kSwapMax; s += 32) {
        row_of[s] = s < w ? k0 + s : -1;
        content[s] = s;
    }
    if (lane == 0) n_slots = w;
    __syncwarp();
    for (int64_t r = k0; r < k1; ++r) {
        const int64_t p = pv[r - k0];
        if (!(p != r && p > r && p < n)) continue;
        int sp;
        if (p < k1) {
            sp = (int)(p - k0);
        } else {
            const int ns = n_slots;
            int found = -1;
            for (int base = w; base < ns && found < 0; base += 32) {
                const int s = base + lane;
                const unsigned hit = __ballot_sync(0xffffffffu, s < ns && row_of[s] == p);
                if (hit) found = base + __ffs(hit) - 1;
            }
            if (found < 0) {
                found = ns;
                if (lane == 0) {
                    row_of[ns] = p;
                    n_slots = ns + 1;
                }
            }
            sp = found;
        }
        __syncwarp();
        if (lane == 0) {
            const int sr = (int)(r - k0);
            const int t = content[sr];
            content[sr] = content[sp];
            content[sp] = t;
        }
        __syncwarp();
    }
    // moved rows: (dst, src) pairs after the count
    if (lane == 0) {
        int c = 0;
        for (int s = 0; s < n_slots; ++s)
            if (content[s] != s) {
                perm[1 + 2 * c] = (int32_t)row_of[s];
                perm[2 + 2 * c] = (int32_t)row_of[content[s]];
                ++c;
            }
        perm[0] = c;
    }
}

// The composed swaps applied to every column outside the panel: each thread loads all the
// moved values of its column (independent loads, staged in shared memory), then stores
// them; the result equals the swaps applied one after the other.
constexpr int kSwapThreads = 64;

template <typename T>
__global__ void __launch_bounds__(kSwapThreads) k_laswp(T* __restrict__ A, int64_t n, int64_t k0, int64_t k1,
                                                        const int32_t* __restrict__ perm) {
    extern __shared__ __align__(16) unsigned char swap_sm[];
    T* vals = reinterpret_cast<T*>(swap_sm);  // [kSwapMax][kSwapThreads]
    const int cnt = perm[0];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || (c >= k0 && c < k1)) return;
    T* col = A + c * n;
    // loads in batches of 16 held in registers, so that they are in flight together
    for (int i0 = 0; i0 < cnt; i0 += 16) {
        T v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (i0 + q < cnt) v[q] = col[perm[2 + 2 * (i0 + q)]];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (i0 + q < cnt) vals[(i0 + q) * kSwapThreads + threadIdx.x] = v[q];
    }
    for (int i = 0; i < cnt; ++i) col[perm[1 + 2 * i]] = vals[i * kSwapThreads + threadIdx.x];
}

// Inverse of the unit-lower nb x nb diagonal block at (k0, k0) into W (nb x nb, ld nb):
// X = I, then for q = 0 .. nb-2 (row q of X is final) X[r][c] -= L[r][q] X[q][c] for
// r > q, c <= q -- forward substitution of all columns at once, one block barrier per q,
// L and X in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_trtri_unit_lower(const T* __restrict__ A, int64_t n, int64_t k0, int nb,
                                                          T* __restrict__ W) {
    extern __shared__ unsigned char smem_raw[];
    const int ld = nb + 1;
    T* L = reinterpret_cast<T*>(smem_raw);  // nb x (nb+1)
    T* X = L + nb * ld;                       // nb x (nb+1)
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx % nb, c = idx / nb;
        L[r + c * ld] = A[(k0 + r) + (k0 + c) * n];
        X[r + c * ld] = (r == c) ? (T)1 : (T)0;
    }
    __syncthreads();
    for (int q = 0; q + 1 < nb; ++q) {
        const int rows = nb - 1 - q;
        for (int idx = threadIdx.x; idx < rows * (q + 1); idx += blockDim.x) {
            const int r = q + 1 + idx % rows, c = idx / rows;
            X[r + c * ld] -= L[r + q * ld] * X[q + c * ld];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx % nb, c = idx / nb;
        W[r + (int64_t)c * nb] = X[r + c * ld];
    }
}

// C = alpha * A * B + beta * C; column-major, M x N x K; 64 x 64 tiles, 256 threads, 4x4
// register tile per thread.
// U12 of a block row: X = L^-1 A[K0 : K0 + 64 nbk, c0 : c1] for the unit-lower L of nbk
// diagonal 64-blocks at (K0, K0), by block forward substitution
//   X_i = Linv_i (A_i - sum_{j < i} L_ij X_j),
// with Linv_i (nbk blocks of 64 x 64, ld 64) from k_trtri_unit_lower and L_ij read from A.
// One CTA per kTrsmCols columns holds its tile of the block row in shared memory (all nbk
// blocks), staging one 64 x 64 block of L (or Linv) at a time; thread t owns row t % 64 and
// columns 8 (t / 64) .. + 7 of the current 64-row block.  Dynamic shared memory:
// trsm_block_smem<T>(nbk).
constexpr int kTrsmCols = 32;

template <typename T>
__host__ __device__ constexpr size_t trsm_block_smem(int nbk) {
    return sizeof(T) * ((size_t)64 * nbk * (kTrsmCols + 1) + (size_t)64 * 65);
}

template <typename T>
__global__ void __launch_bounds__(256) k_trsm_block(T* __restrict__ A, int64_t n, int64_t K0, int nbk,
                                                    const T* __restrict__ Linv, int64_t c0, int64_t c1) {
    extern __shared__ __align__(16) unsigned char trsm_blk_sm[];
    T(*X)[kTrsmCols + 1] = reinterpret_cast<T(*)[kTrsmCols + 1]>(trsm_blk_sm);
    T(*L)[65] = reinterpret_cast<T(*)[65]>(trsm_blk_sm + sizeof(T) * 64 * nbk * (kTrsmCols + 1));
    const int64_t cb = c0 + (int64_t)blockIdx.x * kTrsmCols;
    const int wc = (int)min((int64_t)kTrsmCols, c1 - cb);
    const int rows = 64 * nbk;
    const int r = threadIdx.x % 64, g = threadIdx.x / 64;
    for (int idx = threadIdx.x; idx < rows * kTrsmCols; idx += 256) {
        const int rr = idx % rows, cc = idx / rows;
        X[rr][cc] = cc < wc ? A[(K0 + rr) + (cb + cc) * n] : (T)0;
    }
    T acc[8];
    for (int i = 0; i < nbk; ++i) {
        // X_i -= L_ij X_j, j < i
        for (int j = 0; j < i; ++j) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
                const int rr = idx % 64, q = idx / 64;
                L[rr][q] = A[(K0 + 64 * i + rr) + (K0 + 64 * j + q) * n];
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = (T)0;
            for (int q = 0; q < 64; ++q) {
                const T l = L[r][q];
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = fma(l, X[64 * j + q][8 * g + c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) X[64 * i + r][8 * g + c] -= acc[c];
        }
        // X_i = Linv_i X_i
        __syncthreads();
        for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
            const int rr = idx % 64, q = idx / 64;
            L[rr][q] = Linv[(size_t)i * 64 * 64 + rr + q * 64];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (T)0;
        for (int q = 0; q < 64; ++q) {
            const T l = L[r][q];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = fma(l, X[64 * i + q][8 * g + c], acc[c]);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 8; ++c) X[64 * i + r][8 * g + c] = acc[c];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * kTrsmCols; idx += 256) {
        const int rr = idx % rows, cc = idx / rows;
        if (cc < wc) A[(K0 + rr) + (cb + cc) * n] = X[rr][cc];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* __restrict__ A,
                                              int64_t lda, const T* __restrict__ B, int64_t ldb, T beta,
                                              T* __restrict__ C, int64_t ldc) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
            const int r = idx % BM, kk = idx / BM;
            const int64_t gr = m0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr + gk * lda] : (T)0;
        }
        for (int idx = threadIdx.x; idx < BN * BK; idx += 256) {
            const int kk = idx % BK, c = idx / BK;
            const int64_t gk = k0 + kk, gc = n0 + c;
            Bs[kk][c] = (gk < K && gc < N) ? B[gk + gc * ldb] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][tx + 16 * q];
                b[q] = Bs[kk][ty + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t gr = m0 + tx + 16 * p, gc = n0 + ty + 16 * q;
            if (gr < M && gc < N) {
                T* c = C + gr + gc * ldc;
                *c = (beta == (T)0) ? alpha * acc[p][q] : fma(alpha, acc[p][q], beta * *c);
            }
        }
}

template <typename T>
__global__ void k_copy_block(const T* __restrict__ W, int64_t ldw, T* __restrict__ A, int64_t lda, int64_t rows,
                             int64_t cols) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * cols) return;
    const int64_t r = t % rows, c = t / rows;
    A[r + c * lda] = W[r + c * ldw];
}

template <typename T>
cudaError_t gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B, int64_t ldb, T beta,
                 T* C, int64_t ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64));
    k_gemm<T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

#define NB_TRY(x)                              \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

constexpr int kSuperPanels = 4;  // panels per super-panel of the two-level FP32 factorisation

// work layout: [0, 4 nb*nb) unit-lower inverses; then nb*n U12 staging;
// then kPivBlocks doubles + kPivBlocks int64 for the pivot search and one int ticket.
template <typename T>
cudaError_t lu_factor(T* A, int64_t n, int32_t* piv, int nb, T* work, int* d_info, void* split, void* coop,
                      cudaStream_t s, long long polls) {
    // d_info[0]: first zero pivot (1-based) or 0; d_info[1]: a bounded wait gave up (the
    // tensor-core update or the cooperative panel's barrier); polls > 0: the barrier's
    // poll limit (default kCoopSpinLimit)
    NB_TRY(cudaMemsetAsync(d_info, 0, 2 * sizeof(int), s));
    T* Linv = work;                                         // kSuperPanels unit-lower inverses
    T* W = work + (size_t)kSuperPanels * nb * nb;
    char* tail = reinterpret_cast<char*>(W + (size_t)nb * n);
    size_t off = ((uintptr_t)tail + 15) & ~(uintptr_t)15;
    double* pval = reinterpret_cast<double*>(off);
    int64_t* pidx = reinterpret_cast<int64_t*>(pval + kPivBlocks);
    int* ticket = reinterpret_cast<int*>(pidx + kPivBlocks);
    int32_t* swap_perm = reinterpret_cast<int32_t*>(ticket + 4);  // 1 + 2 kSwapMax ints
    NB_TRY(cudaMemsetAsync(ticket, 0, sizeof(int), s));
    const int swap_smem = (int)(sizeof(T) * kSwapMax * kSwapThreads);
    NB_TRY(cudaFuncSetAttribute(k_laswp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, swap_smem));
    if (nb > 64) return cudaErrorInvalidValue;  // k_panel_col stages at most 64 row values
    // FP32: the whole panel in one cooperative launch when every CTA's rows fit in shared
    // memory (R rows x 64 columns, R = max(64, rows / SMs)) and all CTAs can be resident
    int gmax = 0;
    CoopScratch* cs = static_cast<CoopScratch*>(coop);
    if constexpr (sizeof(T) == 4) {
        int dev = 0, sms = 0, can = 0;
        if (cs && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&can, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && can) {
            const int g = std::min(kCoopMaxG, sms);
            const int64_t R0 = std::max<int64_t>(64, (n + g - 1) / g);
            const int smem0 = (int)(R0 * 64 * sizeof(float));
            int per_sm = 0;
            if (smem0 <= 200 * 1024 &&
                cudaFuncSetAttribute(k_panel_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem0) ==
                    cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_coop, kCoopThreads, smem0) ==
                    cudaSuccess &&
                per_sm >= 1) {
                gmax = g;
                NB_TRY(cudaMemsetAsync(cs, 0, sizeof(CoopScratch), s));
            }
        }
        cudaGetLastError();  // a refused attribute or query leaves the per-column path
    }
    unsigned int arrivals = 0;  // grid-barrier arrivals of the cooperative panels so far
    // FP32 with the bulk tensor-core path: two-level blocking.  Super-panels of kSuperPanels
    // panels; inside one, each panel's U12 and update stop at the super-panel's last column;
    // after it, the block row's U12 by block forward substitution and one trailing update of
    // depth kSuperPanels * nb, so C is read and written once per super-panel.
    bool super = false;
    if constexpr (sizeof(T) == 4) super = split && nb == 64 && (n % 4) == 0 && n > (int64_t)kSuperPanels * nb;
    const int64_t sp = super ? (int64_t)kSuperPanels * nb : (int64_t)nb;
    auto trsm_rows = [&](int64_t r0, int wr, int64_t c0, int64_t c1) -> cudaError_t {
        // A[r0 : r0 + wr, c0 : c1] = L(r0 block)^-1 A[r0 : r0 + wr, c0 : c1] (unit lower wr x wr)
        const int64_t m = c1 - c0;
        const int tri_smem = (int)(2 * sizeof(T) * wr * (wr + 1));
        NB_TRY(cudaFuncSetAttribute(k_trtri_unit_lower<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, tri_smem));
        k_trtri_unit_lower<T><<<1, 256, tri_smem, s>>>(A, n, r0, wr, Linv);
        NB_TRY(gemm<T>(wr, m, wr, (T)1, Linv, wr, A + r0 + c0 * n, n, (T)0, W, wr, s));
        k_copy_block<T><<<(unsigned)((wr * m + 255) / 256), 256, 0, s>>>(W, wr, A + r0 + c0 * n, n, wr, m);
        return cudaGetLastError();
    };
    auto trsm_block = [&](int64_t r0, int nbk, const T* inv, int64_t c0, int64_t c1) -> cudaError_t {
        const int smem = (int)trsm_block_smem<T>(nbk);
        NB_TRY(cudaFuncSetAttribute(k_trsm_block<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_trsm_block<T><<<(unsigned)((c1 - c0 + kTrsmCols - 1) / kTrsmCols), 256, smem, s>>>(A, n, r0, nbk, inv, c0,
                                                                                            c1);
        return cudaGetLastError();
    };
    for (int64_t K0 = 0; K0 < n; K0 += sp) {
        const int64_t K1 = std::min<int64_t>(n, K0 + sp);
        const int64_t e1 = super ? K1 : n;  // last column (exclusive) the panels' updates reach
        for (int64_t k0 = K0; k0 < K1; k0 += nb) {
            const int64_t k1 = std::min<int64_t>(n, k0 + nb);
            const int w = (int)(k1 - k0);
            if (gmax > 0) {
                const int64_t rows = n - k0;
                const int R = (int)std::max<int64_t>(64, (rows + gmax - 1) / gmax);
                const int G = (int)((rows + R - 1) / R);
                float* Af = reinterpret_cast<float*>(A);
                int64_t nn = n, kk0 = k0, kk1 = k1;
                int RR = R;
                int* tmo = d_info + 1;
                unsigned int base = arrivals;
                long long lim = polls > 0 ? polls : kCoopSpinLimit;
                void* args[] = {&Af, &nn, &kk0, &kk1, &RR, &piv, &d_info, &tmo, &cs, &base, &lim};
                NB_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_coop, dim3((unsigned)G), dim3(kCoopThreads),
                                                   args, (size_t)R * w * sizeof(float), s));
                arrivals += (unsigned int)G * (unsigned int)w;
            } else {
                // columns k0..k1-1: update by the previous column + pivot of this one; then the
                // last column's scaling of the rows below the panel
                for (int64_t j = k0; j <= k1; ++j) {
                    if (j == n) break;
                    const int64_t rows = n - j;
                    const int pb = (int)std::min<int64_t>(kPivBlocks, (rows + kPivThreads - 1) / kPivThreads);
                    k_panel_col<T><<<pb, kPivThreads, 0, s>>>(A, n, j, k0, k1, j < k1 ? 1 : 0, pval, pidx, ticket,
                                                              piv, d_info);
                }
            }
            NB_TRY(cudaGetLastError());
            k_swap_perm<<<1, 32, 0, s>>>(piv, n, k0, k1, swap_perm);
            k_laswp<T><<<(unsigned)((n + kSwapThreads - 1) / kSwapThreads), kSwapThreads, swap_smem, s>>>(A, n, k0,
                                                                                                    k1, swap_perm);
            if (super && (k1 < K1 || K1 < n)) {
                // the panel's unit-lower inverse, kept in its slot for the block row's U12
                T* slot = Linv + (size_t)((k0 - K0) / nb) * nb * nb;
                const int tri_smem = (int)(2 * sizeof(T) * w * (w + 1));
                NB_TRY(cudaFuncSetAttribute(k_trtri_unit_lower<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tri_smem));
                k_trtri_unit_lower<T><<<1, 256, tri_smem, s>>>(A, n, k0, w, slot);
            }
            if (k1 < e1) {
                const int64_t m = n - k1, mc = e1 - k1;
                if (super)
                    NB_TRY(trsm_block(k0, 1, Linv + (size_t)((k0 - K0) / nb) * nb * nb, k1, e1));
                else
                    NB_TRY(trsm_rows(k0, w, k1, e1));
                // A22 -= L21 * U12 over the columns up to e1: tensor cores (TF32 x3) for the
                // FP32 factorisation's 64-wide panels, FP64 FMA for the FP64 factorisation
                if constexpr (sizeof(T) == 4) {
                    if (w == 64) {
                        NB_TRY(tc_update_f32(m, mc, reinterpret_cast<const float*>(A + k1 + k0 * n), n,
                                             reinterpret_cast<const float*>(A + k0 + k1 * n), n,
                                             reinterpret_cast<float*>(A + k1 + k1 * n), n, split, d_info + 1, s));
                        continue;
                    }
                }
                NB_TRY(gemm<T>(m, mc, w, (T)-1, A + k1 + k0 * n, n, A + k0 + k1 * n, n, (T)1, A + k1 + k1 * n, n, s));
            }
            NB_TRY(cudaGetLastError());
        }
        if constexpr (sizeof(T) == 4) {
            if (super && K1 < n) {
                const int64_t m = n - K1;
                // U12 of the block row [K0, K1) over the trailing columns: block forward
                // substitution with the super-panel's unit-lower blocks and their inverses
                NB_TRY(trsm_block(K0, kSuperPanels, Linv, K1, n));
                NB_TRY(tc_update_f32_k(m, m, K1 - K0, reinterpret_cast<const float*>(A + K1 + K0 * n), n,
                                       reinterpret_cast<const float*>(A + K0 + K1 * n), n,
                                       reinterpret_cast<float*>(A + K1 + K1 * n), n, split, d_info + 1, s));
            }
        }
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- triangular solves
constexpr int kTB = 64;          // solve block
constexpr int kResRows = 256;    // residual: rows per CTA
constexpr int kResChunk = 512;   // residual: columns per partial sum (enough (row, chunk) threads to keep HBM busy)

// Row permutation of the pivots: applying the swaps (k, piv[k]), k = 0..n-1, to b gives
// b'[i] = b[perm[i]].  The swaps are sequential; they run on an index array in shared
// memory (one thread) when it fits, else in global memory.
__global__ void k_make_perm_smem(const int32_t* __restrict__ piv, int64_t n, int32_t* __restrict__ perm) {
    extern __shared__ int32_t sp[];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) sp[i] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int64_t k = 0; k < n; ++k) {
            const int32_t p = (piv[k] >= k && piv[k] < n) ? piv[k] : (int32_t)k;  // caller pivots: stay in range
            if (p != k) {
                const int32_t t = sp[k];
                sp[k] = sp[p];
                sp[p] = t;
            }
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = sp[i];
}

__global__ void k_make_perm_global(const int32_t* __restrict__ piv, int64_t n, int32_t* __restrict__ perm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t k = 0; k < n; ++k) {
        const int32_t p = (piv[k] >= k && piv[k] < n) ? piv[k] : (int32_t)k;
        if (p != k) {
            const int32_t t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
        }
    }
}

template <typename T>
__global__ void k_permute(const T* __restrict__ b, const int32_t* __restrict__ perm, int64_t n, T* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = b[perm[i]];
}

// One triangular sweep in one launch.  Block rows of kTB rows; the CTA with ticket t (taken
// from an atomic counter, so tickets follow the order in which CTAs start) solves block k =
// t (lower sweep, unit-diagonal L) or nblk-1-t (upper sweep, U):
//   x_k = D_k^-1 (rhs_k - sum_c M_kc x_c),  c < k (lower) or c > k (upper),
// taking the blocks c in sweep order as their solutions are published (flags[c] set with
// release semantics after x_c is written); when more than one block may be ready, one poll
// reads the flags of the next blockDim.x blocks and the ready prefix is consumed.  A CTA
// only waits for blocks of lower tickets, whose CTAs have started, so the waits end.  Each
// thread owns one row of the block and a quarter of its columns; the matrix values of the
// next block are loaded before its flag is awaited, so only x_c is read after it.  The
// four partial sums are added in a fixed order, so the result does not depend on timing.
// Diagonal block: FP64 sweeps solve it by substitution in one warp (lanes in step with
// __syncwarp, one synchronisation per column; U's diagonal through reciprocals); FP32
// sweeps (the inner solves of the iterative refinement) invert it in shared memory while
// the CTA waits, so that the step on the critical path is a 64 x 64 matrix-vector product.  Every wait is bounded: on
// giving up the CTA records *err, writes NaN for its block and still publishes it.
constexpr int kSvThreads = 256;
constexpr long long kSvSpinLimit = 1ll << 22;

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(kSvThreads) k_trsv(const T* __restrict__ LU, int64_t n, int64_t nblk, int lower,
                                                     const T* __restrict__ rhs, T* x, int* flags, int* ticket,
                                                     int* err, long long limit) {
    constexpr bool kInv = sizeof(T) == 4;  // explicit inverse of the diagonal block (FP32)
    __shared__ T D[kTB][kTB + 1];
    __shared__ T Xi[kInv ? kTB : 1][kTB + 1];
    __shared__ T part[kSvThreads / kTB][kTB];
    __shared__ T xs[kTB];
    __shared__ T xo[kInv ? 1 : kTB];
    __shared__ T dinv[kTB];
    __shared__ int s_t, s_ready, s_ok;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int64_t t = s_t;
    const int64_t k = lower ? t : nblk - 1 - t;
    const int64_t r0 = k * kTB, r1 = min(n, r0 + (int64_t)kTB);
    const int w = (int)(r1 - r0);
    constexpr int kGroups = kSvThreads / kTB, kCols = kTB / kGroups;
    const int row = threadIdx.x % kTB, grp = threadIdx.x / kTB;
    for (int idx = threadIdx.x; idx < w * w; idx += kSvThreads) {
        const int r = idx % w, c = idx / w;
        D[r][c] = LU[(r0 + r) + (r0 + c) * n];
    }
    // independent of the other blocks: the block's right-hand side and, for U, the
    // reciprocals of its diagonal
    const T rhs_own = (threadIdx.x < w) ? rhs[r0 + threadIdx.x] : (T)0;
    if (!lower && threadIdx.x < w) dinv[threadIdx.x] = (T)1 / LU[(r0 + threadIdx.x) + (r0 + threadIdx.x) * n];
    if constexpr (kInv) {
        // X = D^-1 by forward (L, unit diagonal) or backward (U) substitution of all
        // columns at once, one block barrier per step
        __syncthreads();
        for (int idx = threadIdx.x; idx < kTB * kTB; idx += kSvThreads) {
            const int r = idx % kTB, c = idx / kTB;
            Xi[r][c] = (r == c && r < w) ? (T)1 : (T)0;
        }
        __syncthreads();
        if (lower) {
            for (int q = 0; q + 1 < w; ++q) {
                const int rows = w - 1 - q;
                for (int idx = threadIdx.x; idx < rows * (q + 1); idx += kSvThreads) {
                    const int r = q + 1 + idx % rows, c = idx / rows;
                    Xi[r][c] -= D[r][q] * Xi[q][c];
                }
                __syncthreads();
            }
        } else {
            for (int q = w - 1; q >= 0; --q) {
                // row q of X is final once scaled by 1 / U[q][q]; then eliminate above
                const int cols = w - q;
                for (int c = q + threadIdx.x; c < w; c += kSvThreads) Xi[q][c] *= dinv[q];
                __syncthreads();
                for (int idx = threadIdx.x; idx < q * cols; idx += kSvThreads) {
                    const int r = idx % q, c = q + idx / q;
                    Xi[r][c] -= D[r][q] * Xi[q][c];
                }
                __syncthreads();
            }
        }
    }
    T acc = (T)0;
    const int64_t total = lower ? k : nblk - 1 - k;
    // matrix values of block i (sweep order) for this thread: row `row`, kCols columns
    T mv[kCols];
    auto load_block = [&](int64_t i) {
        const int64_t c0 = (lower ? i : nblk - 1 - i) * kTB + grp * kCols;
        const T* col = LU + (r0 + row) + c0 * n;
        const int wc = (int)min((int64_t)kCols, n - c0);
#pragma unroll
        for (int q = 0; q < kCols; ++q) mv[q] = (row < w && q < wc) ? col[(int64_t)q * n] : (T)0;
    };
    auto use_block = [&](int64_t i) {
        const int64_t c0 = (lower ? i : nblk - 1 - i) * kTB + grp * kCols;
        const int wc = (int)min((int64_t)kCols, n - c0);
#pragma unroll
        for (int q = 0; q < kCols; ++q)
            if (q < wc) acc = fma(mv[q], __ldcg(x + c0 + q), acc);
    };
    if (total > 0) load_block(0);
    int64_t done = 0;
    long long spins = 0;  // used by thread 0
    bool ok = true;
    while (done < total) {
        // one thread waits (bounded) for the next block in sweep order; if more blocks may
        // be ready, all threads read the flags of the following ones and take the ready prefix
        if (threadIdx.x == 0) {
            const int* fp = flags + (lower ? done : nblk - 1 - done);
            int f = ld_acquire(fp);
            while (!f && ++spins <= limit) {
                __nanosleep(32);
                f = ld_acquire(fp);
            }
            s_ok = f != 0;
            s_ready = kSvThreads;
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        int64_t ready = 1;
        if (total - done > 1) {
            const int64_t idx = done + threadIdx.x;
            if (threadIdx.x > 0 && idx < total && ld_acquire(flags + (lower ? idx : nblk - 1 - idx)) == 0)
                atomicMin(&s_ready, (int)threadIdx.x);
            __syncthreads();
            ready = min((int64_t)s_ready, total - done);
        }
        __syncthreads();  // s_ready and s_ok are rewritten by the next poll
        use_block(done);
        for (int64_t i = done + 1; i < done + ready; ++i) {
            load_block(i);
            use_block(i);
        }
        done += ready;
        if (done < total) load_block(done);  // in flight while the next flag is awaited
    }
    if (!ok) atomicExch(err, 1);
    part[grp][row] = acc;
    __syncthreads();
    if (threadIdx.x < w) {
        T sum = part[0][threadIdx.x];
#pragma unroll
        for (int g = 1; g < kGroups; ++g) sum += part[g][threadIdx.x];
        xs[threadIdx.x] = rhs_own - sum;
    }
    __syncthreads();
    if constexpr (kInv) {
        // x = X (rhs - sum): row `row`, columns of group grp, then the groups in order
        T v = (T)0;
        if (row < w) {
#pragma unroll
            for (int q = 0; q < kCols; ++q) {
                const int c = grp * kCols + q;
                if (c < w) v = fma(Xi[row][c], xs[c], v);
            }
        }
        part[grp][row] = v;
        __syncthreads();
        if (threadIdx.x < w) {
            T sum = part[0][threadIdx.x];
#pragma unroll
            for (int g = 1; g < kGroups; ++g) sum += part[g][threadIdx.x];
            xs[threadIdx.x] = sum;
        }
    } else {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            if (lower) {
                for (int c = 0; c < w; ++c) {
                    const T xc = xs[c];
                    for (int r = lane; r < w; r += 32)
                        if (r > c) xs[r] -= D[r][c] * xc;
                    __syncwarp();
                }
            } else {
                // every lane scales x_c itself (the same rounded product), the owner lane
                // keeps it in xo: one warp synchronisation per column
                for (int c = w - 1; c >= 0; --c) {
                    const T xc = xs[c] * dinv[c];
                    if (lane == (c & 31)) xo[c] = xc;
                    for (int r = lane; r < c; r += 32) xs[r] -= D[r][c] * xc;
                    __syncwarp();
                }
                for (int r = lane; r < w; r += 32) xs[r] = xo[r];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < w) x[r0 + threadIdx.x] = ok ? xs[threadIdx.x] : (T)NAN;
    // the block barrier orders the CTA's stores before thread 0's release (cumulative)
    __syncthreads();
    if (threadIdx.x == 0) st_release(flags + k, 1);
}

// The same sweep for nr <= kMR right-hand sides at once (columns of rhs and x, leading
// dimension n; used for the weighting fields of several readouts, Sec. 2.1).  Each factor
// block is read once for all columns, and the columns share every block barrier.  Per
// column the arithmetic is k_trsv's, in its order (the fma chain over blocks and columns,
// the four group sums in order, the diagonal block: FP64 substitution, one warp per column;
// FP32 explicit inverse), so column j equals k_trsv on that column bit for bit.  Waits,
// give-up and publication as in k_trsv.  Dynamic shared memory, trsm_smem_bytes<T>():
//   D[kTB][kTB+1], Xi[kTB][kTB+1] (FP32 only), part[groups][kMR][kTB] (FP64: shared with
//   the substitution's xo[kMR][kTB]), xs[kMR][kTB] (the block's right-hand sides, then its
//   solution), dinv[kTB].
constexpr int kMR = 8;

template <typename T>
__host__ __device__ constexpr size_t trsm_smem_bytes() {
    return sizeof(T) * ((size_t)kTB * (kTB + 1) * (sizeof(T) == 4 ? 2 : 1) + (size_t)(kSvThreads / kTB) * kMR * kTB +
                        (size_t)kMR * kTB + kTB);
}

template <typename T>
__global__ void __launch_bounds__(kSvThreads) k_trsm(const T* __restrict__ LU, int64_t n, int64_t nblk, int lower,
                                                     const T* __restrict__ rhs, T* x, int nr, int* flags,
                                                     int* ticket, int* err, long long limit) {
    constexpr bool kInv = sizeof(T) == 4;
    constexpr int kGroups = kSvThreads / kTB, kCols = kTB / kGroups;
    extern __shared__ __align__(16) unsigned char trsm_sm[];
    T(*D)[kTB + 1] = reinterpret_cast<T(*)[kTB + 1]>(trsm_sm);
    T(*Xi)[kTB + 1] = D + kTB;  // FP32 only
    T(*part)[kMR][kTB] = reinterpret_cast<T(*)[kMR][kTB]>(reinterpret_cast<T*>(D + (kInv ? 2 : 1) * kTB));
    T(*xo)[kTB] = part[0];  // FP64 substitution, after the group sums
    T(*xs)[kTB] = reinterpret_cast<T(*)[kTB]>(reinterpret_cast<T*>(part + kGroups));
    T* dinv = reinterpret_cast<T*>(xs + kMR);
    __shared__ int s_t, s_ready, s_ok;
    if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int64_t t = s_t;
    const int64_t k = lower ? t : nblk - 1 - t;
    const int64_t r0 = k * kTB, r1 = min(n, r0 + (int64_t)kTB);
    const int w = (int)(r1 - r0);
    const int row = threadIdx.x % kTB, grp = threadIdx.x / kTB;
    for (int idx = threadIdx.x; idx < w * w; idx += kSvThreads) {
        const int r = idx % w, c = idx / w;
        D[r][c] = LU[(r0 + r) + (r0 + c) * n];
    }
    for (int idx = threadIdx.x; idx < w * nr; idx += kSvThreads) {
        const int j = idx / w, r = idx - j * w;
        xs[j][r] = rhs[r0 + r + (int64_t)j * n];
    }
    if (!lower && threadIdx.x < w) dinv[threadIdx.x] = (T)1 / LU[(r0 + threadIdx.x) + (r0 + threadIdx.x) * n];
    if constexpr (kInv) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < kTB * kTB; idx += kSvThreads) {
            const int r = idx % kTB, c = idx / kTB;
            Xi[r][c] = (r == c && r < w) ? (T)1 : (T)0;
        }
        __syncthreads();
        if (lower) {
            for (int q = 0; q + 1 < w; ++q) {
                const int rows = w - 1 - q;
                for (int idx = threadIdx.x; idx < rows * (q + 1); idx += kSvThreads) {
                    const int r = q + 1 + idx % rows, c = idx / rows;
                    Xi[r][c] -= D[r][q] * Xi[q][c];
                }
                __syncthreads();
            }
        } else {
            for (int q = w - 1; q >= 0; --q) {
                const int cols = w - q;
                for (int c = q + threadIdx.x; c < w; c += kSvThreads) Xi[q][c] *= dinv[q];
                __syncthreads();
                for (int idx = threadIdx.x; idx < q * cols; idx += kSvThreads) {
                    const int r = idx % q, c = q + idx / q;
                    Xi[r][c] -= D[r][q] * Xi[q][c];
                }
                __syncthreads();
            }
        }
    }
    T acc[kMR];
#pragma unroll
    for (int j = 0; j < kMR; ++j) acc[j] = (T)0;
    const int64_t total = lower ? k : nblk - 1 - k;
    T mv[kCols];
    auto load_block = [&](int64_t i) {
        const int64_t c0 = (lower ? i : nblk - 1 - i) * kTB + grp * kCols;
        const T* col = LU + (r0 + row) + c0 * n;
        const int wc = (int)min((int64_t)kCols, n - c0);
#pragma unroll
        for (int q = 0; q < kCols; ++q) mv[q] = (row < w && q < wc) ? col[(int64_t)q * n] : (T)0;
    };
    auto use_block = [&](int64_t i) {
        const int64_t c0 = (lower ? i : nblk - 1 - i) * kTB + grp * kCols;
        const int wc = (int)min((int64_t)kCols, n - c0);
#pragma unroll
        for (int q = 0; q < kCols; ++q)
            if (q < wc) {
#pragma unroll
                for (int j = 0; j < kMR; ++j)
                    if (j < nr) acc[j] = fma(mv[q], __ldcg(x + c0 + q + (int64_t)j * n), acc[j]);
            }
    };
    if (total > 0) load_block(0);
    int64_t done = 0;
    long long spins = 0;
    bool ok = true;
    while (done < total) {
        if (threadIdx.x == 0) {
            const int* fp = flags + (lower ? done : nblk - 1 - done);
            int f = ld_acquire(fp);
            while (!f && ++spins <= limit) {
                __nanosleep(32);
                f = ld_acquire(fp);
            }
            s_ok = f != 0;
            s_ready = kSvThreads;
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        int64_t ready = 1;
        if (total - done > 1) {
            const int64_t idx = done + threadIdx.x;
            if (threadIdx.x > 0 && idx < total && ld_acquire(flags + (lower ? idx : nblk - 1 - idx)) == 0)
                atomicMin(&s_ready, (int)threadIdx.x);
            __syncthreads();
            ready = min((int64_t)s_ready, total - done);
        }
        __syncthreads();
        use_block(done);
        for (int64_t i = done + 1; i < done + ready; ++i) {
            load_block(i);
            use_block(i);
        }
        done += ready;
        if (done < total) load_block(done);
    }
    if (!ok) atomicExch(err, 1);
    // every column's four group sums, in order, subtracted from its right-hand side
#pragma unroll
    for (int j = 0; j < kMR; ++j)
        if (j < nr) part[grp][j][row] = acc[j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nr; idx += kSvThreads) {
        const int j = idx / w, r = idx - j * w;
        T sum = part[0][j][r];
#pragma unroll
        for (int g = 1; g < kGroups; ++g) sum += part[g][j][r];
        xs[j][r] = xs[j][r] - sum;
    }
    __syncthreads();
    if constexpr (kInv) {
        // x_j = X (rhs_j - sum_j): row `row`, columns of group grp, then the groups in order
        T v[kMR];
#pragma unroll
        for (int j = 0; j < kMR; ++j) {
            v[j] = (T)0;
            if (j < nr && row < w) {
#pragma unroll
                for (int q = 0; q < kCols; ++q) {
                    const int c = grp * kCols + q;
                    if (c < w) v[j] = fma(Xi[row][c], xs[j][c], v[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kMR; ++j)
            if (j < nr) part[grp][j][row] = v[j];
        __syncthreads();
        for (int idx = threadIdx.x; idx < w * nr; idx += kSvThreads) {
            const int j = idx / w, r = idx - j * w;
            T sum = part[0][j][r];
#pragma unroll
            for (int g = 1; g < kGroups; ++g) sum += part[g][j][r];
            xs[j][r] = sum;
        }
    } else {
        const int j = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (j < nr) {
            if (lower) {
                for (int c = 0; c < w; ++c) {
                    const T xc = xs[j][c];
                    for (int r = lane; r < w; r += 32)
                        if (r > c) xs[j][r] -= D[r][c] * xc;
                    __syncwarp();
                }
            } else {
                for (int c = w - 1; c >= 0; --c) {
                    const T xc = xs[j][c] * dinv[c];
                    if (lane == (c & 31)) xo[j][c] = xc;
                    for (int r = lane; r < c; r += 32) xs[j][r] -= D[r][c] * xc;
                    __syncwarp();
                }
                for (int r = lane; r < w; r += 32) xs[j][r] = xo[j][r];
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * nr; idx += kSvThreads) {
        const int j = idx / w, r = idx - j * w;
        x[r0 + r + (int64_t)j * n] = ok ? xs[j][r] : (T)NAN;
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release(flags + k, 1);
}

template <typename T>
__global__ void k_permute_m(const T* __restrict__ b, const int32_t* __restrict__ perm, int64_t n, int nr,
                            T* __restrict__ y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nr) return;
    const int64_t j = idx / n, i = idx - j * n;
    y[idx] = b[perm[i] + j * n];
}

template <typename T>
cudaError_t lu_solve(const T* LU, int64_t n, const int32_t* perm, T* b, T* work, cudaStream_t s, long long polls) {
    if (n == 0) return cudaSuccess;
    const int64_t nblk = (n + kTB - 1) / kTB;
    T* y = work;
    T* z = work + n;
    // flags of both sweeps, their tickets and the error flag (16-byte aligned after z)
    const uintptr_t fo = ((uintptr_t)(z + n) + 15) & ~(uintptr_t)15;
    int* flags = reinterpret_cast<int*>(fo);
    int* tickets = flags + 2 * nblk;
    int* err = tickets + 2;
    NB_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * (2 * nblk + 3), s));
    const unsigned g = (unsigned)((n + 255) / 256);
    k_permute<T><<<g, 256, 0, s>>>(b, perm, n, y);
    const long long limit = polls > 0 ? polls : kSvSpinLimit;
    k_trsv<T><<<(unsigned)nblk, kSvThreads, 0, s>>>(LU, n, nblk, 1, y, z, flags, tickets, err, limit);
    k_trsv<T><<<(unsigned)nblk, kSvThreads, 0, s>>>(LU, n, nblk, 0, z, b, flags + nblk, tickets + 1, err, limit);
    return cudaGetLastError();
}

// r = b - K x for column-major K: partial sums over column chunks of kResChunk (one CTA per
// rows x chunk), then the chunks added in order per row.
__global__ void __launch_bounds__(kResRows) k_residual_partial(const double* __restrict__ K, int64_t n,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * kResRows + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * kResChunk, j1 = min(n, j0 + (int64_t)kResChunk);
    __shared__ double xs[kResChunk];
    for (int64_t j = j0 + threadIdx.x; j < j1; j += kResRows) xs[j - j0] = x[j];
    __syncthreads();
    if (i >= n) return;
    double s = 0.0;
#pragma unroll 8
    for (int64_t j = j0; j < j1; ++j) s = fma(K[i + j * n], xs[j - j0], s);
    part[(int64_t)blockIdx.y * n + i] = s;
}

__global__ void k_residual_final(const double* __restrict__ part, int64_t nchunk, int64_t n,
                                 const double* __restrict__ b, double* __restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) s += part[c * n + i];
    r[i] = b[i] - s;
}

// r_j = b_j - K x_j for nr <= kMR columns at once (leading dimension n): K is read once for
// all columns; per column the sums are k_residual_partial's (an fma chain over the chunk's
// columns in order) and k_residual_final's (the chunks in order), so column j equals the
// single-column residual bit for bit.  x is staged in shared memory kResTile columns at a time.
constexpr int kResTile = 512;

template <int NR>
__global__ void __launch_bounds__(kResRows) k_residual_partial_m(const double* __restrict__ K, int64_t n,
                                                                 const double* __restrict__ x,
                                                                 double* __restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * kResRows + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * kResChunk, j1 = min(n, j0 + (int64_t)kResChunk);
    constexpr int kUnroll = NR > 4 ? 4 : 8;  // loads in flight, within the register budget
    __shared__ double xs[kResTile][NR];
    double s[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] = 0.0;
    for (int64_t t0 = j0; t0 < j1; t0 += kResTile) {
        const int64_t t1 = min(j1, t0 + (int64_t)kResTile);
        __syncthreads();
        for (int64_t idx = threadIdx.x; idx < (t1 - t0) * NR; idx += kResRows) {
            const int64_t c = idx / (t1 - t0), j = idx - c * (t1 - t0);
            xs[j][c] = x[t0 + j + c * n];
        }
        __syncthreads();
        if (i < n)
#pragma unroll kUnroll
            for (int64_t j = t0; j < t1; ++j) {
                const double kv = K[i + j * n];
#pragma unroll
                for (int c = 0; c < NR; ++c) s[c] = fma(kv, xs[j - t0][c], s[c]);
            }
    }
    if (i < n)
#pragma unroll
        for (int c = 0; c < NR; ++c) part[((int64_t)blockIdx.y * kMR + c) * n + i] = s[c];
}

template <int NR>
static void launch_residual_partial_m(dim3 grid, cudaStream_t s, const double* K, int64_t n, const double* x,
                                      double* part) {
    k_residual_partial_m<NR><<<grid, kResRows, 0, s>>>(K, n, x, part);
}

__global__ void k_residual_final_m(const double* __restrict__ part, int64_t nchunk, int64_t n, int nr,
                                   const double* __restrict__ b, double* __restrict__ r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nr) return;
    const int64_t c = idx / n, i = idx - c * n;
    double s = 0.0;
    for (int64_t q = 0; q < nchunk; ++q) s += part[(q * kMR + c) * n + i];
    r[idx] = b[idx] - s;
}

// x_j += d_j for the columns j whose bit is set in `active`; norms[2j] = max|d_j|,
// norms[2j + 1] = max|x_j| (as k_ir_update, one column per blockIdx.y).
__global__ void k_ir_update_m(double* __restrict__ x, const float* __restrict__ d, int64_t n, uint32_t active,
                              double* norms) {
    const int64_t c = blockIdx.y;
    if (!((active >> c) & 1u)) return;
    double md = 0.0, mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double di = (double)d[i + c * n];
        const double xi = x[i + c * n] + di;
        x[i + c * n] = xi;
        md = fmax(md, fabs(di));
        mx = fmax(mx, fabs(xi));
    }
    for (int o = 16; o > 0; o >>= 1) {
        md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(norms + 2 * c), __double_as_longlong(md));
        atomicMax(reinterpret_cast<unsigned long long*>(norms + 2 * c + 1), __double_as_longlong(mx));
    }
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// x += d; norms[0] = max|d|, norms[1] = max|x| (atomicMax on the bit patterns of
// non-negative doubles, which order like the values).
__global__ void k_ir_update(double* __restrict__ x, const float* __restrict__ d, int64_t n, double* norms) {
    double md = 0.0, mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double di = (double)d[i];
        const double xi = x[i] + di;
        x[i] = xi;
        md = fmax(md, fabs(di));
        mx = fmax(mx, fabs(xi));
    }
    for (int o = 16; o > 0; o >>= 1) {
        md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(norms), __double_as_longlong(md));
        atomicMax(reinterpret_cast<unsigned long long*>(norms + 1), __double_as_longlong(mx));
    }
}

__global__ void k_absmax(const double* __restrict__ a, int64_t n, double* out) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(out), __double_as_longlong(m));
}

__global__ void k_gather(const double* __restrict__ a, const int64_t* __restrict__ idx, int64_t n,
                         double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[idx[i]];
}

}  // namespace

cudaError_t launch_gather(const double* a, const int64_t* idx, int64_t n, double* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, idx, n, out);
    return cudaGetLastError();
}

size_t lu_work_elems(int64_t n, int nb) {
    // L11^-1 + U12 staging + pivot partials, the ticket and the composed row swaps (in
    // 4-byte units rounded up, which covers both types)
    return (size_t)kSuperPanels * nb * nb + (size_t)nb * (size_t)n + 16 + (size_t)kPivBlocks * 4 + 16 +
           (2 * kSwapMax + 16);
}

cudaError_t lu_factor_f64(double* A, int64_t n, int32_t* piv, int nb, double* work, int* d_info, cudaStream_t s) {
    return lu_factor<double>(A, n, piv, nb, work, d_info, nullptr, nullptr, s, 0);
}
static size_t split_offset(int64_t n, int nb) { return (sizeof(float) * lu_work_elems(n, nb) + 255) & ~(size_t)255; }
static size_t coop_offset(int64_t n, int nb) {
    return (split_offset(n, nb) + tc_split_bytes(n, n, kSuperPanels) + 255) & ~(size_t)255;
}
size_t lu_work_bytes_f32(int64_t n, int nb) { return coop_offset(n, nb) + sizeof(CoopScratch); }
cudaError_t lu_factor_f32(float* A, int64_t n, int32_t* piv, int nb, float* work, int* d_info, cudaStream_t s,
                          long long polls) {
    // work: lu_work_bytes_f32(n, nb) bytes, 256-byte aligned: panel staging, then the
    // tensor-core split operands, then the cooperative panel's candidates and barrier
    void* split = reinterpret_cast<char*>(work) + split_offset(n, nb);
    void* coop = reinterpret_cast<char*>(work) + coop_offset(n, nb);
    return lu_factor<float>(A, n, piv, nb, work, d_info, split, coop, s, polls);
}
size_t lu_solve_work_bytes(int64_t n, size_t tsize) {
    return 2 * tsize * (size_t)n + 16 + sizeof(int) * (size_t)(2 * ((n + kTB - 1) / kTB) + 3) + 256;
}

size_t residual_work_bytes(int64_t n) {
    return sizeof(double) * (size_t)((n + kResChunk - 1) / kResChunk) * (size_t)n + 256;
}

cudaError_t lu_make_perm(const int32_t* piv, int64_t n, int32_t* perm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t bytes = sizeof(int32_t) * (size_t)n;
    if (bytes <= 200 * 1024) {
        // set for the current device on every call (an attribute is per device)
        NB_TRY(cudaFuncSetAttribute(k_make_perm_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        k_make_perm_smem<<<1, 1024, bytes, s>>>(piv, n, perm);
    } else {
        k_make_perm_global<<<1, 1, 0, s>>>(piv, n, perm);
    }
    return cudaGetLastError();
}

cudaError_t lu_solve_f64(const double* LU, int64_t n, const int32_t* perm, double* b, void* work, cudaStream_t s,
                         long long polls) {
    return lu_solve<double>(LU, n, perm, b, static_cast<double*>(work), s, polls);
}
cudaError_t lu_solve_f32(const float* LU, int64_t n, const int32_t* perm, float* b, void* work, cudaStream_t s,
                         long long polls) {
    return lu_solve<float>(LU, n, perm, b, static_cast<float*>(work), s, polls);
}
const int* lu_solve_err_flag(const void* work, int64_t n, size_t tsize) {
    // as laid out by lu_solve: y, z (n values each), then 16-byte aligned flags of both
    // sweeps (nblk each), the two tickets and the error flag
    const uintptr_t fo = ((uintptr_t)static_cast<const char*>(work) + 2 * tsize * (size_t)n + 15) & ~(uintptr_t)15;
    const int64_t nblk = (n + kTB - 1) / kTB;
    return reinterpret_cast<const int*>(fo) + 2 * nblk + 2;
}
cudaError_t gemv_residual(const double* K, int64_t n, const double* x, const double* b, double* r, void* work,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t nchunk = (n + kResChunk - 1) / kResChunk;
    double* part = static_cast<double*>(work);
    dim3 grid((unsigned)((n + kResRows - 1) / kResRows), (unsigned)nchunk);
    k_residual_partial<<<grid, kResRows, 0, s>>>(K, n, x, part);
    k_residual_final<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, nchunk, n, b, r);
    return cudaGetLastError();
}
cudaError_t copy_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_f64_to_f32<<<(unsigned)std::min<int64_t>(65535, (n + 255) / 256), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}
cudaError_t ir_update(double* x, const float* d, int64_t n, double* d_norms, cudaStream_t s) {
    NB_TRY(cudaMemsetAsync(d_norms, 0, 2 * sizeof(double), s));
    k_ir_update<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(x, d, n, d_norms);
    return cudaGetLastError();
}
cudaError_t vec_absmax(const double* a, int64_t n, double* out, cudaStream_t s) {
    NB_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    k_absmax<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(a, n, out);
    return cudaGetLastError();
}

// ---- several right-hand sides (columns of leading dimension n), kMR per pass
size_t lu_solve_multi_work_bytes(int64_t n, size_t tsize) {
    return 2 * tsize * (size_t)n * kMR + 16 + sizeof(int) * (size_t)(2 * ((n + kTB - 1) / kTB) + 3) + 256;
}
static int* multi_flags(const void* work, int64_t n, size_t tsize) {
    // y, z (n x kMR values each), then 16-byte aligned flags of both sweeps, the two
    // tickets and the error flag
    const uintptr_t fo =
        ((uintptr_t)static_cast<const char*>(work) + 2 * tsize * (size_t)n * kMR + 15) & ~(uintptr_t)15;
    return reinterpret_cast<int*>(fo);
}
const int* lu_solve_multi_err_flag(const void* work, int64_t n, size_t tsize) {
    return multi_flags(work, n, tsize) + 2 * ((n + kTB - 1) / kTB) + 2;
}
template <typename T>
static cudaError_t lu_solve_multi(const T* LU, int64_t n, const int32_t* perm, T* B, int64_t nrhs, void* work,
                                  cudaStream_t s, long long polls) {
    if (n == 0 || nrhs == 0) return cudaSuccess;
    const int64_t nblk = (n + kTB - 1) / kTB;
    T* y = static_cast<T*>(work);
    T* z = y + n * kMR;
    int* flags = multi_flags(work, n, sizeof(T));
    int* tickets = flags + 2 * nblk;
    int* err = tickets + 2;
    NB_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    const long long limit = polls > 0 ? polls : kSvSpinLimit;
    // set for the current device on every call (an attribute is per device)
    const size_t smem = trsm_smem_bytes<T>();
    NB_TRY(cudaFuncSetAttribute(k_trsm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int64_t c0 = 0; c0 < nrhs; c0 += kMR) {
        const int nr = (int)std::min<int64_t>(kMR, nrhs - c0);
        T* b = B + c0 * n;
        NB_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * (2 * nblk + 2), s));
        k_permute_m<T><<<(unsigned)((n * nr + 255) / 256), 256, 0, s>>>(b, perm, n, nr, y);
        k_trsm<T><<<(unsigned)nblk, kSvThreads, smem, s>>>(LU, n, nblk, 1, y, z, nr, flags, tickets, err, limit);
        k_trsm<T><<<(unsigned)nblk, kSvThreads, smem, s>>>(LU, n, nblk, 0, z, b, nr, flags + nblk, tickets + 1, err,
                                                           limit);
        NB_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}
cudaError_t lu_solve_multi_f64(const double* LU, int64_t n, const int32_t* perm, double* B, int64_t nrhs, void* work,
                               cudaStream_t s, long long polls) {
    return lu_solve_multi<double>(LU, n, perm, B, nrhs, work, s, polls);
}
cudaError_t lu_solve_multi_f32(const float* LU, int64_t n, const int32_t* perm, float* B, int64_t nrhs, void* work,
                               cudaStream_t s, long long polls) {
    return lu_solve_multi<float>(LU, n, perm, B, nrhs, work, s, polls);
}
size_t residual_multi_work_bytes(int64_t n) {
    return sizeof(double) * (size_t)((n + kResChunk - 1) / kResChunk) * kMR * (size_t)n + 256;
}
cudaError_t gemv_residual_multi(const double* K, int64_t n, const double* X, int64_t nrhs, const double* B, double* R,
                                void* work, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t nchunk = (n + kResChunk - 1) / kResChunk;
    double* part = static_cast<double*>(work);
    for (int64_t c0 = 0; c0 < nrhs; c0 += kMR) {
        const int nr = (int)std::min<int64_t>(kMR, nrhs - c0);
        dim3 grid((unsigned)((n + kResRows - 1) / kResRows), (unsigned)nchunk);
        switch (nr) {  // the column count as a template argument: no predicated lanes
            case 1: launch_residual_partial_m<1>(grid, s, K, n, X + c0 * n, part); break;
            case 2: launch_residual_partial_m<2>(grid, s, K, n, X + c0 * n, part); break;
            case 3: launch_residual_partial_m<3>(grid, s, K, n, X + c0 * n, part); break;
            case 4: launch_residual_partial_m<4>(grid, s, K, n, X + c0 * n, part); break;
            case 5: launch_residual_partial_m<5>(grid, s, K, n, X + c0 * n, part); break;
            case 6: launch_residual_partial_m<6>(grid, s, K, n, X + c0 * n, part); break;
            case 7: launch_residual_partial_m<7>(grid, s, K, n, X + c0 * n, part); break;
            default: launch_residual_partial_m<8>(grid, s, K, n, X + c0 * n, part); break;
        }
        k_residual_final_m<<<(unsigned)((n * nr + 255) / 256), 256, 0, s>>>(part, nchunk, n, nr, B + c0 * n,
                                                                           R + c0 * n);
        NB_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}
cudaError_t ir_update_multi(double* X, const float* D, int64_t n, int64_t nrhs, uint64_t active, double* d_norms,
                            cudaStream_t s) {
    if (nrhs > 64) return cudaErrorInvalidValue;
    NB_TRY(cudaMemsetAsync(d_norms, 0, 2 * sizeof(double) * (size_t)nrhs, s));
    if (n == 0) return cudaSuccess;
    for (int64_t c0 = 0; c0 < nrhs; c0 += kMR) {
        const int nr = (int)std::min<int64_t>(kMR, nrhs - c0);
        const uint32_t act = (uint32_t)((active >> c0) & ((1ull << nr) - 1ull));
        if (!act) continue;
        dim3 grid((unsigned)std::min<int64_t>(1024, (n + 255) / 256), (unsigned)nr);
        k_ir_update_m<<<grid, 256, 0, s>>>(X + c0 * n, D + c0 * n, n, act, d_norms + 2 * c0);
        NB_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace nb
