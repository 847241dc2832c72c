// lu_tc.cu -- trailing-matrix update of the mixed (FP32) LU on the 5th-generation tensor
// cores: C[M x N] -= A[M x 64] * B[64 x N] (column-major FP32), the rank-64 update that
// follows each panel of the blocked factorisation (Sec. 4.1 / Alg. 1: LU; the trailing
// update carries almost all of its 2/3 N^3 flops).
//
// Each CTA (128 threads) owns a 128-row strip of C and walks four 64-column tiles of it
// (two CTAs fit per SM); its A tile is staged once.  A and B are split into TF32 pairs
// (hi = x rounded to TF32, lo = x - hi) and staged in shared memory in the
// canonical K-major, non-swizzled UMMA layout (8-row x 16-byte core matrices; core
// matrices adjacent along K are LBO = 128 B apart, 8-row groups SBO = 2048 B apart).
// One elected thread issues tcgen05.mma kind::tf32 (M = 128, N = 64, K = 8 per
// instruction) for lo*hi, hi*lo and hi*hi -- 24 instructions accumulating in FP32 in
// tensor memory -- then commits to an mbarrier.  Two accumulators (128 lanes x 64 columns
// each) alternate between the tiles, so the write-back of tile t-1 (C fetched into
// registers, the product read with tcgen05.ld -- warp w owns TMEM lanes 32w..32w+31 = rows
// of C -- and subtracted) overlaps the MMAs of tile t.  Operand tiles are loaded with
// float4 loads when the leading dimension and pointers allow it.  The three-term split keeps the product within a
// few FP32 units of roundoff, which the FP64 iterative refinement of the solve expects.
//
// The mbarrier wait is bounded: after kSpinLimit polls the CTA records an error flag,
// skips the epilogue, still frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>

#include "nb_internal.h"

namespace nb {

namespace {

constexpr int kTM = 128, kTN = 64, kTK = 64;
constexpr uint32_t kCoreBytes = 128;                 // 8 rows x 16 bytes
constexpr uint32_t kLBO = kCoreBytes;                // next core matrix along K
constexpr uint32_t kSBO = (kTK / 4) * kCoreBytes;    // next 8-row group: 2048 B
constexpr uint32_t kABytes = kTM * kTK * 4;          // 32 KB per A operand tile
constexpr uint32_t kBBytes = kTN * kTK * 4;          // 16 KB per B operand tile
constexpr uint32_t kSmemBytes = 2 * kABytes + 2 * kBBytes + 64;
constexpr long long kSpinLimit = 1ll << 24;
constexpr int kTilesN = 4;                           // 64-column tiles of C per CTA

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row r, k) in a K-major non-swizzled operand tile
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
    return (uint32_t)(r >> 3) * kSBO + (uint32_t)(k >> 2) * kLBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4
// (32-45), fixed 0b001 at bits 46-48, base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kLBO >> 4) << 16;
    d |= (uint64_t)(kSBO >> 4) << 32;
    d |= 1ull << 46;
    return d;
}

// instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9,
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void put_pair(unsigned char* hi, unsigned char* lo, uint32_t o, float x) {
    const float h = tf32_hi(x);
    *reinterpret_cast<float*>(hi + o) = h;
    *reinterpret_cast<float*>(lo + o) = x - h;
}

// Stage B (64 k x 64 columns from column n0) as TF32 hi/lo pairs in the K-major layout.
__device__ __forceinline__ void stage_b(const float* __restrict__ B, int64_t ldb, int64_t N, int64_t n0, bool fast,
                                        unsigned char* b_hi, unsigned char* b_lo, int tid) {
    if (fast) {
        float4 vb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = tid / 16 + 8 * j;
            vb[j] = *reinterpret_cast<const float4*>(B + 4 * (tid % 16) + (n0 + c) * ldb);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = tid / 16 + 8 * j, k = 4 * (tid % 16);
            put_pair(b_hi, b_lo, kmajor_off(c, k), vb[j].x);
            put_pair(b_hi, b_lo, kmajor_off(c, k + 1), vb[j].y);
            put_pair(b_hi, b_lo, kmajor_off(c, k + 2), vb[j].z);
            put_pair(b_hi, b_lo, kmajor_off(c, k + 3), vb[j].w);
        }
    } else {
        for (int idx = tid; idx < kTN * kTK; idx += 128) {
            const int k = idx % kTK, c = idx / kTK;
            const int64_t gn = n0 + c;
            put_pair(b_hi, b_lo, kmajor_off(c, k), (gn < N) ? B[k + gn * ldb] : 0.f);
        }
    }
}

// C[row, n0 .. n0+63] -= accumulator columns [col0, col0 + 64) of TMEM (warp w owns lanes
// 32w .. 32w+31 = rows of the tile), 32 columns at a time, each C segment fetched before
// its TMEM read.
__device__ __forceinline__ void epilogue(float* __restrict__ C, int64_t ldc, int64_t M, int64_t N, int64_t row,
                                         int64_t n0, uint32_t tmem, uint32_t col0, int warp) {
#pragma unroll
    for (int cb = 0; cb < kTN; cb += 32) {
        float cv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int64_t col = n0 + cb + j;
            cv[j] = (row < M && col < N) ? C[row + col * ldc] : 0.f;
        }
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + col0 + (uint32_t)cb;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (row < M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t col = n0 + cb + j;
                if (col < N) C[row + col * ldc] = cv[j] - __uint_as_float(v[j]);
            }
        }
    }
}

// Each CTA stages its 128-row A tile once and walks kTilesN consecutive 64-column tiles of
// C.  Two accumulators in tensor memory (columns 0..63 and 64..127) alternate, so while the
// tensor core runs the MMAs of tile t the threads write tile t-1 back.
__global__ void __launch_bounds__(128, 2) k_tc_update(int64_t M, int64_t N, const float* __restrict__ A, int64_t lda,
                                                       const float* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                                       int64_t ldc, int vec, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + kABytes;
    unsigned char* b_hi = smem + 2 * kABytes;
    unsigned char* b_lo = smem + 2 * kABytes + kBBytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kABytes + 2 * kBBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kABytes + 2 * kBBytes + 16);

    const int64_t m0 = (int64_t)blockIdx.x * kTM;
    const int64_t tiles_n = (N + kTN - 1) / kTN;
    const int64_t t0 = (int64_t)blockIdx.y * kTilesN;
    const int nt = (int)min((int64_t)kTilesN, tiles_n - t0);
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool full_m = m0 + kTM <= M;

    // ---- stage A (128 rows x 64 k, column-major source) once
    if (vec && full_m) {
        float4 va[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k = tid / 32 + 4 * j;
            va[j] = *reinterpret_cast<const float4*>(A + m0 + 4 * (tid % 32) + (int64_t)k * lda);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k = tid / 32 + 4 * j, r = 4 * (tid % 32);
            put_pair(a_hi, a_lo, kmajor_off(r, k), va[j].x);
            put_pair(a_hi, a_lo, kmajor_off(r + 1, k), va[j].y);
            put_pair(a_hi, a_lo, kmajor_off(r + 2, k), va[j].z);
            put_pair(a_hi, a_lo, kmajor_off(r + 3, k), va[j].w);
        }
    } else {
        for (int idx = tid; idx < kTM * kTK; idx += 128) {
            const int r = idx % kTM, k = idx / kTM;
            const int64_t gm = m0 + r;
            put_pair(a_hi, a_lo, kmajor_off(r, k), (gm < M) ? A[gm + (int64_t)k * lda] : 0.f);
        }
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const int64_t row = m0 + warp * 32 + (tid & 31);

    int ok = 1;
    for (int t = 0; t < nt; ++t) {
        const int64_t n0 = (t0 + t) * kTN;
        // the MMAs of tile t-1 have completed (waited below), so B may be overwritten
        stage_b(B, ldb, N, n0, vec && full_m && (n0 + kTN <= N), b_hi, b_lo, tid);
        // make the generic-proxy smem writes visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t col0 = (uint32_t)(t & 1) * (uint32_t)kTN;
        // ---- 24 MMAs from one thread into accumulator t & 1: lo*hi, hi*lo, hi*hi, 8 K-steps
        if (tid == 0) {
            const unsigned char* As[3] = {a_lo, a_hi, a_hi};
            const unsigned char* Bs[3] = {b_hi, b_lo, b_hi};
            uint32_t first = 1;
            for (int q = 0; q < 3; ++q) {
                for (int ks = 0; ks < kTK / 8; ++ks) {
                    const uint64_t ad = make_desc(smem_u32(As[q]) + (uint32_t)ks * 2u * kLBO);
                    const uint64_t bd = make_desc(smem_u32(Bs[q]) + (uint32_t)ks * 2u * kLBO);
                    const uint32_t acc = first ? 0u : 1u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + col0),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                    first = 0;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar)));
        }
        // ---- write back tile t-1 while the tensor core works on tile t
        if (t > 0) epilogue(C, ldc, M, N, row, n0 - kTN, tmem, (uint32_t)((t - 1) & 1) * (uint32_t)kTN, warp);
        // ---- bounded wait for the MMAs of tile t (the t-th completion: parity t & 1)
        uint32_t done = 0;
        const uint32_t parity = (uint32_t)(t & 1);
        for (long long it = 0; it < kSpinLimit && !done; ++it) {
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(smem_u32(mbar)), "r"(parity));
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        ok = __syncthreads_and((int)done);
        if (!ok) break;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else if (nt > 0) {
        epilogue(C, ldc, M, N, row, (t0 + nt - 1) * kTN, tmem, (uint32_t)((nt - 1) & 1) * (uint32_t)kTN, warp);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTN));
}

// ---------------------------------------------------------------- bulk-asynchronous path
// Operands are split once per panel (k_split_ab) into TF32 hi/lo tiles already in the UMMA
// K-major layout, A negated, so a CTA moves them with single bulk copies and the MMAs
// accumulate -A B.  C is never loaded by the SMs: each finished 128 x 64 product tile goes
// from tensor memory to shared memory and is added to C by a TMA reduce-add (a 2-D tensor
// map over C; the read-modify-write happens in L2, out-of-range elements are skipped).
// c + (-v) rounds exactly like c - v, so the factors equal those of the register-staged
// kernel.  One CTA per SM walks tiles_per_cta column tiles of its 128-row strip:
//   smem  A hi/lo (64 KB) | B hi/lo x 2 buffers (64 KB) | product x 2 buffers (64 KB) | barriers
//   tile t: wait B(t) -> 24 MMAs into accumulator t & 1; wait MMAs(t-1) -> prefetch B(t+1);
//           product(t-1) -> shared buffer (t-1) & 1 (once the reduce of tile t-3 has read
//           it) -> TMA reduce-add into C.
constexpr uint32_t kASplit = 2 * kABytes;            // 64 KB per 128-row operand tile
constexpr uint32_t kBSplit = 2 * kBBytes;            // 32 KB per 64-column operand tile
constexpr uint32_t kCTile = kTM * kTN * 4;           // 32 KB
constexpr uint32_t kBulkSmem = kASplit + 2 * kBSplit + 2 * kCTile + 128;

__device__ __forceinline__ void mbar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)));
}
__device__ __forceinline__ void mbar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// bounded wait for completion `parity` of barrier b; 1 = completed
__device__ __forceinline__ int mbar_wait(uint64_t* b, uint32_t parity) {
    uint32_t done = 0;
    for (long long it = 0; it < kSpinLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
    }
    return (int)done;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}
__device__ __forceinline__ void tma_reduce_add_c(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// -A (M x K, column-major) and B (K x N) into TF32 hi/lo operand tiles, in kc chunks of 64
// along K (K <= 64 kc): A tile (tm, chunk c) at asplit + (tm kc + c) * 64 KB (hi, then lo),
// B tile (tn, c) at bsplit + (tn kc + c) * 32 KB; rows of A beyond M, columns of B beyond
// N and depths beyond K are zero.  The TF32 split of -x is the negated split of x.
__global__ void k_split_ab(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
                           int64_t M, int64_t N, int64_t K, int kc, int64_t tiles_m, int64_t tiles_n,
                           unsigned char* __restrict__ asplit, unsigned char* __restrict__ bsplit) {
    const int64_t na = tiles_m * kc * (kTM * kTK), nb = tiles_n * kc * (kTN * kTK);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na + nb;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < na) {
            const int64_t tc = idx / (kTM * kTK);  // tm * kc + c
            const int e = (int)(idx - tc * (kTM * kTK));
            const int r = e % kTM, k = e / kTM;
            const int64_t gm = (tc / kc) * kTM + r, gk = (tc % kc) * kTK + k;
            const float x = (gm < M && gk < K) ? -A[gm + gk * lda] : 0.f;
            unsigned char* t = asplit + tc * kASplit;
            put_pair(t, t + kABytes, kmajor_off(r, k), x);
        } else {
            const int64_t i2 = idx - na;
            const int64_t tc = i2 / (kTN * kTK);  // tn * kc + c
            const int e = (int)(i2 - tc * (kTN * kTK));
            const int k = e % kTK, col = e / kTK;
            const int64_t gn = (tc / kc) * kTN + col, gk = (tc % kc) * kTK + k;
            const float x = (gn < N && gk < K) ? B[gk + gn * ldb] : 0.f;
            unsigned char* t = bsplit + tc * kBSplit;
            put_pair(t, t + kBBytes, kmajor_off(col, k), x);
        }
    }
}

__global__ void __launch_bounds__(128, 1)
    k_tc_update_bulk(const __grid_constant__ CUtensorMap cmap, int64_t M, int64_t N,
                     const unsigned char* __restrict__ asplit, const unsigned char* __restrict__ bsplit, int tpc,
                     int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB0 = smem + kASplit;
    unsigned char* sP0 = smem + kASplit + 2 * kBSplit;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kASplit + 2 * kBSplit + 2 * kCTile);
    uint64_t* barA = bar;
    uint64_t* barB = bar + 1;  // [2]
    uint64_t* barM = bar + 3;  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 6);

    const int64_t tiles_n = (N + kTN - 1) / kTN;
    const int64_t t0 = (int64_t)blockIdx.y * tpc;
    const int nt = (int)min((int64_t)tpc, tiles_n - t0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = (int)(blockIdx.x * kTM);
    auto sB = [&](int s) { return sB0 + s * kBSplit; };
    auto sP = [&](int s) { return reinterpret_cast<float*>(sP0 + s * kCTile); };
    auto load_b = [&](int t) {
        const int s = t & 1;
        mbar_expect(barB + s, kBSplit);
        bulk_load(sB(s), bsplit + (t0 + t) * (int64_t)kBSplit, kBSplit, barB + s);
    };

    if (tid == 0) {
        for (int b = 0; b < 5; ++b) mbar_init(bar + b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(barA, kASplit);
        bulk_load(sA, asplit + (int64_t)blockIdx.x * kASplit, kASplit, barA);
        if (nt > 0) load_b(0);
        if (nt > 1) load_b(1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    // completions consumed per barrier (the next wait's parity), loads / commits issued
    int used_b0 = 0, used_b1 = 0, used_m0 = 0, used_m1 = 0;
    int iss_b0 = nt > 0, iss_b1 = nt > 1, iss_m0 = 0, iss_m1 = 0, a_used = 0;
    int ok = 1;

    // product tile t (accumulator t & 1 = -(A B) for the tile) -> shared buffer t & 1 -> reduce-add into C
    auto finish_tile = [&](int t) -> int {
        const int s = t & 1;
        int& used_m = s ? used_m1 : used_m0;
        int w = mbar_wait(barM + s, (uint32_t)(used_m & 1));
        if (!__syncthreads_and(w)) return 0;
        ++used_m;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // the MMAs of tile t have read B buffer s: prefetch B(t + 2); the reduce of tile
        // t - 2 must have read product buffer s before it is rewritten
        if (tid == 0) {
            if (t + 2 < nt) {
                load_b(t + 2);
                (s ? iss_b1 : iss_b0)++;
            }
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        }
        __syncthreads();
        float* pbuf = sP(s);
        const int r = warp * 32 + lane;
#pragma unroll
        for (int cb = 0; cb < kTN; cb += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kTN + cb);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) pbuf[(cb + j) * kTM + r] = __uint_as_float(v[j]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) tma_reduce_add_c(&cmap, m0, (int)((t0 + t) * kTN), pbuf);
        return 1;
    };

    for (int t = 0; t < nt && ok; ++t) {
        const int s = t & 1;
        int& used_b = s ? used_b1 : used_b0;
        int w = mbar_wait(barB + s, (uint32_t)(used_b & 1));
        if (t == 0) w = w && mbar_wait(barA, 0);
        if (!__syncthreads_and(w)) {
            ok = 0;
            break;
        }
        ++used_b;
        a_used = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const unsigned char* As[3] = {sA + kABytes, sA, sA};
            const unsigned char* Bs[3] = {sB(s), sB(s) + kBBytes, sB(s)};
            uint32_t first = 1;
            for (int q = 0; q < 3; ++q) {
                for (int ks = 0; ks < kTK / 8; ++ks) {
                    const uint64_t ad = make_desc(smem_u32(As[q]) + (uint32_t)ks * 2u * kLBO);
                    const uint64_t bd = make_desc(smem_u32(Bs[q]) + (uint32_t)ks * 2u * kLBO);
                    const uint32_t acc = first ? 0u : 1u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(s * kTN)),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                    first = 0;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(barM + s)));
        }
        (s ? iss_m1 : iss_m0)++;
        if (t > 0 && !finish_tile(t - 1)) ok = 0;
    }
    if (ok && nt > 0 && !finish_tile(nt - 1)) ok = 0;

    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // let every transfer and MMA this CTA started finish (bounded) before its shared
        // and tensor memory go away
        if (tid == 0) {
            if (!a_used) mbar_wait(barA, 0);
            if (iss_b0 > used_b0) mbar_wait(barB, (uint32_t)(used_b0 & 1));
            if (iss_b1 > used_b1) mbar_wait(barB + 1, (uint32_t)(used_b1 & 1));
            if (iss_m0 > used_m0) mbar_wait(barM, (uint32_t)(used_m0 & 1));
            if (iss_m1 > used_m1) mbar_wait(barM + 1, (uint32_t)(used_m1 & 1));
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTN));
}

// ---- rank-K update in one pass over C (K <= 256): the trailing update of a super-panel.
// Wide tiles: each MMA is M = 128 x N = 256 x K = 8 (a 64-wide tile leaves the tensor core
// mostly idle).  Operands are split in chunks of 16 along K (canonical K-major layout,
// SBO = 512 B): A tile (tm, chunk c) 16 KB (hi 8 KB, lo 8 KB), B tile (256-column tile
// tn, c) 32 KB (hi 16 KB, lo 16 KB).
constexpr int kKT = 16;                                    // chunk depth
constexpr int kTW = 256;                                   // columns per accumulator tile
constexpr uint32_t kSBO16 = (kKT / 4) * kCoreBytes;        // 512 B
constexpr uint32_t kABytes16 = kTM * kKT * 4;              // 8 KB
constexpr uint32_t kBBytes16 = kTW * kKT * 4;              // 16 KB
constexpr uint32_t kASplit16 = 2 * kABytes16;              // 16 KB
constexpr uint32_t kBSplit16 = 2 * kBBytes16;              // 32 KB
// instruction descriptor as kIdesc, N = 256
constexpr uint32_t kIdescW = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTW >> 3) << 17) |
                             ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ uint32_t kmajor_off16(int r, int k) {
    return (uint32_t)(r >> 3) * kSBO16 + (uint32_t)(k >> 2) * kLBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 3) * 4u;
}
__device__ __forceinline__ uint64_t make_desc16(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kLBO >> 4) << 16;
    d |= (uint64_t)(kSBO16 >> 4) << 32;
    d |= 1ull << 46;
    return d;
}

// -A (M x K) and B (K x N) into 16-deep TF32 hi/lo tiles, kc = ceil(K / 16) chunks: A tile
// (tm, c) at asplit + (tm kc + c) * 16 KB, B tile (tn, c) (256 columns) at
// bsplit + (tn kc + c) * 32 KB; entries beyond M, N or K are zero.
__global__ void k_split_ab16(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
                             int64_t M, int64_t N, int64_t K, int kc, int64_t tiles_m, int64_t tiles_n,
                             unsigned char* __restrict__ asplit, unsigned char* __restrict__ bsplit) {
    const int64_t na = tiles_m * kc * (kTM * kKT), nb = tiles_n * kc * (kTW * kKT);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na + nb;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < na) {
            const int64_t tc = idx / (kTM * kKT);  // tm * kc + c
            const int e = (int)(idx - tc * (kTM * kKT));
            const int r = e % kTM, k = e / kTM;
            const int64_t gm = (tc / kc) * kTM + r, gk = (tc % kc) * kKT + k;
            const float x = (gm < M && gk < K) ? -A[gm + gk * lda] : 0.f;
            unsigned char* t = asplit + tc * kASplit16;
            put_pair(t, t + kABytes16, kmajor_off16(r, k), x);
        } else {
            const int64_t i2 = idx - na;
            const int64_t tc = i2 / (kTW * kKT);  // tn * kc + c
            const int e = (int)(i2 - tc * (kTW * kKT));
            const int k = e % kKT, col = e / kKT;
            const int64_t gn = (tc / kc) * kTW + col, gk = (tc % kc) * kKT + k;
            const float x = (gn < N && gk < K) ? B[gk + gn * ldb] : 0.f;
            unsigned char* t = bsplit + tc * kBSplit16;
            put_pair(t, t + kBBytes16, kmajor_off16(col, k), x);
        }
    }
}

// One CTA per SM owns a 128-row strip of C and nt <= kAccTiles 256-column tiles, each with
// its own accumulator (up to all 512 TMEM columns), so C is read and written once for the
// whole depth instead of once per panel.  Work items (chunk c, tile t) run chunk-major,
// i = c nt + t; an item is 6 MMAs (lo hi, hi lo, hi hi over 2 steps of 8) into
// accumulator t, overwriting it at c = 0.  Warp-specialised, no block barrier in the
// steady state:
//   warp 4 (one lane)  producer: A chunks into a ring of kRA slots (16 KB), B items into a
//                      ring of kRB slots (32 KB), each slot refilled once emptyA / emptyB
//                      says the MMAs that read it are done;
//   warp 5 (one lane)  MMA issue: waits fullB (and fullA at t = 0), issues the item,
//                      commits to emptyB, to emptyA when it closes a chunk, and to accf[t]
//                      when it is of the last chunk;
//   warps 0-3          epilogue (warp w reads TMEM lanes 32w..): per tile, waits accf[t],
//                      moves the accumulator 64 columns at a time through the product
//                      buffer (once the previous reduce has read it; a named barrier among
//                      these four warps) into TMA reduce-adds into C.
// The u-th use of a ring slot completes its phase u, so every wait's parity follows from
// the item or chunk number.  Waits are bounded: a role that gives up records *err and
// raises the CTA's abort flag, the others stop at their next step; before the tensor
// memory is freed, every copy and MMA that was started is waited for (bounded).
constexpr int kAccTiles = 2;
constexpr int kRA = 4, kRB = 4;
constexpr int kUpdThreads = 192;
constexpr uint32_t kKSmem = kRA * kASplit16 + kRB * kBSplit16 + kCTile + 512;

__device__ __forceinline__ void named_sync_epilogue() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// barrier 1 among the 128 epilogue threads, returning the OR of v over them (the same
// value in every one of them)
__device__ __forceinline__ int named_sync_or_epilogue(int v) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v)
        : "memory");
    return r;
}
// bounded wait that also gives up once the CTA's abort flag is raised
__device__ __forceinline__ int mbar_wait_ab(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    uint32_t done = 0;
    for (long long it = 0; it < kSpinLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
        if (!done && (it & 63) == 63 && *abort_flag) return 0;
    }
    return (int)done;
}

__global__ void __launch_bounds__(kUpdThreads, 1)
    k_tc_update_k(const __grid_constant__ CUtensorMap cmap, int64_t M, int64_t N, int kc,
                  const unsigned char* __restrict__ asplit, const unsigned char* __restrict__ bsplit, int tpc,
                  int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA0 = smem;
    unsigned char* sB0 = smem + kRA * kASplit16;
    float* pbuf = reinterpret_cast<float*>(smem + kRA * kASplit16 + kRB * kBSplit16);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kRA * kASplit16 + kRB * kBSplit16 + kCTile);
    uint64_t* fullA = bar;                 // [kRA]
    uint64_t* emptyA = bar + kRA;          // [kRA]
    uint64_t* fullB = bar + 2 * kRA;       // [kRB]
    uint64_t* emptyB = bar + 2 * kRA + kRB;  // [kRB]
    uint64_t* accf = bar + 2 * kRA + 2 * kRB;  // [kAccTiles]
    constexpr int kBars = 2 * kRA + 2 * kRB + kAccTiles;
    int* sh = reinterpret_cast<int*>(bar + kBars);  // tmem address, abort, progress counters
    volatile int* abort_flag = sh + 1;
    int* prog = sh + 2;  // loadsA, loadsB, waitedA, waitedB, issued

    const int64_t tiles_n = (N + kTW - 1) / kTW;
    const int64_t t0 = (int64_t)blockIdx.y * tpc;
    const int nt = (int)max((int64_t)0, min((int64_t)tpc, tiles_n - t0));
    const int items = nt * kc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = (int)(blockIdx.x * kTM);
    uint32_t ncols = 64;  // tensor-memory columns: a power of two >= nt * 256
    while (ncols < (uint32_t)(nt * kTW)) ncols *= 2;
    auto fail = [&]() {
        atomicExch(err, 1);
        *abort_flag = 1;
    };

    if (tid == 0) {
        for (int b = 0; b < kBars; ++b) mbar_init(bar + b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
        for (int q = 0; q < 5; ++q) prog[q] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sh)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = static_cast<uint32_t>(sh[0]);

    if (warp == 4) {
        // ---- producer
        if (lane == 0) {
            int la = 0, lb = 0;
            for (int i = 0; i < items && !*abort_flag; ++i) {
                const int c = i / nt, t = i - c * nt;
                if (t == 0) {
                    const int a = c % kRA;
                    if (c >= kRA && !mbar_wait_ab(emptyA + a, (uint32_t)(((c / kRA) - 1) & 1), abort_flag)) {
                        fail();
                        break;
                    }
                    mbar_expect(fullA + a, kASplit16);
                    bulk_load(sA0 + a * kASplit16, asplit + ((int64_t)blockIdx.x * kc + c) * kASplit16, kASplit16,
                              fullA + a);
                    la = c + 1;
                }
                const int b = i % kRB;
                if (i >= kRB && !mbar_wait_ab(emptyB + b, (uint32_t)(((i / kRB) - 1) & 1), abort_flag)) {
                    fail();
                    break;
                }
                mbar_expect(fullB + b, kBSplit16);
                bulk_load(sB0 + b * kBSplit16, bsplit + ((t0 + t) * kc + c) * (int64_t)kBSplit16, kBSplit16,
                          fullB + b);
                lb = i + 1;
            }
            prog[0] = la;
            prog[1] = lb;
        }
    } else if (warp == 5) {
        // ---- MMA issue
        if (lane == 0) {
            int wa = 0, wb = 0, iss = 0;
            for (int i = 0; i < items && !*abort_flag; ++i) {
                const int c = i / nt, t = i - c * nt;
                const int a = c % kRA, b = i % kRB;
                if (!mbar_wait_ab(fullB + b, (uint32_t)((i / kRB) & 1), abort_flag)) {
                    fail();
                    break;
                }
                wb = i + 1;
                if (t == 0) {
                    if (!mbar_wait_ab(fullA + a, (uint32_t)((c / kRA) & 1), abort_flag)) {
                        fail();
                        break;
                    }
                    wa = c + 1;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned char* sA = sA0 + a * kASplit16;
                const unsigned char* sB = sB0 + b * kBSplit16;
                const unsigned char* As[3] = {sA + kABytes16, sA, sA};
                const unsigned char* Bs[3] = {sB, sB + kBBytes16, sB};
                uint32_t first = (c == 0) ? 1u : 0u;
                for (int q = 0; q < 3; ++q) {
                    for (int ks = 0; ks < kKT / 8; ++ks) {
                        const uint64_t ad = make_desc16(smem_u32(As[q]) + (uint32_t)ks * 2u * kLBO);
                        const uint64_t bd = make_desc16(smem_u32(Bs[q]) + (uint32_t)ks * 2u * kLBO);
                        const uint32_t acc = first ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)(t * kTW)),
                            "l"(ad), "l"(bd), "r"(kIdescW), "r"(acc));
                        first = 0;
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(emptyB + b)));
                if (t == nt - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(emptyA + a)));
                if (c == kc - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(accf + t)));
                iss = i + 1;
            }
            prog[2] = wa;
            prog[3] = wb;
            prog[4] = iss;
        }
    } else {
        // ---- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31 = rows of the strip
        const int r = warp * 32 + lane;
        for (int t = 0; t < nt; ++t) {
            const int w = mbar_wait_ab(accf + t, 0u, abort_flag);
            if (!w && !*abort_flag) fail();
            // one decision for all four warps (the flag may be raised between their reads)
            if (named_sync_or_epilogue(!w || *abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int pc = 0; pc < kTW / kTN; ++pc) {
                const int64_t col0 = (t0 + t) * kTW + pc * kTN;
                if (col0 >= N) break;  // the same for every epilogue thread
                // the previous piece's reduce-add has read the product buffer
                if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                named_sync_epilogue();
#pragma unroll
                for (int cb = 0; cb < kTN; cb += 32) {
                    uint32_t v[32];
                    const uint32_t taddr =
                        tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * kTW + pc * kTN + cb);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
                        "%30, %31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 32; ++q) pbuf[(cb + q) * kTM + r] = __uint_as_float(v[q]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                named_sync_epilogue();
                if (tid == 0) tma_reduce_add_c(&cmap, m0, (int)col0, pbuf);
            }
        }
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    // before the shared and tensor memory go away: every copy that was started has landed
    // (loads no MMA waited for, after an abort), and every commit the MMA thread issued has
    // arrived (the last use of each ring slot and accumulator is waited for by no one else)
    if (tid == 128 && *abort_flag) {
        for (int c = prog[2]; c < prog[0]; ++c) mbar_wait(fullA + c % kRA, (uint32_t)((c / kRA) & 1));
        for (int i = prog[3]; i < prog[1]; ++i) mbar_wait(fullB + i % kRB, (uint32_t)((i / kRB) & 1));
    }
    if (tid == 160) {
        const int iss = prog[4], closed = nt > 0 ? iss / nt : 0;
        for (int j = max(0, iss - kRB); j < iss; ++j) mbar_wait(emptyB + j % kRB, (uint32_t)((j / kRB) & 1));
        for (int c = max(0, closed - kRA); c < closed; ++c) mbar_wait(emptyA + c % kRA, (uint32_t)((c / kRA) & 1));
        for (int t = 0; t < nt; ++t)
            if ((kc - 1) * nt + t < iss) mbar_wait(accf + t, 0u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

size_t tc_split_bytes(int64_t M, int64_t N, int kc) {
    // kc 64-deep chunks; B counted in whole 256-column tiles, which covers both layouts
    return ((size_t)((M + kTM - 1) / kTM) * kASplit + (size_t)((N + kTW - 1) / kTW) * 4 * kBSplit) * (size_t)kc;
}

cudaError_t tc_update_f32(int64_t M, int64_t N, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                          int64_t ldc, void* split, int* err, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // bulk-asynchronous path: C rows in 16-byte units (TMA strides and coordinates)
    EncodeTiledFn enc = split ? encode_tiled() : nullptr;
    if (enc && (ldc % 4) == 0 && (((uintptr_t)C & 15) == 0) && M <= INT32_MAX && N <= INT32_MAX) {
        CUtensorMap map;
        const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)N};
        const cuuint64_t strides[1] = {(cuuint64_t)ldc * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kTM, (cuuint32_t)kTN};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
            const int64_t tiles_m = (M + kTM - 1) / kTM, tiles_n = (N + kTN - 1) / kTN;
            unsigned char* asplit = static_cast<unsigned char*>(split);
            unsigned char* bsplit = asplit + (size_t)tiles_m * kASplit;
            const int64_t total = tiles_m * kTM * kTK + tiles_n * kTN * kTK;
            k_split_ab<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(
                A, lda, B, ldb, M, N, kTK, 1, tiles_m, tiles_n, asplit, bsplit);
            cudaError_t e = cudaFuncSetAttribute(k_tc_update_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kBulkSmem);
            if (e != cudaSuccess) return e;
            // column tiles per CTA: enough CTAs for two waves of the SMs, at most 16 tiles each
            int64_t tpc = (tiles_m * tiles_n) / (2 * 152);
            tpc = std::max<int64_t>(1, std::min<int64_t>(16, tpc));
            dim3 grid((unsigned)tiles_m, (unsigned)((tiles_n + tpc - 1) / tpc));
            k_tc_update_bulk<<<grid, 128, kBulkSmem, s>>>(map, M, N, asplit, bsplit, (int)tpc, err);
            return cudaGetLastError();
        }
    }
    // set for the current device on every call (an attribute is per device)
    cudaError_t e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // vector loads need 16-byte aligned columns
    const int vec = (lda % 4 == 0) && (ldb % 4 == 0) && (((uintptr_t)A & 15) == 0) && (((uintptr_t)B & 15) == 0);
    const int64_t tiles_n = (N + kTN - 1) / kTN;
    dim3 grid((unsigned)((M + kTM - 1) / kTM), (unsigned)((tiles_n + kTilesN - 1) / kTilesN));
    k_tc_update<<<grid, 128, kSmemBytes, s>>>(M, N, A, lda, B, ldb, C, ldc, vec, err);
    return cudaGetLastError();
}

cudaError_t tc_update_f32_k(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                            int64_t ldb, float* C, int64_t ldc, void* split, int* err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const int kc = (int)((K + kKT - 1) / kKT);  // 16-deep chunks
    EncodeTiledFn enc = split ? encode_tiled() : nullptr;
    if (K <= 256 && enc && (ldc % 4) == 0 && (((uintptr_t)C & 15) == 0) && M <= INT32_MAX && N <= INT32_MAX) {
        CUtensorMap map;
        const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)N};
        const cuuint64_t strides[1] = {(cuuint64_t)ldc * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kTM, (cuuint32_t)kTN};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
            const int64_t tiles_m = (M + kTM - 1) / kTM, tiles_n = (N + kTW - 1) / kTW;
            unsigned char* asplit = static_cast<unsigned char*>(split);
            unsigned char* bsplit = asplit + (size_t)tiles_m * kc * kASplit16;
            const int64_t total = (tiles_m * kTM * kKT + tiles_n * kTW * kKT) * kc;
            k_split_ab16<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(
                A, lda, B, ldb, M, N, K, kc, tiles_m, tiles_n, asplit, bsplit);
            cudaError_t e =
                cudaFuncSetAttribute(k_tc_update_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKSmem);
            if (e != cudaSuccess) return e;
            // column tiles per CTA: enough CTAs for two waves of the SMs, at most kAccTiles
            int64_t tpc = (tiles_m * tiles_n) / (2 * 152);
            tpc = std::max<int64_t>(1, std::min<int64_t>(kAccTiles, tpc));
            dim3 grid((unsigned)tiles_m, (unsigned)((tiles_n + tpc - 1) / tpc));
            k_tc_update_k<<<grid, kUpdThreads, kKSmem, s>>>(map, M, N, kc, asplit, bsplit, (int)tpc, err);
            return cudaGetLastError();
        }
    }
    // no bulk path: one rank-64 pass per chunk
    for (int64_t k0 = 0; k0 < K; k0 += kTK) {
        const int64_t kw = std::min<int64_t>(kTK, K - k0);
        if (kw != kTK) return cudaErrorInvalidValue;
        cudaError_t e = tc_update_f32(M, N, A + k0 * lda, lda, B + k0, ldb, C, ldc, split, err, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace nb
