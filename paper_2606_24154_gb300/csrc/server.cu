// server.cu -- persistent batched evaluation kernel of the field-query server.
//
// Work items (up to kEvalThreads points of one request) are published by the host into
// a ring in host-mapped memory: the host writes the items, then advances `tail` with a
// release store.  Each CTA claims the next item with a CAS on a device-memory `head`,
// evaluates its points with the same block bodies as the standalone kernels (so a
// request's results do not depend on which requests share the launch), and decrements
// the request's remaining-item count; the CTA that finishes the last item publishes the
// request's generation number to a host-mapped completion word.
//
// Every wait is bounded: a CTA that finds no claimable item for `idle_ns` (read from
// %globaltimer) exits, and the kernel ends when all CTAs have; the host relaunches it
// when new work arrives.  No CTA ever waits on another.
#include <cuda/atomic>

#include "eval_blocks.cuh"
#include "server_internal.h"

namespace nb {

namespace {

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kEvalThreads) k_serve(const ServeGeom* __restrict__ geoms, const WorkItem* ring,
                                                        int64_t ring_cap, int64_t* tail_mapped,
                                                        unsigned long long* head, const double* __restrict__ arena_pts,
                                                        double* __restrict__ arena_phi, double* __restrict__ arena_E,
                                                        int* remaining, int64_t* done_mapped, uint64_t idle_ns) {
    __shared__ WorkItem it;
    __shared__ int have;
    for (;;) {
        if (threadIdx.x == 0) {
            have = 0;
            const uint64_t t0 = global_ns();
            cuda::atomic_ref<int64_t, cuda::thread_scope_system> tail(*tail_mapped);
            for (;;) {
                const int64_t t = tail.load(cuda::memory_order_acquire);
                const unsigned long long h = atomicAdd(head, 0ull);
                if ((int64_t)h < t) {
                    if (atomicCAS(head, h, h + 1) == h) {
                        it = ring[h % (unsigned long long)ring_cap];
                        have = 1;
                        break;
                    }
                    continue;
                }
                if (global_ns() - t0 > idle_ns) break;
                __nanosleep(2000);
            }
        }
        __syncthreads();
        if (!have) return;
        const ServeGeom& G = geoms[it.geom];
        const double* pts = arena_pts + 3 * it.offset;
        double* phi = arena_phi + it.offset;
        double* E = arena_E + 3 * it.offset;
        if (it.precision == NEBEM_MIXED) {
            far_block(G.view, arena_pts, nullptr, it.offset, it.count, arena_phi, arena_E);
            if ((int)threadIdx.x < it.count) near_point(G.view, G.img, arena_pts, it.offset + threadIdx.x, arena_phi, arena_E);
        } else {
            f64_block(G.view.el, G.view.sigma, G.view.n_el, G.img, pts, it.count, phi, E);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicSub(&remaining[it.slot], 1) == 1) {
                __threadfence_system();
                cuda::atomic_ref<int64_t, cuda::thread_scope_system> d(done_mapped[it.slot]);
                d.store(it.gen, cuda::memory_order_release);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_serve(const ServeGeom* geoms, const WorkItem* ring, int64_t ring_cap, int64_t* tail_mapped,
                         unsigned long long* head, const double* arena_pts, double* arena_phi, double* arena_E,
                         int* remaining, int64_t* done_mapped, uint64_t idle_ns, int workers, cudaStream_t s) {
    k_serve<<<workers, kEvalThreads, 0, s>>>(geoms, ring, ring_cap, tail_mapped, head, arena_pts, arena_phi, arena_E,
                                             remaining, done_mapped, idle_ns);
    return cudaGetLastError();
}

ServeGeom make_serve_geom(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma, int64_t n_el,
                          const ImageTable& img, const NearGrid& grid, const int32_t* cell_start,
                          const int32_t* cell_items) {
    ServeGeom g;
    g.view = make_view(el, far, cjk, sigma, n_el, img, grid, cell_start, cell_items);
    g.img = img;
    return g;
}

}  // namespace nb
