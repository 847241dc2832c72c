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
// Every wait is bounded.  A CTA that has found no claimable item for `idle_ns` (read from
// %globaltimer), at a moment when every item claimed so far has finished (head[1] counts
// finished items), closes the launch: it sets head[2], and every CTA that sees it leaves
// without claiming more, so the whole kernel ends and the host relaunches it, with all its
// CTAs, when new work arrives (items published meanwhile wait in the ring for that
// launch).  Leaving together matters: if CTAs left one by one, a trickle of requests could
// keep a few of them, and so the kernel, alive, and no relaunch would restore the rest.
// While any item is still being evaluated, idle CTAs stay.  No CTA ever waits on another:
// an item's processing has no waits of its own.  Idle polls of the host-mapped tail back
// off from 1 to 32 us.
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

static_assert(kChunkElements == kChunkEl, "server chunk width must match the evaluation bodies");

__global__ void __launch_bounds__(kEvalThreads) k_serve(const ServeGeom* __restrict__ geoms, const WorkItem* ring,
                                                        int64_t ring_cap, int64_t* tail_mapped,
                                                        unsigned long long* head, const double* __restrict__ arena_pts,
                                                        double* __restrict__ arena_phi, double* __restrict__ arena_E,
                                                        float4* __restrict__ arena_bound, int* remaining, int64_t* done_mapped, double* partials,
                                                        int* pblock_count, int max_chunks, uint64_t idle_ns) {
    __shared__ WorkItem it;
    __shared__ int have;
    __shared__ int last;
    for (;;) {
        if (threadIdx.x == 0) {
            have = 0;
            uint64_t t0 = global_ns();
            unsigned sleep_ns = 1000;  // back-off between polls of the host-mapped tail
            cuda::atomic_ref<int64_t, cuda::thread_scope_system> tail(*tail_mapped);
            for (;;) {
                if (atomicAdd(head + 2, 0ull) != 0ull) break;  // the launch is closing
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
                if (global_ns() - t0 > idle_ns) {
                    if (atomicAdd(head + 1, 0ull) >= h) {  // every claimed item has finished
                        atomicExch(head + 2, 1ull);        // close the launch for every CTA
                        break;
                    }
                    t0 = global_ns();  // items still in progress: stay for what may arrive
                }
                __nanosleep(sleep_ns);
                sleep_ns = min(2u * sleep_ns, 32000u);
            }
        }
        __syncthreads();
        if (!have) return;
        const ServeGeom& G = geoms[it.geom];
        bool block_done = true;
        const bool mixed = it.precision == NEBEM_MIXED;
        if (it.chunk < 0 && !mixed) {
            f64_block(G.view.el, G.view.sigma, G.view.n_el, G.img, arena_pts + 3 * it.offset, it.count,
                      arena_phi + it.offset, arena_E + 3 * it.offset);
        } else if (it.chunk < 0) {
            far_block(G.view, arena_pts, nullptr, it.offset, it.count, arena_phi, arena_E, arena_bound);
            if ((int)threadIdx.x < it.count)
                near_point(G.view, G.img, arena_pts, it.offset + threadIdx.x, arena_phi, arena_E);
        } else {
            // one element chunk of a point block: raw sums to the partial area; the CTA that
            // finishes the block's last chunk adds the chunks in order (as far_block and
            // f64_block do), stores ke * sum and (mixed) adds the near pairs
            const bool active = (int)threadIdx.x < it.count;
            const int64_t p = it.offset + threadIdx.x;
            const int64_t e0 = (int64_t)it.chunk * kChunkEl;
            const int64_t e1 = min(e0 + (int64_t)kChunkEl, G.view.n_el);
            Sum4 c;
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mixed) {
                float phx, phy, phz, plx, ply, plz;
                load_point_2f(arena_pts, p, active, phx, phy, phz, plx, ply, plz);
                bound_reset();
                c = far_range(G.view, phx, phy, phz, plx, ply, plz, e0, e1);
                b = *bound_slot();
            } else {
                const double Px = active ? arena_pts[3 * p] : 0.0, Py = active ? arena_pts[3 * p + 1] : 0.0,
                             Pz = active ? arena_pts[3 * p + 2] : 0.0;
                c = f64_range(G.view.el, G.view.sigma, e0, e1, G.img, Px, Py, Pz);
            }
            constexpr int kP = kPartialDoubles;
            double* part = partials + ((int64_t)it.pblock * max_chunks + it.chunk) * (kP * kEvalThreads);
            part[kP * threadIdx.x] = c.phi;
            part[kP * threadIdx.x + 1] = c.x;
            part[kP * threadIdx.x + 2] = c.y;
            part[kP * threadIdx.x + 3] = c.z;
            part[kP * threadIdx.x + 4] = (double)b.x;  // exact
            part[kP * threadIdx.x + 5] = (double)b.y;
            part[kP * threadIdx.x + 6] = (double)b.z;
            part[kP * threadIdx.x + 7] = (double)b.w;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) last = (atomicAdd(&pblock_count[it.pblock], 1) == it.nchunks - 1);
            __syncthreads();
            block_done = last;
            if (last) {
                __threadfence();
                Sum4 tot{0.0, 0.0, 0.0, 0.0};
                float4 btot = make_float4(0.f, 0.f, 0.f, 0.f);  // FP32 sums in chunk order, as far_block
                for (int k = 0; k < it.nchunks; ++k) {
                    const double* q = partials + ((int64_t)it.pblock * max_chunks + k) * (kP * kEvalThreads) +
                                      kP * threadIdx.x;
                    tot.phi += __ldcg(q);
                    tot.x += __ldcg(q + 1);
                    tot.y += __ldcg(q + 2);
                    tot.z += __ldcg(q + 3);
                    btot.x += (float)__ldcg(q + 4);
                    btot.y += (float)__ldcg(q + 5);
                    btot.z += (float)__ldcg(q + 6);
                    btot.w += (float)__ldcg(q + 7);
                }
                if (active) {
                    store_far(arena_pts, arena_phi, arena_E, p, tot);
                    if (mixed) store_bound(arena_bound, p, btot);
                    if (mixed) near_point(G.view, G.img, arena_pts, p, arena_phi, arena_E);
                }
                if (threadIdx.x == 0) pblock_count[it.pblock] = 0;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && block_done) {
            __threadfence();
            if (atomicSub(&remaining[it.slot], 1) == 1) {
                __threadfence_system();
                cuda::atomic_ref<int64_t, cuda::thread_scope_system> d(done_mapped[it.slot]);
                d.store(it.gen, cuda::memory_order_release);
            }
        }
        if (threadIdx.x == 0) atomicAdd(head + 1, 1ull);  // one more item finished
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_serve(const ServeGeom* geoms, const WorkItem* ring, int64_t ring_cap, int64_t* tail_mapped,
                         unsigned long long* head, const double* arena_pts, double* arena_phi, double* arena_E,
                         float4* arena_bound, int* remaining, int64_t* done_mapped, double* partials,
                         int* pblock_count, int max_chunks, uint64_t idle_ns, int workers, cudaStream_t s) {
    k_serve<<<workers, kEvalThreads, 0, s>>>(geoms, ring, ring_cap, tail_mapped, head, arena_pts, arena_phi, arena_E,
                                             arena_bound, remaining, done_mapped, partials, pblock_count, max_chunks, idle_ns);
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
