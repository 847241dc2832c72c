// server_internal.h -- types shared by the serving kernel (server.cu) and its host side
// (server.cpp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nb_internal.h"

namespace nb {

// One work item: up to 128 points of one request, at `offset` in the point arena, over
// all elements (chunk < 0) or over one chunk of kChunkEl elements (requests up to 16384 points:
// every chunk of a point block is a separate item, so a few points still spread over many
// CTAs; the block's partial sums live in partial block `pblock`).
struct WorkItem {
    int32_t slot;       // request slot (remaining point-block counter, completion word)
    int32_t geom;       // geometry index
    int32_t precision;  // NEBEM_FP64 / NEBEM_MIXED
    int32_t count;      // points in this item
    int64_t offset;     // first point in the arena
    int64_t gen;        // generation number the completion word receives
    int32_t chunk;      // element chunk, or -1 for all elements
    int32_t nchunks;    // chunks of this geometry (chunked items)
    int32_t pblock;     // partial-sum block (chunked items)
    int32_t pad;
};

// Device-side geometry record of the server (one per context).
struct ServeGeom {
    GeomView view;
    ImageTable img;
};

ServeGeom make_serve_geom(const Elem* el, const FarNodes* far, const float4* cjk, const double* sigma, int64_t n_el,
                          const ImageTable& img, const NearGrid& grid, const int32_t* cell_start,
                          const int32_t* cell_items);

// Partial sums of chunked items: pblock p, chunk c, point t at partials[(p * max_chunks + c) *
// 128 + t] (kPartialDoubles each: phi, E, and the chunk's raw error scales of bound_slot());
// pblock_count[p] counts finished chunks.
constexpr int kChunkElements = 1024;  // = kChunkEl of the evaluation bodies
constexpr int kPartialDoubles = 8;
// arena_bound: the FP32 pass's error scales of every mixed point (arena index), for the
// refinement the host launches when a request's items are done.
cudaError_t launch_serve(const ServeGeom* geoms, const WorkItem* ring, int64_t ring_cap, int64_t* tail_mapped,
                         unsigned long long* head, const double* arena_pts, double* arena_phi, double* arena_E,
                         float4* arena_bound, int* remaining, int64_t* done_mapped, double* partials,
                         int* pblock_count, int max_chunks, uint64_t idle_ns, int workers, cudaStream_t s);

}  // namespace nb
