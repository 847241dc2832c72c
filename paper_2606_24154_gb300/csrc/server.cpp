// server.cpp -- continuous-batching field-query server over several resident solved
// contexts (C-ABI in include/nebem.h; persistent kernel in server.cu).
//
// Requests enter a host FIFO.  A request is admitted when a slot is free, the device
// point arena has room for its points and the work ring has room for its items: its
// points are copied into the arena, its remaining point-block counter is set, and its
// items are appended to the ring in host-mapped memory before `tail` is advanced.  An
// item is 128 points over all elements; a request of up to 16384 points instead gets one
// item per (point block, chunk of 1024 elements), so that its points still spread over
// many CTAs (its latency would otherwise be one CTA's pass over all elements).  A persistent kernel (relaunched whenever admitted work exists and no
// instance is running) claims items as they appear, so requests admitted while others
// run join the running launch.  On completion the outputs are copied to the caller's
// buffers and the arena range, slot and ring items are released.
//
// Mixed requests on a context whose mixed_point_tol is > 0 get the refinement of the
// standalone evaluation: once their items are done, the host launches the flag and
// two-float re-evaluation kernels (eval_acc.cu) on the request's arena range on a second
// stream, and the request completes when that work has finished.  The kernels and the
// error scales are those of nebem_eval, so every point gets the same bits either way.
//
// The server is driven from the caller's thread: submit, poll and wait each run one
// round of completion -> admission -> launch.  Calls on one server must be serialised.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "context.h"
#include "server_internal.h"

namespace nb {

namespace {

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);               \
    } while (0)

constexpr int kItemPoints = 128;
// Requests up to this many points are split by element chunks (when the partial-sum blocks
// are free), so that a request of a few hundred point blocks still spreads over every SM; a
// point's chunk sums are added in a fixed order, so the split does not change its bits.
constexpr int64_t kSmallPoints = 16384;     // mixed
constexpr int64_t kSmallPointsF64 = 16384;  // FP64
constexpr int kPartialBlocks = 512;     // point blocks with chunk partial sums in flight

struct Interval {
    int64_t start, len;
};

// First-fit allocator over [0, cap) points.
struct Arena {
    int64_t cap = 0;
    std::vector<Interval> free_list;
    void reset(int64_t c) {
        cap = c;
        free_list.assign(1, Interval{0, c});
    }
    int64_t alloc(int64_t n) {
        for (size_t i = 0; i < free_list.size(); ++i)
            if (free_list[i].len >= n) {
                const int64_t s = free_list[i].start;
                free_list[i].start += n;
                free_list[i].len -= n;
                if (free_list[i].len == 0) free_list.erase(free_list.begin() + (long)i);
                return s;
            }
        return -1;
    }
    void release(int64_t s, int64_t n) {
        size_t i = 0;
        while (i < free_list.size() && free_list[i].start < s) ++i;
        free_list.insert(free_list.begin() + (long)i, Interval{s, n});
        if (i + 1 < free_list.size() && free_list[i].start + free_list[i].len == free_list[i + 1].start) {
            free_list[i].len += free_list[i + 1].len;
            free_list.erase(free_list.begin() + (long)i + 1);
        }
        if (i > 0 && free_list[i - 1].start + free_list[i - 1].len == free_list[i].start) {
            free_list[i - 1].len += free_list[i].len;
            free_list.erase(free_list.begin() + (long)i);
        }
    }
};

struct Request {
    int64_t id = 0;
    int32_t geom = 0, precision = 0;
    const double* pts = nullptr;
    int64_t n = 0;
    double* phi = nullptr;
    double* E = nullptr;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int32_t slot = -1;
    int64_t offset = -1, items = 0, gen = 0;
    std::vector<int32_t> pblocks;  // partial-sum blocks of a chunked request
    int state = 0;  // 0 queued, 1 admitted, 2 done, 3 refining (items done, refinement queued)
};

}  // namespace

struct Server {
    int device = 0;
    nebem_server_options opt{};
    std::vector<Ctx*> ctxs;
    cudaStream_t compute = nullptr, copy = nullptr, refine = nullptr;
    cudaEvent_t kernel_done = nullptr;
    std::vector<cudaEvent_t> refine_done;  // per slot
    bool kernel_launched = false;
    DevBuf d_geoms, d_pts, d_phi, d_E, d_head, d_remaining, d_partials, d_pcount;
    DevBuf d_rpart;                           // refinement partial sums (groups split over chunks)
    // refinement: error scales, the lists of the two levels (level 1 in three: phi and E,
    // phi only, E only; arena indices), their counts (four per slot)
    DevBuf d_bound, d_list, d_list2, d_list_p, d_list_e, d_nlist;
    std::vector<int32_t> nchunks;  // element chunks per geometry
    int32_t max_chunks = 1;
    std::vector<int32_t> free_pblocks;
    WorkItem* h_ring = nullptr;
    int64_t* h_tail = nullptr;
    int64_t* h_done = nullptr;
    int64_t ring_cap = 0, published = 0, in_flight_items = 0;
    Arena arena;
    std::vector<int32_t> free_slots;
    std::vector<int64_t> slot_gen;
    std::deque<Request*> queue;
    std::vector<Request*> admitted;
    std::unordered_map<int64_t, Request*> reqs;
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    ~Server() {
        cudaSetDevice(device);
        if (compute) cudaStreamSynchronize(compute);  // the device buffers free themselves after this body
        if (h_ring) cudaFreeHost(h_ring);
        if (h_tail) cudaFreeHost(h_tail);
        if (h_done) cudaFreeHost(h_done);
        if (refine) cudaStreamSynchronize(refine);
        for (cudaEvent_t e : refine_done)
            if (e) cudaEventDestroy(e);
        if (kernel_done) cudaEventDestroy(kernel_done);
        if (refine) cudaStreamDestroy(refine);
        if (compute) cudaStreamDestroy(compute);
        if (copy) cudaStreamDestroy(copy);
        for (auto& kv : reqs) delete kv.second;
    }

    bool refines(const Request* r) const {
        return r->precision == NEBEM_MIXED && ctxs[r->geom]->opt.mixed_point_tol > 0.0;
    }

    // the flag and re-evaluation kernels of the standalone evaluation on r's arena range
    int launch_refine(Request* r) {
        Ctx* c = ctxs[r->geom];
        AccView A;
        A.view = make_view(c->d_el.as<Elem>(), c->d_far.as<FarNodes>(), c->d_cjk.as<float4>(), c->d_sigma.as<double>(),
                           c->n, c->img, c->grid, c->d_cell_start.as<int32_t>(), c->d_cell_items.as<int32_t>());
        A.far = c->d_far.as<FarNodes>();
        A.el = c->d_el.as<Elem>();
        A.fe = c->d_fill_el.as<FillEl>();
        A.nodes = c->d_fill_nodes.as<float4>();
        A.tau = c->d_fill_tau.as<float4>();
        A.cjk = c->d_cjk.as<float4>();
        A.sigma = c->d_sigma.as<double>();
        A.n_el = c->n;
        A.grid = c->fill_grid;
        A.cell_start = c->d_fill_cell_start.as<int32_t>();
        A.cell_items = c->d_fill_cell_items.as<int32_t>();
        MixedScratch ms{};
        ms.order = nullptr;
        ms.bound = d_bound.as<float4>() + r->offset;
        ms.list = d_list.as<int32_t>() + r->offset;
        ms.list2 = d_list2.as<int32_t>() + r->offset;
        ms.list_p = d_list_p.as<int32_t>() + r->offset;
        ms.list_e = d_list_e.as<int32_t>() + r->offset;
        ms.n_list = d_nlist.as<int32_t>() + 4 * r->slot;
        // the refine stream runs one request at a time, so one partial-sum area serves them all
        void* part = d_rpart.ptr;
        CK(launch_eval_refine(A, c->img, d_pts.as<double>() + 3 * r->offset, r->n,
                              r->phi ? d_phi.as<double>() + r->offset : nullptr,
                              r->E ? d_E.as<double>() + 3 * r->offset : nullptr, nullptr, c->opt.mixed_point_tol,
                              c->err_model, ms, c->props.multiProcessorCount, refine, nullptr, part));
        CK(cudaEventRecord(refine_done[r->slot], refine));
        return 0;
    }

    int complete() {
        for (size_t i = 0; i < admitted.size();) {
            Request* r = admitted[i];
            if (r->state == 3) {
                const cudaError_t q = cudaEventQuery(refine_done[r->slot]);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                if (q != cudaSuccess) return cuda_fail(q, "refinement kernels");
            } else {
                const int64_t done = __atomic_load_n(&h_done[r->slot], __ATOMIC_ACQUIRE);
                if (done != r->gen) {
                    ++i;
                    continue;
                }
                if (refines(r)) {
                    int rc = launch_refine(r);
                    if (rc) return rc;
                    r->state = 3;
                    ++i;
                    continue;
                }
            }
            if (r->phi)
                CK(cudaMemcpyAsync(r->phi, d_phi.as<double>() + r->offset,
                                   sizeof(double) * r->n, cudaMemcpyDeviceToHost, copy));
            if (r->E)
                CK(cudaMemcpyAsync(r->E, d_E.as<double>() + 3 * r->offset, sizeof(double) * 3 * r->n,
                                   cudaMemcpyDeviceToHost, copy));
            CK(cudaStreamSynchronize(copy));
            arena.release(r->offset, r->n);
            for (int32_t pb : r->pblocks) free_pblocks.push_back(pb);
            r->pblocks.clear();
            free_slots.push_back(r->slot);
            in_flight_items -= r->items;
            r->state = 2;
            r->t_done = now();
            admitted.erase(admitted.begin() + (long)i);
        }
        return 0;
    }

    int admit() {
        while (!queue.empty()) {
            Request* r = queue.front();
            const int64_t blocks = (r->n + kItemPoints - 1) / kItemPoints;
            const int32_t nch = nchunks[r->geom];
            const int64_t small = (r->precision == NEBEM_MIXED) ? kSmallPoints : kSmallPointsF64;
            const bool chunked = r->n <= small && nch > 1 && (int64_t)free_pblocks.size() >= blocks;
            const int64_t items = chunked ? blocks * nch : blocks;
            if (free_slots.empty() || in_flight_items + items > ring_cap) break;
            const int64_t off = arena.alloc(r->n);
            if (off < 0) break;
            queue.pop_front();
            const int32_t slot = free_slots.back();
            free_slots.pop_back();
            r->slot = slot;
            r->offset = off;
            r->items = items;
            r->gen = ++slot_gen[slot];
            if (chunked)
                for (int64_t b = 0; b < blocks; ++b) {
                    r->pblocks.push_back(free_pblocks.back());
                    free_pblocks.pop_back();
                }
            const int cnt = (int)blocks;  // the kernel counts finished point blocks
            CK(cudaMemcpyAsync(d_pts.as<double>() + 3 * off, r->pts, sizeof(double) * 3 * r->n,
                               cudaMemcpyHostToDevice, copy));
            CK(cudaMemcpyAsync(d_remaining.as<int>() + slot, &cnt, sizeof(int), cudaMemcpyHostToDevice, copy));
            CK(cudaStreamSynchronize(copy));
            int64_t k = 0;
            for (int64_t b = 0; b < blocks; ++b)
                for (int32_t c = 0; c < (chunked ? nch : 1); ++c, ++k) {
                    WorkItem& w = h_ring[(published + k) % ring_cap];
                    w.slot = slot;
                    w.geom = r->geom;
                    w.precision = r->precision;
                    w.count = (int32_t)std::min<int64_t>(kItemPoints, r->n - b * kItemPoints);
                    w.offset = off + b * kItemPoints;
                    w.gen = r->gen;
                    w.chunk = chunked ? c : -1;
                    w.nchunks = nch;
                    w.pblock = chunked ? r->pblocks[b] : -1;
                    w.pad = 0;
                }
            published += items;
            __atomic_store_n(h_tail, published, __ATOMIC_RELEASE);
            in_flight_items += items;
            r->state = 1;
            r->t_admit = now();
            admitted.push_back(r);
        }
        return 0;
    }

    int launch_if_needed() {
        if (admitted.empty()) return 0;
        if (kernel_launched) {
            const cudaError_t q = cudaEventQuery(kernel_done);
            if (q == cudaErrorNotReady) return 0;
            if (q != cudaSuccess) return cuda_fail(q, "serving kernel");
        }
        // a new launch is open (the last one closed itself when it ran dry)
        CK(cudaMemsetAsync(d_head.as<unsigned long long>() + 2, 0, sizeof(unsigned long long), compute));
        CK(launch_serve(d_geoms.as<ServeGeom>(), h_ring, ring_cap, h_tail, d_head.as<unsigned long long>(),
                        d_pts.as<double>(), d_phi.as<double>(), d_E.as<double>(), d_bound.as<float4>(),
                        d_remaining.as<int>(), h_done,
                        d_partials.as<double>(), d_pcount.as<int>(), max_chunks, (uint64_t)opt.idle_us * 1000ull,
                        opt.workers, compute));
        CK(cudaEventRecord(kernel_done, compute));
        kernel_launched = true;
        return 0;
    }

    int drive() {
        CK(cudaSetDevice(device));
        int rc = complete();
        if (rc) return rc;
        rc = admit();
        if (rc) return rc;
        return launch_if_needed();
    }
};

}  // namespace nb

using namespace nb;

extern "C" {

int nebem_server_default_options(nebem_server_options* opt) {
    if (!opt) return fail(NEBEM_INVALID_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->arena_points = 4194304;
    opt->chunk_points = kItemPoints;
    opt->max_requests = 256;
    opt->workers = 0;
    opt->idle_us = 2000;
    return NEBEM_OK;
}

int nebem_server_create(nebem_server** out, nebem_ctx* const* ctxs, int32_t n_ctx, const nebem_server_options* opt) {
    if (!out || !ctxs || n_ctx <= 0) return fail(NEBEM_INVALID_ARG, "need contexts");
    *out = nullptr;
    nebem_server_options o;
    nebem_server_default_options(&o);
    if (opt) o = *opt;
    if (o.arena_points <= 0 || o.max_requests <= 0 || o.idle_us <= 0 || o.workers < 0)
        return fail(NEBEM_INVALID_ARG, "bad server options");
    if (o.chunk_points != kItemPoints) return fail(NEBEM_INVALID_ARG, "chunk_points must be 128");
    std::vector<Ctx*> cs;
    for (int32_t i = 0; i < n_ctx; ++i) {
        Ctx* c = reinterpret_cast<Ctx*>(ctxs[i]);
        if (!c) return fail(NEBEM_INVALID_ARG, "NULL context");
        if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "context " + std::to_string(i) + " has no charge densities");
        if (c->n_car > 0 || c->am_on)
            return fail(NEBEM_BAD_STATE, "context " + std::to_string(i) +
                                             " has known charges or Adaptive Modelling, which the server does not apply");
        if (c->device != reinterpret_cast<Ctx*>(ctxs[0])->device)
            return fail(NEBEM_INVALID_ARG, "all contexts must share one device");
        if (c->opt.mixed_point_tol > 0.0) {  // tables of the refinement, built before any request
            const cudaError_t e = cudaSetDevice(c->device);
            if (e != cudaSuccess) return cuda_fail(e, "nebem_server_create");
            const int rc = ensure_fill_tables(c);
            if (rc) return rc;
        }
        cs.push_back(c);
    }
    Server* s = new (std::nothrow) Server();
    if (!s) return fail(NEBEM_OUT_OF_MEMORY, "host allocation failed");
    s->opt = o;
    s->device = cs[0]->device;
    s->ctxs = cs;
    s->t0 = std::chrono::steady_clock::now();
    auto bail = [&](int rc) {
        delete s;
        return rc;
    };
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->refine, cudaStreamNonBlocking);
    s->refine_done.assign((size_t)o.max_requests, nullptr);
    for (int32_t i = 0; i < o.max_requests && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->refine_done[(size_t)i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(e, "nebem_server_create"));
    if (s->opt.workers == 0) s->opt.workers = 2 * cs[0]->props.multiProcessorCount;
    const int64_t cap = o.arena_points;
    std::vector<ServeGeom> geoms;
    for (Ctx* c : cs)
        geoms.push_back(make_serve_geom(c->d_el.as<Elem>(), c->d_far.as<FarNodes>(), c->d_cjk.as<float4>(),
                                        c->d_sigma.as<double>(), c->n, c->img, c->grid,
                                        c->d_cell_start.as<int32_t>(), c->d_cell_items.as<int32_t>()));
    int64_t max_el = 1;
    for (Ctx* c : cs) max_el = std::max<int64_t>(max_el, c->n);
    for (Ctx* c : cs) {
        const int32_t nc = (int32_t)((c->n + kChunkElements - 1) / kChunkElements);
        s->nchunks.push_back(nc);
        s->max_chunks = std::max(s->max_chunks, nc);
    }
    s->ring_cap = std::max<int64_t>(4096 + (int64_t)kPartialBlocks * s->max_chunks,
                                    2 * (cap + kItemPoints - 1) / kItemPoints);
    if ((e = s->d_geoms.ensure(sizeof(ServeGeom) * geoms.size())) != cudaSuccess ||
        (e = s->d_pts.ensure(sizeof(double) * 3 * cap)) != cudaSuccess ||
        (e = s->d_phi.ensure(sizeof(double) * cap)) != cudaSuccess ||
        (e = s->d_E.ensure(sizeof(double) * 3 * cap)) != cudaSuccess ||
        (e = s->d_head.ensure(3 * sizeof(unsigned long long))) != cudaSuccess ||  // claimed, finished, closing
        (e = s->d_remaining.ensure(sizeof(int) * o.max_requests)) != cudaSuccess ||
        (e = s->d_partials.ensure(sizeof(double) * kPartialDoubles * kItemPoints * (size_t)kPartialBlocks *
                                  s->max_chunks)) != cudaSuccess ||
        (e = s->d_bound.ensure(sizeof(float4) * cap)) != cudaSuccess ||
        (e = s->d_list.ensure(sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = s->d_list2.ensure(sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = s->d_list_p.ensure(sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = s->d_list_e.ensure(sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = s->d_rpart.ensure(refine_part_bytes(cap, cs[0]->props.multiProcessorCount, max_el))) != cudaSuccess ||
        (e = s->d_nlist.ensure(4 * sizeof(int32_t) * o.max_requests)) != cudaSuccess ||
        (e = s->d_pcount.ensure(sizeof(int) * kPartialBlocks)) != cudaSuccess)
        return bail(cuda_fail(e, "server device buffers"));
    if ((e = cudaHostAlloc(&s->h_ring, sizeof(WorkItem) * s->ring_cap, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(&s->h_tail, 64, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(&s->h_done, sizeof(int64_t) * o.max_requests, cudaHostAllocMapped)) != cudaSuccess)
        return bail(cuda_fail(e, "server mapped buffers"));
    std::memset(s->h_ring, 0, sizeof(WorkItem) * s->ring_cap);
    std::memset(s->h_tail, 0, 64);
    std::memset(s->h_done, 0, sizeof(int64_t) * o.max_requests);
    if ((e = cudaMemcpy(s->d_geoms.ptr, geoms.data(), sizeof(ServeGeom) * geoms.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemset(s->d_head.ptr, 0, 3 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(s->d_pcount.ptr, 0, sizeof(int) * kPartialBlocks)) != cudaSuccess)
        return bail(cuda_fail(e, "server setup copies"));
    for (int32_t i = kPartialBlocks - 1; i >= 0; --i) s->free_pblocks.push_back(i);
    s->arena.reset(cap);
    s->slot_gen.assign((size_t)o.max_requests, 0);
    for (int32_t i = o.max_requests - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = reinterpret_cast<nebem_server*>(s);
    return NEBEM_OK;
}

int nebem_server_submit(nebem_server* srv, int32_t geometry, const double* pts, int64_t n, double* phi, double* E,
                        int32_t precision, int64_t* req_id) {
    if (!srv || !req_id) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(srv);
    if (geometry < 0 || geometry >= (int32_t)s->ctxs.size()) return fail(NEBEM_INVALID_ARG, "bad geometry index");
    {
        const Ctx* c = s->ctxs[geometry];
        if (!c->sigma_valid) return fail(NEBEM_BAD_STATE, "the geometry's charge densities are no longer valid");
        if (c->n_car > 0 || c->am_on)
            return fail(NEBEM_BAD_STATE, "the geometry has known charges or Adaptive Modelling, which the server does not apply");
    }
    if (n <= 0 || !pts) return fail(NEBEM_INVALID_ARG, "need n > 0 points");
    if (precision != NEBEM_FP64 && precision != NEBEM_MIXED) return fail(NEBEM_INVALID_ARG, "bad precision");
    if (n > s->opt.arena_points) return fail(NEBEM_TOO_LARGE, "request larger than the point arena");
    Request* r = new (std::nothrow) Request();
    if (!r) return fail(NEBEM_OUT_OF_MEMORY, "host allocation failed");
    r->id = s->next_id++;
    r->geom = geometry;
    r->precision = precision;
    r->pts = pts;
    r->n = n;
    r->phi = phi;
    r->E = E;
    r->t_submit = s->now();
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *req_id = r->id;
    return s->drive();
}

int nebem_server_poll(nebem_server* srv, int64_t req_id, int32_t* done) {
    if (!srv || !done) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(srv);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(NEBEM_INVALID_ARG, "unknown request");
    int rc = s->drive();
    if (rc) return rc;
    *done = it->second->state == 2 ? 1 : 0;
    return NEBEM_OK;
}

int nebem_server_wait(nebem_server* srv, int64_t req_id, int64_t timeout_ms) {
    if (!srv) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(srv);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(NEBEM_INVALID_ARG, "unknown request");
    const double deadline = s->now() + 1e-3 * (double)timeout_ms;
    for (;;) {
        int rc = s->drive();
        if (rc) return rc;
        if (it->second->state == 2) return NEBEM_OK;
        if (s->now() > deadline) return fail(NEBEM_TIMEOUT, "request not complete within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int nebem_server_request_times(nebem_server* srv, int64_t req_id, double* t_submit, double* t_admit, double* t_done) {
    if (!srv) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Server* s = reinterpret_cast<Server*>(srv);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(NEBEM_INVALID_ARG, "unknown request");
    const Request* r = it->second;
    if (r->state != 2) return fail(NEBEM_BAD_STATE, "request not complete");
    if (t_submit) *t_submit = r->t_submit;
    if (t_admit) *t_admit = r->t_admit;
    if (t_done) *t_done = r->t_done;
    return NEBEM_OK;
}

int nebem_server_destroy(nebem_server* srv) {
    if (!srv) return NEBEM_OK;
    Server* s = reinterpret_cast<Server*>(srv);
    // finish admitted work (the kernel idles out once the ring is drained); queued
    // requests that were never admitted are dropped
    s->queue.clear();
    for (int guard = 0; guard < 600000 && !s->admitted.empty(); ++guard) {
        if (s->drive()) break;
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    delete s;
    return NEBEM_OK;
}

}  // extern "C"
