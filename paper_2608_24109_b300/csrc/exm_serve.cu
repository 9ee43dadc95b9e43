// Relight serving (the relighting use of the exported asset, Sec. 6.6): resident assets,
// HBM-budget admission and continuous batching into persistent launches.
//
// A request names a resident asset (mesh + BVH + UV maps), an environment map, cameras and
// an output size.  Requests wait in a FIFO queue.  Whenever one of the server's batch streams
// is free, the scheduler takes requests from the head of the queue as long as a request slot
// is free and the request's device footprint (computed before any allocation) fits the
// remaining budget, and runs them as one batch on that stream: each request's own setup
// (environment distribution, raster, pixel records, secondary rays), then ONE persistent
// closest-hit tracer launch over the secondary-ray queues of every request in the batch, the
// shadow rays of each, ONE persistent any-hit tracer launch over all their shadow-ray queues,
// and each request's shading.  The tracer's warps claim pools of rays from the queues in turn
// and each lane traces its ray through the BVH of its own asset, so assets of different mesh
// sizes, map sizes and output resolutions share the launches.  Requests that arrive while a
// batch runs go into the next batch, on another stream, so the GPU keeps working on several
// batches at once.  Each request's completion is an event recorded after its shading; latency
// is measured from submission to the observation of that event on the host's steady clock.
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace {

using clk = std::chrono::steady_clock;
constexpr uint64_t kBatchQueueMax = 1ull << 27;  // rays a batched request's queue holds at most

struct Asset {
    const exm_mesh* mesh;
    const void* maps;
    exm_dtype dtype;
    int mapW, mapH;
};

struct Pending {
    uint64_t ticket;
    exm_relight_req req;
    std::vector<exm_camera> cams;
    size_t footprint;
    clk::time_point arrival;
    clk::time_point ready;  // not launched before (the slow-request injector)
};

// The render state of one request in flight: frames and environment tables, one per output
// size and environment size the slot has served (allocated on first use, so that steady-state
// requests allocate nothing).
struct Slot {
    std::vector<std::pair<uint64_t, exm_frame*>> frames;
    std::vector<std::pair<uint64_t, exm_env*>> envs;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool cancelled = false;
    uint64_t ticket = 0;
    size_t footprint = 0;
    clk::time_point arrival;
};

// A batch stream with its job tables for the batched tracer launches (closest, any).
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    ExmTraceJob* h_jobs = nullptr;  // pinned host, 2 x kJobLayouts x kMaxBatch (closest / any, per layout)
    ExmTraceJob* d_jobs = nullptr;  // device, the same
};

struct Result {
    bool done = false;
    exm_status status = EXM_OK;
    double latency_ms = 0.0;
};

}  // namespace

struct exm_server {
    exm_ctx* ctx = nullptr;
    size_t budget = 0;
    size_t used = 0;
    std::vector<Asset> assets;
    std::vector<Slot> slots;
    std::vector<Lane> lanes;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    uint64_t completed = 0, batches = 0, batched_requests = 0;
    std::mutex mu;
};

// Device bytes of one frame: visibility keys and pixel list, pixel records (the 112-byte
// shading record and the 48-byte adjoint sums), the texel of each direct sample and of each
// secondary light sample (nbs = N_b N_s of them), snapped vertices, visibility bits, secondary
// hit ids, the ray queue of a chunk, cameras, counters, the large-triangle list of the raster.
static size_t frame_bytes(size_t P, size_t views, size_t nv, int wd, int ws, int nb, int nbs, size_t ray_cap) {
    return P * (8 + 4 + 16 * kPrec + 48) + P * (size_t)wd * 32 * 4 + P * (size_t)nbs * 4 + views * nv * 12 +
           P * (size_t)(wd + ws) * 4 + P * (size_t)nb * 4 + ray_cap * 32 + views * 80 + 64 + (size_t)kBigTriCap * 8;
}

// The queue a request's frame needs: all its rays (one chunk) when they fit a batched queue,
// else the chunked default.
static size_t request_queue(const exm_relight_req& r, const exm_params& p) {
    const uint64_t rays = relight_queue_rays(r.views, r.width, r.height, &p);
    return rays <= kBatchQueueMax ? (size_t)rays : (size_t)kBatchQueueMax;
}

static size_t request_footprint(const exm_server* s, const exm_relight_req& r) {
    const size_t P = (size_t)r.views * r.width * r.height;
    const size_t nv = (size_t)s->assets[r.asset].mesh->nv;
    const int wd = (r.params.n_direct + 31) / 32;
    const bool ind = r.params.n_bounce > 0 && r.params.lambda_ind != 0.0f;
    const int ws = ind ? (r.params.n_bounce * r.params.n_light + 31) / 32 : 0;
    size_t frame;
    if (ind && (r.params.flags & EXM_FLAG_HALF_RES_INDIRECT)) {
        // direct-only frame, plus the half-resolution child frame and its image
        exm_params pd = r.params, ph = r.params;
        pd.n_bounce = 0;
        ph.n_direct = 0;
        const size_t Ph = (size_t)r.views * ((r.width + 1) / 2) * ((r.height + 1) / 2);
        frame = frame_bytes(P, r.views, nv, wd, 0, 0, 0, request_queue(r, pd)) +
                frame_bytes(Ph, r.views, nv, 0, ws, r.params.n_bounce, r.params.n_bounce * r.params.n_light,
                            kBatchQueueMax) + Ph * 12;
    } else {
        frame = frame_bytes(P, r.views, nv, wd, ws, ind ? r.params.n_bounce : 0,
                            ind ? r.params.n_bounce * r.params.n_light : 0, request_queue(r, r.params));
    }
    const size_t n = (size_t)r.env_w * r.env_h;
    int rb = 1, cb = 1;
    while ((1 << rb) < r.env_h && rb < 20) ++rb;
    while ((1 << cb) < r.env_w && cb < 20) ++cb;
    size_t env = n * (16 + 4 + 8 + 4) + (size_t)r.env_h * 16 + (((size_t)1 << (rb + 1)) + 1) * 4 +
                 (size_t)r.env_h * (((size_t)1 << (cb + 1)) + 1) * 4 + 16;
    return frame + env;
}

// The slot's frame and environment tables for this request (created on first use).
static exm_status slot_state(exm_server* s, Slot& sl, const exm_relight_req& r, exm_frame** frame, exm_env** env) {
    const uint64_t fkey = ((uint64_t)r.views << 40) | ((uint64_t)r.width << 20) | (uint64_t)r.height;
    const uint64_t ekey = ((uint64_t)r.env_w << 32) | (uint64_t)r.env_h;
    *frame = nullptr;
    *env = nullptr;
    for (auto& kv : sl.frames)
        if (kv.first == fkey) *frame = kv.second;
    if (!*frame) {
        exm_status st = exm_frame_create(s->ctx, r.views, r.width, r.height, frame);
        if (st != EXM_OK) return st;
        sl.frames.push_back({fkey, *frame});
    }
    for (auto& kv : sl.envs)
        if (kv.first == ekey) *env = kv.second;
    if (!*env) {
        exm_status st = exm_env_create(s->ctx, r.env_w, r.env_h, env);
        if (st != EXM_OK) return st;
        sl.envs.push_back({ekey, *env});
    }
    return EXM_OK;
}

// Enqueues one batch on `lane`: every request's setup, the batched tracer launches, every
// request's shading and completion event.  A request whose rays exceed one queue, or that
// asks for half-resolution indirect light, runs its whole (chunked) forward pass in the batch's
// stream instead.  Returns per request the status of its enqueueing.
static void launch_batch(exm_server* s, Lane& lane, const std::vector<int>& slot_ids, std::vector<Pending>& reqs,
                         std::vector<exm_status>& status) {
    ExmRange range("relight batch");
    exm_ctx* ctx = s->ctx;
    cudaStream_t st_ = lane.stream;
    const size_t n = reqs.size();
    status.assign(n, EXM_OK);
    std::vector<exm_relight_pass*> pass(n, nullptr);
    std::vector<exm_frame*> frames(n, nullptr);
    for (size_t i = 0; i < n; ++i) {
        Slot& sl = s->slots[slot_ids[i]];
        const exm_relight_req& r = reqs[i].req;
        const Asset& a = s->assets[r.asset];
        exm_env* env = nullptr;
        exm_status st = slot_state(s, sl, r, &frames[i], &env);
        if (st == EXM_OK) st = exm_env_prepare(env, r.env, r.env_dtype, st_);
        const bool batchable = !((r.params.flags & EXM_FLAG_HALF_RES_INDIRECT) && r.params.n_bounce > 0 &&
                                 r.params.lambda_ind != 0.0f) &&
                               relight_queue_rays(r.views, r.width, r.height, &r.params) <= kBatchQueueMax;
        if (st == EXM_OK && !batchable) {
            frames[i]->ray_cap = 0;
            st = exm_render_forward(ctx, a.mesh, a.maps, a.dtype, a.mapW, a.mapH, env, reqs[i].cams.data(), r.views,
                                    &r.params, frames[i], r.out_rgb, st_);
        } else if (st == EXM_OK) {
            frames[i]->ray_cap = (uint32_t)kBatchQueueMax;
            st = check_render(ctx, a.mesh, a.maps, a.dtype, a.mapW, a.mapH, env, reqs[i].cams.data(), r.views,
                              &r.params, frames[i], "relight");
            if (st == EXM_OK) st = upload_cameras(frames[i], reqs[i].cams.data(), r.views, st_);
            if (st == EXM_OK) st = exm_raster_impl(ctx, a.mesh, frames[i], r.views, st_);
            if (st == EXM_OK)
                st = relight_pass_begin(ctx, a.mesh, a.maps, a.dtype, a.mapW, a.mapH, env, frames[i], &r.params,
                                        r.out_rgb, st_, &pass[i]);
        }
        status[i] = st;
    }
    std::vector<exm_relight_pass*> live;
    for (size_t i = 0; i < n; ++i)
        if (pass[i]) live.push_back(pass[i]);
    exm_status bst = EXM_OK;
    if (!live.empty()) {
        bst = relight_trace_batch(ctx, live.data(), (int)live.size(), true, lane.h_jobs, lane.d_jobs, st_);
        for (exm_relight_pass* rp : live) relight_pass_shadow_rays(ctx, rp, st_);
        if (bst == EXM_OK)
            bst = relight_trace_batch(ctx, live.data(), (int)live.size(), false, lane.h_jobs + kJobLayouts * kMaxBatch,
                                      lane.d_jobs + kJobLayouts * kMaxBatch, st_);
    }
    for (size_t i = 0; i < n; ++i) {
        if (pass[i]) {
            exm_status st = bst == EXM_OK ? relight_pass_shade(ctx, pass[i], frames[i], st_) : bst;
            if (status[i] == EXM_OK) status[i] = st;
            relight_pass_free(pass[i]);
        }
        cudaEventRecord(s->slots[slot_ids[i]].done, st_);
    }
    cudaEventRecord(lane.done, st_);
}

static void finish(exm_server* s, uint64_t ticket, exm_status st, clk::time_point arrival) {
    Result& res = s->results[ticket];
    res.done = true;
    res.status = st;
    res.latency_ms = std::chrono::duration<double, std::milli>(clk::now() - arrival).count();
}

// Retires finished requests and batches, then forms batches from the head of the queue while a
// batch stream is free: requests join in arrival order as long as a slot is free and the
// request's footprint fits the remaining budget.
static exm_status progress_locked(exm_server* s) {
    for (Slot& sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        exm_status st = q == cudaSuccess ? EXM_OK : exm_cuda_check(q, "relight request");
        if (sl.cancelled) st = exm_fail(EXM_ERR_CANCELLED, "relight request cancelled");
        finish(s, sl.ticket, st, sl.arrival);
        s->used -= sl.footprint;
        sl.busy = false;
        sl.cancelled = false;
        ++s->completed;
    }
    for (Lane& ln : s->lanes) {
        if (!ln.busy) continue;
        if (cudaEventQuery(ln.done) != cudaErrorNotReady) ln.busy = false;
    }
    const clk::time_point now = clk::now();
    for (Lane& ln : s->lanes) {
        if (ln.busy || s->queue.empty()) continue;
        std::vector<int> ids;
        std::vector<Pending> batch;
        size_t used = s->used;
        while (!s->queue.empty() && (int)batch.size() < kMaxBatch) {
            Pending& p = s->queue.front();
            if (p.ready > now || used + p.footprint > s->budget) break;
            int free_slot = -1;
            for (size_t k = 0; k < s->slots.size(); ++k) {
                bool taken = s->slots[k].busy;
                for (int id : ids) taken = taken || id == (int)k;
                if (!taken) { free_slot = (int)k; break; }
            }
            if (free_slot < 0) break;
            ids.push_back(free_slot);
            used += p.footprint;
            batch.push_back(std::move(p));
            s->queue.pop_front();
        }
        if (batch.empty()) break;
        std::vector<exm_status> status;
        launch_batch(s, ln, ids, batch, status);
        ln.busy = true;
        ++s->batches;
        s->batched_requests += batch.size();
        for (size_t i = 0; i < batch.size(); ++i) {
            if (status[i] != EXM_OK) {
                finish(s, batch[i].ticket, status[i], batch[i].arrival);
                continue;
            }
            Slot& sl = s->slots[ids[i]];
            sl.busy = true;
            sl.cancelled = false;
            sl.ticket = batch[i].ticket;
            sl.footprint = batch[i].footprint;
            sl.arrival = batch[i].arrival;
            s->used += batch[i].footprint;
        }
    }
    return EXM_OK;
}

extern "C" {

exm_status exm_server_create(exm_ctx* ctx, uint64_t hbm_budget_bytes, int max_slots, exm_server** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_server_create: out is NULL");
    *out = nullptr;
    if (!ctx || max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0)
        return exm_fail(EXM_ERR_ARG, "exm_server_create: bad argument");
    exm_server* s = new (std::nothrow) exm_server();
    if (!s) return exm_fail(EXM_ERR_OOM, "exm_server_create: host allocation");
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
    DeviceGuard g(ctx->device);
    s->slots.resize(max_slots);
    s->lanes.resize(max_slots < 3 ? max_slots : 3);
    bool ok = true;
    for (Slot& sl : s->slots)
        ok = ok && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
    for (Lane& ln : s->lanes)
        ok = ok && cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) == cudaSuccess &&
             cudaHostAlloc((void**)&ln.h_jobs, 2 * kJobLayouts * kMaxBatch * sizeof(ExmTraceJob), cudaHostAllocDefault) ==
                 cudaSuccess &&
             exm_malloc((void**)&ln.d_jobs, 2 * kJobLayouts * kMaxBatch * sizeof(ExmTraceJob)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        exm_server_destroy(s);
        return exm_fail(EXM_ERR_OOM, "exm_server_create: streams, events or job tables");
    }
    *out = s;
    return EXM_OK;
}

void exm_server_destroy(exm_server* s) {
    if (!s) return;
    DeviceGuard g(s->ctx->device);
    for (Lane& ln : s->lanes)
        if (ln.stream) cudaStreamSynchronize(ln.stream);
    for (Slot& sl : s->slots) {
        for (auto& kv : sl.frames) exm_frame_destroy(kv.second);
        for (auto& kv : sl.envs) exm_env_destroy(kv.second);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (Lane& ln : s->lanes) {
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.stream) cudaStreamDestroy(ln.stream);
        cudaFreeHost(ln.h_jobs);
        cudaFree(ln.d_jobs);
    }
    delete s;
}

exm_status exm_server_add_asset(exm_server* s, const exm_mesh* mesh, const void* maps, exm_dtype dtype, int mapW,
                                int mapH, int32_t* asset_id) {
    if (!s || !mesh || !maps || !asset_id || mapW < 1 || mapH < 1)
        return exm_fail(EXM_ERR_ARG, "exm_server_add_asset: bad argument");
    if (dtype != EXM_F32 && dtype != EXM_BF16 && dtype != EXM_F16)
        return exm_fail(EXM_ERR_ARG, "exm_server_add_asset: map dtype");
    std::lock_guard<std::mutex> lock(s->mu);
    s->assets.push_back(Asset{mesh, maps, dtype, mapW, mapH});
    *asset_id = (int32_t)s->assets.size() - 1;
    return EXM_OK;
}

exm_status exm_relight_submit(exm_server* s, const exm_relight_req* r, uint64_t* ticket) {
    if (!s || !r || !ticket || !r->cams || !r->env || !r->out_rgb)
        return exm_fail(EXM_ERR_ARG, "exm_relight_submit: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->asset < 0 || r->asset >= (int)s->assets.size()) return exm_fail(EXM_ERR_ARG, "exm_relight_submit: asset id");
    if (r->views < 1 || r->width < 1 || r->height < 1 || r->env_w < 1 || r->env_h < 1 || r->params.n_direct < 1)
        return exm_fail(EXM_ERR_ARG, "exm_relight_submit: sizes");
    Pending p;
    p.req = *r;
    p.cams.assign(r->cams, r->cams + r->views);
    p.req.cams = nullptr;
    p.footprint = request_footprint(s, *r);
    if (p.footprint > s->budget)
        return exm_fail(EXM_ERR_BUSY, "exm_relight_submit: the request alone exceeds the server's HBM budget");
    if (exm_fault_take(kFaultAdmit)) return exm_fail(EXM_ERR_BUSY, "exm_relight_submit: admission refused (injected)");
    DeviceGuard g(s->ctx->device);
    p.arrival = clk::now();
    p.ready = p.arrival + std::chrono::milliseconds(exm_fault_value(kFaultSlow));
    p.ticket = s->next_ticket++;
    s->results[p.ticket] = Result{};
    *ticket = p.ticket;
    if (exm_fault_take(kFaultCancel)) {  // a client that cancels right after submitting
        finish(s, p.ticket, EXM_ERR_CANCELLED, p.arrival);
        return progress_locked(s);
    }
    s->queue.push_back(std::move(p));
    return progress_locked(s);
}

exm_status exm_server_progress(exm_server* s) {
    if (!s) return exm_fail(EXM_ERR_ARG, "exm_server_progress: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    DeviceGuard g(s->ctx->device);
    return progress_locked(s);
}

exm_status exm_relight_cancel(exm_server* s, uint64_t ticket) {
    if (!s) return exm_fail(EXM_ERR_ARG, "exm_relight_cancel: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return exm_fail(EXM_ERR_ARG, "exm_relight_cancel: unknown ticket");
    if (it->second.done) return EXM_OK;  // finished already: its result stands
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (q->ticket == ticket) {
            finish(s, ticket, EXM_ERR_CANCELLED, q->arrival);
            s->queue.erase(q);
            return EXM_OK;
        }
    for (Slot& sl : s->slots)
        if (sl.busy && sl.ticket == ticket) sl.cancelled = true;  // its kernels finish; the result is dropped
    return EXM_OK;
}

exm_status exm_relight_wait(exm_server* s, uint64_t ticket, double timeout_ms, double* latency_ms) {
    if (!s || !(timeout_ms >= 0.0)) return exm_fail(EXM_ERR_ARG, "exm_relight_wait: bad argument");
    const clk::time_point deadline =
        clk::now() + std::chrono::microseconds((long long)(timeout_ms < 1e9 ? timeout_ms * 1000.0 : 1e12));
    while (true) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            DeviceGuard g(s->ctx->device);
            progress_locked(s);
            auto it = s->results.find(ticket);
            if (it == s->results.end()) return exm_fail(EXM_ERR_ARG, "exm_relight_wait: unknown ticket");
            if (it->second.done) {
                if (latency_ms) *latency_ms = it->second.latency_ms;
                const exm_status st = it->second.status;
                s->results.erase(it);
                return st == EXM_OK ? EXM_OK : exm_fail(st, st == EXM_ERR_CANCELLED ? "relight request cancelled"
                                                                                      : "relight request failed");
            }
        }
        if (clk::now() >= deadline) return exm_fail(EXM_ERR_TIMEOUT, "exm_relight_wait: the request is not done");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

exm_status exm_relight_poll(exm_server* s, uint64_t ticket, int* done, double* latency_ms) {
    if (!s || !done) return exm_fail(EXM_ERR_ARG, "exm_relight_poll: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    DeviceGuard g(s->ctx->device);
    progress_locked(s);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return exm_fail(EXM_ERR_ARG, "exm_relight_poll: unknown ticket");
    *done = it->second.done ? 1 : 0;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    if (it->second.done) {
        exm_status st = it->second.status;
        s->results.erase(it);
        return st == EXM_OK ? EXM_OK : exm_fail(st, st == EXM_ERR_CANCELLED ? "relight request cancelled"
                                                                              : "relight request failed");
    }
    return EXM_OK;
}

exm_status exm_server_batches(exm_server* s, uint64_t* batches, uint64_t* batched_requests) {
    if (!s) return exm_fail(EXM_ERR_ARG, "exm_server_batches: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    if (batches) *batches = s->batches;
    if (batched_requests) *batched_requests = s->batched_requests;
    return EXM_OK;
}

exm_status exm_server_stats(exm_server* s, uint64_t* queued, uint64_t* in_flight, uint64_t* bytes_in_use,
                            uint64_t* completed) {
    if (!s) return exm_fail(EXM_ERR_ARG, "exm_server_stats: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    uint64_t busy = 0;
    for (const Slot& sl : s->slots) busy += sl.busy ? 1 : 0;
    if (queued) *queued = s->queue.size();
    if (in_flight) *in_flight = busy;
    if (bytes_in_use) *bytes_in_use = s->used;
    if (completed) *completed = s->completed;
    return EXM_OK;
}

exm_status exm_relight_footprint(exm_server* s, const exm_relight_req* r, uint64_t* bytes) {
    if (!s || !r || !bytes) return exm_fail(EXM_ERR_ARG, "exm_relight_footprint: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->asset < 0 || r->asset >= (int)s->assets.size()) return exm_fail(EXM_ERR_ARG, "exm_relight_footprint: asset");
    *bytes = request_footprint(s, *r);
    return EXM_OK;
}

}  // extern "C"
