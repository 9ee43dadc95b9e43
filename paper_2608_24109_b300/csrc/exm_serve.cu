// Relight serving (the relighting use of the exported asset, Sec. 6.6): resident assets,
// HBM-budget admission and continuous batching.
//
// A request names a resident asset (mesh + BVH + UV maps), an environment map, cameras and
// an output size.  Requests wait in a FIFO queue; the scheduler admits the head of the
// queue as soon as a slot is free and the request's device footprint fits the remaining
// budget, so requests that arrive while others run are admitted as slots and memory free
// up.  Each slot owns a CUDA stream and its reusable render state (environment tables and a
// frame); an admitted request's whole forward pass (environment distribution, raster,
// shading) is enqueued on its slot's stream, so the work of all in-flight requests overlaps
// on the device.  Completion is observed by polling each slot's event; latency is measured
// from submission to that observation on the host's steady clock.
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace {

using clk = std::chrono::steady_clock;

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
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // reusable render state, one per output size / environment size this slot has served
    // (allocated on first use, so steady-state requests allocate nothing)
    std::vector<std::pair<uint64_t, exm_frame*>> frames;
    std::vector<std::pair<uint64_t, exm_env*>> envs;
    bool busy = false;
    uint64_t ticket = 0;
    size_t footprint = 0;
    clk::time_point arrival;
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
    uint32_t ray_cap = 1u << 25;  // rays per chunk of a slot's frame (1 GiB): fewer chunks, fewer tracer tails
    std::vector<Asset> assets;
    std::vector<Slot> slots;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    uint64_t completed = 0;
    std::mutex mu;
};

// Device bytes a request needs while it runs: the frame (visibility buffer, pixel list,
// snapped vertices, visibility bits, secondary hits, ray queue) and the environment tables.
// Device bytes of one frame: visibility keys and pixel list, pixel records (the 112-byte
// shading record and the 48-byte adjoint sums), the texel of each direct sample, snapped
// vertices, visibility bits, secondary hit ids, the ray queue of a chunk, cameras, counters.
static size_t frame_bytes(size_t P, size_t views, size_t nv, int wd, int ws, int nb, size_t ray_cap) {
    return P * (8 + 4 + 16 * kPrec + 48) + P * (size_t)wd * 32 * 4 + views * nv * 12 + P * (size_t)(wd + ws) * 4 + P * (size_t)nb * 4 + ray_cap * 32 +
           views * 80 + 64;
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
        const size_t Ph = (size_t)r.views * ((r.width + 1) / 2) * ((r.height + 1) / 2);
        frame = frame_bytes(P, r.views, nv, wd, 0, 0, s->ray_cap) +
                frame_bytes(Ph, r.views, nv, 0, ws, r.params.n_bounce, s->ray_cap) + Ph * 12;
    } else {
        frame = frame_bytes(P, r.views, nv, wd, ws, ind ? r.params.n_bounce : 0, s->ray_cap);
    }
    const size_t n = (size_t)r.env_w * r.env_h;
    int rb = 1, cb = 1;
    while ((1 << rb) < r.env_h && rb < 20) ++rb;
    while ((1 << cb) < r.env_w && cb < 20) ++cb;
    size_t env = n * (16 + 4 + 8 + 4) + (size_t)r.env_h * 16 + (((size_t)1 << (rb + 1)) + 1) * 4 +
                 (size_t)r.env_h * (((size_t)1 << (cb + 1)) + 1) * 4 + 16;
    return frame + env;
}

static exm_status launch_request(exm_server* s, Slot& sl, Pending& p) {
    exm_ctx* ctx = s->ctx;
    const exm_relight_req& r = p.req;
    const Asset& a = s->assets[r.asset];
    exm_status st = EXM_OK;
    const uint64_t fkey = ((uint64_t)r.views << 40) | ((uint64_t)r.width << 20) | (uint64_t)r.height;
    const uint64_t ekey = ((uint64_t)r.env_w << 32) | (uint64_t)r.env_h;
    exm_frame* frame = nullptr;
    for (auto& kv : sl.frames)
        if (kv.first == fkey) frame = kv.second;
    if (!frame) {
        st = exm_frame_create(ctx, r.views, r.width, r.height, &frame);
        if (st != EXM_OK) return st;
        frame->ray_cap = s->ray_cap;
        sl.frames.push_back({fkey, frame});
    }
    exm_env* env = nullptr;
    for (auto& kv : sl.envs)
        if (kv.first == ekey) env = kv.second;
    if (!env) {
        st = exm_env_create(ctx, r.env_w, r.env_h, &env);
        if (st != EXM_OK) return st;
        sl.envs.push_back({ekey, env});
    }
    st = exm_env_prepare(env, r.env, r.env_dtype, sl.stream);
    if (st != EXM_OK) return st;
    st = exm_render_forward(ctx, a.mesh, a.maps, a.dtype, a.mapW, a.mapH, env, p.cams.data(), r.views, &r.params,
                            frame, r.out_rgb, sl.stream);
    if (st != EXM_OK) return st;
    return exm_cuda_check(cudaEventRecord(sl.done, sl.stream), "relight completion event");
}

// Retires finished slots, then admits queued requests in arrival order while a slot is free
// and the head request's footprint fits the remaining budget.
static exm_status progress_locked(exm_server* s) {
    for (Slot& sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        Result& res = s->results[sl.ticket];
        res.done = true;
        res.status = q == cudaSuccess ? EXM_OK : exm_cuda_check(q, "relight request");
        res.latency_ms = std::chrono::duration<double, std::milli>(clk::now() - sl.arrival).count();
        s->used -= sl.footprint;
        sl.busy = false;
        ++s->completed;
    }
    while (!s->queue.empty()) {
        Pending& p = s->queue.front();
        if (s->used + p.footprint > s->budget) break;
        Slot* free_slot = nullptr;
        for (Slot& sl : s->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        if (!free_slot) break;
        exm_status st = launch_request(s, *free_slot, p);
        if (st != EXM_OK) {
            Result& res = s->results[p.ticket];
            res.done = true;
            res.status = st;
            s->queue.pop_front();
            continue;
        }
        free_slot->busy = true;
        free_slot->ticket = p.ticket;
        free_slot->footprint = p.footprint;
        free_slot->arrival = p.arrival;
        s->used += p.footprint;
        s->queue.pop_front();
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
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    s->slots.resize(max_slots);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            exm_server_destroy(s);
            if (prev >= 0) cudaSetDevice(prev);
            return exm_fail(EXM_ERR_CUDA, "exm_server_create: stream/event creation");
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = s;
    return EXM_OK;
}

void exm_server_destroy(exm_server* s) {
    if (!s) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->ctx->device);
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        for (auto& kv : sl.frames) exm_frame_destroy(kv.second);
        for (auto& kv : sl.envs) exm_env_destroy(kv.second);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (prev >= 0) cudaSetDevice(prev);
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
    p.arrival = clk::now();
    p.ticket = s->next_ticket++;
    s->results[p.ticket] = Result{};
    s->queue.push_back(std::move(p));
    *ticket = s->queue.back().ticket;
    return progress_locked(s);
}

exm_status exm_server_progress(exm_server* s) {
    if (!s) return exm_fail(EXM_ERR_ARG, "exm_server_progress: NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    return progress_locked(s);
}

exm_status exm_relight_poll(exm_server* s, uint64_t ticket, int* done, double* latency_ms) {
    if (!s || !done) return exm_fail(EXM_ERR_ARG, "exm_relight_poll: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    progress_locked(s);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return exm_fail(EXM_ERR_ARG, "exm_relight_poll: unknown ticket");
    *done = it->second.done ? 1 : 0;
    if (latency_ms) *latency_ms = it->second.latency_ms;
    if (it->second.done) {
        exm_status st = it->second.status;
        s->results.erase(it);
        return st;
    }
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
