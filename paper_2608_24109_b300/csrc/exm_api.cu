// C ABI of libexmesh (include/exmesh.h): object lifetimes, argument checks, launches.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "exm_device.cuh"
#include "exm_internal.h"

#include <atomic>

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_stamp{0};

uint64_t exm_next_stamp() { return ++g_stamp; }

// ------------------------------------------------------------ host-side fault injection

static std::atomic<uint32_t> g_fault[kFaultKinds];

static void parse_fault_env() {
    static std::atomic<bool> parsed{false};
    if (parsed.exchange(true)) return;  // once per process
    const char* v = getenv("EXM_FAULT");
    if (!v) return;
    static const char* names[kFaultKinds] = {"alloc", "admit", "slow", "cancel", "corrupt"};
    std::string s(v);
    size_t pos = 0;
    while (pos < s.size()) {
        size_t end = s.find(',', pos);
        if (end == std::string::npos) end = s.size();
        const std::string item = s.substr(pos, end - pos);
        const size_t colon = item.find(':');
        const std::string name = item.substr(0, colon);
        const uint32_t count = colon == std::string::npos ? 1u : (uint32_t)strtoul(item.c_str() + colon + 1, nullptr, 10);
        for (int k = 0; k < kFaultKinds; ++k)
            if (name == names[k]) g_fault[k] = count;
        pos = end + 1;
    }
}

bool exm_fault_take(int kind) {
    uint32_t c = g_fault[kind].load();
    while (c > 0)
        if (g_fault[kind].compare_exchange_weak(c, c - 1)) return true;
    return false;
}

uint32_t exm_fault_value(int kind) { return g_fault[kind].load(); }

cudaError_t exm_malloc(void** p, size_t bytes) {
    if (exm_fault_take(kFaultAlloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

exm_status exm_fail(exm_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

exm_status exm_cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return EXM_OK;
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EXM_ERR_OOM : EXM_ERR_CUDA;
}

#define EXM_TRY_ALLOC(ptr, bytes, what)                                              \
    do {                                                                             \
        if (exm_malloc((void**)&(ptr), (bytes)) != cudaSuccess) {                    \
            cudaGetLastError();                                                      \
            return exm_fail(EXM_ERR_OOM, std::string("allocation failed: ") + what); \
        }                                                                            \
    } while (0)

namespace {
}  // namespace

__global__ void exm_l1_kernel(const float* __restrict__ pred, const float* __restrict__ target, long long n,
                              float inv_n, float* loss, float* grad) {
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float d = pred[i] - target[i];
        acc += fabsf(d);
        grad[i] = d > 0.0f ? inv_n : (d < 0.0f ? -inv_n : 0.0f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float part[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(loss, acc * inv_n);
    }
}

// Uploads the cameras unless they equal the frame's last upload (a copy from pageable host
// memory waits for the stream to drain, so repeated renders of the same views skip it).
exm_status upload_cameras(exm_frame* f, const exm_camera* cams, int views, cudaStream_t s) {
    const size_t bytes = (size_t)views * sizeof(exm_camera);
    if (f->cams_host.size() == bytes && memcmp(f->cams_host.data(), cams, bytes) == 0) return EXM_OK;
    f->cams_host.assign((const unsigned char*)cams, (const unsigned char*)cams + bytes);
    return exm_cuda_check(cudaMemcpyAsync(f->cams, cams, bytes, cudaMemcpyHostToDevice, s), "camera upload");
}

extern "C" {

const char* exm_last_error(void) { return g_last_error.c_str(); }

exm_status exm_debug_fault(int kind, uint32_t count) {
    if (kind < EXM_FAULT_ALLOC || kind > EXM_FAULT_CORRUPT) return exm_fail(EXM_ERR_ARG, "exm_debug_fault: kind");
    g_fault[kind - EXM_FAULT_ALLOC] = count;
    return EXM_OK;
}

exm_status exm_create(int device, exm_ctx** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_create: out is NULL");
    parse_fault_env();
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return exm_fail(EXM_ERR_ARG, "exm_create: no such CUDA device");
    DeviceGuard g(device);
    exm_ctx* c = new (std::nothrow) exm_ctx();
    if (!c) return exm_fail(EXM_ERR_OOM, "exm_create: host allocation");
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (const char* w = getenv("EXM_BVH_WIDTH")) c->bvh_layout = atoi(w) == 8 ? EXM_BVH_8Q : (atoi(w) == 4 ? EXM_BVH_4 : 0);
    if (const char* k = getenv("EXM_BVH_COLLAPSE")) {
        const std::string v(k);
        c->bvh_collapse = v == "greedy" ? EXM_BVH_COLLAPSE_GREEDY : (v == "sah" ? EXM_BVH_COLLAPSE_SAH : 0);
    }
    if (const char* l = getenv("EXM_BVH_LAYOUT")) {
        const std::string v(l);
        c->bvh_layout = v == "4" ? EXM_BVH_4 : v == "4q" ? EXM_BVH_4Q : v == "8" ? EXM_BVH_8Q : c->bvh_layout;
    }
    if (exm_malloc((void**)&c->d_status, sizeof(uint32_t)) != cudaSuccess) {
        delete c;
        return exm_fail(EXM_ERR_OOM, "exm_create: status word");
    }
    cudaMemset(c->d_status, 0, sizeof(uint32_t));
    *out = c;
    return exm_cuda_check(cudaDeviceSynchronize(), "exm_create");
}

void exm_destroy(exm_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaFree(c->d_status);
    cudaFree(c->d_acc);
    cudaFree(c->scratch);
    delete c;
}

exm_status exm_ctx_set_bvh_layout(exm_ctx* c, int layout) {
    if (!c || layout < EXM_BVH_AUTO || layout > EXM_BVH_8Q) return exm_fail(EXM_ERR_ARG, "exm_ctx_set_bvh_layout");
    c->bvh_layout = layout;
    return EXM_OK;
}

exm_status exm_ctx_set_bvh_collapse(exm_ctx* c, int mode) {
    if (!c || mode < EXM_BVH_COLLAPSE_AUTO || mode > EXM_BVH_COLLAPSE_SAH)
        return exm_fail(EXM_ERR_ARG, "exm_ctx_set_bvh_collapse");
    c->bvh_collapse = mode;
    return EXM_OK;
}

exm_status exm_ctx_set_bvh_width(exm_ctx* c, int width) {
    if (!c || (width != 0 && width != 4 && width != 8)) return exm_fail(EXM_ERR_ARG, "exm_ctx_set_bvh_width");
    c->bvh_layout = width == 8 ? EXM_BVH_8Q : (width == 4 ? EXM_BVH_4 : EXM_BVH_AUTO);
    return EXM_OK;
}

exm_status exm_sync(exm_ctx* c, void* stream) {
    if (!c) return exm_fail(EXM_ERR_ARG, "exm_sync: ctx is NULL");
    DeviceGuard g(c->device);
    exm_status st = exm_cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "exm_sync");
    if (st != EXM_OK) return st;
    uint32_t bits = 0;
    st = exm_cuda_check(cudaMemcpy(&bits, c->d_status, 4, cudaMemcpyDeviceToHost), "exm_sync status read");
    if (st != EXM_OK) return st;
    if (bits) cudaMemset(c->d_status, 0, 4);
    if (bits & exm::ERRBIT_INDEX) return exm_fail(EXM_ERR_ARG, "index out of range in the mesh");
    if (bits & exm::ERRBIT_GUARD)
        return exm_fail(EXM_ERR_GUARDBAND, "a vertex lies behind the near plane or outside the guard band");
    if (bits & exm::ERRBIT_QUEUE)
        return exm_fail(EXM_ERR_QUEUE_OVERFLOW, "a ray queue chunk overflowed; the rays beyond it were not traced");
    if (bits & exm::ERRBIT_TRAVERSAL) return exm_fail(EXM_ERR_TRAVERSAL_LIMIT, "BVH traversal step/stack limit");
    return EXM_OK;
}

// ------------------------------------------------------------------------ mesh

static void mesh_free(exm_mesh* m) {
    void* ptrs[] = {m->V, m->F, m->UV, m->Fuv, m->nacc, m->nrm, m->tacc, m->tan, m->fsign, m->nfix, m->tfix,
                    m->tris, m->codes, m->codes_sorted, m->ids, m->ids_sorted, m->child, m->bounds,
                    m->scene_box, m->sort_tmp, m->nodes4, m->sphere, m->frontier, m->frontier_cnt, m->nodes8,
                    m->tris8, m->n_tris8, m->nodesq, m->sah_cost, m->sah_code, m->sah_span,
                    m->ploc_c, m->ploc_nn, m->ploc_flag, m->ploc_scan, m->scan_tmp};
    for (void* p : ptrs) cudaFree(p);
}

exm_status exm_mesh_create(exm_ctx* c, const float* V, int nv, const int32_t* F, int nf, const float* UV, int nuv,
                           const int32_t* Fuv, void* stream, exm_mesh** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_mesh_create: out is NULL");
    *out = nullptr;
    if (!c || !V || !F || !UV || !Fuv) return exm_fail(EXM_ERR_ARG, "exm_mesh_create: NULL argument");
    if (nv < 3 || nf < 1 || nuv < 3) return exm_fail(EXM_ERR_ARG, "exm_mesh_create: empty mesh");
    if (nf > (1 << 28) || nv > (1 << 28) || nuv > (1 << 28)) return exm_fail(EXM_ERR_ARG, "exm_mesh_create: mesh too large");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    exm_mesh* m = new (std::nothrow) exm_mesh();
    if (!m) return exm_fail(EXM_ERR_OOM, "exm_mesh_create: host allocation");
    m->ctx = c;
    m->nv = nv; m->nf = nf; m->nuv = nuv;
    auto alloc = [&](void** p, size_t bytes) { return exm_malloc((void**)p, bytes) == cudaSuccess; };
    bool ok = alloc((void**)&m->V, (size_t)nv * 12) && alloc((void**)&m->F, (size_t)nf * 12) &&
              alloc((void**)&m->UV, (size_t)nuv * 8) && alloc((void**)&m->Fuv, (size_t)nf * 12) &&
              alloc((void**)&m->nacc, (size_t)nv * 12) && alloc((void**)&m->nrm, (size_t)nv * 12) &&
              alloc((void**)&m->tacc, (size_t)nuv * 12) && alloc((void**)&m->tan, (size_t)nuv * 12) &&
              alloc((void**)&m->fsign, (size_t)nf * 4) && alloc((void**)&m->nfix, (size_t)nv * 24) &&
              alloc((void**)&m->tfix, (size_t)nuv * 24);
    if (!ok) {
        cudaGetLastError();
        mesh_free(m);
        delete m;
        return exm_fail(EXM_ERR_OOM, "exm_mesh_create: device allocation");
    }
    cudaMemcpyAsync(m->V, V, (size_t)nv * 12, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->F, F, (size_t)nf * 12, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->UV, UV, (size_t)nuv * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->Fuv, Fuv, (size_t)nf * 12, cudaMemcpyDeviceToDevice, s);
    m->stamp = exm_next_stamp();
    exm_status st = exm_frames_build(m, s);
    if (st == EXM_OK) st = exm_bvh_build_impl(m, s);
    if (st != EXM_OK) {
        mesh_free(m);
        delete m;
        return st;
    }
    *out = m;
    return EXM_OK;
}

exm_status exm_mesh_update_vertices(exm_mesh* m, const float* V, void* stream) {
    if (!m || !V) return exm_fail(EXM_ERR_ARG, "exm_mesh_update_vertices: NULL argument");
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyAsync(m->V, V, (size_t)m->nv * 12, cudaMemcpyDeviceToDevice, s);
    m->stamp = exm_next_stamp();
    exm_status st = exm_frames_build(m, s);
    if (st != EXM_OK) return st;
    return exm_bvh_build_impl(m, s);
}

exm_status exm_bvh_build(exm_mesh* m, void* stream) {
    if (!m) return exm_fail(EXM_ERR_ARG, "exm_bvh_build: mesh is NULL");
    DeviceGuard g(m->ctx->device);
    m->stamp = exm_next_stamp();
    return exm_bvh_build_impl(m, (cudaStream_t)stream);
}

void exm_mesh_destroy(exm_mesh* m) {
    if (!m) return;
    DeviceGuard g(m->ctx->device);
    mesh_free(m);
    delete m;
}

exm_status exm_mesh_frames(const exm_mesh* m, const float** normals, const float** tangents) {
    if (!m || !normals || !tangents) return exm_fail(EXM_ERR_ARG, "exm_mesh_frames: NULL argument");
    *normals = m->nrm;
    *tangents = m->tan;
    return EXM_OK;
}

// ------------------------------------------------------------------------ env

static void env_free(exm_env* e) {
    void* ptrs[] = {e->texel, e->q, e->cdf, e->rowsum, e->rowpre, e->rguide, e->cguide, e->wbuf, e->wmax, e->total};
    for (void* p : ptrs) cudaFree(p);
}

exm_status exm_env_create(exm_ctx* c, int W, int H, exm_env** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_env_create: out is NULL");
    *out = nullptr;
    if (!c || W < 1 || H < 1 || (long long)W * H > (1 << 22)) return exm_fail(EXM_ERR_ARG, "exm_env_create: bad size");
    DeviceGuard g(c->device);
    exm_env* e = new (std::nothrow) exm_env();
    if (!e) return exm_fail(EXM_ERR_OOM, "exm_env_create: host allocation");
    e->ctx = c;
    e->W = W; e->H = H;
    size_t n = (size_t)W * H;
    int rb = 1, cb = 1;
    while ((1 << rb) < H && rb < 20) ++rb;
    while ((1 << cb) < W && cb < 20) ++cb;
    e->rbits = rb + 1;
    e->cbits = cb + 1;
    size_t Gr = ((size_t)1 << e->rbits) + 1, Gc = (size_t)H * (((size_t)1 << e->cbits) + 1);
    bool ok = exm_malloc((void**)&e->texel, n * sizeof(float4)) == cudaSuccess && exm_malloc((void**)&e->q, n * 4) == cudaSuccess &&
              exm_malloc((void**)&e->cdf, n * 8) == cudaSuccess && exm_malloc((void**)&e->rowsum, (size_t)H * 8) == cudaSuccess &&
              exm_malloc((void**)&e->rowpre, (size_t)H * 8) == cudaSuccess && exm_malloc((void**)&e->rguide, Gr * 4) == cudaSuccess &&
              exm_malloc((void**)&e->cguide, Gc * 4) == cudaSuccess && exm_malloc((void**)&e->wbuf, n * 4) == cudaSuccess &&
              exm_malloc((void**)&e->wmax, 4) == cudaSuccess && exm_malloc((void**)&e->total, 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        env_free(e);
        delete e;
        return exm_fail(EXM_ERR_OOM, "exm_env_create: device allocation");
    }
    *out = e;
    return EXM_OK;
}

exm_status exm_env_prepare(exm_env* e, const void* E, exm_dtype dtype, void* stream) {
    if (!e || !E) return exm_fail(EXM_ERR_ARG, "exm_env_prepare: NULL argument");
    if (dtype != EXM_F32 && dtype != EXM_BF16 && dtype != EXM_F16) return exm_fail(EXM_ERR_ARG, "exm_env_prepare: dtype");
    DeviceGuard g(e->ctx->device);
    e->stamp = exm_next_stamp();
    return exm_env_prepare_impl(e, E, dtype, (cudaStream_t)stream);
}

void exm_env_destroy(exm_env* e) {
    if (!e) return;
    DeviceGuard g(e->ctx->device);
    env_free(e);
    delete e;
}

exm_status exm_env_total(exm_env* e, uint64_t* Q) {
    if (!e || !Q) return exm_fail(EXM_ERR_ARG, "exm_env_total: NULL argument");
    DeviceGuard g(e->ctx->device);
    return exm_cuda_check(cudaMemcpy(Q, e->total, 8, cudaMemcpyDeviceToHost), "exm_env_total");
}

// ---------------------------------------------------------------------- frame

static void frame_free(exm_frame* f) {
    void* ptrs[] = {f->visbuf, f->pixels, f->counters, f->samples, f->work, f->cams, f->XY,   f->Zq,
                    f->genv,   f->gnrm,   f->gtan,     f->bits,    f->hits, f->rays, f->ctr, f->prec,
                    f->pacc,   f->tsel, f->tv_gbuf, f->tv_inv, f->half_img, f->half_grad, f->big_tris, f->tsel2};
    for (void* p : ptrs) cudaFree(p);
    if (f->half) {
        frame_free(f->half);
        delete f->half;
        f->half = nullptr;
    }
    for (auto& t : f->timers) {
        cudaEventDestroy(t.begin);
        cudaEventDestroy(t.end);
    }
    f->timers.clear();
}

exm_status exm_frame_create(exm_ctx* c, int views, int width, int height, exm_frame** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_frame_create: out is NULL");
    *out = nullptr;
    if (!c || views < 1 || width < 1 || height < 1 || width > 16384 || height > 16384 ||
        (long long)views * width * height >= (1ll << 31))
        return exm_fail(EXM_ERR_ARG, "exm_frame_create: bad size");
    DeviceGuard g(c->device);
    exm_frame* f = new (std::nothrow) exm_frame();
    if (!f) return exm_fail(EXM_ERR_OOM, "exm_frame_create: host allocation");
    f->ctx = c;
    f->views = views; f->W = width; f->H = height;
    size_t n = (size_t)views * width * height;
    bool ok = exm_malloc((void**)&f->visbuf, n * 8) == cudaSuccess && exm_malloc((void**)&f->pixels, n * 4) == cudaSuccess &&
              exm_malloc((void**)&f->counters, 16) == cudaSuccess && exm_malloc((void**)&f->samples, 8) == cudaSuccess &&
              exm_malloc((void**)&f->work, 32) == cudaSuccess &&
              exm_malloc((void**)&f->cams, (size_t)views * sizeof(exm_camera)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        frame_free(f);
        delete f;
        return exm_fail(EXM_ERR_OOM, "exm_frame_create: device allocation");
    }
    cudaMemset(f->counters, 0, 16);
    cudaMemset(f->samples, 0, 8);
    cudaMemset(f->work, 0, 32);
    *out = f;
    return EXM_OK;
}

void exm_frame_destroy(exm_frame* f) {
    if (!f) return;
    DeviceGuard g(f->ctx->device);
    frame_free(f);
    delete f;
}

exm_status exm_frame_set_limits(exm_frame* f, uint32_t ray_cap, uint64_t saved_budget_bytes) {
    if (!f) return exm_fail(EXM_ERR_ARG, "exm_frame_set_limits: frame is NULL");
    if (ray_cap > (1u << 27)) return exm_fail(EXM_ERR_ARG, "exm_frame_set_limits: ray_cap above 2^27");
    f->ray_cap = ray_cap;
    f->saved_budget = saved_budget_bytes;
    return EXM_OK;
}

exm_status exm_frame_stats(exm_frame* f, uint64_t* covered, uint64_t* samples) {
    if (!f) return exm_fail(EXM_ERR_ARG, "exm_frame_stats: frame is NULL");
    DeviceGuard g(f->ctx->device);
    uint32_t cnt = 0;
    unsigned long long smp = 0;
    exm_status st = exm_cuda_check(cudaMemcpy(&cnt, f->counters, 4, cudaMemcpyDeviceToHost), "frame stats");
    if (st == EXM_OK) st = exm_cuda_check(cudaMemcpy(&smp, f->samples, 8, cudaMemcpyDeviceToHost), "frame stats");
    if (st == EXM_OK && f->half) {  // samples of the half-resolution indirect pass
        unsigned long long hs = 0;
        st = exm_cuda_check(cudaMemcpy(&hs, f->half->samples, 8, cudaMemcpyDeviceToHost), "frame stats");
        smp += hs;
    }
    if (covered) *covered = cnt;
    if (samples) *samples = smp;
    return st;
}

exm_status exm_frame_work(exm_frame* f, uint64_t counts[4]) {
    if (!f || !counts) return exm_fail(EXM_ERR_ARG, "exm_frame_work: NULL argument");
    DeviceGuard g(f->ctx->device);
    exm_status st = exm_cuda_check(cudaMemcpy(counts, f->work, 32, cudaMemcpyDeviceToHost), "frame work counters");
    if (st == EXM_OK && f->half) {
        uint64_t h[4];
        st = exm_cuda_check(cudaMemcpy(h, f->half->work, 32, cudaMemcpyDeviceToHost), "frame work counters");
        for (int k = 0; k < 4; ++k) counts[k] += h[k];
    }
    return st;
}

exm_status exm_frame_kernel_ms(exm_frame* f, float ms[4]) {
    if (!f || !ms) return exm_fail(EXM_ERR_ARG, "exm_frame_kernel_ms: NULL argument");
    DeviceGuard g(f->ctx->device);
    for (int k = 0; k < 4; ++k) ms[k] = 0.0f;
    exm_status st = EXM_OK;
    for (auto& t : f->timers) {
        float x = 0.0f;
        if (st == EXM_OK) st = exm_cuda_check(cudaEventSynchronize(t.end), "kernel timer");
        if (st == EXM_OK) st = exm_cuda_check(cudaEventElapsedTime(&x, t.begin, t.end), "kernel timer");
        if (t.which >= 0 && t.which < 4) ms[t.which] += x;
        cudaEventDestroy(t.begin);
        cudaEventDestroy(t.end);
    }
    f->timers.clear();
    if (st == EXM_OK && f->half) {
        float h[4];
        st = exm_frame_kernel_ms(f->half, h);
        for (int k = 0; k < 4; ++k) ms[k] += h[k];
    }
    return st;
}

exm_status exm_launch_count(exm_ctx* c, uint64_t* launches) {
    if (!c || !launches) return exm_fail(EXM_ERR_ARG, "exm_launch_count: NULL argument");
    *launches = c->launches;
    return EXM_OK;
}

exm_status exm_frame_visbuf(exm_frame* f, const uint64_t** keys) {
    if (!f || !keys) return exm_fail(EXM_ERR_ARG, "exm_frame_visbuf: NULL argument");
    *keys = f->visbuf;
    return EXM_OK;
}

// --------------------------------------------------------------------- render

}  // extern "C"

exm_status check_render(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                        const exm_env* e, const exm_camera* cams, int views, const exm_params* p,
                        const exm_frame* f, const char* who) {
    std::string w(who);
    if (!c || !m || !maps || !e || !cams || !p || !f) return exm_fail(EXM_ERR_ARG, w + ": NULL argument");
    if (dt != EXM_F32 && dt != EXM_BF16 && dt != EXM_F16) return exm_fail(EXM_ERR_ARG, w + ": map dtype");
    if (mapW < 1 || mapH < 1 || (long long)mapW * mapH > (1ll << 28)) return exm_fail(EXM_ERR_ARG, w + ": map size");
    if (views != f->views) return exm_fail(EXM_ERR_ARG, w + ": views differ from the frame's");
    if (p->n_direct < 1 || p->n_direct > 65536) return exm_fail(EXM_ERR_ARG, w + ": n_direct must be in [1, 65536]");
    if (p->n_bounce < 0 || p->n_bounce > 4096) return exm_fail(EXM_ERR_ARG, w + ": n_bounce must be in [0, 4096]");
    if (p->n_bounce > 0 && (p->n_light < 1 || p->n_light > 4096))
        return exm_fail(EXM_ERR_ARG, w + ": n_light must be in [1, 4096] with secondary rays");
    if ((long long)p->n_bounce * (p->n_light > 0 ? p->n_light : 1) > (1ll << 31))
        return exm_fail(EXM_ERR_ARG, w + ": n_bounce * n_light too large");
    if (m->ctx != c || e->ctx != c || f->ctx != c) return exm_fail(EXM_ERR_ARG, w + ": objects of another context");
    for (int v = 0; v < views; ++v)
        if (!(cams[v].kx > 0.0f) || !(cams[v].ky > 0.0f) || !(cams[v].near_plane > 0.0f))
            return exm_fail(EXM_ERR_ARG, w + ": camera kx, ky and near_plane must be positive");
    return EXM_OK;
}

extern "C" {

exm_status exm_render_forward(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                              const exm_env* e, const exm_camera* cams, int views, const exm_params* p,
                              exm_frame* f, float* out_rgb, void* stream) {
    ExmRange range("exm_render_forward");
    exm_status st = check_render(c, m, maps, dt, mapW, mapH, e, cams, views, p, f, "exm_render_forward");
    if (st != EXM_OK) return st;
    if (!out_rgb) return exm_fail(EXM_ERR_ARG, "exm_render_forward: out_rgb is NULL");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((p->flags & EXM_FLAG_HALF_RES_INDIRECT) && p->n_bounce > 0 && p->lambda_ind != 0.0f)
        return exm_render_forward_halfres(c, m, maps, dt, mapW, mapH, e, cams, views, p, f, out_rgb, s);
    st = upload_cameras(f, cams, views, s);
    if (st != EXM_OK) return st;
    {
        ExmRange r("raster");
        st = exm_raster_impl(c, m, f, views, s);
    }
    if (st != EXM_OK) return st;
    return exm_shade_forward_impl(c, m, maps, dt, mapW, mapH, e, f, p, out_rgb, s);
}

exm_status exm_render_backward(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                               const exm_env* e, const exm_camera* cams, int views, const exm_params* p,
                               exm_frame* f, const float* grad_rgb, float* grad_maps, float* grad_env, float* grad_V,
                               void* stream) {
    ExmRange range("exm_render_backward");
    exm_status st = check_render(c, m, maps, dt, mapW, mapH, e, cams, views, p, f, "exm_render_backward");
    if (st != EXM_OK) return st;
    if (!grad_rgb) return exm_fail(EXM_ERR_ARG, "exm_render_backward: grad_rgb is NULL");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((p->flags & EXM_FLAG_HALF_RES_INDIRECT) && p->n_bounce > 0 && p->lambda_ind != 0.0f)
        return exm_render_backward_halfres(c, m, maps, dt, mapW, mapH, e, cams, views, p, f, grad_rgb, grad_maps,
                                           grad_env, grad_V, s);
    st = exm_check_backward(f, m, e, mapW, mapH, cams, views, p);
    if (st != EXM_OK) return st;
    return exm_shade_backward_impl(c, m, maps, dt, mapW, mapH, e, f, p, grad_rgb, grad_maps, grad_env, grad_V, s);
}

exm_status exm_l1_loss(const float* pred, const float* target, int64_t n, float* loss, float* grad, void* stream) {
    if (!pred || !target || !loss || !grad || n < 1) return exm_fail(EXM_ERR_ARG, "exm_l1_loss: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    exm_l1_kernel<<<(int)blocks, 256, 0, s>>>(pred, target, (long long)n, 1.0f / (float)n, loss, grad);
    return exm_cuda_check(cudaGetLastError(), "exm_l1_loss launch");
}

// ------------------------------------------------------ Stage-II objective (Sec. 5.4)

exm_status exm_image_loss(exm_ctx* c, const float* pred, const float* target, int views, int width, int height,
                          float lambda_ssim, float* loss, float* grad_rgb, void* stream) {
    if (!c || !pred || !target || !loss || !grad_rgb || views < 1 || width < 1 || height < 1)
        return exm_fail(EXM_ERR_ARG, "exm_image_loss: bad argument");
    if ((size_t)views * 3 > 65535) return exm_fail(EXM_ERR_ARG, "exm_image_loss: more than 21845 views");
    if (!(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f)) return exm_fail(EXM_ERR_ARG, "exm_image_loss: lambda_ssim");
    DeviceGuard g(c->device);
    return exm_image_loss_impl(c, pred, target, views, width, height, lambda_ssim, loss, grad_rgb,
                               (cudaStream_t)stream);
}

exm_status exm_material_tv(exm_ctx* c, const void* maps, exm_dtype map_dtype, int mapW, int mapH, exm_frame* frame,
                           uint32_t flags, float lambda_mat, float* loss, float* grad_maps, void* stream) {
    if (!c || !maps || !frame || !loss || mapW < 1 || mapH < 1) return exm_fail(EXM_ERR_ARG, "exm_material_tv: bad argument");
    if (map_dtype != EXM_F32 && map_dtype != EXM_BF16 && map_dtype != EXM_F16)
        return exm_fail(EXM_ERR_ARG, "exm_material_tv: map dtype");
    if (frame->ctx != c) return exm_fail(EXM_ERR_ARG, "exm_material_tv: frame of another context");
    DeviceGuard g(c->device);
    return exm_material_tv_impl(c, maps, map_dtype, mapW, mapH, frame, flags, lambda_mat, loss, grad_maps,
                                (cudaStream_t)stream);
}

exm_status exm_env_regularizers(exm_ctx* c, const float* E, int envW, int envH, float lambda_env, float lambda_chroma,
                                float* loss, float* grad_env, void* stream) {
    if (!c || !E || !loss || !grad_env || envW < 1 || envH < 1)
        return exm_fail(EXM_ERR_ARG, "exm_env_regularizers: bad argument");
    DeviceGuard g(c->device);
    return exm_env_regularizers_impl(c, E, envW, envH, lambda_env, lambda_chroma, loss, grad_env, (cudaStream_t)stream);
}

exm_status exm_adam_step(exm_ctx* c, float* param, const float* grad, float* m, float* v, int64_t rows, int channels,
                         float lr, float beta1, float beta2, float eps, int step, const float* lo, const float* hi,
                         void* stream) {
    if (!c || !param || !grad || !m || !v || rows < 0 || channels < 1 || channels > 8 || step < 1)
        return exm_fail(EXM_ERR_ARG, "exm_adam_step: bad argument");
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f))
        return exm_fail(EXM_ERR_ARG, "exm_adam_step: beta outside [0, 1)");
    if (rows == 0) return EXM_OK;
    DeviceGuard g(c->device);
    return exm_adam_step_impl(c, param, grad, m, v, (size_t)rows, channels, lr, beta1, beta2, eps, step, lo, hi,
                              (cudaStream_t)stream);
}

}  // extern "C"
