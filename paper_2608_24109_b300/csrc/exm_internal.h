// Host-side internals of libexmesh: object layouts and kernel launchers shared by the
// translation units.  Not part of the public ABI (include/exmesh.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/exmesh.h"

// A named NVTX range over a scope of host code: the library's entry points and stages show up
// as ranges in Nsight tools (and ncu can select kernels by them: --nvtx --nvtx-include).
// Without a tool attached the calls return at once.
struct ExmRange {
    explicit ExmRange(const char* name) { nvtxRangePushA(name); }
    ~ExmRange() { nvtxRangePop(); }
    ExmRange(const ExmRange&) = delete;
    ExmRange& operator=(const ExmRange&) = delete;
};

struct exm_ctx {
    int device = 0;
    int num_sms = 0;
    int bvh_layout = 0;            // BVH layout of new meshes: EXM_BVH_4 / _4Q / _8Q, 0 = the default
    int bvh_collapse = 0;          // 4-wide collapse: EXM_BVH_COLLAPSE_GREEDY / _SAH, 0 = the default
    uint32_t* d_status = nullptr;  // latched device error bits
    unsigned long long launches = 0;  // kernels launched by the library on this context
    unsigned long long* d_acc = nullptr;  // 64-bit fixed-point accumulators of the objective calls
    float* scratch = nullptr;         // objective scratch (SSIM coefficients)
    size_t scratch_cap = 0;
};

// Stamps of object contents: every mesh upload or vertex update, BVH build and environment
// preparation takes a new process-wide stamp, so a frame can tell whether the objects handed to a
// backward pass are the ones its forward pass used, unchanged (exm_api.cu).
uint64_t exm_next_stamp();

struct exm_mesh {
    exm_ctx* ctx = nullptr;
    uint64_t stamp = 0;        // contents stamp (upload, vertex update, BVH build)
    int nv = 0, nf = 0, nuv = 0;
    float* V = nullptr;        // [nv,3]
    int32_t* F = nullptr;      // [nf,3]
    float* UV = nullptr;       // [nuv,2]
    int32_t* Fuv = nullptr;    // [nf,3]
    float* nacc = nullptr;     // [nv,3] sum of incident face cross products
    float* nrm = nullptr;      // [nv,3] unit vertex normals
    float* tacc = nullptr;     // [nuv,3] sum of incident face tangents
    float* tan = nullptr;      // [nuv,3] unit UV-vertex tangents
    float* fsign = nullptr;    // [nf] UV handedness (+1 / -1)
    unsigned long long* nfix = nullptr;  // [nv,3] fixed-point normal sums
    unsigned long long* tfix = nullptr;  // [nuv,3] fixed-point tangent sums
    // BVH
    float4* tris = nullptr;    // [nf * 4] triangle records in leaf order (64 B: three vertices, padding)
    float4* nodes4 = nullptr;  // [max(nf-1,1) * 8] 4-wide nodes
    float4* sphere = nullptr;  // [1] bounding sphere of the triangles: centre, inflated R^2
    uint32_t n_nodes = 0;      // nodes of the BVH in use (in nodes4, nodesq or nodes8)
    int layout = EXM_BVH_4;    // BVH in use: EXM_BVH_4 (nodes4, tris), _4Q (nodesq, tris), _8Q (nodes8, tris8)
    float4* nodesq = nullptr;  // [n_nodes * 4] 4-wide nodes with quantised child boxes
    float4* sah_cost = nullptr;   // [nf - 1] SAH collapse: C(x, 1..4) per binary node (exm_bvh.cu)
    uint32_t* sah_code = nullptr; // [nf - 1] SAH collapse: the choices behind them
    int2* sah_span = nullptr;     // [nf - 1] SAH collapse: first leaf record and leaf count
    float4* nodes8 = nullptr;  // [n_nodes * 5] 8-wide compressed nodes
    float4* tris8 = nullptr;   // [nf * 4] triangle records in the 8-wide nodes' order
    uint32_t* n_tris8 = nullptr;
    int2* frontier = nullptr;  // [2 * nf] collapse frontier (binary node, 4-wide node)
    uint32_t* frontier_cnt = nullptr;
    // build scratch
    uint32_t* codes = nullptr;
    uint32_t* codes_sorted = nullptr;
    uint32_t* ids = nullptr;
    uint32_t* ids_sorted = nullptr;
    int32_t* child = nullptr;      // [2*(nf-1)] encoded children
    float* bounds = nullptr;       // [(2nf-1) * 6]
    float* scene_box = nullptr;    // [6] (ordered-int encoded min/max)
    int32_t* ploc_c = nullptr;     // [2nf] cluster arrays (ping-pong)
    int32_t* ploc_nn = nullptr;    // [nf] nearest neighbour of each cluster
    unsigned long long* ploc_flag = nullptr;  // [nf] merges << 32 | keeps
    unsigned long long* ploc_scan = nullptr;  // [nf] exclusive scan of ploc_flag
    void* scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    void* sort_tmp = nullptr;
    size_t sort_tmp_bytes = 0;
};

struct exm_env {
    exm_ctx* ctx = nullptr;
    uint64_t stamp = 0;           // contents stamp (exm_env_prepare)
    int W = 0, H = 0;
    int rbits = 0, cbits = 0;
    float4* texel = nullptr;      // [H*W] E.rgb, (q/Q) W H / (2 pi^2)
    uint32_t* q = nullptr;        // [H*W]
    uint64_t* cdf = nullptr;      // [H*W] inclusive prefix, row-major
    uint64_t* rowsum = nullptr;   // [H]
    uint64_t* rowpre = nullptr;   // [H] exclusive prefix of the row sums
    uint32_t* rguide = nullptr;   // [2^rbits + 1] row guide
    uint32_t* cguide = nullptr;   // [H * (2^cbits + 1)] per-row column guides
    float* wbuf = nullptr;        // [H*W] FP32 weights
    uint32_t* wmax = nullptr;     // [1] max weight bits
    uint64_t* total = nullptr;    // [1] Q on the device
};

// float4 per pixel record: [0..4] the camera-ray geometry (pixel_prep_kernel), [5..6] the
// material and shading normal (pixel_surface_kernel)
constexpr int kPrec = 7;
constexpr uint32_t kBigTriCap = 1u << 18;  // entries of a frame's large-triangle list (exm_raster.cu)

struct exm_frame {
    exm_ctx* ctx = nullptr;
    int views = 0, W = 0, H = 0;
    uint64_t* visbuf = nullptr;   // [views*H*W]
    uint32_t* pixels = nullptr;   // [views*H*W] covered pixel ids (view*H*W + py*W + px)
    uint32_t* counters = nullptr; // [0] covered count, [1] work cursor, [2] large triangles listed
    uint2* big_tris = nullptr;    // (view, face) of the triangles with large pixel boxes (exm_raster.cu)
    unsigned long long* samples = nullptr;  // [1] shaded samples of the last forward
    unsigned long long* work = nullptr;     // [4] work counters of the last counted pass
    void* cams = nullptr;         // device copy of the cameras [views]
    std::vector<unsigned char> cams_host;  // host copy of the last uploaded cameras
    int32_t* XY = nullptr;        // [views*nv*2] snapped coordinates (sized on demand)
    uint32_t* Zq = nullptr;       // [views*nv]
    size_t snap_capacity = 0;     // vertices * views the snap buffers hold
    float4* genv = nullptr;       // [envW*envH] env gradient accumulator (padded)
    size_t genv_capacity = 0;
    float4* gnrm = nullptr;       // [nv] vertex-normal adjoint
    float4* gtan = nullptr;       // [nuv] tangent adjoint
    size_t gframe_capacity = 0;
    size_t gtan_capacity = 0;
    // wavefront state of the last forward
    float4* prec = nullptr;       // [P * kPrec] per-pixel shading records
    size_t prec_cap = 0;
    float* pacc = nullptr;        // [P * 12] per-pixel sums of the backward's sample adjoints
    size_t pacc_cap = 0;
    uint32_t* tsel = nullptr;     // [P * Nd] texel picked by each queued direct sample
    size_t tsel_cap = 0;
    uint32_t* tsel2 = nullptr;    // [P * Nb * Ns] texel picked by each queued secondary light sample
    size_t tsel2_cap = 0;
    uint32_t* bits = nullptr;     // visibility bits: [P * wd] direct, then [P * ws] secondary
    size_t bits_cap = 0;
    int32_t* hits = nullptr;      // [P * Nb] secondary closest front-facing hit, -1 if none
    size_t hits_cap = 0;
    float4* rays = nullptr;       // ray queue of one chunk
    size_t rays_cap = 0;
    uint32_t ray_cap = 0;         // rays per chunk at most (0: the library's default of 2^27)
    uint32_t* ctr = nullptr;      // per chunk: queued / fetched counters
    size_t ctr_cap = 0;
    int last_nd = -1, last_nb = -1, last_ns = -1, last_wd = 0, last_ws = 0;
    // what the last forward pass used: the backward pass must be given the same objects,
    // unchanged, because the recorded texels, visibility bits, hit ids and pixel records
    // index into them
    uint64_t fwd_mesh_stamp = 0, fwd_env_stamp = 0;
    int fwd_env_W = 0, fwd_env_H = 0, fwd_mapW = 0, fwd_mapH = 0;
    uint32_t fwd_flags = 0;
    // per-sample saved state: whole frame (stored) or one chunk at a time (recomputed by the
    // backward pass, exm_frame_set_limits / EXM_FLAG_RECOMPUTE)
    bool fwd_recompute = false;
    uint32_t fwd_chunk = 0;        // pixels per chunk of the last forward
    uint32_t fwd_ray_cap = 0;      // queue entries per chunk of the last forward
    uint64_t fwd_seed = 0;
    uint64_t saved_budget = 0;     // bytes of per-sample state kept for the whole frame (0: default)
    exm_frame* half = nullptr;    // half-resolution indirect pass (EXM_FLAG_HALF_RES_INDIRECT)
    float* half_img = nullptr;    // [views*H'*W'*3] its lambda_ind L_ind image
    size_t half_img_cap = 0;
    float* half_grad = nullptr;   // [views*H'*W'*3] adjoint of the upsampling
    size_t half_grad_cap = 0;
    float* tv_gbuf = nullptr;     // [P * 8] projected material of the material TV
    size_t tv_gbuf_cap = 0;
    int32_t* tv_inv = nullptr;    // [views*H*W] covered index of each screen pixel
    size_t tv_inv_cap = 0;
    struct Timer { int which; cudaEvent_t begin, end; };
    std::vector<Timer> timers;    // EXM_FLAG_TIME_KERNELS
};

// Makes `dev` current for a scope and restores the caller's device on exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Host-side fault injection (failure tests; no GPU fault is made).  Set from the environment
// variable EXM_FAULT ("alloc:N,admit:N,slow:MS,cancel:N,corrupt:N", read by exm_create) or by
// exm_debug_fault; process-wide counters (exm_api.cu).
enum ExmFault { kFaultAlloc = 0, kFaultAdmit, kFaultSlow, kFaultCancel, kFaultCorrupt, kFaultKinds };
// True (and one count used up) when an injected fault of `kind` is due.
bool exm_fault_take(int kind);
// The current value of a fault setting (the slow-request delay in milliseconds).
uint32_t exm_fault_value(int kind);

// cudaMalloc through the allocation-failure injector: cudaErrorMemoryAllocation (nothing
// allocated) when an injected failure is due.
cudaError_t exm_malloc(void** p, size_t bytes);

// Grows a device buffer to hold `need` elements (contents are not kept); false on OOM.
template <typename TT>
inline bool ensure(TT** ptr, size_t* cap, size_t need) {
    if (need <= *cap && *ptr) return true;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (exm_malloc((void**)ptr, need * sizeof(TT)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *cap = need;
    return true;
}

// Batched relight forward (exm_shade.cu; used by the relight server, exm_serve.cu): one
// request's forward pass split at its two tracer launches, which the server makes once for a
// whole batch of requests.  A request's rays must fit one queue chunk (relight_queue_rays at
// most 2^27).
struct exm_relight_pass;
// One ray queue of a batched tracer launch: the queue of one request, the BVH of its asset and
// the outputs its rays write.
constexpr int kJobLayouts = 3;  // BVH layouts EXM_BVH_4, _4Q, _8Q: one batched launch each
struct ExmTraceJob {
    const float4* nodes4;
    const float4* tris;
    const float4* sphere;
    const float4* rays;
    const uint32_t* qcount;  // rays queued
    uint32_t ray_cap;
    uint32_t* visbits;
    uint32_t* secbits;
    int32_t* hits;
};
constexpr int kMaxBatch = 32;  // queues per batched tracer launch
// Setup on `s`: pixel records, surface records and (indirect) the secondary rays.
exm_status relight_pass_begin(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                              const exm_env* e, exm_frame* f, const exm_params* p, float* out, cudaStream_t s,
                              exm_relight_pass** out_pass);
bool relight_pass_indirect(const exm_relight_pass* rp);
// Shadow rays of the direct samples and of the secondary hits' light samples.
void relight_pass_shadow_rays(exm_ctx* ctx, exm_relight_pass* rp, cudaStream_t s);
// The sample loops (Eqs. 17-20) into the request's image.
exm_status relight_pass_shade(exm_ctx* ctx, exm_relight_pass* rp, exm_frame* f, cudaStream_t s);
void relight_pass_free(exm_relight_pass* rp);
uint64_t relight_queue_rays(int views, int W, int H, const exm_params* p);
// One persistent tracer launch over the queues of `passes` (closest: secondary rays, else shadow
// rays); the job table goes through h_jobs (pinned host) to d_jobs (device), kMaxBatch entries.
exm_status relight_trace_batch(exm_ctx* ctx, exm_relight_pass* const* passes, int n, bool closest,
                               ExmTraceJob* h_jobs, ExmTraceJob* d_jobs, cudaStream_t s);

// argument checks shared by the render entry points (exm_api.cu)
exm_status check_render(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                        const exm_env* e, const exm_camera* cams, int views, const exm_params* p, const exm_frame* f,
                        const char* who);

// The backward pass's checks of the frame's saved forward state against its arguments
// (exm_shade.cu): cameras, mesh, environment, map size, seed and sample counts.
exm_status exm_check_backward(const exm_frame* f, const exm_mesh* m, const exm_env* e, int mapW, int mapH,
                              const exm_camera* cams, int views, const exm_params* p);

// error helpers (exm_api.cu)
exm_status exm_fail(exm_status code, const std::string& msg);
exm_status exm_cuda_check(cudaError_t e, const char* what);

exm_status upload_cameras(exm_frame* f, const exm_camera* cams, int views, cudaStream_t s);

// the half-resolution indirect pass (exm_halfres.cu)
exm_status exm_render_forward_halfres(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                      int mapH, const exm_env* e, const exm_camera* cams, int views,
                                      const exm_params* p, exm_frame* f, float* out, cudaStream_t s);
exm_status exm_render_backward_halfres(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                       int mapH, const exm_env* e, const exm_camera* cams, int views,
                                       const exm_params* p, exm_frame* f, const float* grad_rgb, float* grad_maps,
                                       float* grad_env, float* grad_V, cudaStream_t s);

// Stage-II objective (exm_objective.cu)
exm_status exm_image_loss_impl(exm_ctx* ctx, const float* pred, const float* target, int views, int W, int H,
                               float lambda_ssim, float* loss, float* grad, cudaStream_t s);
exm_status exm_material_tv_impl(exm_ctx* ctx, const void* maps, exm_dtype dt, int mapW, int mapH, exm_frame* f,
                                uint32_t flags, float lambda_mat, float* loss, float* grad_maps, cudaStream_t s);
exm_status exm_env_regularizers_impl(exm_ctx* ctx, const float* E, int W, int H, float lambda_env,
                                     float lambda_chroma, float* loss, float* grad_env, cudaStream_t s);
exm_status exm_adam_step_impl(exm_ctx* ctx, float* param, const float* grad, float* m, float* v, size_t rows,
                              int channels, float lr, float beta1, float beta2, float eps, int step, const float* lo,
                              const float* hi, cudaStream_t s);

// kernels launchers
exm_status exm_frames_build(exm_mesh* m, cudaStream_t s);
exm_status exm_bvh_build_impl(exm_mesh* m, cudaStream_t s);
exm_status exm_env_prepare_impl(exm_env* e, const void* E, exm_dtype dt, cudaStream_t s);
exm_status exm_raster_impl(exm_ctx* ctx, const exm_mesh* m, exm_frame* f, int views, cudaStream_t s);
exm_status exm_shade_forward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                  int mapH, const exm_env* e, exm_frame* f, const exm_params* p, float* out,
                                  cudaStream_t s);
exm_status exm_frames_adjoint(exm_mesh* m, float4* gn, float4* gt, float* gV, cudaStream_t s);
exm_status exm_shade_backward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                   int mapH, const exm_env* e, exm_frame* f, const exm_params* p,
                                   const float* grad_rgb, float* grad_maps, float* grad_env, float* grad_V,
                                   cudaStream_t s);

inline int exm_blocks(size_t n, int threads) { return (int)((n + threads - 1) / threads); }
