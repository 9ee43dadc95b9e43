/*
 * exmesh.h -- C ABI of the B300 (sm_103a) Stage-II differentiable UV-PBR renderer.
 *
 * The library implements the data-parallel hot path of the UV-PBR decomposition stage
 * (Sec. 5 of "ExMesh++", arxiv 2608.24109): rasterise a fixed triangle mesh into a
 * visibility buffer, query UV-space PBR maps (Sec. 5.1, Eqs. 10-11), shade with a
 * Lambert + GGX microfacet BRDF under an importance-sampled lat-long environment map
 * with ray-traced visibility (Sec. 5.2, Eqs. 12-17), add one-bounce diffuse indirect
 * light from secondary rays that hit the same mesh and read the same maps (Sec. 5.3,
 * Eqs. 18-20), and run the adjoint that scatters gradients into the maps, the
 * environment map and the vertex positions.
 *
 * Conventions (all entry points):
 *  - Every pointer argument named as "device" is a CUDA device pointer on the context's
 *    device; "host" pointers are ordinary host memory read before the call returns.
 *  - The caller owns every input, output and gradient buffer.  The library owns the
 *    objects it creates (mesh, BVH, environment tables, frames) and frees them in the
 *    matching *_destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *    device work is enqueued on it; calls return once the work is enqueued.
 *  - Argument errors are returned synchronously and nothing is enqueued.  Errors found on
 *    the device (guard band, traversal step limit) are latched in the context and
 *    returned by exm_sync.
 *  - Nothing crosses the ABI as an exception; every device loop is bounded.
 *  - Gradients are ACCUMULATED (+=) into caller-zeroed FP32 buffers.
 */
#ifndef EXMESH_H
#define EXMESH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int exm_status;
#define EXM_OK 0
#define EXM_ERR_ARG (-1)             /* invalid argument (nothing enqueued) */
#define EXM_ERR_OOM (-2)             /* device allocation failed */
#define EXM_ERR_CUDA (-3)            /* a CUDA runtime call failed */
#define EXM_ERR_GUARDBAND (-4)       /* a vertex behind the near plane / outside +-16384 px,
                                        or a front face with doubled area >= 2^38 (1/256 px units) */
#define EXM_ERR_TRAVERSAL_LIMIT (-5) /* a BVH traversal exceeded its step cap (corrupt BVH) */
#define EXM_ERR_TIMEOUT (-6)         /* a bounded wait ran out (exm_relight_wait) */
#define EXM_ERR_BUSY (-7)            /* admission refused: not enough budget or slots */
#define EXM_ERR_QUEUE_OVERFLOW (-8)  /* a ray-queue chunk overflowed (exm_frame_set_limits' ray_cap below one
                                        chunk's rays); the rays beyond it were not traced */
#define EXM_ERR_CANCELLED (-9)       /* a relight request was cancelled (exm_relight_cancel) */

typedef enum { EXM_F32 = 0, EXM_BF16 = 1, EXM_F16 = 2 } exm_dtype;

/* Render flags. */
#define EXM_FLAG_WRAP_U 1u       /* bilinear fetch wraps in u (spherical UV seam); else clamps */
#define EXM_FLAG_NO_METALLIC 2u  /* metallic read as 0: the dielectric model (Sec. 5, Sec. 6.1) */
#define EXM_FLAG_COUNT_WORK 4u   /* also count BVH nodes, triangle tests, BRDF evaluations and rays
                                    (exm_frame_work); a slower instrumented kernel, same results */
#define EXM_FLAG_ZERO_GRADS 8u   /* exm_render_backward zeroes the gradient buffers before accumulating */
#define EXM_FLAG_TIME_KERNELS 16u /* record CUDA events around the trace and shade launches
                                     (exm_frame_kernel_ms) */
#define EXM_FLAG_NO_SECONDARY_MATERIAL 32u /* the "No Secondary Material" ablation (Sec. 6.4): secondary
                                     hits read no map and take a constant diffuse material (albedo 0.5,
                                     roughness 0.5, metallic 0, flat normal map, so n_s(y) is the
                                     interpolated vertex normal); no map gradient flows from y */
#define EXM_FLAG_HALF_RES_INDIRECT 64u /* indirect light at half resolution (Sec. 6.1 implementation
                                     details): the frame renders direct light; a child frame of
                                     ceil(W/2) x ceil(H/2) pixels renders the same cameras with halved
                                     intrinsics (pixel (i, j) centred on full-resolution (2i+1, 2j+1))
                                     and the indirect term only; each covered pixel adds its bilinear
                                     interpolation at ((x + 1/2)/2 - 1/2, (y + 1/2)/2 - 1/2), taps
                                     clamped to the image.  Not offered by exm_render_backward_noalloc */
#define EXM_FLAG_RECOMPUTE 128u /* keep the per-sample state (recorded texels, visibility bits, secondary
                                     hit ids) one chunk of pixels at a time instead of for the whole frame:
                                     the forward pass shades each chunk right after tracing it, and the
                                     backward pass generates and traces each chunk's rays again before its
                                     adjoint (the same decisions: the sample streams are counter-based and
                                     the traversal deterministic).  A frame also switches to it by itself
                                     when the whole-frame state would exceed its budget
                                     (exm_frame_set_limits) */

typedef struct exm_ctx exm_ctx;
typedef struct exm_mesh exm_mesh;
typedef struct exm_env exm_env;
typedef struct exm_frame exm_frame;

/* Pinhole camera (80 bytes).  A point p has camera coordinates x = (p-eye).right,
 * y = (p-eye).up, w = (p-eye).fwd and projects to pixel (cx + kx*x/w, cy - ky*y/w);
 * pixel (px, py) has its centre at (px + 0.5, py + 0.5).  near_plane bounds w from below. */
typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float kx, ky, cx, cy, near_plane;
    float pad[3];
} exm_camera;

/* Estimator parameters (Sec. 5.2-5.3): N_d direct environment samples per pixel, N_b
 * secondary rays per pixel, N_s light samples per valid secondary hit, lambda_ind of
 * Eq. 20, flags, and the 64-bit seed of the counter-based sample streams. */
typedef struct {
    int32_t n_direct;
    int32_t n_bounce;
    int32_t n_light;
    float lambda_ind;
    uint32_t flags;
    uint32_t reserved;
    uint64_t seed;
} exm_params;

/* ----------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`.  *out receives the handle. */
exm_status exm_create(int device, exm_ctx** out);
void exm_destroy(exm_ctx* ctx);
/* Message of the last error raised on the calling thread (library-owned string). */
const char* exm_last_error(void);
/* Waits for `stream` and returns the first device-side error latched since the last
 * exm_sync (EXM_ERR_GUARDBAND, EXM_ERR_TRAVERSAL_LIMIT), then clears it. */
exm_status exm_sync(exm_ctx* ctx, void* stream);

/* ------------------------------------------------------------------- mesh (S1) */

/* BVH node layout of the meshes `ctx` builds from now on (uploads, vertex updates, rebuilds):
 *   EXM_BVH_4   4-wide nodes of 128 bytes, FP32 child boxes;
 *   EXM_BVH_4Q  4-wide nodes of 64 bytes, child boxes quantised to 8 bits per plane on a per-node
 *               power-of-two grid, rounded outwards by one grid step (the same tree as EXM_BVH_4);
 *   EXM_BVH_8Q  8-wide nodes of 80 bytes with 8-bit quantised child boxes;
 *   EXM_BVH_AUTO the library's default (EXM_BVH_4).
 * The environment variable EXM_BVH_LAYOUT (4, 4q or 8) sets it at exm_create.  All layouts take
 * the same decisions (the box tests are conservative; the triangle tests are the same), so they
 * render the same images bit for bit. */
#define EXM_BVH_AUTO 0
#define EXM_BVH_4 1
#define EXM_BVH_4Q 2
#define EXM_BVH_8Q 3
exm_status exm_ctx_set_bvh_layout(exm_ctx* ctx, int layout);
/* The same by node width: 4 (EXM_BVH_4), 8 (EXM_BVH_8Q) or 0 (EXM_BVH_AUTO); EXM_BVH_WIDTH (4 or
 * 8) in the environment sets it at exm_create. */
exm_status exm_ctx_set_bvh_width(exm_ctx* ctx, int width);
/* How the binary tree is cut into 4-wide nodes (layouts EXM_BVH_4 and EXM_BVH_4Q) for the meshes
 * `ctx` builds from now on: EXM_BVH_COLLAPSE_GREEDY opens the child with the largest box until a
 * node holds four; EXM_BVH_COLLAPSE_SAH minimises the surface-area cost of the node and triangle
 * visits by dynamic programming over the slots each subtree may take, and may cut a subtree of
 * up to four consecutive triangle records as one leaf; EXM_BVH_COLLAPSE_AUTO is
 * the library's default (EXM_BVH_COLLAPSE_SAH).  EXM_BVH_COLLAPSE (greedy or sah) in the
 * environment sets it at exm_create.  Both render the same images bit for bit. */
#define EXM_BVH_COLLAPSE_AUTO 0
#define EXM_BVH_COLLAPSE_GREEDY 1
#define EXM_BVH_COLLAPSE_SAH 2
exm_status exm_ctx_set_bvh_collapse(exm_ctx* ctx, int mode);

/* Uploads the fixed mesh-UV carrier (V*, F*, U*, Phi* of Sec. 5): V float32 [nv,3],
 * F int32 [nf,3] (counter-clockwise seen from outside), UV float32 [nuv,2] (u right,
 * v down), Fuv int32 [nf,3] -- all DEVICE pointers, copied.  Computes the per-vertex
 * normals and per-UV-vertex tangents of the interpolated tangent frame (Sec. 5.1) and
 * builds the BVH.  Indices are checked on the device; an out-of-range index is an
 * EXM_ERR_ARG returned by exm_sync. */
exm_status exm_mesh_create(exm_ctx* ctx, const float* V, int nv, const int32_t* F, int nf,
                           const float* UV, int nuv, const int32_t* Fuv, void* stream, exm_mesh** out);
/* Replaces the vertex positions (DEVICE float32 [nv,3]), recomputes frames and BVH. */
exm_status exm_mesh_update_vertices(exm_mesh* mesh, const float* V, void* stream);
/* Rebuilds the BVH (Morton order, locally-ordered clustering, then 4- or 8-wide nodes in the
 * context's layout (exm_ctx_set_bvh_layout); one triangle per leaf). */
exm_status exm_bvh_build(exm_mesh* mesh, void* stream);
void exm_mesh_destroy(exm_mesh* mesh);
/* Device pointers to the mesh's per-vertex unit normals [nv,3] and per-UV-vertex unit
 * tangents [nuv,3] (read-only views, valid until the mesh changes). */
exm_status exm_mesh_frames(const exm_mesh* mesh, const float** normals, const float** tangents);

/* Asset export and import (no counterpart in the paper: the serving registry's reload path).
 * An exported asset is the mesh-UV carrier and its BVH in EXM_ASSET_SECTIONS little-endian
 * sections: V float32 [nv,3], F int32 [nf,3], UV float32 [nuv,2], Fuv int32 [nf,3], the BVH's
 * nodes (node 0 is the root), its triangle records (four float4 per triangle: the three vertices,
 * the original face id in the first .w, then padding to 64 bytes) and its bounding sphere (float4
 * centre, R^2).  Triangle record k holds its two 32-byte halves swapped when bit 1 of k is set.
 * A node of node_bytes 128 is 4-wide: child boxes lo.x[4] lo.y[4] lo.z[4] hi.x[4] hi.y[4]
 * hi.z[4], then four int32 child references (>= 0 a node; < 0 a leaf ~(k | (c - 1) << 28) of the
 * c = 1..4 consecutive triangle records from k; 0x7fffffff an empty slot), padded to 128 bytes; node q stores its 32-byte quarter j (j = 0..3
 * in that order) at quarter j xor (q mod 4) of its 128 bytes (node 0 as listed).
 * A node of node_bytes 80 is 8-wide compressed: float origin p.xyz and the biased exponents e of
 * the per-axis grid steps 2^(e-127) in bytes 0-2 of word 3; then uint32 child_base, tri_base and
 * ni | nt << 8; then the child boxes quantised on that grid, qlo.x[8] qlo.y[8] qlo.z[8] qhi.x[8]
 * qhi.y[8] qhi.z[8] (bytes; plane = p + q 2^(e-127)): slots 0..ni-1 are the nodes child_base + c,
 * slots ni..ni+nt-1 the triangle records tri_base + c - ni. */
#define EXM_ASSET_VERSION 4
#define EXM_ASSET_SECTIONS 7
typedef struct {
    uint32_t version;    /* EXM_ASSET_VERSION */
    uint32_t node_bytes; /* bytes of one BVH node (128) */
    int32_t nv, nf, nuv;
    uint32_t n_nodes;    /* BVH nodes */
    uint64_t bytes[EXM_ASSET_SECTIONS];
} exm_asset_info;
/* Sizes of `mesh`'s export. */
exm_status exm_mesh_export_info(const exm_mesh* mesh, exm_asset_info* info);
/* Copies the sections into caller buffers (HOST or DEVICE, of info.bytes each); synchronous. */
exm_status exm_mesh_export(const exm_mesh* mesh, void* const sections[EXM_ASSET_SECTIONS], void* stream);
/* A mesh from exported sections (HOST or DEVICE; copied): the carrier's frames are computed and
 * the imported BVH is used as it is.  Before it is used every face index and every node
 * reference is checked to lie in range (EXM_ERR_ARG otherwise, nothing created); a tree with a
 * cycle is not detected here, and its rays end at the traversal's caps (EXM_ERR_TRAVERSAL_LIMIT
 * from exm_sync after a render).  Synchronous. */
exm_status exm_mesh_import(exm_ctx* ctx, const exm_asset_info* info, const void* const sections[EXM_ASSET_SECTIONS],
                           void* stream, exm_mesh** out);

/* Host-side fault injection for failure tests (no counterpart in the paper; it makes no GPU
 * fault).  The next `count` events of `kind` fail: EXM_FAULT_ALLOC a device allocation by the
 * library (EXM_ERR_OOM); EXM_FAULT_ADMIT a relight submission (EXM_ERR_BUSY); EXM_FAULT_CANCEL a
 * submitted relight request is cancelled right after it is queued (EXM_ERR_CANCELLED);
 * EXM_FAULT_CORRUPT an imported BVH gets a cycle (the root's first node child points back to the
 * root).  EXM_FAULT_SLOW holds every relight request `count` milliseconds on the host before
 * its work is enqueued.  count 0 clears a kind.  The same settings come from the environment
 * variable EXM_FAULT ("alloc:N,admit:N,slow:MS,cancel:N,corrupt:N"), read by the process's
 * first exm_create.  Process-wide. */
#define EXM_FAULT_ALLOC 1
#define EXM_FAULT_ADMIT 2
#define EXM_FAULT_SLOW 3
#define EXM_FAULT_CANCEL 4
#define EXM_FAULT_CORRUPT 5
exm_status exm_debug_fault(int kind, uint32_t count);

/* ------------------------------------------------------- environment (Sec. 5.2) */

/* Creates environment tables for a W x H lat-long map (row 0 = +y). */
exm_status exm_env_create(exm_ctx* ctx, int W, int H, exm_env** out);
/* Builds the importance distribution from E (DEVICE, [H,W,3] of `dtype`): integer
 * weights q = 1 + floor(lum * sin(theta_row) * 2^24 / max), exact 64-bit prefix sums and
 * the sampling guide table; keeps an FP32 copy of E for shading. */
exm_status exm_env_prepare(exm_env* env, const void* E, exm_dtype dtype, void* stream);
void exm_env_destroy(exm_env* env);
/* Total Q of the integer weights (synchronous read, for tests). */
exm_status exm_env_total(exm_env* env, uint64_t* Q);

/* --------------------------------------------------------- render (Sec. 5.1-5.3) */

/* Per-render saved state: visibility buffer (u64 depth<<32|tri per pixel, all ones when
 * empty), covered-pixel list, counters, device copy of the cameras. */
exm_status exm_frame_create(exm_ctx* ctx, int views, int width, int height, exm_frame** out);
void exm_frame_destroy(exm_frame* frame);
/* Memory limits of a frame's wavefront state.  ray_cap: queued rays per chunk at most (0: the
 * default of 2^27 = 4 GiB of 32-byte rays; at most 2^27); a chunk is the pixels whose worst-case
 * ray count fits it, at least 32 pixels, so a cap below 32 pixels' rays overflows
 * (EXM_ERR_QUEUE_OVERFLOW from exm_sync).  saved_budget_bytes: bytes of per-sample state (4 per
 * direct sample, 4 per secondary light sample when the indirect term is active, 4 per visibility
 * word, 4 per secondary ray, per frame pixel) the frame keeps for the whole frame (0: the
 * default of 16 GiB); above it the frame works as with
 * EXM_FLAG_RECOMPUTE, with chunks whose state fits the budget.  Takes effect at the next forward
 * pass; a backward pass follows the split of its forward pass. */
exm_status exm_frame_set_limits(exm_frame* frame, uint32_t ray_cap, uint64_t saved_budget_bytes);
/* Covered pixels and shaded samples of the last forward (synchronous). */
exm_status exm_frame_stats(exm_frame* frame, uint64_t* covered, uint64_t* samples);
/* Work counters of the last pass run with EXM_FLAG_COUNT_WORK (synchronous): counts[0] BVH
 * nodes visited, [1] ray/triangle tests, [2] BRDF evaluations, [3] rays traced. */
exm_status exm_frame_work(exm_frame* frame, uint64_t counts[4]);
/* Milliseconds spent in the kernels timed since the last call (EXM_FLAG_TIME_KERNELS), summed
 * per kind: ms[0] any-hit trace, [1] closest-hit trace, [2] forward shade, [3] backward shade.
 * Waits for the recorded events. */
exm_status exm_frame_kernel_ms(exm_frame* frame, float ms[4]);
/* Number of kernels the library has launched on this context so far. */
exm_status exm_launch_count(exm_ctx* ctx, uint64_t* launches);
/* DEVICE pointer to the visibility buffer [views, height, width] of u64 keys. */
exm_status exm_frame_visbuf(exm_frame* frame, const uint64_t** keys);

/* Read-only DEVICE views of the per-sample decisions of the frame's last forward pass (for
 * inspection and tests; valid until the frame's next pass).  pixels: the covered-pixel list in
 * shading order (view*H*W + py*W + px; exm_frame_stats gives its length n).  visbits: row i
 * (covered pixel i) of [rows, dims[0]] u32 words holds the direct samples, bit k of word k/32
 * set iff sample k's direction lies above the geometric horizon and its shadow ray escapes
 * (Eq. 17's Vis); then, from visbits + rows*dims[0], [rows, dims[1]] words hold the light samples
 * of the secondary hits, bit j*N_s + s for light sample s of secondary ray j (Eq. 18's Vis).
 * hits: [rows, dims[2]] i32, the closest front-facing triangle of each secondary ray, -1 if none
 * (NULL without an indirect term).  dims = {direct words, secondary words, N_b, rows}.
 * EXM_ERR_ARG when the forward kept its state one chunk at a time (EXM_FLAG_RECOMPUTE). */
exm_status exm_frame_saved_state(exm_frame* frame, const uint32_t** pixels, const uint32_t** visbits,
                                 const int32_t** hits, int dims[4]);

/* Forward render (Eqs. 10-20).  maps: DEVICE [mapH, mapW, 8] texel-interleaved
 * (A rgb, R, M, N xyz) of `map_dtype`; cams: HOST array of `views` cameras; out_rgb:
 * DEVICE float32 [views, height, width, 3] (written; background 0).  The frame keeps
 * the visibility buffer for the backward pass.  The frame grows its wavefront buffers on the
 * first forward of a size and sample count and keeps them until destroyed: per frame pixel
 * 160 bytes (the 112-byte shading record and the backward's 48-byte adjoint sums); the
 * per-sample state -- 4 bytes per direct and per secondary light sample (the texel it picked),
 * one bit per direct and per secondary light sample, and 4 bytes per secondary ray -- per frame
 * pixel, or per pixel of
 * one chunk when it is recomputed (EXM_FLAG_RECOMPUTE, exm_frame_set_limits); plus one ray
 * queue of at most 2^27 rays x 32 bytes (4 GiB), sized down to the rays a chunk can produce. */
exm_status exm_render_forward(exm_ctx* ctx, const exm_mesh* mesh, const void* maps, exm_dtype map_dtype,
                              int mapW, int mapH, const exm_env* env, const exm_camera* cams, int views,
                              const exm_params* params, exm_frame* frame, float* out_rgb, void* stream);

/* Adjoint of exm_render_forward for the same inputs: given grad_rgb (DEVICE float32
 * [views,height,width,3]) accumulates dL/dmaps (DEVICE float32 [mapH,mapW,8]),
 * dL/dE (DEVICE float32 [envH,envW,3]) and dL/dV (DEVICE float32 [nv,3]); any gradient
 * pointer may be NULL to skip it.  The sampling density and every discrete decision are
 * constants of the derivative.  It reads the camera-ray records, recorded texels, visibility
 * bits and secondary hits of the frame's last forward (no ray is traced again, unless that
 * forward kept them per chunk: then each chunk is generated and traced again) and evaluates the
 * material from `maps` as passed.  The cameras, sample counts and seed must be the forward's,
 * and the mesh, the environment and the map size the ones it used, unchanged since (no
 * exm_mesh_update_vertices, exm_bvh_build or exm_env_prepare in between): otherwise EXM_ERR_ARG
 * before anything is enqueued. */
exm_status exm_render_backward(exm_ctx* ctx, const exm_mesh* mesh, const void* maps, exm_dtype map_dtype,
                               int mapW, int mapH, const exm_env* env, const exm_camera* cams, int views,
                               const exm_params* params, exm_frame* frame, const float* grad_rgb,
                               float* grad_maps, float* grad_env, float* grad_V, void* stream);

/* ------------------------------------------------- relight serving (Sec. 6.6 relighting) */

typedef struct exm_server exm_server;

/* One relight request: a resident asset rendered under a new environment map (forward only,
 * Eqs. 10-20).  env: DEVICE [env_h, env_w, 3] of env_dtype and out_rgb: DEVICE float32
 * [views, height, width, 3], both owned by the caller and kept alive until the request
 * completes; cams: HOST array of `views` cameras, copied at submission. */
typedef struct {
    int32_t asset;
    int32_t views, width, height;
    const void* env;
    exm_dtype env_dtype;
    int32_t env_w, env_h;
    const exm_camera* cams;
    exm_params params;
    float* out_rgb;
} exm_relight_req;

/* A relight server on `ctx`: at most `max_slots` requests in flight, an HBM budget (bytes)
 * bounding their device footprint, and min(max_slots, 3) batch streams.  Requests wait in a
 * FIFO queue; whenever a batch stream is free, the requests at the head of the queue that find
 * a free slot and fit the remaining budget are run as one batch on it: each request's own setup
 * (environment distribution, raster, pixel records), then one persistent closest-hit tracer
 * launch over all their secondary rays and one persistent any-hit tracer launch over all their
 * shadow rays -- each ray traced through the BVH of its own asset -- and each request's shading.
 * A request whose rays exceed one 2^27-ray queue, or that asks for half-resolution indirect
 * light, runs its own chunked forward pass inside the batch.  Requests that arrive while a batch
 * runs join the next batch on another stream, so batches overlap on the device.  A request's
 * footprint counts a ray queue sized to its own rays. */
exm_status exm_server_create(exm_ctx* ctx, uint64_t hbm_budget_bytes, int max_slots, exm_server** out);
void exm_server_destroy(exm_server* server);
/* Registers a resident asset (mesh with BVH and DEVICE maps [mapH, mapW, 8]); the caller
 * keeps both alive for the server's lifetime.  *asset_id receives its index. */
exm_status exm_server_add_asset(exm_server* server, const exm_mesh* mesh, const void* maps, exm_dtype map_dtype,
                                int mapW, int mapH, int32_t* asset_id);
/* Queues a request and runs the scheduler; *ticket identifies it.  EXM_ERR_BUSY when the
 * request alone exceeds the budget. */
exm_status exm_relight_submit(exm_server* server, const exm_relight_req* req, uint64_t* ticket);
/* Non-blocking: runs the scheduler, then reports whether `ticket` is done and its latency
 * (submission to observed completion, milliseconds).  A done ticket is forgotten after the
 * call that reports it; that call returns the request's status. */
exm_status exm_relight_poll(exm_server* server, uint64_t ticket, int* done, double* latency_ms);
/* Cancels a request: a queued one is dropped; one in flight finishes on the device but its
 * result is discarded (its output buffer is left undefined).  Either way the ticket reports
 * EXM_ERR_CANCELLED.  A finished ticket keeps its result; an unknown ticket is EXM_ERR_ARG. */
exm_status exm_relight_cancel(exm_server* server, uint64_t ticket);
/* Waits at most timeout_ms for `ticket`, running the scheduler meanwhile: the request's status
 * once it is done (and then forgets it, like exm_relight_poll), or EXM_ERR_TIMEOUT. */
exm_status exm_relight_wait(exm_server* server, uint64_t ticket, double timeout_ms, double* latency_ms);
/* Batches launched so far and the requests they held. */
exm_status exm_server_batches(exm_server* server, uint64_t* batches, uint64_t* batched_requests);
/* Runs the scheduler once (retire finished requests, admit queued ones). */
exm_status exm_server_progress(exm_server* server);
/* Queue length, requests in flight, budgeted bytes in use, requests completed. */
exm_status exm_server_stats(exm_server* server, uint64_t* queued, uint64_t* in_flight, uint64_t* bytes_in_use,
                            uint64_t* completed);
/* Device footprint the server budgets for `req`. */
exm_status exm_relight_footprint(exm_server* server, const exm_relight_req* req, uint64_t* bytes);

/* Backward pass without device allocation (no counterpart in the paper).
 *
 * For callers that must not call cudaMalloc while they run -- a host whose device memory
 * is owned by another allocator (a caching allocator or a pre-reserved arena), or a
 * latency-critical loop that cannot take the implicit synchronisation of cudaMalloc.  It
 * takes the same arguments as exm_render_backward without grad_V, makes the same checks
 * (EXM_ERR_ARG before anything is enqueued, outputs untouched) and accumulates dL/dmaps and
 * dL/dE (either may be NULL) for the last forward of `frame`.  Its environment-gradient
 * accumulator is a static device array of EXM_STATIC_ENV_MAX_TEXELS float4 (4 MiB) that every
 * GPU loading the library holds until exit; a larger environment is rejected with
 * EXM_ERR_ARG.  The array is shared by all calls on a device and keeps the last call's
 * contents (each call clears the part it uses): calls that overlap on the GPU race and must be
 * serialised by the caller.  The first call on a device resolves the array's address
 * (cudaGetSymbolAddress); make it before any stream capture.  The per-pixel and per-chunk
 * buffers it reads and writes belong to `frame` and were allocated by its forward pass.
 * Half-resolution indirect light (EXM_FLAG_HALF_RES_INDIRECT with an active indirect term) is
 * not offered. */
#define EXM_STATIC_ENV_MAX_TEXELS 262144
exm_status exm_render_backward_noalloc(exm_ctx* ctx, const exm_mesh* mesh, const void* maps, exm_dtype map_dtype,
                                       int mapW, int mapH, const exm_env* env, const exm_camera* cams, int views,
                                       const exm_params* params, exm_frame* frame, const float* grad_rgb,
                                       float* grad_maps, float* grad_env, void* stream);

/* L1 image loss of Sec. 6 workloads: *loss (DEVICE float32, written) = mean |pred - target|
 * over n elements; grad (DEVICE float32 [n], written) = sign(pred - target) / n. */
exm_status exm_l1_loss(const float* pred, const float* target, int64_t n, float* loss, float* grad,
                       void* stream);

/* ------------------------------------------------- Stage-II objective (Sec. 5.4, Eqs. 21-24)
 *
 * The objective calls of one context share its fixed-point accumulators and scratch: issue them on
 * one stream (or serialise them).  Loss outputs are DEVICE float32 arrays, written; gradient
 * outputs follow each call's rule (written or accumulated). */

/* Image term of Eq. 21 on pred, target (DEVICE float32 [views,height,width,3], linear RGB):
 * (1 - lambda_ssim) * mean|log(1 + pred) - log(1 + target)| + lambda_ssim * (1 - SSIM) with
 * SSIM on the sRGB-encoded images, per channel, 11 x 11 Gaussian window (sigma 1.5), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2, averaged over views, pixels and channels.
 * loss[3] = {total, log-L1, D-SSIM}; grad_rgb (DEVICE [views,height,width,3]) is WRITTEN with
 * d(total)/d(pred). */
exm_status exm_image_loss(exm_ctx* ctx, const float* pred, const float* target, int views, int width, int height,
                          float lambda_ssim, float* loss, float* grad_rgb, void* stream);

/* L_mat of Eq. 23 for the last exm_render_forward held by `frame`: the total variation of the
 * screen-projected material maps (the bilinear fetch at each pixel's primary hit) of base
 * colour, roughness and normal, plus metallic unless flags has EXM_FLAG_NO_METALLIC; each TV
 * is the mean |difference| over horizontal neighbour pairs (both pixels covered) plus the
 * same over vertical pairs, averaged over the map's channels.  flags' EXM_FLAG_WRAP_U selects
 * the fetch's u rule, as in the render.  loss[1] = L_mat (unweighted); grad_maps (DEVICE
 * float32 [mapH,mapW,8], may be NULL) is ACCUMULATED with lambda_mat * dL_mat/dmaps. */
exm_status exm_material_tv(exm_ctx* ctx, const void* maps, exm_dtype map_dtype, int mapW, int mapH, exm_frame* frame,
                           uint32_t flags, float lambda_mat, float* loss, float* grad_maps, void* stream);

/* L_env (Eq. 23) and L_chroma (Eq. 24) of E (DEVICE float32 [envH,envW,3]): TV with
 * longitude wrap-around; chroma = |mean(E) - mu_E 1|^2, mean over texels.  loss[2] = {TV,
 * chroma} (unweighted); grad_env (DEVICE float32 [envH,envW,3]) is ACCUMULATED with
 * lambda_env dTV/dE + lambda_chroma dchroma/dE (lambda_chroma is the weight at this step,
 * lambda_chroma0 (1 - t/T) in the paper). */
exm_status exm_env_regularizers(exm_ctx* ctx, const float* E, int envW, int envH, float lambda_env, float lambda_chroma,
                                float* loss, float* grad_env, void* stream);

/* One bias-corrected Adam step (step >= 1) on rows x channels FP32 values (DEVICE param,
 * grad, m, v; m and v zero before the first step), then a clamp of channel c to
 * [lo[c], hi[c]] (HOST arrays of `channels` <= 8 entries; NULL for no bound). */
exm_status exm_adam_step(exm_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t rows, int channels,
                         float lr, float beta1, float beta2, float eps, int step, const float* lo, const float* hi,
                         void* stream);

/* ------------------------------------------- Stage-I topology round (Sec. 4.1-4.3, Eqs. 1-6) */

typedef struct {
    float beta_g;          /* EMA coefficient of Eq. 1 (0.95) */
    float w_g, w_k;        /* split-score weights of Eq. 3 (0.6, 0.4) */
    float tau_degen;       /* degeneracy threshold of Eq. 4 (0.05) */
    float tau_uv;          /* UV seam distance of Eqs. 5-6 (1e-4) */
    int32_t split_percent; /* faces tried for splitting per round, percent of the face count (5) */
    int32_t max_faces;     /* face budget (200000) */
    int32_t reserved;
} exm_topology_params;

typedef struct exm_topology exm_topology;
exm_status exm_topology_create(exm_ctx* ctx, exm_topology** out);
void exm_topology_destroy(exm_topology* topo);

/* Per-face count of covered pixels in the frame's last raster (C_rend of Sec. 4.2), ADDED to
 * counts (DEVICE uint32 [nf]). */
exm_status exm_face_render_counts(exm_frame* frame, int nf, uint32_t* counts, void* stream);

/* One topology round on the mesh V [nv,3], F [nf,3], UV [nuv,2], Fuv [nf,3] (DEVICE, read
 * only) with the vertex EMA state ema [nv], this iteration's position gradients grad_V [nv,3]
 * and the render counts [nf] (DEVICE).  Updates the EMA (Eq. 1); scores faces (Eqs. 2-3);
 * splits the best-scoring large faces on their best edge, greedily in rank order with no face
 * modified twice, keeping separate UVs across seams (Eqs. 5-6); then collapses small
 * degenerate or never-rendered faces (Eq. 4) on the split mesh, greedily in rank order; deletes
 * the faces that lose a vertex and compacts vertices, faces and UVs.  Every floating-point
 * decision is taken in FP32 in a fixed operation order (arccos by Abramowitz and Stegun
 * 4.4.46), so the result is deterministic.  Synchronous (it reads sizes back); the result is
 * held by `topo` until its next round. */
exm_status exm_topology_round(exm_topology* topo, const float* V, int nv, const int32_t* F, int nf, const float* UV,
                              int nuv, const int32_t* Fuv, const float* ema, const float* grad_V,
                              const uint32_t* render_counts, const exm_topology_params* params, void* stream);
/* Sizes and DEVICE pointers of the last round's mesh and EMA (valid until the next round or
 * destroy); stats = {splits, merges, faces deleted}.  Any output pointer may be NULL. */
exm_status exm_topology_result(exm_topology* topo, int* nv, int* nf, int* nuv, const float** V, const int32_t** F,
                               const float** UV, const int32_t** Fuv, const float** ema, int stats[3]);

#ifdef __cplusplus
}
#endif
#endif
