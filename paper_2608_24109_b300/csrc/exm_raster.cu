// Primary visibility (Sec. 5.1): per-view vertex snap to 8-bit sub-pixel fixed point,
// triangle setup and rasterisation into a 64-bit (depth << 32 | triangle id) visibility
// buffer, then compaction of the covered pixels into a tile-ordered work list.
#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

constexpr int32_t kBadSnap = INT32_MIN;

// a1: one thread per (view, vertex).  FP32 specification: camera coordinates by rounded
// dot products, sx = cx + kx*(x/w), sy = cy - ky*(y/w), X = rint(256 sx), Y = rint(256 sy),
// Zq = rint(clamp(1 - near/w, 0, 1) * (2^24 - 1)).
__global__ void snap_kernel(const float* __restrict__ V, int nv, const Cam* __restrict__ cams, int views,
                            int2* __restrict__ XY, uint32_t* __restrict__ Zq, uint32_t* status) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (v >= nv || c >= views) return;
    const Cam& cm = cams[c];
    S3 d = ssub3(s3(V[3 * v], V[3 * v + 1], V[3 * v + 2]), s3(cm.eye[0], cm.eye[1], cm.eye[2]));
    float xc = sdot(d, s3(cm.right[0], cm.right[1], cm.right[2]));
    float yc = sdot(d, s3(cm.up[0], cm.up[1], cm.up[2]));
    float w = sdot(d, s3(cm.fwd[0], cm.fwd[1], cm.fwd[2]));
    size_t o = (size_t)c * nv + v;
    if (!(w >= cm.near_plane)) {
        atomicOr(status, ERRBIT_GUARD);
        XY[o] = make_int2(kBadSnap, kBadSnap);
        Zq[o] = 0;
        return;
    }
    float sx = sadd(cm.cx, smul(cm.kx, sdiv(xc, w)));
    float sy = ssub(cm.cy, smul(cm.ky, sdiv(yc, w)));
    if (!(fabsf(sx) < 16384.0f && fabsf(sy) < 16384.0f)) {
        atomicOr(status, ERRBIT_GUARD);
        XY[o] = make_int2(kBadSnap, kBadSnap);
        Zq[o] = 0;
        return;
    }
    XY[o] = make_int2(__float2int_rn(smul(sx, 256.0f)), __float2int_rn(smul(sy, 256.0f)));
    float z = ssub(1.0f, sdiv(cm.near_plane, w));
    z = fminf(fmaxf(z, 0.0f), 1.0f);
    Zq[o] = (uint32_t)__float2uint_rn(smul(z, 16777215.0f));
}

__device__ __forceinline__ bool edge_incl(long long dx, long long dy) { return dy > 0 || (dy == 0 && dx < 0); }

// A snapped triangle set up for rasterisation: integer vertices, twice its area, quantised
// depths, its pixel box (inclusive, clipped to the image) and the fill rule of each edge.
struct TriSetup {
    long long X0, Y0, X1, Y1, X2, Y2, A2, Z0, Z1, Z2;
    int x0, x1, y0, y1;
    bool in0, in1, in2;
};

// false: the triangle is culled (a bad vertex, back-facing or degenerate, or outside the
// guard band, which latches ERRBIT_GUARD) or covers no pixel centre.
__device__ __forceinline__ bool tri_setup(const int32_t* __restrict__ F, int f, int nv, const int2* __restrict__ xy,
                                          const uint32_t* __restrict__ zq, int W, int H, uint32_t* status,
                                          TriSetup* t) {
    const int ia = __ldg(F + 3 * f), ib = __ldg(F + 3 * f + 1), ic = __ldg(F + 3 * f + 2);
    if ((unsigned)ia >= (unsigned)nv || (unsigned)ib >= (unsigned)nv || (unsigned)ic >= (unsigned)nv) return false;
    const int2 a = xy[ia], b = xy[ib], d = xy[ic];
    if (a.x == kBadSnap || b.x == kBadSnap || d.x == kBadSnap) return false;
    t->X0 = a.x; t->Y0 = a.y; t->X1 = b.x; t->Y1 = b.y; t->X2 = d.x; t->Y2 = d.y;
    t->A2 = (t->Y1 - t->Y0) * (t->X2 - t->X0) - (t->X1 - t->X0) * (t->Y2 - t->Y0);
    if (t->A2 <= 0) return false;
    if (t->A2 >= (1ll << 38)) { atomicOr(status, ERRBIT_GUARD); return false; }
    t->Z0 = zq[ia]; t->Z1 = zq[ib]; t->Z2 = zq[ic];
    const long long mnx = min(t->X0, min(t->X1, t->X2)), mxx = max(t->X0, max(t->X1, t->X2));
    const long long mny = min(t->Y0, min(t->Y1, t->Y2)), mxy = max(t->Y0, max(t->Y1, t->Y2));
    const long long x0 = mnx - 128 <= 0 ? 0 : (mnx - 128 + 255) / 256;
    const long long x1 = min(mxx - 128 < 0 ? -1 : (mxx - 128) / 256, (long long)W - 1);
    const long long y0 = mny - 128 <= 0 ? 0 : (mny - 128 + 255) / 256;
    const long long y1 = min(mxy - 128 < 0 ? -1 : (mxy - 128) / 256, (long long)H - 1);
    if (x0 > x1 || y0 > y1) return false;
    t->x0 = (int)x0; t->x1 = (int)x1; t->y0 = (int)y0; t->y1 = (int)y1;
    t->in0 = edge_incl(t->X2 - t->X1, t->Y2 - t->Y1);
    t->in1 = edge_incl(t->X0 - t->X2, t->Y0 - t->Y2);
    t->in2 = edge_incl(t->X1 - t->X0, t->Y1 - t->Y0);
    return true;
}

// Pixel (px, py): the three edge functions at its centre under the fill rule, then depth =
// floor(sum E_i Z_i / A2) and a 64-bit atomicMin of (depth << 32 | f).
__device__ __forceinline__ void raster_pixel(const TriSetup& t, int f, int px, int py, int W,
                                             unsigned long long* __restrict__ vb) {
    const long long Px = (long long)px * 256 + 128, Py = (long long)py * 256 + 128;
    const long long E0 = (t.Y1 - Py) * (t.X2 - Px) - (t.X1 - Px) * (t.Y2 - Py);
    const long long E1 = (t.Y2 - Py) * (t.X0 - Px) - (t.X2 - Px) * (t.Y0 - Py);
    const long long E2 = (t.Y0 - Py) * (t.X1 - Px) - (t.X0 - Px) * (t.Y1 - Py);
    if (!(E0 > 0 || (E0 == 0 && t.in0))) return;
    if (!(E1 > 0 || (E1 == 0 && t.in1))) return;
    if (!(E2 > 0 || (E2 == 0 && t.in2))) return;
    const long long num = E0 * t.Z0 + E1 * t.Z1 + E2 * t.Z2;
    const unsigned long long z = (unsigned long long)(num / t.A2);
    atomicMin(vb + (size_t)py * W + px, (z << 32) | (unsigned long long)(uint32_t)f);
}

// Triangles whose pixel box holds more than kBigTriPixels pixels are handed to
// raster_big_kernel (a warp per triangle) through the frame's list of kBigTriCap (view, face)
// entries; when the list is full, the thread rasterises the triangle itself.  Both paths write
// the same keys by atomicMin, so the visibility buffer does not depend on which path took a
// triangle.
constexpr long long kBigTriPixels = 256;

// a2: one thread per (view, triangle).  Integer edge functions, lexicographic (top-left)
// fill rule, back faces culled, depth = floor(sum E_i Z_i / A2), 64-bit atomicMin.
__global__ void raster_kernel(const int32_t* __restrict__ F, int nf, int nv, const int2* __restrict__ XY,
                              const uint32_t* __restrict__ Zq, int views, int W, int H,
                              unsigned long long* __restrict__ visbuf, uint2* __restrict__ big,
                              uint32_t* __restrict__ big_count, uint32_t* status) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (f >= nf || c >= views) return;
    TriSetup t;
    if (!tri_setup(F, f, nv, XY + (size_t)c * nv, Zq + (size_t)c * nv, W, H, status, &t)) return;
    if ((long long)(t.x1 - t.x0 + 1) * (t.y1 - t.y0 + 1) > kBigTriPixels && big) {
        const uint32_t k = atomicAdd(big_count, 1u);
        if (k < kBigTriCap) {
            big[k] = make_uint2((uint32_t)c, (uint32_t)f);
            return;
        }
    }
    unsigned long long* vb = visbuf + (size_t)c * W * H;
    for (int py = t.y0; py <= t.y1; ++py)
        for (int px = t.x0; px <= t.x1; ++px) raster_pixel(t, f, px, py, W, vb);
}

// The listed large triangles: persistent warps, a triangle per warp at a time, its pixel box
// walked 32 pixels at a time (row-major, so a warp's pixels share rows of the buffer).
__global__ void raster_big_kernel(const int32_t* __restrict__ F, int nv, const int2* __restrict__ XY,
                                  const uint32_t* __restrict__ Zq, int W, int H,
                                  unsigned long long* __restrict__ visbuf, const uint2* __restrict__ big,
                                  const uint32_t* __restrict__ big_count, uint32_t* status) {
    const uint32_t n = min(*big_count, kBigTriCap);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += nwarps) {
        const uint2 e = big[k];
        const int c = (int)e.x, f = (int)e.y;
        TriSetup t;
        if (!tri_setup(F, f, nv, XY + (size_t)c * nv, Zq + (size_t)c * nv, W, H, status, &t)) continue;
        unsigned long long* vb = visbuf + (size_t)c * W * H;
        // the box lies inside the image (at most 16384^2 = 2^28 pixels): 32-bit indices
        const uint32_t bw = (uint32_t)(t.x1 - t.x0 + 1);
        const uint32_t area = bw * (uint32_t)(t.y1 - t.y0 + 1);
        for (uint32_t i = lane; i < area; i += 32)
            raster_pixel(t, f, t.x0 + (int)(i % bw), t.y0 + (int)(i / bw), W, vb);
    }
}

// Covered-pixel compaction: one warp per 8x4 pixel tile, warp-aggregated append, so the
// work list keeps 2D locality within each warp.
__global__ void compact_kernel(const unsigned long long* __restrict__ visbuf, int views, int W, int H,
                               uint32_t* __restrict__ pixels, uint32_t* __restrict__ counters) {
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int tx = (W + 7) / 8, ty = (H + 3) / 4;
    int tiles = tx * ty;
    if (warp >= tiles * views) return;
    int c = warp / tiles, t = warp - c * tiles;
    int px = (t % tx) * 8 + (lane & 7), py = (t / tx) * 4 + (lane >> 3);
    bool cov = false;
    uint32_t id = 0;
    if (px < W && py < H) {
        id = (uint32_t)c * W * H + (uint32_t)py * W + px;
        cov = (uint32_t)(visbuf[id] & 0xffffffffull) != 0xffffffffu;
    }
    unsigned mask = __ballot_sync(0xffffffffu, cov);
    if (!mask) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(counters, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cov) pixels[base + __popc(mask & ((1u << lane) - 1u))] = id;
}

}  // namespace exm

using namespace exm;

exm_status exm_raster_impl(exm_ctx* ctx, const exm_mesh* m, exm_frame* f, int views, cudaStream_t s) {
    size_t need = (size_t)views * m->nv;
    if (need > f->snap_capacity) {
        cudaFree(f->XY);
        cudaFree(f->Zq);
        f->XY = nullptr;
        f->Zq = nullptr;
        if (exm_malloc((void**)&f->XY, need * sizeof(int2)) != cudaSuccess ||
            exm_malloc((void**)&f->Zq, need * sizeof(uint32_t)) != cudaSuccess) {
            f->snap_capacity = 0;
            return exm_fail(EXM_ERR_OOM, "snap buffers");
        }
        f->snap_capacity = need;
    }
    if (!f->big_tris && exm_malloc((void**)&f->big_tris, (size_t)kBigTriCap * sizeof(uint2)) != cudaSuccess) {
        f->big_tris = nullptr;
        return exm_fail(EXM_ERR_OOM, "large-triangle list");
    }
    size_t npx = (size_t)views * f->W * f->H;
    cudaMemsetAsync(f->visbuf, 0xff, npx * sizeof(uint64_t), s);
    cudaMemsetAsync(f->counters, 0, 3 * sizeof(uint32_t), s);  // covered count, work cursor, large triangles
    dim3 g1(exm_blocks(m->nv, 256), views);
    snap_kernel<<<g1, 256, 0, s>>>(m->V, m->nv, (const Cam*)f->cams, views, (int2*)f->XY, f->Zq, ctx->d_status);
    dim3 g2(exm_blocks(m->nf, 128), views);
    raster_kernel<<<g2, 128, 0, s>>>(m->F, m->nf, m->nv, (const int2*)f->XY, f->Zq, views, f->W, f->H,
                                     (unsigned long long*)f->visbuf, f->big_tris, f->counters + 2, ctx->d_status);
    raster_big_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(m->F, m->nv, (const int2*)f->XY, f->Zq, f->W, f->H,
                                                        (unsigned long long*)f->visbuf, f->big_tris, f->counters + 2,
                                                        ctx->d_status);
    size_t tiles = (size_t)((f->W + 7) / 8) * ((f->H + 3) / 4) * views;
    compact_kernel<<<exm_blocks(tiles * 32, 256), 256, 0, s>>>((const unsigned long long*)f->visbuf, views, f->W,
                                                               f->H, f->pixels, f->counters);
    ctx->launches += 4;
    return exm_cuda_check(cudaGetLastError(), "raster launch");
}
