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

// a2: one thread per (view, triangle).  Integer edge functions, lexicographic (top-left)
// fill rule, back faces culled, depth = floor(sum E_i Z_i / A2), 64-bit atomicMin.
__global__ void raster_kernel(const int32_t* __restrict__ F, int nf, int nv, const int2* __restrict__ XY,
                              const uint32_t* __restrict__ Zq, int views, int W, int H,
                              unsigned long long* __restrict__ visbuf, uint32_t* status) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (f >= nf || c >= views) return;
    int ia = __ldg(F + 3 * f), ib = __ldg(F + 3 * f + 1), ic = __ldg(F + 3 * f + 2);
    if ((unsigned)ia >= (unsigned)nv || (unsigned)ib >= (unsigned)nv || (unsigned)ic >= (unsigned)nv) return;
    const int2* xy = XY + (size_t)c * nv;
    const uint32_t* zq = Zq + (size_t)c * nv;
    int2 a = xy[ia], b = xy[ib], d = xy[ic];
    if (a.x == kBadSnap || b.x == kBadSnap || d.x == kBadSnap) return;
    long long X0 = a.x, Y0 = a.y, X1 = b.x, Y1 = b.y, X2 = d.x, Y2 = d.y;
    long long A2 = (Y1 - Y0) * (X2 - X0) - (X1 - X0) * (Y2 - Y0);
    if (A2 <= 0) return;
    if (A2 >= (1ll << 38)) { atomicOr(status, ERRBIT_GUARD); return; }
    long long Z0 = zq[ia], Z1 = zq[ib], Z2 = zq[ic];
    long long mnx = min(X0, min(X1, X2)), mxx = max(X0, max(X1, X2));
    long long mny = min(Y0, min(Y1, Y2)), mxy = max(Y0, max(Y1, Y2));
    long long x0 = mnx - 128 <= 0 ? 0 : (mnx - 128 + 255) / 256;
    long long x1 = mxx - 128 < 0 ? -1 : (mxx - 128) / 256;
    long long y0 = mny - 128 <= 0 ? 0 : (mny - 128 + 255) / 256;
    long long y1 = mxy - 128 < 0 ? -1 : (mxy - 128) / 256;
    x1 = min(x1, (long long)W - 1);
    y1 = min(y1, (long long)H - 1);
    bool in0 = edge_incl(X2 - X1, Y2 - Y1), in1 = edge_incl(X0 - X2, Y0 - Y2), in2 = edge_incl(X1 - X0, Y1 - Y0);
    unsigned long long* vb = visbuf + (size_t)c * W * H;
    for (long long py = y0; py <= y1; ++py) {
        long long Py = py * 256 + 128;
        for (long long px = x0; px <= x1; ++px) {
            long long Px = px * 256 + 128;
            long long E0 = (Y1 - Py) * (X2 - Px) - (X1 - Px) * (Y2 - Py);
            long long E1 = (Y2 - Py) * (X0 - Px) - (X2 - Px) * (Y0 - Py);
            long long E2 = (Y0 - Py) * (X1 - Px) - (X0 - Px) * (Y1 - Py);
            if (!(E0 > 0 || (E0 == 0 && in0))) continue;
            if (!(E1 > 0 || (E1 == 0 && in1))) continue;
            if (!(E2 > 0 || (E2 == 0 && in2))) continue;
            long long num = E0 * Z0 + E1 * Z1 + E2 * Z2;
            unsigned long long z = (unsigned long long)(num / A2);
            unsigned long long key = (z << 32) | (unsigned long long)(uint32_t)f;
            atomicMin(vb + py * W + px, key);
        }
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
    size_t npx = (size_t)views * f->W * f->H;
    cudaMemsetAsync(f->visbuf, 0xff, npx * sizeof(uint64_t), s);
    cudaMemsetAsync(f->counters, 0, 2 * sizeof(uint32_t), s);
    dim3 g1(exm_blocks(m->nv, 256), views);
    snap_kernel<<<g1, 256, 0, s>>>(m->V, m->nv, (const Cam*)f->cams, views, (int2*)f->XY, f->Zq, ctx->d_status);
    dim3 g2(exm_blocks(m->nf, 128), views);
    raster_kernel<<<g2, 128, 0, s>>>(m->F, m->nf, m->nv, (const int2*)f->XY, f->Zq, views, f->W, f->H,
                                     (unsigned long long*)f->visbuf, ctx->d_status);
    size_t tiles = (size_t)((f->W + 7) / 8) * ((f->H + 3) / 4) * views;
    compact_kernel<<<exm_blocks(tiles * 32, 256), 256, 0, s>>>((const unsigned long long*)f->visbuf, views, f->W,
                                                               f->H, f->pixels, f->counters);
    ctx->launches += 3;
    return exm_cuda_check(cudaGetLastError(), "raster launch");
}
