// Environment importance distribution (Sec. 5.2): "brightness of the environment map and
// the spherical area weights".  Integer weights q = 1 + floor(lum * sin(theta_row) * 2^24 /
// max), exact 64-bit prefix sums (so the texel a target picks is independent of summation
// order), a guide table indexed by the top bits of the 32-bit stratified fraction, and a
// per-texel record (E.rgb, (q/Q) * W*H / (2 pi^2)) read once per light sample.
#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename T>
__global__ void env_weight_kernel(const T* __restrict__ E, int W, int H, float4* texel, float* wbuf, uint32_t* wmax) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    float w = 0.0f;
    if (t < W * H) {
        int i = t / W;
        float r = to_f(E[3 * (size_t)t]), g = to_f(E[3 * (size_t)t + 1]), b = to_f(E[3 * (size_t)t + 2]);
        float sn, cs;
        sincos2pi(sdiv((float)(2 * i + 1), (float)(4 * H)), &sn, &cs);
        float lum = sadd(sadd(smul(0x1.b367a0p-3f, r), smul(0x1.6e2eb2p-1f, g)), smul(0x1.27bb30p-4f, b));
        w = smul(lum, sn);
        if (!(w > 0.0f)) w = 0.0f;
        wbuf[t] = w;
        texel[t] = make_float4(r, g, b, 0.0f);
    }
    for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((threadIdx.x & 31) == 0) atomicMax(wmax, __float_as_uint(w));
}

// One block per row: integer weights, inclusive in-row prefix, row sum.
__global__ void env_row_kernel(const float* __restrict__ wbuf, int W, const uint32_t* __restrict__ wmax,
                               uint32_t* q, uint64_t* cdf, uint64_t* rowsum) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    int i = blockIdx.x;
    float wm = __uint_as_float(*wmax);
    float scale = 0.0f;
    if (wm > 0.0f) {
        scale = sdiv(16777216.0f, wm);
        if (!(scale <= 3.4028235e38f)) scale = 3.4028235e38f;
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < W; base += blockDim.x) {
        int j = base + threadIdx.x;
        uint64_t v = 0;
        if (j < W) {
            size_t t = (size_t)i * W + j;
            float w = wbuf[t];
            uint32_t qq = 1;
            if (w > 0.0f) {
                float x = smul(w, scale);
                if (!(x < 16777216.0f)) x = 16777216.0f;
                qq = 1u + (uint32_t)x;
            }
            q[t] = qq;
            v = qq;
        }
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint64_t s = lane < nw ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) warp_tot[lane] = s;
        }
        __syncthreads();
        uint64_t pre = carry + x + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (j < W) cdf[(size_t)i * W + j] = pre;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pre;
        __syncthreads();
    }
    if (threadIdx.x == 0) rowsum[i] = carry;
}

// Single block: exclusive prefix of the row sums and the total Q.
__global__ void env_rows_prefix_kernel(const uint64_t* __restrict__ rowsum, int H, uint64_t* rowpre, uint64_t* total) {
    if (threadIdx.x != 0) return;
    uint64_t acc = 0;
    for (int i = 0; i < H; ++i) { rowpre[i] = acc; acc += rowsum[i]; }
    *total = acc;
}

__global__ void env_finish_kernel(int W, int H, const uint64_t* __restrict__ rowpre, const uint64_t* __restrict__ total,
                                  const uint32_t* __restrict__ q, uint64_t* cdf, float4* texel) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * H) return;
    int i = t / W;
    cdf[t] += rowpre[i];
    float Q = (float)(*total);
    float p = (float)q[t] / Q * ((float)W * (float)H / (2.0f * kPi * kPi));
    texel[t].w = p;
}

// Row guide: the row picked at each U1 = g * 2^(32-rbits); entry Gr is H - 1.
__global__ void env_row_guide_kernel(const uint64_t* __restrict__ cdf, int W, int H, const uint64_t* __restrict__ total,
                                     int rbits, uint32_t* rguide) {
    const uint32_t G = 1u << rbits;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > G) return;
    if (g == G) { rguide[g] = (uint32_t)H - 1; return; }
    const uint64_t t = scaled_target(g << (32 - rbits), *total);
    uint32_t lo = 0, hi = (uint32_t)H - 1;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (cdf[(size_t)mid * W + W - 1] > t) hi = mid; else lo = mid + 1;
    }
    rguide[g] = lo;
}

// Column guides: for each row, the column picked at each U2 = g * 2^(32-cbits).
__global__ void env_col_guide_kernel(const uint64_t* __restrict__ cdf, int W, int H, int cbits, uint32_t* cguide) {
    const uint32_t G = 1u << cbits;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)H * (G + 1)) return;
    const uint32_t row = (uint32_t)(t / (G + 1)), g = (uint32_t)(t % (G + 1));
    if (g == G) { cguide[t] = (uint32_t)W - 1; return; }
    const uint64_t* rc = cdf + (size_t)row * W;
    const uint64_t pre = row ? rc[-1] : 0ull;
    const uint64_t tc = pre + scaled_target(g << (32 - cbits), rc[W - 1] - pre);
    uint32_t lo = 0, hi = (uint32_t)W - 1;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (rc[mid] > tc) hi = mid; else lo = mid + 1;
    }
    cguide[t] = lo;
}

}  // namespace exm

using namespace exm;

exm_status exm_env_prepare_impl(exm_env* e, const void* E, exm_dtype dt, cudaStream_t s) {
    ExmRange range("environment distribution");
    int n = e->W * e->H;
    cudaMemsetAsync(e->wmax, 0, 4, s);
    int blocks = exm_blocks(n, 256);
    switch (dt) {
        case EXM_F32:
            env_weight_kernel<float><<<blocks, 256, 0, s>>>((const float*)E, e->W, e->H, e->texel, e->wbuf, e->wmax);
            break;
        case EXM_BF16:
            env_weight_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)E, e->W, e->H, e->texel,
                                                                     e->wbuf, e->wmax);
            break;
        case EXM_F16:
            env_weight_kernel<__half><<<blocks, 256, 0, s>>>((const __half*)E, e->W, e->H, e->texel, e->wbuf, e->wmax);
            break;
        default:
            return exm_fail(EXM_ERR_ARG, "env dtype");
    }
    int rt = e->W >= 1024 ? 1024 : ((e->W + 31) / 32) * 32;
    env_row_kernel<<<e->H, rt, 0, s>>>(e->wbuf, e->W, e->wmax, e->q, e->cdf, e->rowsum);
    env_rows_prefix_kernel<<<1, 32, 0, s>>>(e->rowsum, e->H, e->rowpre, e->total);
    env_finish_kernel<<<blocks, 256, 0, s>>>(e->W, e->H, e->rowpre, e->total, e->q, e->cdf, e->texel);
    env_row_guide_kernel<<<exm_blocks(((size_t)1 << e->rbits) + 1, 256), 256, 0, s>>>(e->cdf, e->W, e->H, e->total,
                                                                                    e->rbits, e->rguide);
    env_col_guide_kernel<<<exm_blocks((size_t)e->H * (((size_t)1 << e->cbits) + 1), 256), 256, 0, s>>>(
        e->cdf, e->W, e->H, e->cbits, e->cguide);
    e->ctx->launches += 6;
    return exm_cuda_check(cudaGetLastError(), "env prepare launch");
}
