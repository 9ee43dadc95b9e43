// Stage-II objective (Sec. 5.4, Eqs. 21-24) and the Adam step that follows it.
//
//   L_img    = lambda_log |log(1 + I^) - log(1 + I)|_1 + lambda_ssim (1 - SSIM(G(I^), G(I)))
//   L_mat    = sum over P in {A, R, N} (+ M) of TV(P^), P^ the map fetched at the primary hits
//   L_env    = TV(E),  L_chroma = |mean(E) - mu_E 1|^2
//
// with lambda_log = 1 - lambda_ssim, G the sRGB transfer curve, SSIM per channel with an
// 11 x 11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2) averaged over
// views, pixels and channels, TV the mean absolute difference over neighbour pairs (screen
// pairs whose two pixels see the surface; the environment wraps in longitude).
//
// SSIM runs as two tiled kernels per (view, channel) plane.  The first stages a 32 x 16
// output tile plus a 5-texel halo of both sRGB images in shared memory, takes the five local
// moments with a separable pass and writes SSIM's partial derivatives with respect to the
// moments (a, b, c below).  The second convolves a, b, c the same way; the gradient at q is
// conv(a) + x(q) conv(b) + y(q) conv(c), the Gaussian being its own transpose.
#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

constexpr int kWin = 11;
constexpr int kRad = kWin / 2;
constexpr int kTW = 32, kTH = 16;  // SSIM output tile (one thread per output, warp = tile row)
constexpr int kSW = kTW + 2 * kRad, kSH = kTH + 2 * kRad;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Gauss {
    float w[kWin];
};

// accumulator slots of one objective call: signed 64-bit fixed point (integer addition is
// exact and order-independent, so the loss values are deterministic)
enum : int {
    ACC_LOG = 0,
    ACC_SSIM = 1,
    ACC_MAT = 2,    // 8: group * 2 + (0 horizontal, 1 vertical)
    ACC_PAIRS = 10, // 2: horizontal, vertical screen pairs
    ACC_ESUM = 12,  // 3: per-channel sums of E
    ACC_ETV = 15,   // 2: horizontal, vertical
};
constexpr int kAccSlots = 20;

__device__ __forceinline__ float srgb_f(float x) {
    return x <= 0.0031308f ? 12.92f * x : 1.055f * powf(x, 1.0f / 2.4f) - 0.055f;
}
__device__ __forceinline__ float srgb_d(float x) {
    return x <= 0.0031308f ? 12.92f : (1.055f / 2.4f) * powf(x, 1.0f / 2.4f - 1.0f);
}
__device__ __forceinline__ float sgnf(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

// Fixed-point scales of the slots: 2^32 for the image and material sums (terms of magnitude at
// most a few units, at most ~10^8 of them), 1 for the pair counts, 2^16 for the environment
// sums (HDR texel values).
constexpr float kFixImg = 0x1p32f, kFixEnv = 0x1p16f;

// A thread's running sum as a double word (hi + lo), one TwoSum per term.
__device__ __forceinline__ void ff_acc(FF& s, float x) {
    const FF t = ff_two_sum(s.hi, x);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, t.lo);
}

// Warp sum of the lanes' double words in `scale` fixed point, one 64-bit integer atomic per warp
// (every lane of the warp must call it).
__device__ __forceinline__ void warp_add(FF v, float scale, unsigned long long* dst) {
    long long q = __float2ll_rn(__fmul_rn(v.hi, scale)) + __float2ll_rn(__fmul_rn(v.lo, scale));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0 && q != 0) atomicAdd(dst, (unsigned long long)q);
}

// A fixed-point sum back as a double word: the integer split into two floats, then unscaled
// (a power of two: exact).
__device__ __forceinline__ FF fix_ff(unsigned long long a, float inv_scale) {
    const long long q = (long long)a;
    const float hi = __ll2float_rn(q);
    const float lo = __ll2float_rn(q - __float2ll_rn(hi));
    return FF{__fmul_rn(hi, inv_scale), __fmul_rn(lo, inv_scale)};
}
__device__ __forceinline__ float fix_f(unsigned long long a, float inv_scale) { return ff_f(fix_ff(a, inv_scale)); }

// ------------------------------------------------------------------ image term (Eq. 21)

__global__ void log_l1_kernel(const float* __restrict__ pred, const float* __restrict__ target, size_t n,
                              float scale, float* grad, unsigned long long* acc) {
    FF local = ff(0.0f);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float p = pred[i];
        const float d = log1pf(p) - log1pf(target[i]);
        ff_acc(local, fabsf(d));
        grad[i] = scale * sgnf(d) / (1.0f + p);
    }
    warp_add(local, kFixImg, acc + ACC_LOG);
}

// One (view, channel) plane of the interleaved [views, H, W, 3] images per grid z; the tile and
// its halo are read as sRGB, zero outside the image.
__global__ void __launch_bounds__(kTW * kTH) ssim_fwd_kernel(const float* __restrict__ pred,
                                                            const float* __restrict__ target, int H, int W,
                                                            Gauss g, float* coef, size_t plane_total,
                                                            unsigned long long* acc) {
    __shared__ float sx[kSH][kSW], sy[kSH][kSW];
    __shared__ float hs[5][kSH][kTW];
    const int plane = blockIdx.z, v = plane / 3, ch = plane - 3 * v;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int tid = threadIdx.x;
    for (int k = tid; k < kSH * kSW; k += blockDim.x) {
        const int r = k / kSW, c = k - r * kSW;
        const int gy = y0 + r - kRad, gx = x0 + c - kRad;
        float xv = 0.0f, yv = 0.0f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const size_t idx = (((size_t)v * H + gy) * W + gx) * 3 + ch;
            xv = srgb_f(pred[idx]);
            yv = srgb_f(target[idx]);
        }
        sx[r][c] = xv;
        sy[r][c] = yv;
    }
    __syncthreads();
    for (int k = tid; k < kSH * kTW; k += blockDim.x) {
        const int r = k / kTW, c = k - r * kTW;
        float a = 0.f, b = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float w = g.w[t], xv = sx[r][c + t], yv = sy[r][c + t];
            a += w * xv;
            b += w * yv;
            xx += w * xv * xv;
            yy += w * yv * yv;
            xy += w * xv * yv;
        }
        hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = xx; hs[3][r][c] = yy; hs[4][r][c] = xy;
    }
    __syncthreads();
    const int ty = tid / kTW, tx = tid - ty * kTW;
    const int gx = x0 + tx, gy = y0 + ty;
    FF local = ff(0.0f);
    if (gx < W && gy < H) {
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float w = g.w[t];
            mx += w * hs[0][ty + t][tx];
            my += w * hs[1][ty + t][tx];
            exx += w * hs[2][ty + t][tx];
            eyy += w * hs[3][ty + t][tx];
            exy += w * hs[4][ty + t][tx];
        }
        const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        const float A1 = 2.0f * mx * my + kC1, A2 = 2.0f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
        const float inv = 1.0f / (B1 * B2);
        const float S = A1 * A2 * inv;
        local = ff(S);
        // dS / d(mu_x), 2 dS / d(E[x^2]), dS / d(E[xy]) at this output
        const size_t o = ((size_t)plane * H + gy) * W + gx;
        coef[o] = 2.0f * my * (A2 - A1) * inv - 2.0f * mx * S * (1.0f / B1 - 1.0f / B2);
        coef[plane_total + o] = -2.0f * S / B2;
        coef[2 * plane_total + o] = 2.0f * A1 * inv;
    }
    warp_add(local, kFixImg, acc + ACC_SSIM);
}

__global__ void __launch_bounds__(kTW * kTH) ssim_bwd_kernel(const float* __restrict__ pred,
                                                            const float* __restrict__ target, int H, int W,
                                                            Gauss g, const float* __restrict__ coef,
                                                            size_t plane_total, float scale, float* grad) {
    __shared__ float sc[3][kSH][kSW];
    __shared__ float hs[3][kSH][kTW];
    const int plane = blockIdx.z, v = plane / 3, ch = plane - 3 * v;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int tid = threadIdx.x;
    for (int k = tid; k < kSH * kSW; k += blockDim.x) {
        const int r = k / kSW, c = k - r * kSW;
        const int gy = y0 + r - kRad, gx = x0 + c - kRad;
        float a = 0.f, b = 0.f, cc = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const size_t o = ((size_t)plane * H + gy) * W + gx;
            a = coef[o];
            b = coef[plane_total + o];
            cc = coef[2 * plane_total + o];
        }
        sc[0][r][c] = a; sc[1][r][c] = b; sc[2][r][c] = cc;
    }
    __syncthreads();
    for (int k = tid; k < kSH * kTW; k += blockDim.x) {
        const int r = k / kTW, c = k - r * kTW;
        float a = 0.f, b = 0.f, cc = 0.f;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float w = g.w[t];
            a += w * sc[0][r][c + t];
            b += w * sc[1][r][c + t];
            cc += w * sc[2][r][c + t];
        }
        hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = cc;
    }
    __syncthreads();
    const int ty = tid / kTW, tx = tid - ty * kTW;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= W || gy >= H) return;
    float a = 0.f, b = 0.f, cc = 0.f;
#pragma unroll
    for (int t = 0; t < kWin; ++t) {
        const float w = g.w[t];
        a += w * hs[0][ty + t][tx];
        b += w * hs[1][ty + t][tx];
        cc += w * hs[2][ty + t][tx];
    }
    const size_t idx = (((size_t)v * H + gy) * W + gx) * 3 + ch;
    const float p = pred[idx];
    const float G = a + srgb_f(p) * b + srgb_f(target[idx]) * cc;
    grad[idx] += scale * G * srgb_d(p);
}

__global__ void image_loss_finish_kernel(const unsigned long long* acc, float n, float lambda_ssim, float* loss) {
    const float l1 = fix_f(acc[ACC_LOG], 0x1p-32f) / n;
    const float dssim = ff_f(ff_sub(ff(1.0f), ff_div(fix_ff(acc[ACC_SSIM], 0x1p-32f), ff(n))));
    loss[0] = (1.0f - lambda_ssim) * l1 + lambda_ssim * dssim;
    loss[1] = l1;
    loss[2] = dssim;
}

// ------------------------------------------------------------------ material TV (Eq. 23)

struct TvArgs {
    const float4* prec;       // pixel records of the frame's last forward
    const uint32_t* pixels;   // covered pixel ids
    const uint32_t* count;    // covered count (device)
    MapView map;
    int W, H;                 // frame size
    float* gbuf;              // [P, 8] projected material
    int32_t* inv;             // [views*H*W] covered index of a screen pixel, -1 if none
    float* gmaps;
    float lambda;
    bool metallic;
    unsigned long long* acc;
};

template <typename T>
__global__ void tv_gbuf_kernel(TvArgs a) {
    const uint32_t n = *a.count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 r1 = a.prec[kPrec * (size_t)i + 1], r2 = a.prec[kPrec * (size_t)i + 2];
        const Footprint fp = footprint_i(a.map, __float_as_int(r2.y), __float_as_int(r2.z), r1.w, r2.x);
        float att[8];
        fetch8<T>(a.map, fp, att, nullptr, nullptr);
        float4* o = reinterpret_cast<float4*>(a.gbuf) + 2 * (size_t)i;
        o[0] = make_float4(att[0], att[1], att[2], att[3]);
        o[1] = make_float4(att[4], att[5], att[6], att[7]);
        a.inv[a.pixels[i]] = (int32_t)i;
    }
}

__global__ void tv_pairs_kernel(TvArgs a) {
    const uint32_t n = *a.count;
    FF h = ff(0.0f), v = ff(0.0f);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t pid = a.pixels[i];
        const uint32_t rem = pid % (uint32_t)(a.W * a.H);
        const int y = (int)(rem / a.W), x = (int)(rem - (uint32_t)y * a.W);
        if (x + 1 < a.W && a.inv[pid + 1] >= 0) ff_acc(h, 1.0f);
        if (y + 1 < a.H && a.inv[pid + a.W] >= 0) ff_acc(v, 1.0f);
    }
    warp_add(h, 1.0f, a.acc + ACC_PAIRS);
    warp_add(v, 1.0f, a.acc + ACC_PAIRS + 1);
}

// channel groups of the material map: A (0..2), R (3), N (5..7), M (4)
__device__ __forceinline__ int tv_group(int ch) { return ch < 3 ? 0 : ch == 3 ? 1 : ch == 4 ? 3 : 2; }
__device__ __forceinline__ float tv_group_size(int grp) { return grp == 0 || grp == 2 ? 3.0f : 1.0f; }

template <typename T>
__global__ void tv_grad_kernel(TvArgs a) {
    const uint32_t n = *a.count;
    const float ph = fix_f(a.acc[ACC_PAIRS], 1.0f), pv = fix_f(a.acc[ACC_PAIRS + 1], 1.0f);
    const float ih = ph > 0.0f ? 1.0f / ph : 0.0f, iv = pv > 0.0f ? 1.0f / pv : 0.0f;
    FF part[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) part[k] = ff(0.0f);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t pid = a.pixels[i];
        const uint32_t rem = pid % (uint32_t)(a.W * a.H);
        const int y = (int)(rem / a.W), x = (int)(rem - (uint32_t)y * a.W);
        const int nb[4] = {x > 0 ? a.inv[pid - 1] : -1, x + 1 < a.W ? a.inv[pid + 1] : -1,
                           y > 0 ? a.inv[pid - a.W] : -1, y + 1 < a.H ? a.inv[pid + a.W] : -1};
        const float* P = a.gbuf + 8 * (size_t)i;
        float g[8];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            const int grp = tv_group(ch);
            if (grp == 3 && !a.metallic) { g[ch] = 0.0f; continue; }
            const float p = P[ch], inv_c = 1.0f / tv_group_size(grp);
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (nb[k] < 0) continue;
                const float d = p - a.gbuf[8 * (size_t)nb[k] + ch];
                s += sgnf(d) * (k < 2 ? ih : iv);
                if (k == 1) ff_acc(part[2 * grp], fabsf(d));      // pair (x, x + 1), counted once
                if (k == 3) ff_acc(part[2 * grp + 1], fabsf(d));  // pair (y, y + 1)
            }
            g[ch] = a.lambda * s * inv_c;
        }
        if (a.gmaps) {
            const float4 r1 = a.prec[kPrec * (size_t)i + 1], r2 = a.prec[kPrec * (size_t)i + 2];
            const Footprint fp = footprint_i(a.map, __float_as_int(r2.y), __float_as_int(r2.z), r1.w, r2.x);
            scatter8(a.gmaps, fp, g);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) warp_add(part[k], kFixImg, a.acc + ACC_MAT + k);
}

__global__ void tv_finish_kernel(const unsigned long long* acc, bool metallic, float* loss) {
    const float ph = fix_f(acc[ACC_PAIRS], 1.0f), pv = fix_f(acc[ACC_PAIRS + 1], 1.0f);
    const float size[4] = {3.0f, 1.0f, 3.0f, 1.0f};
    FF tot = ff(0.0f);
    for (int grp = 0; grp < 4; ++grp) {
        if (grp == 3 && !metallic) continue;
        if (ph > 0.0f) tot = ff_add(tot, ff_div(fix_ff(acc[ACC_MAT + 2 * grp], 0x1p-32f), ff(ph * size[grp])));
        if (pv > 0.0f) tot = ff_add(tot, ff_div(fix_ff(acc[ACC_MAT + 2 * grp + 1], 0x1p-32f), ff(pv * size[grp])));
    }
    loss[0] = ff_f(tot);
}

// ------------------------------------------------------------- env TV and chroma (Eqs. 23-24)

__global__ void env_sum_kernel(const float* __restrict__ E, size_t texels, unsigned long long* acc) {
    FF s[3] = {ff(0.0f), ff(0.0f), ff(0.0f)};
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < texels; t += (size_t)gridDim.x * blockDim.x) {
        ff_acc(s[0], E[3 * t]);
        ff_acc(s[1], E[3 * t + 1]);
        ff_acc(s[2], E[3 * t + 2]);
    }
    for (int c = 0; c < 3; ++c) warp_add(s[c], kFixEnv, acc + ACC_ESUM + c);
}

__global__ void env_reg_kernel(const float* __restrict__ E, int W, int H, float lambda_env, float lambda_chroma,
                               float* grad, unsigned long long* acc) {
    const size_t texels = (size_t)W * H;
    const float inv_t = 1.0f / (float)texels;
    // channel means as double words, and their differences from the grey mean
    FF mf[3];
    for (int c = 0; c < 3; ++c) mf[c] = ff_div(fix_ff(acc[ACC_ESUM + c], 0x1p-16f), ff((float)texels));
    const FF muf = ff_div(ff_add(ff_add(mf[0], mf[1]), mf[2]), ff(3.0f));
    const float dm[3] = {ff_f(ff_sub(mf[0], muf)), ff_f(ff_sub(mf[1], muf)), ff_f(ff_sub(mf[2], muf))};
    const float ih = 1.0f / (float)(texels * 3), iv = H > 1 ? 1.0f / (float)((size_t)(H - 1) * W * 3) : 0.0f;
    FF ph = ff(0.0f), pv = ff(0.0f);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < texels; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / W), j = (int)(t - (size_t)i * W);
        const size_t l = (size_t)i * W + (j == 0 ? W - 1 : j - 1), r = (size_t)i * W + (j + 1 == W ? 0 : j + 1);
        for (int c = 0; c < 3; ++c) {
            const float e = E[3 * t + c];
            const float dr = E[3 * r + c] - e;
            ff_acc(ph, fabsf(dr));
            float g = (sgnf(e - E[3 * l + c]) - sgnf(dr)) * ih;
            if (i > 0) g += sgnf(e - E[3 * (t - W) + c]) * iv;
            if (i + 1 < H) {
                const float dd = E[3 * (t + W) + c] - e;
                ff_acc(pv, fabsf(dd));
                g -= sgnf(dd) * iv;
            }
            grad[3 * t + c] += lambda_env * g + lambda_chroma * 2.0f * dm[c] * inv_t;
        }
    }
    warp_add(ph, kFixEnv, acc + ACC_ETV);
    warp_add(pv, kFixEnv, acc + ACC_ETV + 1);
}

__global__ void env_reg_finish_kernel(const unsigned long long* acc, int W, int H, float* loss) {
    const float texels = (float)((size_t)W * H);
    FF tv = ff_div(fix_ff(acc[ACC_ETV], 0x1p-16f), ff(__fmul_rn(texels, 3.0f)));
    if (H > 1) tv = ff_add(tv, ff_div(fix_ff(acc[ACC_ETV + 1], 0x1p-16f), ff((float)((size_t)(H - 1) * W * 3))));
    FF m[3];
    for (int c = 0; c < 3; ++c) m[c] = ff_div(fix_ff(acc[ACC_ESUM + c], 0x1p-16f), ff(texels));
    const FF mu = ff_div(ff_add(ff_add(m[0], m[1]), m[2]), ff(3.0f));
    FF ch = ff(0.0f);
    for (int c = 0; c < 3; ++c) {
        const FF d = ff_sub(m[c], mu);
        ch = ff_add(ch, ff_mul(d, d));
    }
    loss[0] = ff_f(tv);
    loss[1] = ff_f(ch);
}

// ------------------------------------------------------------------ Adam

struct AdamArgs {
    float lr, beta1, beta2, eps, bc1, bc2;
    float lo[8], hi[8];
    int channels;
};

__global__ void adam_kernel(float* __restrict__ param, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, size_t n, AdamArgs a) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = a.beta1 * m[i] + (1.0f - a.beta1) * g;
        const float vi = a.beta2 * v[i] + (1.0f - a.beta2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const int ch = (int)(i % (size_t)a.channels);
        const float step = a.lr * (mi / a.bc1) / (sqrtf(vi / a.bc2) + a.eps);
        param[i] = fminf(fmaxf(param[i] - step, a.lo[ch]), a.hi[ch]);
    }
}

static Gauss gaussian() {
    Gauss g;
    double w[kWin], sum = 0.0;
    for (int t = 0; t < kWin; ++t) {
        const double k = t - kRad;
        w[t] = exp(-(k * k) / (2.0 * 1.5 * 1.5));
        sum += w[t];
    }
    for (int t = 0; t < kWin; ++t) g.w[t] = (float)(w[t] / sum);
    return g;
}

static int grid_for(exm_ctx* ctx, size_t n, int threads) {
    const size_t want = (n + threads - 1) / threads;
    const size_t cap = (size_t)ctx->num_sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

static bool ensure_acc(exm_ctx* ctx) {
    if (ctx->d_acc) return true;
    if (exm_malloc((void**)&ctx->d_acc, kAccSlots * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace exm

using namespace exm;

exm_status exm_image_loss_impl(exm_ctx* ctx, const float* pred, const float* target, int views, int W, int H,
                               float lambda_ssim, float* loss, float* grad, cudaStream_t s) {
    ExmRange range("image loss");
    const size_t n = (size_t)views * W * H * 3, planes = (size_t)views * 3, plane_total = planes * W * H;
    if (!ensure_acc(ctx) || !ensure(&ctx->scratch, &ctx->scratch_cap, 3 * plane_total))
        return exm_fail(EXM_ERR_OOM, "exm_image_loss: scratch");
    cudaMemsetAsync(ctx->d_acc, 0, kAccSlots * sizeof(unsigned long long), s);
    log_l1_kernel<<<grid_for(ctx, n, 256), 256, 0, s>>>(pred, target, n, (1.0f - lambda_ssim) / (float)n, grad,
                                                        ctx->d_acc);
    const dim3 tiles((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, (unsigned)planes);
    const Gauss g = gaussian();
    ssim_fwd_kernel<<<tiles, kTW * kTH, 0, s>>>(pred, target, H, W, g, ctx->scratch, plane_total, ctx->d_acc);
    ssim_bwd_kernel<<<tiles, kTW * kTH, 0, s>>>(pred, target, H, W, g, ctx->scratch, plane_total,
                                                -lambda_ssim / (float)n, grad);
    image_loss_finish_kernel<<<1, 1, 0, s>>>(ctx->d_acc, (float)n, lambda_ssim, loss);
    ctx->launches += 4;
    return exm_cuda_check(cudaGetLastError(), "exm_image_loss launch");
}

exm_status exm_material_tv_impl(exm_ctx* ctx, const void* maps, exm_dtype dt, int mapW, int mapH, exm_frame* f,
                                uint32_t flags, float lambda_mat, float* loss, float* grad_maps, cudaStream_t s) {
    if (f->last_nd < 0 || !f->prec) return exm_fail(EXM_ERR_ARG, "exm_material_tv: the frame holds no forward pass");
    const size_t P = (size_t)f->views * f->W * f->H;
    if (!ensure_acc(ctx) || !ensure(&f->tv_gbuf, &f->tv_gbuf_cap, 8 * P) || !ensure(&f->tv_inv, &f->tv_inv_cap, P))
        return exm_fail(EXM_ERR_OOM, "exm_material_tv: scratch");
    cudaMemsetAsync(ctx->d_acc, 0, kAccSlots * sizeof(unsigned long long), s);
    cudaMemsetAsync(f->tv_inv, 0xff, P * sizeof(int32_t), s);
    TvArgs a;
    a.prec = f->prec;
    a.pixels = f->pixels;
    a.count = f->counters;
    a.map.data = maps;
    a.map.W = mapW;
    a.map.H = mapH;
    a.map.wrap_u = (flags & EXM_FLAG_WRAP_U) != 0;
    a.W = f->W;
    a.H = f->H;
    a.gbuf = f->tv_gbuf;
    a.inv = f->tv_inv;
    a.gmaps = grad_maps;
    a.lambda = lambda_mat;
    a.metallic = (flags & EXM_FLAG_NO_METALLIC) == 0;
    a.acc = ctx->d_acc;
    const int grid = grid_for(ctx, P, 256);
    switch (dt) {
        case EXM_F32: tv_gbuf_kernel<float><<<grid, 256, 0, s>>>(a); break;
        case EXM_BF16: tv_gbuf_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(a); break;
        default: tv_gbuf_kernel<__half><<<grid, 256, 0, s>>>(a); break;
    }
    tv_pairs_kernel<<<grid, 256, 0, s>>>(a);
    switch (dt) {
        case EXM_F32: tv_grad_kernel<float><<<grid, 256, 0, s>>>(a); break;
        case EXM_BF16: tv_grad_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(a); break;
        default: tv_grad_kernel<__half><<<grid, 256, 0, s>>>(a); break;
    }
    tv_finish_kernel<<<1, 1, 0, s>>>(ctx->d_acc, a.metallic, loss);
    ctx->launches += 4;
    return exm_cuda_check(cudaGetLastError(), "exm_material_tv launch");
}

exm_status exm_env_regularizers_impl(exm_ctx* ctx, const float* E, int W, int H, float lambda_env,
                                     float lambda_chroma, float* loss, float* grad_env, cudaStream_t s) {
    if (!ensure_acc(ctx)) return exm_fail(EXM_ERR_OOM, "exm_env_regularizers: scratch");
    const size_t texels = (size_t)W * H;
    cudaMemsetAsync(ctx->d_acc, 0, kAccSlots * sizeof(unsigned long long), s);
    env_sum_kernel<<<grid_for(ctx, texels, 256), 256, 0, s>>>(E, texels, ctx->d_acc);
    env_reg_kernel<<<grid_for(ctx, texels, 256), 256, 0, s>>>(E, W, H, lambda_env, lambda_chroma, grad_env,
                                                             ctx->d_acc);
    env_reg_finish_kernel<<<1, 1, 0, s>>>(ctx->d_acc, W, H, loss);
    ctx->launches += 3;
    return exm_cuda_check(cudaGetLastError(), "exm_env_regularizers launch");
}

exm_status exm_adam_step_impl(exm_ctx* ctx, float* param, const float* grad, float* m, float* v, size_t rows,
                              int channels, float lr, float beta1, float beta2, float eps, int step, const float* lo,
                              const float* hi, cudaStream_t s) {
    ExmRange range("Adam step");
    AdamArgs a;
    a.lr = lr;
    a.beta1 = beta1;
    a.beta2 = beta2;
    a.eps = eps;
    a.bc1 = (float)(1.0 - pow((double)beta1, (double)step));
    a.bc2 = (float)(1.0 - pow((double)beta2, (double)step));
    a.channels = channels;
    for (int c = 0; c < 8; ++c) {
        a.lo[c] = (lo && c < channels) ? lo[c] : -INFINITY;
        a.hi[c] = (hi && c < channels) ? hi[c] : INFINITY;
    }
    const size_t n = rows * (size_t)channels;
    adam_kernel<<<grid_for(ctx, n, 256), 256, 0, s>>>(param, grad, m, v, n, a);
    ctx->launches += 1;
    return exm_cuda_check(cudaGetLastError(), "exm_adam_step launch");
}
