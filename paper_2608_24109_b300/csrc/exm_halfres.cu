// Indirect light at half resolution (the paper's implementation details, Sec. 6.1: secondary
// rays are traced at half resolution in both image dimensions and the indirect component is
// upsampled to full resolution).
//
// The full-resolution frame renders the direct term only.  A child frame of W' = ceil(W/2) x
// H' = ceil(H/2) pixels renders the same cameras with halved intrinsics (its pixel (i, j) is
// centred on the full-resolution point (2i + 1, 2j + 1)) with no direct samples, giving
// lambda_ind L_ind at its own primary hits (0 where it sees no surface).  Every covered
// full-resolution pixel then adds the bilinear interpolation of that image at
// x' = (x + 1/2)/2 - 1/2, y' likewise, from the taps floor and floor + 1 clamped to the image.
// The backward runs the direct adjoint on the full frame, scatters the pixel gradients back
// through the interpolation weights onto the half image, and runs the indirect adjoint of
// the child frame on that.
#include <vector>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

__device__ __forceinline__ void half_taps(int x, int n_in, int* i0, int* i1, float* f) {
    const float src = ((float)x + 0.5f) * 0.5f - 0.5f;  // exact: a multiple of 1/4
    const float fl = floorf(src);
    *f = src - fl;
    const int a = (int)fl;
    *i0 = min(max(a, 0), n_in - 1);
    *i1 = min(max(a + 1, 0), n_in - 1);
}

__global__ void upsample_add_kernel(const float* __restrict__ half, int Wh, int Hh, const uint32_t* __restrict__ pixels,
                                    const uint32_t* __restrict__ count, int W, int H, float* out) {
    const uint32_t n = *count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t pid = pixels[i];
        const uint32_t v = pid / (uint32_t)(W * H), rem = pid - v * (uint32_t)(W * H);
        const int y = (int)(rem / W), x = (int)(rem - (uint32_t)y * W);
        int x0, x1, y0, y1;
        float fx, fy;
        half_taps(x, Wh, &x0, &x1, &fx);
        half_taps(y, Hh, &y0, &y1, &fy);
        const float* r0 = half + ((size_t)v * Hh + y0) * Wh * 3;
        const float* r1 = half + ((size_t)v * Hh + y1) * Wh * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float top = (1.0f - fx) * r0[3 * x0 + c] + fx * r0[3 * x1 + c];
            const float bot = (1.0f - fx) * r1[3 * x0 + c] + fx * r1[3 * x1 + c];
            out[3 * (size_t)pid + c] += (1.0f - fy) * top + fy * bot;
        }
    }
}

__global__ void upsample_adjoint_kernel(const float* __restrict__ grad, const uint32_t* __restrict__ pixels,
                                        const uint32_t* __restrict__ count, int W, int H, int Wh, int Hh,
                                        float* ghalf) {
    const uint32_t n = *count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t pid = pixels[i];
        const uint32_t v = pid / (uint32_t)(W * H), rem = pid - v * (uint32_t)(W * H);
        const int y = (int)(rem / W), x = (int)(rem - (uint32_t)y * W);
        int x0, x1, y0, y1;
        float fx, fy;
        half_taps(x, Wh, &x0, &x1, &fx);
        half_taps(y, Hh, &y0, &y1, &fy);
        float* r0 = ghalf + ((size_t)v * Hh + y0) * Wh * 3;
        float* r1 = ghalf + ((size_t)v * Hh + y1) * Wh * 3;
        const float w00 = (1.0f - fy) * (1.0f - fx), w01 = (1.0f - fy) * fx, w10 = fy * (1.0f - fx), w11 = fy * fx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float g = grad[3 * (size_t)pid + c];
            if (g == 0.0f) continue;
            atomicAdd(r0 + 3 * x0 + c, w00 * g);
            atomicAdd(r0 + 3 * x1 + c, w01 * g);
            atomicAdd(r1 + 3 * x0 + c, w10 * g);
            atomicAdd(r1 + 3 * x1 + c, w11 * g);
        }
    }
}

}  // namespace exm

using namespace exm;

// The child frame of `f` at half resolution (created or resized on demand).
static exm_status half_frame(exm_ctx* c, exm_frame* f, exm_frame** out) {
    const int Wh = (f->W + 1) / 2, Hh = (f->H + 1) / 2;
    if (f->half && (f->half->views != f->views || f->half->W != Wh || f->half->H != Hh)) {
        exm_frame_destroy(f->half);
        f->half = nullptr;
    }
    if (!f->half) {
        exm_status st = exm_frame_create(c, f->views, Wh, Hh, &f->half);
        if (st != EXM_OK) return st;
    }
    f->half->ray_cap = f->ray_cap;
    f->half->saved_budget = f->saved_budget;
    *out = f->half;
    return EXM_OK;
}

static std::vector<exm_camera> half_cameras(const exm_camera* cams, int views) {
    std::vector<exm_camera> h(cams, cams + views);
    for (auto& c : h) {
        c.kx *= 0.5f;
        c.ky *= 0.5f;
        c.cx *= 0.5f;
        c.cy *= 0.5f;
    }
    return h;
}

static int grid_pixels(exm_ctx* c, const exm_frame* f) {
    const size_t P = (size_t)f->views * f->W * f->H;
    const size_t want = (P + 255) / 256, cap = (size_t)c->num_sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

exm_status exm_render_forward_halfres(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                      int mapH, const exm_env* e, const exm_camera* cams, int views,
                                      const exm_params* p, exm_frame* f, float* out, cudaStream_t s) {
    exm_params pd = *p;  // full resolution: direct light only
    pd.n_bounce = 0;
    pd.n_light = 0;
    exm_status st = upload_cameras(f, cams, views, s);
    if (st == EXM_OK) st = exm_raster_impl(c, m, f, views, s);
    if (st == EXM_OK) st = exm_shade_forward_impl(c, m, maps, dt, mapW, mapH, e, f, &pd, out, s);
    if (st != EXM_OK) return st;
    exm_frame* h = nullptr;
    st = half_frame(c, f, &h);
    if (st != EXM_OK) return st;
    const size_t nh = (size_t)views * h->W * h->H * 3;
    if (!ensure(&f->half_img, &f->half_img_cap, nh)) return exm_fail(EXM_ERR_OOM, "half-resolution image");
    exm_params ph = *p;  // half resolution: indirect light only
    ph.n_direct = 0;
    const std::vector<exm_camera> hc = half_cameras(cams, views);
    st = upload_cameras(h, hc.data(), views, s);
    if (st == EXM_OK) st = exm_raster_impl(c, m, h, views, s);
    if (st == EXM_OK) st = exm_shade_forward_impl(c, m, maps, dt, mapW, mapH, e, h, &ph, f->half_img, s);
    if (st != EXM_OK) return st;
    upsample_add_kernel<<<grid_pixels(c, f), 256, 0, s>>>(f->half_img, h->W, h->H, f->pixels, f->counters, f->W,
                                                         f->H, out);
    c->launches += 1;
    return exm_cuda_check(cudaGetLastError(), "half-resolution upsampling");
}

exm_status exm_render_backward_halfres(exm_ctx* c, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW,
                                       int mapH, const exm_env* e, const exm_camera* cams, int views,
                                       const exm_params* p, exm_frame* f, const float* grad_rgb, float* grad_maps,
                                       float* grad_env, float* grad_V, cudaStream_t s) {
    exm_frame* h = f->half;
    if (!h || h->views != views || h->W != (f->W + 1) / 2 || h->H != (f->H + 1) / 2 || !f->half_img)
        return exm_fail(EXM_ERR_ARG, "backward: the frame holds no half-resolution forward pass");
    exm_params pd = *p;
    pd.n_bounce = 0;
    pd.n_light = 0;
    exm_params ph = *p;
    ph.n_direct = 0;
    ph.flags &= ~EXM_FLAG_ZERO_GRADS;  // the direct adjoint below zeroes them if asked
    const std::vector<exm_camera> hc = half_cameras(cams, views);
    // both passes' saved state is checked before anything is enqueued
    exm_status st = exm_check_backward(f, m, e, mapW, mapH, cams, views, &pd);
    if (st == EXM_OK) st = exm_check_backward(h, m, e, mapW, mapH, hc.data(), views, &ph);
    if (st != EXM_OK) return st;
    const size_t nh = (size_t)views * h->W * h->H * 3;
    if (!ensure(&f->half_grad, &f->half_grad_cap, nh)) return exm_fail(EXM_ERR_OOM, "half-resolution gradient");
    st = exm_shade_backward_impl(c, m, maps, dt, mapW, mapH, e, f, &pd, grad_rgb, grad_maps, grad_env, grad_V, s);
    if (st != EXM_OK) return st;
    cudaMemsetAsync(f->half_grad, 0, nh * sizeof(float), s);
    upsample_adjoint_kernel<<<grid_pixels(c, f), 256, 0, s>>>(grad_rgb, f->pixels, f->counters, f->W, f->H, h->W,
                                                             h->H, f->half_grad);
    c->launches += 1;
    return exm_shade_backward_impl(c, m, maps, dt, mapW, mapH, e, h, &ph, f->half_grad, grad_maps, grad_env, grad_V,
                                   s);
}
