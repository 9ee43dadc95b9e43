// Tangent frames of the attribute query (Sec. 5.1: the normal map is taken to world space
// "using the tangent frame interpolated on the current face"): per-vertex normals (sum of
// incident face cross products) and per-UV-vertex tangents (sum of incident dP/du
// directions, UV-area weighted), normalised; and their adjoint for vertex gradients.
#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

// UV handedness of a face: sign of the FP32 UV doubled area (one rounding per operation).
__device__ __forceinline__ float uv_sign(const float* UV, int a, int b, int c) {
    float du1 = ssub(UV[2 * b], UV[2 * a]), dv1 = ssub(UV[2 * b + 1], UV[2 * a + 1]);
    float du2 = ssub(UV[2 * c], UV[2 * a]), dv2 = ssub(UV[2 * c + 1], UV[2 * a + 1]);
    float det = ssub(smul(du1, dv2), smul(du2, dv1));
    return det < 0.0f ? -1.0f : 1.0f;
}

// The sums are accumulated in 64-bit fixed point (2^-40 units): integer addition is
// associative, so the frames do not depend on the order in which faces are summed and
// every upload of the same mesh yields bit-identical normals and tangents.
// Scaling by the power of two 2^40 is exact in FP32 (no overflow for |v| < 2^87), and the
// conversions round once, to nearest even: the same integers as rounding the exact products.
constexpr float kFix = 0x1p40f;
constexpr float kInvFix = 0x1p-40f;

__device__ __forceinline__ void fix_add(unsigned long long* p, float v) {
    atomicAdd(p, (unsigned long long)__float2ll_rn(__fmul_rn(v, kFix)));
}
__device__ __forceinline__ float fix_value(unsigned long long x) {
    return __fmul_rn(__ll2float_rn((long long)x), kInvFix);
}

__global__ void frames_accumulate_kernel(const float* __restrict__ V, const int32_t* __restrict__ F,
                                         const float* __restrict__ UV, const int32_t* __restrict__ Fuv, int nf,
                                         int nv, int nuv, unsigned long long* nacc, unsigned long long* tacc,
                                         float* fsign, uint32_t* status) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    int u0 = Fuv[3 * f], u1 = Fuv[3 * f + 1], u2 = Fuv[3 * f + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv || u0 < 0 || u1 < 0 || u2 < 0 ||
        u0 >= nuv || u1 >= nuv || u2 >= nuv) {
        atomicOr(status, ERRBIT_INDEX);
        fsign[f] = 1.0f;
        return;
    }
    float3 p0 = ld3(V + 3 * i0), p1 = ld3(V + 3 * i1), p2 = ld3(V + 3 * i2);
    float3 e1 = p1 - p0, e2 = p2 - p0;
    float3 fn = cross(e1, e2);
    int idx[3] = {i0, i1, i2};
    for (int k = 0; k < 3; ++k) {
        fix_add(nacc + 3 * idx[k], fn.x);
        fix_add(nacc + 3 * idx[k] + 1, fn.y);
        fix_add(nacc + 3 * idx[k] + 2, fn.z);
    }
    float s = uv_sign(UV, u0, u1, u2);
    fsign[f] = s;
    float dv1 = UV[2 * u1 + 1] - UV[2 * u0 + 1], dv2 = UV[2 * u2 + 1] - UV[2 * u0 + 1];
    float3 tf = s * (dv2 * e1 - dv1 * e2);
    int uidx[3] = {u0, u1, u2};
    for (int k = 0; k < 3; ++k) {
        fix_add(tacc + 3 * uidx[k], tf.x);
        fix_add(tacc + 3 * uidx[k] + 1, tf.y);
        fix_add(tacc + 3 * uidx[k] + 2, tf.z);
    }
}

// Fixed-point sums -> float sums (kept for the adjoint) and unit vectors.
__global__ void normalize_rows_kernel(const unsigned long long* __restrict__ fix, int n, float* acc, float* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 a = f3(fix_value(fix[3 * i]), fix_value(fix[3 * i + 1]), fix_value(fix[3 * i + 2]));
    acc[3 * i] = a.x; acc[3 * i + 1] = a.y; acc[3 * i + 2] = a.z;
    float l2 = dot(a, a);
    float3 u = l2 > 0.0f ? rsqrtf(l2) * a : f3(0.0f, 0.0f, 1.0f);
    out[3 * i] = u.x; out[3 * i + 1] = u.y; out[3 * i + 2] = u.z;
}

// Adjoint of u = a / |a|: du -> (du - (du.u) u) / |a|, in place on the float4 buffer.
__global__ void unnormalize_adjoint_kernel(const float* __restrict__ acc, const float* __restrict__ unit, int n,
                                           float4* g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 a = ld3(acc + 3 * i), u = ld3(unit + 3 * i);
    float4 gv = g[i];
    float3 gu = f3(gv.x, gv.y, gv.z);
    float l2 = dot(a, a);
    float3 ga = l2 > 0.0f ? rsqrtf(l2) * (gu - dot(gu, u) * u) : f3(0.0f, 0.0f, 0.0f);
    g[i] = make_float4(ga.x, ga.y, ga.z, 0.0f);
}

// Adjoint of the per-face accumulation: n_acc += e1 x e2 and t_acc += s (dv2 e1 - dv1 e2).
__global__ void frames_adjoint_kernel(const float* __restrict__ V, const int32_t* __restrict__ F,
                                      const float* __restrict__ UV, const int32_t* __restrict__ Fuv,
                                      const float* __restrict__ fsign, int nf, const float4* __restrict__ gn,
                                      const float4* __restrict__ gt, float* gV) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    int u0 = Fuv[3 * f], u1 = Fuv[3 * f + 1], u2 = Fuv[3 * f + 2];
    float3 p0 = ld3(V + 3 * i0), p1 = ld3(V + 3 * i1), p2 = ld3(V + 3 * i2);
    float3 e1 = p1 - p0, e2 = p2 - p0;
    float4 a = gn[i0], b = gn[i1], c = gn[i2];
    float3 gfn = f3(a.x + b.x + c.x, a.y + b.y + c.y, a.z + b.z + c.z);
    float3 ge1 = cross(e2, gfn), ge2 = cross(gfn, e1);
    float4 ta = gt[u0], tb = gt[u1], tc = gt[u2];
    float3 gtf = f3(ta.x + tb.x + tc.x, ta.y + tb.y + tc.y, ta.z + tb.z + tc.z);
    float s = fsign[f];
    float dv1 = UV[2 * u1 + 1] - UV[2 * u0 + 1], dv2 = UV[2 * u2 + 1] - UV[2 * u0 + 1];
    ge1 += (s * dv2) * gtf;
    ge2 += (-s * dv1) * gtf;
    float3 g0 = f3(0.f, 0.f, 0.f) - ge1 - ge2;
    atomicAdd(gV + 3 * i0, g0.x); atomicAdd(gV + 3 * i0 + 1, g0.y); atomicAdd(gV + 3 * i0 + 2, g0.z);
    atomicAdd(gV + 3 * i1, ge1.x); atomicAdd(gV + 3 * i1 + 1, ge1.y); atomicAdd(gV + 3 * i1 + 2, ge1.z);
    atomicAdd(gV + 3 * i2, ge2.x); atomicAdd(gV + 3 * i2 + 1, ge2.y); atomicAdd(gV + 3 * i2 + 2, ge2.z);
}

}  // namespace exm

using namespace exm;

exm_status exm_frames_build(exm_mesh* m, cudaStream_t s) {
    cudaMemsetAsync(m->nfix, 0, (size_t)m->nv * 3 * 8, s);
    cudaMemsetAsync(m->tfix, 0, (size_t)m->nuv * 3 * 8, s);
    frames_accumulate_kernel<<<exm_blocks(m->nf, 256), 256, 0, s>>>(m->V, m->F, m->UV, m->Fuv, m->nf, m->nv, m->nuv,
                                                                   m->nfix, m->tfix, m->fsign, m->ctx->d_status);
    normalize_rows_kernel<<<exm_blocks(m->nv, 256), 256, 0, s>>>(m->nfix, m->nv, m->nacc, m->nrm);
    normalize_rows_kernel<<<exm_blocks(m->nuv, 256), 256, 0, s>>>(m->tfix, m->nuv, m->tacc, m->tan);
    m->ctx->launches += 3;
    return exm_cuda_check(cudaGetLastError(), "frames launch");
}

exm_status exm_frames_adjoint(exm_mesh* m, float4* gn, float4* gt, float* gV, cudaStream_t s) {
    unnormalize_adjoint_kernel<<<exm_blocks(m->nv, 256), 256, 0, s>>>(m->nacc, m->nrm, m->nv, gn);
    unnormalize_adjoint_kernel<<<exm_blocks(m->nuv, 256), 256, 0, s>>>(m->tacc, m->tan, m->nuv, gt);
    frames_adjoint_kernel<<<exm_blocks(m->nf, 256), 256, 0, s>>>(m->V, m->F, m->UV, m->Fuv, m->fsign, m->nf, gn, gt, gV);
    return exm_cuda_check(cudaGetLastError(), "frames adjoint launch");
}
