// Shading and its adjoint (Sec. 5.1-5.3, Eqs. 10-20) as a wavefront pipeline.
//
// Forward, per chunk of covered pixels:
//   gen_secondary  -> one cosine-weighted secondary ray per (pixel, j) about n_g  (Sec. 5.3)
//   trace<closest> -> the closest hit of each; valid iff front-facing              (Sec. 5.3)
//   gen_direct     -> one shadow ray per (pixel, k) above the geometric horizon    (Eq. 17)
//   gen_seclight   -> one shadow ray per (valid hit, s) above its horizon          (Eq. 18)
//   trace<any>     -> any-hit visibility of every queued shadow ray, as bits
// then pixel_surface (a thread per pixel: material and n_s into the pixel record) and one
// shade kernel, a warp per pixel, which enumerates the pixel's unoccluded samples from the
// bits (so every lane evaluates a live sample), evaluates f_r = f_d + f_s (Eqs. 13-16), the
// direct estimator (Eq. 17), L_sec at each valid hit (Eq. 18), the indirect estimator
// (Eq. 19) and the composite (Eq. 20).  gen_direct records the texel each queued direct
// sample picked, so the shade kernels re-derive a sample's direction from its stream and
// that texel without repeating the search.
//
// The backward pass is the same warp-per-pixel kernel with the adjoint: it re-derives each
// sample, reads the saved visibility bits and hit ids (no ray is traced again), scatters
// dL/dE (one padded float4 per texel) and sums the sample adjoints of n_s, w_o, a, r and m per
// pixel; shade_epilogue (a thread per pixel) carries them to dL/d(map texels) (4 bilinear
// taps x 8 channels) and dL/dV (barycentrics, position, view direction, interpolated normals
// and tangents, UV; the frame adjoint finishes it).
//
// The trace kernel is persistent: a warp claims pools of queued rays and its lanes refill
// from the pool between rounds of kRound items.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

constexpr int kShadeWarps = 4;        // warps per block of the shade kernel
constexpr int kListMax = 1024;        // sample slots enumerated per round (32 bit words)
// Queued rays per chunk at most (2 float4 each: 4 GiB).  Few, large chunks keep the persistent
// tracer's launch tails small: the geometry workload's forward takes 8 chunks (64 at 2^24 rays).
constexpr uint32_t kRayCapDefault = 1u << 27;

struct ShadeArgs {
    // mesh
    const float* V;
    const int32_t* F;
    const float* UV;
    const int32_t* Fuv;
    const float* nrm;
    const float* tan;
    const float* fsign;
    BvhView bvh;
    int bvh_layout;  // EXM_BVH_4: bvh.nodes4, _4Q: bvh.nodesq, _8Q: bvh.nodes8 (and bvh.tris in its order)
    // maps, env, frame
    MapView map;
    EnvView env;
    uint32_t env_smem;  // bytes of shared memory that stage the row phase of the texel search, 0: none
    const Cam* cams;
    const unsigned long long* visbuf;
    const uint32_t* pixels;
    const uint32_t* count;
    int W, H;
    // params
    int Nd, Nb, Ns;
    int wd, ws;        // 32-bit words per pixel of the direct / secondary visibility bits
    uint32_t nxd, nyd, nxs, nys;  // 2D strata of the direct and secondary light samples
    float lambda;
    bool metallic;
    bool sec_material;  // false: secondary hits take the constant default material
    uint2 key;
    // wavefront state
    uint32_t* visbits;   // [P * wd]
    uint32_t* secbits;   // [P * ws]
    int32_t* hits;       // [P * Nb] closest front-facing hit of each secondary ray, -1 if none
    float4* prec;        // [P * kPrec] per-pixel shading record
    float* pacc;         // [P * 12] backward: per-pixel sums of the sample adjoints
    uint32_t* tsel;      // [P * Nd] texel picked by each queued direct sample (gen_direct)
    uint32_t* tsel2;     // [P * Nb * Ns] texel picked by each queued secondary light sample (gen_seclight)
    float4* rays;        // queue: [ray_cap * 2]
    uint32_t ray_cap;
    uint32_t* ctr;       // per chunk: [0] queued, [1] fetch cursor (x2: closest, any)
    uint32_t chunk_begin, chunk_pixels;
    // per-sample state (tsel, tsel2, visibility bits, hits) holds pixels [state_base, ...): the whole
    // frame (state_base 0) or, when it is recomputed chunk by chunk, the current chunk
    uint32_t state_base;
    uint32_t shade_begin, shade_end;  // covered-pixel range of a shade launch
    // outputs
    float* out;
    unsigned long long* samples;
    unsigned long long* work;  // [4] nodes, triangle tests, BRDF evaluations, rays (COUNT)
    uint32_t* status;
    // backward
    const float* grad_rgb;
    float* gmaps;
    float4* genv;
    float* gV;
    float4* gnrm;
    float4* gtan;
};

__device__ __forceinline__ void pixel_of(const ShadeArgs& A, uint32_t pid, int* c, int* px, int* py, uint32_t* rem) {
    const uint32_t per_view = (uint32_t)A.W * (uint32_t)A.H;
    *c = (int)(pid / per_view);
    *rem = pid - (uint32_t)(*c) * per_view;
    *py = (int)(*rem / (uint32_t)A.W);
    *px = (int)(*rem - (uint32_t)(*py) * (uint32_t)A.W);
}

// Spec geometry of a covered pixel: the shading point, its geometric normal and the
// offset origin of its shadow and secondary rays (all decisions hang on these).
__device__ __forceinline__ void pixel_geometry(const ShadeArgs& A, uint32_t pid, S3* org, S3* ngs) {
    int c, px, py;
    uint32_t rem;
    pixel_of(A, pid, &c, &px, &py, &rem);
    const int f = (int)(uint32_t)(A.visbuf[pid] & 0xffffffffull);
    const int i0 = __ldg(A.F + 3 * f), i1 = __ldg(A.F + 3 * f + 1), i2 = __ldg(A.F + 3 * f + 2);
    S3 o, d, xs;
    float bs[3];
    camera_ray(A.cams[c], px, py, &o, &d);
    surface_point(o, d, s3(__ldg(A.V + 3 * i0), __ldg(A.V + 3 * i0 + 1), __ldg(A.V + 3 * i0 + 2)),
                  s3(__ldg(A.V + 3 * i1), __ldg(A.V + 3 * i1 + 1), __ldg(A.V + 3 * i1 + 2)),
                  s3(__ldg(A.V + 3 * i2), __ldg(A.V + 3 * i2 + 1), __ldg(A.V + 3 * i2 + 2)), &xs, ngs, bs);
    *org = offset_origin(xs, *ngs);
}

// The j-th secondary direction of a pixel (stream 1) and xi1 (for p_b).
__device__ __forceinline__ S3 secondary_dir(const ShadeArgs& A, uint32_t pixel, int c, int j, S3 ngs, float* xi1) {
    const uint4 h = philox(make_uint4(pixel, (uint32_t)c, (uint32_t)j, 1u), A.key);
    *xi1 = smul(__uint2float_rn(stratified32((uint32_t)j, (uint32_t)A.Nb, h.x) >> 8), 0x1p-24f);
    return cosine_dir(ngs, *xi1, unit24(h.y));
}

// The hit point y of a valid secondary ray (spec), its geometric normal and offset origin.
__device__ __forceinline__ void secondary_point(const ShadeArgs& A, int g, S3 org, S3 wjs, S3* ys, S3* ngy, S3* yorg,
                                                float3* Q) {
    const int j0 = __ldg(A.F + 3 * g), j1 = __ldg(A.F + 3 * g + 1), j2 = __ldg(A.F + 3 * g + 2);
    Q[0] = ld3(A.V + 3 * j0);
    Q[1] = ld3(A.V + 3 * j1);
    Q[2] = ld3(A.V + 3 * j2);
    float bys[3];
    surface_point(org, wjs, s3(Q[0].x, Q[0].y, Q[0].z), s3(Q[1].x, Q[1].y, Q[1].z), s3(Q[2].x, Q[2].y, Q[2].z), ys,
                  ngy, bys);
    *yorg = offset_origin(*ys, *ngy);
}

__device__ __forceinline__ void push_ray(float4* rays, uint32_t idx, S3 o, S3 d, uint64_t slot) {
    rays[2 * (size_t)idx] = make_float4(o.x, o.y, o.z, d.x);
    rays[2 * (size_t)idx + 1] = make_float4(d.y, d.z, __uint_as_float((uint32_t)slot), __uint_as_float((uint32_t)(slot >> 32)));
}

// Warp-aggregated append of the lanes with `want` set; returns this lane's queue index.
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (mask) {
        if (lane == __ffs(mask) - 1) base = atomicAdd(counter, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    }
    return base + __popc(mask & ((1u << lane) - 1u));
}

// sqrt of a positive shading quantity (the BRDF weights are estimator values, not decisions:
// approximate reciprocals and square roots are within a few ulp)
__device__ __forceinline__ float fsqrt_pos(float q) { return q * rsqrtf(q); }

// (f_d + f_s) * max(n.wi, 0), Eqs. 13-16 (FP32).  The GGX denominator uses
// |n x h|^2 + alpha^2 (n.h)^2, equal to (n.h)^2 (alpha^2 - 1) + 1 for unit vectors.
__device__ __forceinline__ float3 brdf_cos(float3 ns, float3 wi, float3 wo, float3 a, float r, float m) {
    float ci = dot(ns, wi), co = dot(ns, wo);
    if (ci <= 0.0f) return f3(0.f, 0.f, 0.f);
    float om = 1.0f - m;
    float3 res = (om * kInvPi) * a;
    if (co > 0.0f) {
        float rc = fminf(fmaxf(r, kRMin), 1.0f);
        float al = rc * rc, a2 = al * al;
        float3 hu = wi + wo;
        float3 h = rsqrtf(dot(hu, hu)) * hu;
        float nh = dot(ns, h), vh = dot(wi, h);
        float3 cx = cross(ns, h);
        float k = dot(cx, cx) + a2 * nh * nh;
        float D = __fdividef(a2, kPi * k * k);
        float sqi = fsqrt_pos(a2 + (1.0f - a2) * ci * ci), sqo = fsqrt_pos(a2 + (1.0f - a2) * co * co);
        float G = __fdividef(2.0f * ci, ci + sqi) * __fdividef(2.0f * co, co + sqo);
        float om5 = 1.0f - vh, w2 = om5 * om5, w5 = w2 * w2 * om5;
        float3 F0 = f3(om * kFDielectric + m * a.x, om * kFDielectric + m * a.y, om * kFDielectric + m * a.z);
        float3 Fr = f3(F0.x + (1.f - F0.x) * w5, F0.y + (1.f - F0.y) * w5, F0.z + (1.f - F0.z) * w5);
        float P = __fdividef(D * G, 4.0f * ci * co + kSpecEps);
        res += P * Fr;
    }
    return ci * res;
}

// Adjoint of brdf_cos for an upstream RGB gradient G3; accumulates into gns, gwo, ga, gr, gm and
// returns the value brdf_cos would (computed on the way, through reciprocals: equal to it up to
// rounding), so the backward pass needs no separate forward evaluation.
__device__ __forceinline__ float3 brdf_cos_adjoint(float3 ns, float3 wi, float3 wo, float3 a, float r, float m,
                                                   float3 G3, float3& gns, float3& gwo, float3& ga, float& gr,
                                                   float& gm) {
    float ci = dot(ns, wi), co = dot(ns, wo);
    if (ci <= 0.0f) return f3(0.f, 0.f, 0.f);
    float om = 1.0f - m;
    float3 fd = (om * kInvPi) * a;
    float3 res = fd;
    float gci = 0.0f, gco = 0.0f;
    float3 gres = ci * G3;
    ga += (om * kInvPi) * gres;
    gm += -dot(gres, a) * kInvPi;
    if (co > 0.0f) {
        float rc = fminf(fmaxf(r, kRMin), 1.0f);
        float al = rc * rc, a2 = al * al;
        float3 hu = wi + wo;
        float hl = rsqrtf(dot(hu, hu));
        float3 h = hl * hu;
        float nh = dot(ns, h), vh = dot(wi, h);
        float3 cx = cross(ns, h);
        float k = dot(cx, cx) + a2 * nh * nh;
        const float ipk2 = __fdividef(1.0f, kPi * k * k);
        float D = a2 * ipk2;
        float sqi = fsqrt_pos(a2 + (1.0f - a2) * ci * ci), sqo = fsqrt_pos(a2 + (1.0f - a2) * co * co);
        const float ici2 = __fdividef(1.0f, ci + sqi), ico2 = __fdividef(1.0f, co + sqo);
        float G1i = 2.0f * ci * ici2, G1o = 2.0f * co * ico2;
        float G = G1i * G1o;
        float om5 = 1.0f - vh, w2 = om5 * om5, w4 = w2 * w2, w5 = w4 * om5;
        float3 F0 = f3(om * kFDielectric + m * a.x, om * kFDielectric + m * a.y, om * kFDielectric + m * a.z);
        float3 Fr = f3(F0.x + (1.f - F0.x) * w5, F0.y + (1.f - F0.y) * w5, F0.z + (1.f - F0.z) * w5);
        float den = 4.0f * ci * co + kSpecEps;
        const float iden = __fdividef(1.0f, den);
        float P = D * G * iden;
        res += P * Fr;
        float S = dot(gres, Fr);
        float3 gF = P * gres;
        float gD = S * G * iden, gG = S * D * iden, gden = -S * P * iden;
        gci += gden * 4.0f * co;
        gco += gden * 4.0f * ci;
        float3 gF0 = f3(gF.x * (1.f - w5), gF.y * (1.f - w5), gF.z * (1.f - w5));
        float gw5 = gF.x * (1.f - F0.x) + gF.y * (1.f - F0.y) + gF.z * (1.f - F0.z);
        float gvh = -5.0f * w4 * gw5;
        gm += gF0.x * (a.x - kFDielectric) + gF0.y * (a.y - kFDielectric) + gF0.z * (a.z - kFDielectric);
        ga += m * gF0;
        float gk = -2.0f * gD * D * __fdividef(1.0f, k);
        float ga2 = gD * ipk2 + gk * nh * nh;
        float gnh = gk * 2.0f * nh * (a2 - 1.0f);
        const float di = __fdividef(ici2 * ici2, sqi), dq = __fdividef(ico2 * ico2, sqo);  // 1/(sq (c+sq)^2)
        gci += gG * G1o * (2.0f * a2 * di);
        gco += gG * G1i * (2.0f * a2 * dq);
        ga2 += gG * G1o * (-ci * (1.0f - ci * ci) * di);
        ga2 += gG * G1i * (-co * (1.0f - co * co) * dq);
        if (r >= kRMin && r <= 1.0f) gr += ga2 * 4.0f * rc * rc * rc;
        gns += gnh * h;
        float3 gh = gnh * ns + gvh * wi;
        gwo += hl * (gh - dot(gh, h) * h);
        gns += gco * wo;
        gwo += gco * ns;
    }
    gci += dot(G3, res);
    gns += gci * wi;
    return ci * res;
}

// Material and shading normal from 8 fetched channels and the interpolated frame.
struct Surface {
    float3 a;
    float r, m;
    float3 n, T, B, nt, ns;
    float3 ni, u;  // unnormalised interpolants (adjoint)
    float ql;      // |q|
    float s;
};

__device__ __forceinline__ Surface make_surface(const float att[8], float3 ni, float3 ti, float s, bool metallic) {
    Surface su;
    su.a = f3(att[0], att[1], att[2]);
    su.r = att[3];
    su.m = metallic ? att[4] : 0.0f;
    su.ni = ni;
    su.n = normalize(ni);
    su.u = ti - dot(su.n, ti) * su.n;
    su.T = normalize(su.u);
    su.s = s;
    su.B = s * cross(su.n, su.T);
    float3 q = f3(att[5], att[6], att[7]);
    su.ql = sqrtf(dot(q, q));
    su.nt = (1.0f / su.ql) * q;
    su.ns = su.nt.x * su.T + su.nt.y * su.B + su.nt.z * su.n;
    return su;
}


// ------------------------------------------------------------------ ray generation

// Ray queues are written in coherent order: a warp's lanes are 32 neighbouring pixels of the
// tile-ordered pixel list, and consecutive queue entries hold the same sample index k of
// those pixels, so the 32 rays a warp later traces start close together and point the
// same way (the same stratum of the same CDF).
constexpr int kGenK = 32;     // sample indices per warp of gen_direct
constexpr int kGenBatch = 8;  // sample indices per queue append of a warp
constexpr int kGenThreads = 256;
// Shared memory the ray generation kernels may take for the row phase of the texel search
// (env_rows_to_shared), beside their 24 KB of staged directions: 16 KB holds it for environments
// of up to 1024 rows; taller ones search global memory.
constexpr size_t kEnvSharedMax = 20u << 10;

// One shadow ray per (pixel, k) whose direction is above the geometric horizon (Eq. 17).
// A warp appends the rays of kGenBatch sample indices at once: their directions wait in
// shared memory (each lane its own column) while one atomic on the chunk's queue counter
// reserves their slots, so the counter sees one request per batch instead of one per sample.
template <bool SR>
__global__ void __launch_bounds__(kGenThreads) gen_direct_kernel(ShadeArgs A) {
    __shared__ float s_dir[kGenThreads / 32][kGenBatch][3][32];
    extern __shared__ __align__(8) unsigned char s_env_rows[];
    EnvView env = A.env;
    env.Q = *A.env.Qp;
    if (SR) env_rows_to_shared(env, s_env_rows);  // before any thread returns
    const uint32_t total = *A.count;
    const uint32_t end = min(A.chunk_begin + A.chunk_pixels, total);
    if (A.chunk_begin >= end) return;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nkc = (uint32_t)(A.Nd + kGenK - 1) / kGenK;
    const uint32_t group = warp / nkc, kc = warp % nkc;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (A.chunk_begin + group * 32 >= end) return;
    float (*sd)[3][32] = s_dir[threadIdx.x >> 5];
    const uint32_t i = A.chunk_begin + group * 32 + lane;
    const bool valid = i < end;
    int c = 0, px, py;
    uint32_t rem = 0;
    S3 org = s3(0.f, 0.f, 0.f), ngs = s3(0.f, 0.f, 1.f);
    if (valid) {
        const uint32_t pid = A.pixels[i];
        pixel_of(A, pid, &c, &px, &py, &rem);
        const float4 r3 = A.prec[kPrec * (size_t)i + 3], r4 = A.prec[kPrec * (size_t)i + 4];
        org = s3(r3.x, r3.y, r3.z);
        ngs = s3(r3.w, r4.x, r4.y);
    }
    const int k0 = (int)kc * kGenK, k1 = min(A.Nd, k0 + kGenK);
    for (int kb = k0; kb < k1; kb += kGenBatch) {
        const int kn = min(kGenBatch, k1 - kb);  // warp-uniform
        uint32_t want = 0;                       // bit u: the ray of sample kb + u is queued
        // samples k and k + 1 together (their texel searches overlap)
        for (int u = 0; u < kn; u += 2) {
            if (!valid) continue;
            const int k = kb + u;
            const bool two = u + 1 < kn;
            const int k2 = two ? k + 1 : k;
            const uint4 ha = philox(make_uint4(rem, (uint32_t)c, (uint32_t)k, 0u), A.key);
            const uint4 hb = philox(make_uint4(rem, (uint32_t)c, (uint32_t)k2, 0u), A.key);
            LightSample sa, sb;
            light_sample2<SR>(env, ha, (uint32_t)k, hb, (uint32_t)k2, A.nxd, A.nyd, &sa, &sb);
            if (sdot(ngs, sa.dir) > 0.0f) {
                want |= 1u << u;
                A.tsel[(size_t)(i - A.state_base) * A.Nd + k] = sa.texel;
                sd[u][0][lane] = sa.dir.x; sd[u][1][lane] = sa.dir.y; sd[u][2][lane] = sa.dir.z;
            }
            if (two && sdot(ngs, sb.dir) > 0.0f) {
                want |= 2u << u;
                A.tsel[(size_t)(i - A.state_base) * A.Nd + k2] = sb.texel;
                sd[u + 1][0][lane] = sb.dir.x; sd[u + 1][1][lane] = sb.dir.y; sd[u + 1][2][lane] = sb.dir.z;
            }
        }
        // one reservation for the batch; within it the rays keep the order (k, lane)
        uint32_t cnt = 0;
#pragma unroll
        for (int u = 0; u < kGenBatch; ++u) cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, (want >> u) & 1u));
        if (cnt == 0) continue;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(A.ctr + 2, cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
        for (int u = 0; u < kGenBatch; ++u) {
            const unsigned mu = __ballot_sync(0xffffffffu, (want >> u) & 1u);
            if ((want >> u) & 1u) {
                const uint32_t idx = base + (uint32_t)__popc(mu & lt);
                const S3 d = s3(sd[u][0][lane], sd[u][1][lane], sd[u][2][lane]);
                if (idx < A.ray_cap)
                    push_ray(A.rays, idx, org, d,
                             (uint64_t)(i - A.state_base) * (uint32_t)A.wd * 32u + (uint32_t)(kb + u));
                else atomicOr(A.status, ERRBIT_QUEUE);
            }
            base += (uint32_t)__popc(mu);
        }
    }
}

// One closest-hit ray per (pixel, j): cosine-weighted about n_g (Sec. 5.3).
__global__ void __launch_bounds__(256) gen_secondary_kernel(ShadeArgs A) {
    const uint32_t total = *A.count;
    const uint32_t end = min(A.chunk_begin + A.chunk_pixels, total);
    if (A.chunk_begin >= end) return;
    const uint32_t group = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (A.chunk_begin + group * 32 >= end) return;
    const uint32_t i = A.chunk_begin + group * 32 + lane;
    const bool valid = i < end;
    int c = 0, px, py;
    uint32_t rem = 0;
    S3 org = s3(0.f, 0.f, 0.f), ngs = s3(0.f, 0.f, 1.f);
    if (valid) {
        const uint32_t pid = A.pixels[i];
        pixel_of(A, pid, &c, &px, &py, &rem);
        const float4 r3 = A.prec[kPrec * (size_t)i + 3], r4 = A.prec[kPrec * (size_t)i + 4];
        org = s3(r3.x, r3.y, r3.z);
        ngs = s3(r3.w, r4.x, r4.y);
    }
    for (int j = 0; j < A.Nb; ++j) {
        S3 wjs = s3(0.f, 0.f, 0.f);
        if (valid) {
            float xi1;
            wjs = secondary_dir(A, rem, c, j, ngs, &xi1);
        }
        const uint32_t idx = warp_append(A.ctr, valid);
        if (valid) {
            if (idx < A.ray_cap)
                push_ray(A.rays, idx, org, wjs, (uint64_t)(i - A.state_base) * (uint32_t)A.Nb + (uint32_t)j);
            else atomicOr(A.status, ERRBIT_QUEUE);
        }
    }
}

// One shadow ray per (valid secondary hit, s) above the hit's geometric horizon (Eq. 18),
// appended kGenBatch light samples at a time like gen_direct's.
template <bool SR>
__global__ void __launch_bounds__(kGenThreads) gen_seclight_kernel(ShadeArgs A) {
    __shared__ float s_dir[kGenThreads / 32][kGenBatch][3][32];
    extern __shared__ __align__(8) unsigned char s_env_rows[];
    EnvView env = A.env;
    env.Q = *A.env.Qp;
    if (SR) env_rows_to_shared(env, s_env_rows);  // before any thread returns
    const uint32_t total = *A.count;
    const uint32_t end = min(A.chunk_begin + A.chunk_pixels, total);
    if (A.chunk_begin >= end) return;
    const uint32_t group = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (A.chunk_begin + group * 32 >= end) return;
    float (*sd)[3][32] = s_dir[threadIdx.x >> 5];
    const uint32_t i = A.chunk_begin + group * 32 + lane;
    const bool valid = i < end;
    int c = 0, px, py;
    uint32_t rem = 0;
    S3 org = s3(0.f, 0.f, 0.f), ngs = s3(0.f, 0.f, 1.f);
    if (valid) {
        const uint32_t pid = A.pixels[i];
        pixel_of(A, pid, &c, &px, &py, &rem);
        const float4 r3 = A.prec[kPrec * (size_t)i + 3], r4 = A.prec[kPrec * (size_t)i + 4];
        org = s3(r3.x, r3.y, r3.z);
        ngs = s3(r3.w, r4.x, r4.y);
    }
    for (int j = 0; j < A.Nb; ++j) {
        const int g = valid ? A.hits[(size_t)(i - A.state_base) * A.Nb + j] : -1;
        S3 yorg = s3(0.f, 0.f, 0.f), ngy = s3(0.f, 0.f, 1.f);
        if (g >= 0) {
            float xi1;
            const S3 wjs = secondary_dir(A, rem, c, j, ngs, &xi1);
            S3 ys;
            float3 Q[3];
            secondary_point(A, g, org, wjs, &ys, &ngy, &yorg, Q);
        }
        for (int sb = 0; sb < A.Ns; sb += kGenBatch) {
            const int sn = min(kGenBatch, A.Ns - sb);  // warp-uniform
            uint32_t want = 0;
            if (g >= 0) {
                for (int u = 0; u < sn; ++u) {
                    const int s = sb + u;
                    const uint4 h = philox(make_uint4(rem, (uint32_t)c, (uint32_t)(j * A.Ns + s), 2u), A.key);
                    const LightSample ls = light_sample<SR>(env, h, (uint32_t)s, A.nxs, A.nys);
                    if (sdot(ngy, ls.dir) > 0.0f) {
                        want |= 1u << u;
                        A.tsel2[(size_t)(i - A.state_base) * A.Nb * A.Ns + j * A.Ns + s] = ls.texel;
                        sd[u][0][lane] = ls.dir.x; sd[u][1][lane] = ls.dir.y; sd[u][2][lane] = ls.dir.z;
                    }
                }
            }
            uint32_t cnt = 0;
#pragma unroll
            for (int u = 0; u < kGenBatch; ++u) cnt += (uint32_t)__popc(__ballot_sync(0xffffffffu, (want >> u) & 1u));
            if (cnt == 0) continue;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(A.ctr + 2, cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
            for (int u = 0; u < kGenBatch; ++u) {
                const unsigned mu = __ballot_sync(0xffffffffu, (want >> u) & 1u);
                if ((want >> u) & 1u) {
                    const uint32_t idx = base + (uint32_t)__popc(mu & lt);
                    const S3 d = s3(sd[u][0][lane], sd[u][1][lane], sd[u][2][lane]);
                    const uint64_t slot =
                        (uint64_t)(i - A.state_base) * (uint32_t)A.ws * 32u + (uint32_t)(j * A.Ns + sb + u);
                    if (idx < A.ray_cap) push_ray(A.rays, idx, yorg, d, slot | (1ull << 63));
                    else atomicOr(A.status, ERRBIT_QUEUE);
                }
                base += (uint32_t)__popc(mu);
            }
        }
    }
}

// ------------------------------------------------------------------ persistent tracer
// Any-hit (shadow rays -> visibility bits) or closest-hit (secondary rays -> hit ids) over
// the chunk's ray queue.  A warp claims a pool of kPool consecutive queue entries (the same
// few sample indices of 32 neighbouring pixels), so the rays a warp holds stay local to one
// group of pixels.  Its lanes run rounds of kRound items (a 4-wide node or a triangle each)
// and the lanes whose ray ended refill from the pool between rounds: a lane waits at most
// the rest of a round, never for the longest ray of the warp.  Longer rounds idle more
// lanes, shorter ones refill more often; 24 measured best.  Each ray is clipped where it
// leaves the triangles' bounding sphere (sphere_exit).
constexpr uint32_t kPool = 256;
constexpr int kRound = 32;  // traversal iterations between refills

constexpr int kTraceThreads = 128;
// Resident tracer blocks per SM (the persistent grid is this many per SM): 9 blocks of 4 warps
// hold the registers to 56 per thread with a few bytes of spills, and traced the 2M-triangle
// workload 0.9% faster than 8 blocks at 64 registers; 10 blocks (48 registers) were 6% slower.
// The batched tracer, whose lanes also carry their ray's BVH, keeps 8 blocks (64 registers).
constexpr int kTraceBlocksPerSM = 9;
constexpr int kTraceBatchBlocksPerSM = 8;

// Byte c of a pair of words (children 0-3 in .x, 4-7 in .y) as a float: one byte permutation
// puts it under the exponent of 2^23, and subtracting 2^23 leaves the byte's value (exact).
__device__ __forceinline__ float q8(uint2 w, int c) {
    return __uint_as_float(__byte_perm(c < 4 ? w.x : w.y, 0x4B000000u, 0x7540u + (uint32_t)(c & 3))) - 8388608.0f;
}

// Box tests of the eight children of an 8-wide compressed node (exm_bvh.cu): a child's plane is
// p + q 2^e, and its ray parameter fma(q, 2^e / d, (p - o) / d) (the same conservative slab test
// as the 4-wide nodes': the build's padding of the leaf boxes absorbs its rounding).  Returns the
// node's child groups: node children gbase + bit, triangle children tbase + bit.
__device__ __forceinline__ void node8_hits(const float4* N, const Ray& r, float tmax, uint32_t* gbase, uint32_t* tbase,
                                           uint32_t* gmask, uint32_t* tmask) {
    const float4 w0 = __ldg(N);
    const uint4 w1 = __ldg(reinterpret_cast<const uint4*>(N) + 1);
    const uint4 w2 = __ldg(reinterpret_cast<const uint4*>(N) + 2);
    const uint4 w3 = __ldg(reinterpret_cast<const uint4*>(N) + 3);
    const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(N) + 4);
    const uint32_t eb = __float_as_uint(w0.w);
    const float sx = r.inv.x * __uint_as_float((eb & 0xffu) << 23);
    const float sy = r.inv.y * __uint_as_float(((eb >> 8) & 0xffu) << 23);
    const float sz = r.inv.z * __uint_as_float(((eb >> 16) & 0xffu) << 23);
    const float bx = fmaf(w0.x, r.inv.x, r.oinv.x), by = fmaf(w0.y, r.inv.y, r.oinv.y), bz = fmaf(w0.z, r.inv.z, r.oinv.z);
    const uint2 lox = make_uint2(w2.x, w2.y), loy = make_uint2(w2.z, w2.w), loz = make_uint2(w3.x, w3.y);
    const uint2 hix = make_uint2(w3.z, w3.w), hiy = make_uint2(w4.x, w4.y), hiz = make_uint2(w4.z, w4.w);
    // near / far planes of each axis chosen by the ray's direction signs
    const uint2 nx = r.nx ? hix : lox, fx = r.nx ? lox : hix;
    const uint2 ny = r.ny ? hiy : loy, fy = r.ny ? loy : hiy;
    const uint2 nz = r.nz ? hiz : loz, fz = r.nz ? loz : hiz;
    uint32_t h = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float t0 = fmaxf(fmax3(fmaf(q8(nx, c), sx, bx), fmaf(q8(ny, c), sy, by), fmaf(q8(nz, c), sz, bz)), 0.0f);
        const float t1 = fminf(fmin3(fmaf(q8(fx, c), sx, bx), fmaf(q8(fy, c), sy, by), fmaf(q8(fz, c), sz, bz)), tmax);
        h |= (t0 <= t1 ? 1u : 0u) << c;
    }
    const uint32_t ni = w1.z & 0xffu, nt = (w1.z >> 8) & 0xffu;
    h &= (1u << (ni + nt)) - 1u;
    *gbase = w1.x;
    *tbase = w1.y;
    *gmask = h & ((1u << ni) - 1u);
    *tmask = h >> ni;
}

using TraceJob = ExmTraceJob;

// Plane byte c of a word of quantised planes, as the float 2^23 + q (exact).
__device__ __forceinline__ float qplane(uint32_t w, int c) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + (uint32_t)c));
}

// Box tests of the four children of 4-wide node `node`: their entry distances tc, which of
// them the ray enters before tmax (hc) and their references.
template <int LAYOUT>
__device__ __forceinline__ void node4_test(const BvhView& bvh, int node, const Ray& r, float tmax, float tc[4],
                                           bool hc[4], int ref[4]) {
    if constexpr (LAYOUT == EXM_BVH_4Q) {
        // two 32-byte loads (chunks skewed by bit 1 of the node index).  Plane q of axis a lies
        // at t = q s_a + b_a with s_a = step_a / d_a (exact scaling by a power of two) and
        // b_a = (p_a - o_a) / d_a; it is evaluated as fma(2^23 + q, s_a, b_a - 2^23 s_a), the
        // byte placed under the exponent of 2^23 by one permutation.  The folded constant's
        // rounding is at most half a grid step, inside the one-step margin the build adds.
        const float4* N = bvh.nodesq + kNodeQ4 * (size_t)node;
        const unsigned x = ((unsigned)node & 2u) << 4;
        float4 a0, a1, b0, b1;
        ldg32(chunk_at(N, x), a0, a1);
        ldg32(chunk_at(N, x ^ 32u), b0, b1);
        const float sx = a0.w * r.inv.x, sy = b1.z * r.inv.y, sz = b1.w * r.inv.z;
        const float cx = fmaf(-8388608.0f, sx, fmaf(a0.x, r.inv.x, r.oinv.x));
        const float cy = fmaf(-8388608.0f, sy, fmaf(a0.y, r.inv.y, r.oinv.y));
        const float cz = fmaf(-8388608.0f, sz, fmaf(a0.z, r.inv.z, r.oinv.z));
        const uint32_t lox = __float_as_uint(b0.x), loy = __float_as_uint(b0.y), loz = __float_as_uint(b0.z);
        const uint32_t hix = __float_as_uint(b0.w), hiy = __float_as_uint(b1.x), hiz = __float_as_uint(b1.y);
        // near / far plane words of each axis, by the ray's direction signs (four children at once)
        const uint32_t nx = r.nx ? hix : lox, fx = r.nx ? lox : hix;
        const uint32_t ny = r.ny ? hiy : loy, fy = r.ny ? loy : hiy;
        const uint32_t nz = r.nz ? hiz : loz, fz = r.nz ? loz : hiz;
        ref[0] = __float_as_int(a1.x); ref[1] = __float_as_int(a1.y);
        ref[2] = __float_as_int(a1.z); ref[3] = __float_as_int(a1.w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float t0 = fmaxf(fmax3(fmaf(qplane(nx, c), sx, cx), fmaf(qplane(ny, c), sy, cy),
                                         fmaf(qplane(nz, c), sz, cz)), 0.0f);
            const float t1 = fminf(fmin3(fmaf(qplane(fx, c), sx, cx), fmaf(qplane(fy, c), sy, cy),
                                         fmaf(qplane(fz, c), sz, cz)), tmax);
            tc[c] = t0;
            hc[c] = t0 <= t1 && ref[c] != kEmptyChild;
        }
    } else {
        // the six plane vectors in three 32-byte loads (chunks skewed by the node index), then
        // the near / far planes of each axis chosen by the ray's direction signs
        const float4* N = bvh.nodes4 + 8 * (size_t)node;
        const unsigned sk = ((unsigned)node & 3u) << 5;
        float4 lx, ly, lz, hx, hy, hz;
        ldg32(chunk_at(N, sk), lx, ly);
        ldg32(chunk_at(N, sk ^ 32u), lz, hx);
        ldg32(chunk_at(N, sk ^ 64u), hy, hz);
        const float4 rf = __ldg(chunk_at(N, sk ^ 96u));
        const float4 qx = r.nx ? hx : lx, qy = r.ny ? hy : ly, qz = r.nz ? hz : lz;
        const float4 fx = r.nx ? lx : hx, fy = r.ny ? ly : hy, fz = r.nz ? lz : hz;
        ref[0] = __float_as_int(rf.x); ref[1] = __float_as_int(rf.y);
        ref[2] = __float_as_int(rf.z); ref[3] = __float_as_int(rf.w);
#define EXM_BOX(C, c)                                                                                              \
    {                                                                                                              \
        const float t0 = fmaxf(fmax3(fmaf(qx.c, r.inv.x, r.oinv.x), fmaf(qy.c, r.inv.y, r.oinv.y),                    \
                                     fmaf(qz.c, r.inv.z, r.oinv.z)), 0.0f);                                        \
        const float t1 = fminf(fmin3(fmaf(fx.c, r.inv.x, r.oinv.x), fmaf(fy.c, r.inv.y, r.oinv.y),                    \
                                     fmaf(fz.c, r.inv.z, r.oinv.z)), tmax);                                        \
        tc[C] = t0;                                                                                                \
        hc[C] = t0 <= t1 && ref[C] != kEmptyChild;                                                                 \
    }
        EXM_BOX(0, x)
        EXM_BOX(1, y)
        EXM_BOX(2, z)
        EXM_BOX(3, w)
#undef EXM_BOX
    }
}

// The traversal loop.  Single queue (BATCH false): the chunk's queue of A, claimed kPool rays at
// a time.  Batched: the queues of `jobs`, whose pools are numbered one after another; a warp
// claims a pool number, finds its queue, and each lane keeps the BVH of the queue its ray came
// from, so the lanes of a warp may trace rays of different assets.
template <bool CLOSEST, bool COUNT, bool BATCH, int LAYOUT>
__device__ __forceinline__ void trace_body(const ShadeArgs& A, const TraceJob* __restrict__ jobs, int njobs,
                                           uint32_t* batch_cursor) {
    constexpr bool W8 = LAYOUT == EXM_BVH_8Q;
    int stack[W8 ? kStackSize8 : kStackSize4];
    // closest hit, 4-wide: the entry distance of each stacked box, so that a pop skips the boxes
    // that begin beyond the nearest hit found since the push without loading them

    __shared__ uint32_t s_pool_end[BATCH ? kMaxBatch : 1];  // BATCH: pools of queues 0..j
    __shared__ uint32_t s_count[BATCH ? kMaxBatch : 1];     // BATCH: rays of queue j
    uint32_t n = 0;          // single queue: its rays
    uint32_t* cursor = nullptr;
    if (BATCH) {
        if (threadIdx.x < (unsigned)njobs)
            s_count[threadIdx.x] = min(__ldg(jobs[threadIdx.x].qcount), jobs[threadIdx.x].ray_cap);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int j = 0; j < njobs; ++j) {
                acc += (s_count[j] + kPool - 1) / kPool;
                s_pool_end[j] = acc;
            }
        }
        __syncthreads();
        if (njobs == 0 || s_pool_end[njobs - 1] == 0) return;
        cursor = batch_cursor;
    } else {
        n = min(*(A.ctr + (CLOSEST ? 0 : 2)), A.ray_cap);  // an overflowed queue holds ray_cap rays (ERRBIT_QUEUE)
        if (n == 0) return;
        cursor = A.ctr + (CLOSEST ? 1 : 3);
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t err = 0, c_nodes = 0, c_tris = 0, c_rays = 0;
    int sp = 0, node = 0, best = -1, steps = 0;
    int leaf = INT_MIN;  // any hit, 4-wide: the leaf set aside while the lane opens nodes (none: INT_MIN)
    // 8-wide traversal: the current group of node children (base, mask of those left to visit)
    // and of triangle children (base, mask of those left to test)
    uint32_t gbase = 0, gmask = 0, tbase = 0, tmask = 0;
    float bt = INFINITY, bdet = 0.0f;
    float tclip = 0.0f;  // where the ray leaves the triangles' bounding sphere
    bool active = false;
    Ray r;
    r.o = s3(0.f, 0.f, 0.f); r.d = s3(0.f, 0.f, 1.f);
    r.kx = 0; r.ky = 1; r.kz = 2; r.Sx = r.Sy = 0.f; r.Sz = 1.f; r.inv = make_float3(0.f, 0.f, 1.f);
    r.oinv = make_float3(0.f, 0.f, 0.f);
    uint64_t slot = 0;
    uint32_t pnext = 0, pend = 0;  // warp-uniform pool [pnext, pend)
    int pjob = 0;                  // BATCH, warp-uniform: the queue of the pool
    int job = 0;                   // BATCH: the queue of this lane's ray
    BvhView bvh = A.bvh;           // BATCH: the BVH of this lane's ray
    bool drained = false;          // warp-uniform: the queue has no more pools
    while (true) {
        const unsigned need = __ballot_sync(0xffffffffu, !active);
        if (need && pnext >= pend && !drained) {
            if (BATCH) {
                uint32_t g = 0;
                if (lane == 0) g = atomicAdd(cursor, 1u);
                g = __shfl_sync(0xffffffffu, g, 0);
                if (g >= s_pool_end[njobs - 1]) {
                    drained = true;
                } else {
                    int j = 0;
                    while (s_pool_end[j] <= g) ++j;
                    const uint32_t first = (g - (j ? s_pool_end[j - 1] : 0u)) * kPool;
                    pjob = j;
                    pnext = first;
                    pend = min(first + kPool, s_count[j]);
                }
            } else {
                uint32_t b = 0;
                if (lane == 0) b = atomicAdd(cursor, kPool);
                b = __shfl_sync(0xffffffffu, b, 0);
                if (b >= n) drained = true;
                else { pnext = b; pend = min(b + kPool, n); }
            }
        }
        if (need && pnext < pend) {
            const uint32_t my = pnext + (uint32_t)__popc(need & lt);
            if (!active && my < pend) {
                const float4* rays = A.rays;
                if (BATCH) {
                    job = pjob;
                    rays = jobs[job].rays;
                    bvh.nodes4 = jobs[job].nodes4;
                    bvh.nodes8 = jobs[job].nodes4;
                    bvh.nodesq = jobs[job].nodes4;
                    bvh.tris = jobs[job].tris;
                    bvh.sphere = jobs[job].sphere;
                }
                float4 a, b;
                ldg32(rays + 2 * (size_t)my, a, b);
                r = make_ray(s3(a.x, a.y, a.z), s3(a.w, b.x, b.y));
                tclip = sphere_exit(r.o, r.d, __ldg(bvh.sphere));
                slot = (uint64_t)__float_as_uint(b.z) | ((uint64_t)__float_as_uint(b.w) << 32);
                sp = 0; node = 0; leaf = INT_MIN; best = -1; steps = 0; bt = INFINITY; bdet = 0.0f;
                gbase = 0; gmask = 1u; tmask = 0u;  // 8-wide: the root alone
                active = true;
                ++c_rays;
            }
            pnext = min(pnext + (uint32_t)__popc(need), pend);
        }
        if (!__any_sync(0xffffffffu, active)) {
            if (drained) break;
            continue;
        }
        if (!active) continue;
        bool done = false, hit = false;
        // a round of at most kRound iterations, each one traversal item (a node or a triangle)
        // per lane that takes part
        steps += kRound;  // the cap is checked once per round: at most kTraversalCap + kRound iterations
        if (steps > kTraversalCap) { err |= ERRBIT_TRAVERSAL; hit = true; done = true; }
        if constexpr (W8) {
            // one item per iteration: an 8-wide node (the next child of the current node group)
            // or one triangle of the current triangle group; a visited node's remaining group is
            // pushed as one stack entry (base << 8 | mask)
            for (int it = 0; it < kRound && !done; ++it) {
                if (tmask) {
                    const int k = __ffs(tmask) - 1;
                    tmask &= tmask - 1u;
                    ++c_tris;
                    float T, det;
                    int id;
                    if (tri_test(bvh, (int)(tbase + k), r, &T, &det, &id)) {
                        if (!CLOSEST) { hit = true; done = true; break; }
                        const float t = sdiv(T, det);
                        if (t < bt || (t == bt && id < best)) { bt = t; best = id; bdet = det; }
                    }
                    continue;
                }
                if (!gmask) {
                    if (sp == 0) { done = true; break; }
                    const uint32_t e = (uint32_t)stack[--sp];
                    gbase = e >> 8;
                    gmask = e & 0xffu;
                }
                const uint32_t nd = gbase + (uint32_t)(__ffs(gmask) - 1);
                gmask &= gmask - 1u;
                if (gmask) {
                    if (sp >= kStackSize8) { err |= ERRBIT_TRAVERSAL; hit = true; done = true; break; }
                    stack[sp++] = (int)((gbase << 8) | gmask);
                }
                ++c_nodes;
                node8_hits(bvh.nodes8 + kNode8 * (size_t)nd, r, CLOSEST ? fminf(bt, tclip) : tclip, &gbase, &tbase,
                           &gmask, &tmask);
            }
        } else if constexpr (!CLOSEST) {
            // any hit: a leaf met while opening nodes is set aside in `leaf` and the lane goes on
            // opening nodes (an unoccluded ray opens every box it crosses in any order, so the
            // work is wasted only on rays that turn out occluded).  Each iteration the warp runs
            // node tests or triangle tests, not both: triangles once the lanes holding a leaf
            // are at least 3/4 of those with a node to open (a triangle test costs less than a
            // node test; 1/2 and 1 measured slower, and so did a second leaf in hand).  `node`
            // holds the next node, or a second leaf that waits for the first, or none.
            for (int it = 0; it < kRound; ++it) {
                if (node == INT_MIN && sp > 0) node = stack[--sp];
                if (leaf == INT_MIN && node < 0 && node != INT_MIN) { leaf = node; node = INT_MIN; }
                if (node == INT_MIN && leaf == INT_MIN) { done = true; break; }
                const unsigned m = __activemask();
                const int ntri = __popc(__ballot_sync(m, leaf != INT_MIN));
                const int nnode = __popc(__ballot_sync(m, node >= 0));
                if (4 * ntri >= 3 * nnode) {
                    if (leaf != INT_MIN) {
                        // a leaf of c consecutive triangle records from k, ~(k | (c - 1) << 28): one
                        // triangle per iteration, the rest of the leaf kept in the hand
                        const uint32_t lt = ~(uint32_t)leaf;
                        ++c_tris;
                        float T, det;
                        int id;
                        if (tri_test(bvh, (int)(lt & ((1u << kLeafCountShift) - 1u)), r, &T, &det, &id)) {
                            hit = true; done = true; break;
                        }
                        leaf = (lt >> kLeafCountShift) ? (int)~(lt - ((1u << kLeafCountShift) - 1u)) : INT_MIN;
                    }
                } else if (node >= 0) {
                    ++c_nodes;
                    float tc[4];
                    int ref[4];
                    bool hc[4];
                    node4_test<LAYOUT>(bvh, node, r, tclip, tc, hc, ref);
                    if (sp > kStackSize4 - 3) { err |= ERRBIT_TRAVERSAL; hit = true; done = true; break; }
                    // the first hit child in slot order goes on, the others are pushed
                    int nc = -1;
#pragma unroll
                    for (int c = 3; c >= 0; --c)
                        if (hc[c]) nc = c;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (hc[c] && c != nc) stack[sp++] = ref[c];
                    node = nc < 0 ? INT_MIN : nc == 0 ? ref[0] : nc == 1 ? ref[1] : nc == 2 ? ref[2] : ref[3];
                }
            }
        } else {
            // closest hit: one item per iteration, a 4-wide node (node >= 0) or one triangle
            // (node < 0); hit leaves are pushed like inner nodes
            for (int it = 0; it < kRound && !done; ++it) {
                int next = INT_MIN;  // none: pop (a leaf reference is negative, ~0 == -1)
                if (node < 0) {
                    // a leaf of c consecutive triangle records from k, ~(k | (c - 1) << 28): one
                    // triangle per iteration, the rest of the leaf as the next item
                    const uint32_t lt = ~(uint32_t)node;
                    ++c_tris;
                    float T, det;
                    int id;
                    if (tri_test(bvh, (int)(lt & ((1u << kLeafCountShift) - 1u)), r, &T, &det, &id)) {
                        const float t = sdiv(T, det);
                        if (t < bt || (t == bt && id < best)) { bt = t; best = id; bdet = det; }
                    }
                    if (lt >> kLeafCountShift) next = (int)~(lt - ((1u << kLeafCountShift) - 1u));
                } else {
                    ++c_nodes;
                    float tc[4];
                    int ref[4];
                    bool hc[4];
                    node4_test<LAYOUT>(bvh, node, r, fminf(bt, tclip), tc, hc, ref);
                    // a node pushes at most 3 children; the build keeps 3 entries per level within the stack
                    if (sp > kStackSize4 - 3) { err |= ERRBIT_TRAVERSAL; hit = true; done = true; break; }
                    // continue with the nearest hit child; push the others (storing their entry
                    // distances to skip boxes beyond the nearest hit at pop time, or pushing them
                    // farthest first, cost more than they saved: the secondary rays mostly leave
                    // the mesh)
                    int nc = -1;
                    float tn = INFINITY;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (hc[c] && tc[c] < tn) { tn = tc[c]; nc = c; }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (hc[c] && c != nc) stack[sp++] = ref[c];
                    if (nc >= 0) next = nc == 0 ? ref[0] : nc == 1 ? ref[1] : nc == 2 ? ref[2] : ref[3];
                }
                if (next == INT_MIN) {
                    if (sp == 0) { done = true; break; }
                    next = stack[--sp];
                }
                node = next;
            }
        }
        if (done) {
            if (CLOSEST) {
                int32_t* hits = BATCH ? jobs[job].hits : A.hits;
                hits[slot] = (best >= 0 && bdet > 0.0f) ? best : -1;
            } else if (!hit) {
                const uint64_t bit = slot & ~(1ull << 63);
                uint32_t* words = (slot >> 63) ? (BATCH ? jobs[job].secbits : A.secbits)
                                               : (BATCH ? jobs[job].visbits : A.visbits);
                atomicOr(words + (bit >> 5), 1u << (uint32_t)(bit & 31));
            }
            active = false;
        }
    }
    if (err) atomicOr(A.status, err);
    if (COUNT) {
        atomicAdd(A.work, (unsigned long long)c_nodes);
        atomicAdd(A.work + 1, (unsigned long long)c_tris);
        atomicAdd(A.work + 3, (unsigned long long)c_rays);
    }
}

template <bool CLOSEST, bool COUNT, int LAYOUT>
__global__ void __launch_bounds__(kTraceThreads, kTraceBlocksPerSM) trace_kernel(ShadeArgs A) {
    trace_body<CLOSEST, COUNT, false, LAYOUT>(A, nullptr, 0, nullptr);
}

// The batched tracer: one persistent launch over the ray queues of several relight requests
// (whose assets all use one BVH layout).
template <bool CLOSEST, int LAYOUT>
__global__ void __launch_bounds__(kTraceThreads, kTraceBatchBlocksPerSM) trace_batch_kernel(ShadeArgs A, const TraceJob* __restrict__ jobs,
                                                                       int njobs, uint32_t* cursor) {
    trace_body<CLOSEST, false, true, LAYOUT>(A, jobs, njobs, cursor);
}

// ------------------------------------------------------------------ shading (warp per pixel)

// Appends the set bits of `words` [wbase, min(wbase + 32, nwords)) of a pixel to the warp's
// list (bit index relative to wbase*32) and returns how many were appended.  Word k goes to
// all lanes at once: lane l writes bit l of it, if set, at the count of the set bits below.
__device__ __forceinline__ int enumerate_bits(const uint32_t* words, int wbase, int nwords, uint16_t* list) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int n = min(32, nwords - wbase);
    const uint32_t mine = lane < n ? words[wbase + lane] : 0u;
    int tot = 0;
    for (int k = 0; k < n; ++k) {
        const uint32_t w = __shfl_sync(0xffffffffu, mine, k);
        if ((w >> lane) & 1u) list[tot + __popc(w & lt)] = (uint16_t)(k * 32 + lane);
        tot += __popc(w);
    }
    __syncwarp();
    return tot;
}

// As enumerate_bits, over words [wbase, min(wbase + 32, wend)) and keeping only the bits whose
// index lies in [lo, hi).
__device__ __forceinline__ int enumerate_bits_in(const uint32_t* words, int wbase, int wend, int lo, int hi,
                                                 uint16_t* list) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int n = min(32, wend - wbase);
    uint32_t mine = 0u;
    if (lane < n) {
        const int b0 = (wbase + lane) * 32;  // index of the word's bit 0
        mine = words[wbase + lane];
        if (lo > b0) mine = lo - b0 >= 32 ? 0u : mine & (0xffffffffu << (lo - b0));
        if (hi < b0 + 32) mine = hi <= b0 ? 0u : mine & (0xffffffffu >> (b0 + 32 - hi));
    }
    int tot = 0;
    for (int k = 0; k < n; ++k) {
        const uint32_t w = __shfl_sync(0xffffffffu, mine, k);
        if ((w >> lane) & 1u) list[tot + __popc(w & lt)] = (uint16_t)(k * 32 + lane);
        tot += __popc(w);
    }
    __syncwarp();
    return tot;
}

// Warp sum of N values (N a power of two, at most 32).  Each step halves the values a lane
// holds: the lanes with bit `ofs` set keep the upper half and add their partner's, the others
// the lower half; once one value is left the remaining steps are a plain butterfly.  Lane l
// returns the total of v[l >> (5 - log2 N)].  N - 1 + 5 - log2 N shuffles instead of 5 N.
template <int N>
__device__ __forceinline__ float warp_sum_spread(float (&v)[N]) {
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N: a power of two up to 32");
    const int lane = threadIdx.x & 31;
    int ofs = 16;
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2) {
        const bool up = (lane & ofs) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = up ? v[k] : v[k + h];
            const float keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, ofs);
        }
        ofs >>= 1;
    }
    float t = v[0];
#pragma unroll
    for (; ofs > 0; ofs >>= 1) t += __shfl_xor_sync(0xffffffffu, t, ofs);
    return t;
}

// Per-pixel record, computed once per covered pixel (one thread each) so that the
// double-word shading geometry is not repeated by every lane of the warp-per-pixel kernels:
//   [0] b0 b1 b2 |eye-x|   [1] w_o.xyz fs   [2] ft i0 j0 -   [3] org.xyz ng.x   [4] ng.y ng.z - -
// (b: barycentrics of the camera ray; (i0 + fs, j0 + ft): texel-space position of the shading
// point; org / ng: the spec ray origin and geometric normal).
__global__ void __launch_bounds__(256) pixel_prep_kernel(ShadeArgs A) {
    const uint32_t total = *A.count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t pid = A.pixels[i];
        int c, px, py;
        uint32_t rem;
        pixel_of(A, pid, &c, &px, &py, &rem);
        const int f = (int)(uint32_t)(A.visbuf[pid] & 0xffffffffull);
        const Cam& cam = A.cams[c];
        S3 org, ngs;
        pixel_geometry(A, pid, &org, &ngs);
        const int i0 = __ldg(A.F + 3 * f), i1 = __ldg(A.F + 3 * f + 1), i2 = __ldg(A.F + 3 * f + 2);
        const int u0 = __ldg(A.Fuv + 3 * f), u1 = __ldg(A.Fuv + 3 * f + 1), u2 = __ldg(A.Fuv + 3 * f + 2);
        const float3 P0 = ld3(A.V + 3 * i0), P1 = ld3(A.V + 3 * i1), P2 = ld3(A.V + 3 * i2);
        // the camera ray through the pixel centre, d = fwd + dx right + dy up with
        // dx = (px + 1/2 - cx) / kx and dy = (cy - py - 1/2) / ky, as double-words
        const FF dx = ff_div(ff_two_sum((float)px + 0.5f, -cam.cx), ff(cam.kx));
        const FF dy = ff_div(ff_two_sum(cam.cy, -((float)py + 0.5f)), ff(cam.ky));
        FF3 d;
        d.x = ff_add(ff_add(ff(cam.fwd[0]), ff_mul_f(dx, cam.right[0])), ff_mul_f(dy, cam.up[0]));
        d.y = ff_add(ff_add(ff(cam.fwd[1]), ff_mul_f(dx, cam.right[1])), ff_mul_f(dy, cam.up[1]));
        d.z = ff_add(ff_add(ff(cam.fwd[2]), ff_mul_f(dx, cam.right[2])), ff_mul_f(dy, cam.up[2]));
        const float3 eye = f3(cam.eye[0], cam.eye[1], cam.eye[2]);
        const FF3 so = ff3_sub(eye, P0);
        FF b[3];
        bary_ff(so, d, P0, P1, P2, b);
        int ii, jj;
        float fs, ft;
        texel_coord(b, __ldg(A.UV + 2 * u0), __ldg(A.UV + 2 * u1), __ldg(A.UV + 2 * u2), A.map.W, &ii, &fs);
        texel_coord(b, __ldg(A.UV + 2 * u0 + 1), __ldg(A.UV + 2 * u1 + 1), __ldg(A.UV + 2 * u2 + 1), A.map.H, &jj,
                    &ft);
        // view vector eye - x = (eye - p0) - b1 e1 - b2 e2 and its length
        const FF3 e1 = ff3_sub(P1, P0), e2 = ff3_sub(P2, P0);
        FF3 v;
        v.x = ff_sub(so.x, ff_add(ff_mul(b[1], e1.x), ff_mul(b[2], e2.x)));
        v.y = ff_sub(so.y, ff_add(ff_mul(b[1], e1.y), ff_mul(b[2], e2.y)));
        v.z = ff_sub(so.z, ff_add(ff_mul(b[1], e1.z), ff_mul(b[2], e2.z)));
        const FF l2 = ff3_dot(v, v);
        const float r0 = __fsqrt_rn(l2.hi);  // one Newton step: |v| = r0 + (l2 - r0^2) / (2 r0)
        const FF len = ff_fast_two_sum(r0, __fdiv_rn(ff_f(ff_sub(l2, ff_two_prod(r0, r0))), __fmul_rn(2.0f, r0)));
        float4* R = A.prec + kPrec * (size_t)i;
        R[0] = make_float4(ff_f(b[0]), ff_f(b[1]), ff_f(b[2]), ff_f(len));
        R[1] = make_float4(ff_f(ff_div(v.x, len)), ff_f(ff_div(v.y, len)), ff_f(ff_div(v.z, len)), fs);
        R[2] = make_float4(ft, __int_as_float(ii), __int_as_float(jj), 0.0f);
        R[3] = make_float4(org.x, org.y, org.z, ngs.x);
        R[4] = make_float4(ngs.y, ngs.z, 0.0f, 0.0f);
    }
}

// Shading state of a covered pixel (Eqs. 10-11) from its record: fetched channels (and their
// texel-space derivatives when `deriv`), the interpolated frame, the material and n_s.
struct PixelShade {
    int i0, i1, i2, u0, u1, u2;
    float3 P0, P1, P2;
    float b[3];
    float2 uv0, uv1, uv2;
    Footprint fp;
    float att[8], dfs[8], dft[8];
    float3 N0, N1, N2, T0, T1, T2, ni, ti;
    Surface su;
    float vol;
    float3 wo;
};

template <typename T>
__device__ __forceinline__ void pixel_shade(const ShadeArgs& A, uint32_t i, int f, bool deriv, PixelShade& S) {
    const float4* R = A.prec + kPrec * (size_t)i;
    const float4 r0 = R[0], r1 = R[1], r2 = R[2];
    S.i0 = __ldg(A.F + 3 * f); S.i1 = __ldg(A.F + 3 * f + 1); S.i2 = __ldg(A.F + 3 * f + 2);
    S.u0 = __ldg(A.Fuv + 3 * f); S.u1 = __ldg(A.Fuv + 3 * f + 1); S.u2 = __ldg(A.Fuv + 3 * f + 2);
    S.b[0] = r0.x; S.b[1] = r0.y; S.b[2] = r0.z;
    S.vol = r0.w;
    S.wo = f3(r1.x, r1.y, r1.z);
    S.fp = footprint_i(A.map, __float_as_int(r2.y), __float_as_int(r2.z), r1.w, r2.x);
    fetch8<T>(A.map, S.fp, S.att, deriv ? S.dfs : nullptr, S.dft);
    S.N0 = ld3(A.nrm + 3 * S.i0); S.N1 = ld3(A.nrm + 3 * S.i1); S.N2 = ld3(A.nrm + 3 * S.i2);
    S.T0 = ld3(A.tan + 3 * S.u0); S.T1 = ld3(A.tan + 3 * S.u1); S.T2 = ld3(A.tan + 3 * S.u2);
    S.ni = S.b[0] * S.N0 + S.b[1] * S.N1 + S.b[2] * S.N2;
    S.ti = S.b[0] * S.T0 + S.b[1] * S.T1 + S.b[2] * S.T2;
    S.su = make_surface(S.att, S.ni, S.ti, __ldg(A.fsign + f), A.metallic);
    if (deriv) {
        S.P0 = ld3(A.V + 3 * S.i0); S.P1 = ld3(A.V + 3 * S.i1); S.P2 = ld3(A.V + 3 * S.i2);
        S.uv0 = make_float2(__ldg(A.UV + 2 * S.u0), __ldg(A.UV + 2 * S.u0 + 1));
        S.uv1 = make_float2(__ldg(A.UV + 2 * S.u1), __ldg(A.UV + 2 * S.u1 + 1));
        S.uv2 = make_float2(__ldg(A.UV + 2 * S.u2), __ldg(A.UV + 2 * S.u2 + 1));
    }
}

// Resident blocks per SM the register allocation must allow.  The sample loops are latency-bound,
// so more resident warps pay until spills cost more: measured on the 2M-triangle workload, the
// indirect forward ran 8.16 / 7.50 / 7.25 ms at 5 / 6 / 7 blocks and the indirect backward
// 12.31 / 11.92 / 12.46 ms at 5 / 6 / 5 (direct-only / with indirect).
constexpr int shade_min_blocks(bool bwd, bool ind) { return bwd ? 6 : (ind ? 7 : 8); }

// Material and shading normal of each covered pixel from the maps of the pass that runs it,
// one thread per pixel, into its record: [5] a.xyz r, [6] m n_s.xyz.  The warp-per-pixel
// sample loops below read them instead of evaluating Eqs. 10-11 once per warp.
template <typename T>
__global__ void __launch_bounds__(256) pixel_surface_kernel(ShadeArgs A) {
    const uint32_t total = *A.count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t pid = A.pixels[i];
        const int f = (int)(uint32_t)(A.visbuf[pid] & 0xffffffffull);
        PixelShade S;
        pixel_shade<T>(A, i, f, false, S);
        float4* R = A.prec + kPrec * (size_t)i;
        R[5] = make_float4(S.su.a.x, S.su.a.y, S.su.a.z, S.su.r);
        R[6] = make_float4(S.su.m, S.su.ns.x, S.su.ns.y, S.su.ns.z);
    }
}

// Sample loops, one warp per pixel: the forward sums the pixel's estimator (Eqs. 17-20); the
// backward sums, over the pixel's samples, the adjoints of E (scattered per sample) and of
// n_s, w_o, a, r and m, which shade_epilogue_kernel carries back to the maps and vertices.
// Fields of the per-hit records of the indirect loop (one column per secondary ray of a batch of
// 32 rays, of one pixel or of a group of pixels): the forward's first seven, then the
// backward's hit state and its adjoint sums.
enum : int {
    HWB, HF_X, HF_Y, HF_Z, HN_X, HN_Y, HN_Z, kHitFwd,
    HJ_X = kHitFwd, HJ_Y, HJ_Z, HPBS, HA_X, HA_Y, HA_Z, HM, HT_X, HT_Y, HT_Z, HB_X, HB_Y, HB_Z, HN_X2, HN_Y2, HN_Z2,
    HNT_X, HNT_Y, HNT_Z, HQL, HFP0, HFP1, HFP2, HFP3, HFS, HFT, GFD_X, GFD_Y, GFD_Z, GNS_X, GNS_Y, GNS_Z, kHitBwd
};

// Hit record of secondary ray j of a pixel (what depends on j alone: its direction, the hit
// point's double-word barycentrics, the material and frame at y) into column `col` of the
// warp's records.  wb = 0 marks a ray without live samples (no valid hit, or n_s(x).w_j <= 0).
template <typename T, bool BWD>
__device__ __forceinline__ void ind_record(const ShadeArgs& A, size_t si, uint32_t rem, int c, int j, S3 org, S3 ngs,
                                           float3 sns, float (*hr)[32], int col) {
    const int gtri = A.hits[si * A.Nb + j];
    float wb = 0.0f;
    float3 fdy = f3(0.f, 0.f, 0.f), nsy = f3(0.f, 0.f, 1.f);
    if (gtri >= 0) {
        float xi1;
        const S3 wjs = secondary_dir(A, rem, c, j, ngs, &xi1);
        const float3 wj = normalize(tof(wjs));
        const float cxj = dot(sns, wj);
        if (cxj > 0.0f) {
            const float pbs = (A.lambda / (float)A.Nb) * (kPi / __fsqrt_rn(ssub(1.0f, xi1)));  // lambda / (N_b p_b)
            wb = pbs * cxj;
            const int q0 = __ldg(A.F + 3 * gtri), q1 = __ldg(A.F + 3 * gtri + 1), q2 = __ldg(A.F + 3 * gtri + 2);
            const int v0 = __ldg(A.Fuv + 3 * gtri), v1 = __ldg(A.Fuv + 3 * gtri + 1), v2 = __ldg(A.Fuv + 3 * gtri + 2);
            const float3 Q0 = ld3(A.V + 3 * q0), Q1 = ld3(A.V + 3 * q1), Q2 = ld3(A.V + 3 * q2);
            FF by[3];
            bary_ff(ff3_sub(f3(org.x, org.y, org.z), Q0), FF3{ff(wjs.x), ff(wjs.y), ff(wjs.z)}, Q0, Q1, Q2, by);
            int ti, tj;
            float fs, ft;
            texel_coord(by, __ldg(A.UV + 2 * v0), __ldg(A.UV + 2 * v1), __ldg(A.UV + 2 * v2), A.map.W, &ti, &fs);
            texel_coord(by, __ldg(A.UV + 2 * v0 + 1), __ldg(A.UV + 2 * v1 + 1), __ldg(A.UV + 2 * v2 + 1), A.map.H,
                        &tj, &ft);
            const Footprint fpy = footprint_i(A.map, ti, tj, fs, ft);
            float atty[8];
            if (A.sec_material) {
                fetch8<T>(A.map, fpy, atty, nullptr, nullptr);
            } else {
                // constant default material: grey diffuse, flat tangent-space normal
                atty[0] = atty[1] = atty[2] = 0.5f;
                atty[3] = 0.5f;
                atty[4] = 0.0f;
                atty[5] = atty[6] = 0.0f;
                atty[7] = 1.0f;
            }
            const float b0 = ff_f(by[0]), b1 = ff_f(by[1]), b2 = ff_f(by[2]);
            const float3 niy = b0 * ld3(A.nrm + 3 * q0) + b1 * ld3(A.nrm + 3 * q1) + b2 * ld3(A.nrm + 3 * q2);
            const float3 tiy = b0 * ld3(A.tan + 3 * v0) + b1 * ld3(A.tan + 3 * v1) + b2 * ld3(A.tan + 3 * v2);
            const Surface sy = make_surface(atty, niy, tiy, __ldg(A.fsign + gtri), A.metallic);
            fdy = ((1.0f - sy.m) * kInvPi) * sy.a;
            nsy = sy.ns;
            if (BWD) {
                hr[HJ_X][col] = wj.x; hr[HJ_Y][col] = wj.y; hr[HJ_Z][col] = wj.z;
                hr[HPBS][col] = pbs;
                hr[HA_X][col] = sy.a.x; hr[HA_Y][col] = sy.a.y; hr[HA_Z][col] = sy.a.z;
                hr[HM][col] = sy.m;
                hr[HT_X][col] = sy.T.x; hr[HT_Y][col] = sy.T.y; hr[HT_Z][col] = sy.T.z;
                hr[HB_X][col] = sy.B.x; hr[HB_Y][col] = sy.B.y; hr[HB_Z][col] = sy.B.z;
                hr[HN_X2][col] = sy.n.x; hr[HN_Y2][col] = sy.n.y; hr[HN_Z2][col] = sy.n.z;
                hr[HNT_X][col] = sy.nt.x; hr[HNT_Y][col] = sy.nt.y; hr[HNT_Z][col] = sy.nt.z;
                hr[HQL][col] = sy.ql;
                hr[HFP0][col] = __uint_as_float(fpy.t[0]); hr[HFP1][col] = __uint_as_float(fpy.t[1]);
                hr[HFP2][col] = __uint_as_float(fpy.t[2]); hr[HFP3][col] = __uint_as_float(fpy.t[3]);
                hr[HFS][col] = fpy.fs; hr[HFT][col] = fpy.ft;
                hr[GFD_X][col] = 0.f; hr[GFD_Y][col] = 0.f; hr[GFD_Z][col] = 0.f;
                hr[GNS_X][col] = 0.f; hr[GNS_Y][col] = 0.f; hr[GNS_Z][col] = 0.f;
            }
        }
    }
    hr[HWB][col] = wb;
    hr[HF_X][col] = fdy.x; hr[HF_Y][col] = fdy.y; hr[HF_Z][col] = fdy.z;
    hr[HN_X][col] = nsy.x; hr[HN_Y][col] = nsy.y; hr[HN_Z][col] = nsy.z;
}

// The backward's last step for one hit record: its summed material adjoint to the map
// footprint at y, once per hit.
__device__ __forceinline__ void ind_scatter(const ShadeArgs& A, const float (*hr)[32], int col) {
    const float3 gfd = f3(hr[GFD_X][col], hr[GFD_Y][col], hr[GFD_Z][col]);
    const float3 gny = f3(hr[GNS_X][col], hr[GNS_Y][col], hr[GNS_Z][col]);
    const float my = hr[HM][col];
    const float3 ay = f3(hr[HA_X][col], hr[HA_Y][col], hr[HA_Z][col]);
    const float3 nty = f3(hr[HNT_X][col], hr[HNT_Y][col], hr[HNT_Z][col]);
    float gy[8];
    const float3 gay = ((1.0f - my) * kInvPi) * gfd;
    gy[0] = gay.x; gy[1] = gay.y; gy[2] = gay.z; gy[3] = 0.0f;
    gy[4] = A.metallic ? -dot(gfd, ay) * kInvPi : 0.0f;
    const float3 gnt = f3(dot(f3(hr[HT_X][col], hr[HT_Y][col], hr[HT_Z][col]), gny),
                          dot(f3(hr[HB_X][col], hr[HB_Y][col], hr[HB_Z][col]), gny),
                          dot(f3(hr[HN_X2][col], hr[HN_Y2][col], hr[HN_Z2][col]), gny));
    const float3 gq = (1.0f / hr[HQL][col]) * (gnt - dot(gnt, nty) * nty);
    gy[5] = gq.x; gy[6] = gq.y; gy[7] = gq.z;
    Footprint fpy;
    fpy.t[0] = __float_as_uint(hr[HFP0][col]); fpy.t[1] = __float_as_uint(hr[HFP1][col]);
    fpy.t[2] = __float_as_uint(hr[HFP2][col]); fpy.t[3] = __float_as_uint(hr[HFP3][col]);
    fpy.fs = hr[HFS][col];
    fpy.ft = hr[HFT][col];
    scatter8(A.gmaps, fpy, gy);
}

// The live (j, s) light samples of secondary rays jb .. jend - 1 of one pixel (bits
// [jb N_s, jend N_s) of its secondary visibility words), one per lane; ray jj's record sits in
// column cb + jj - jb.  The forward adds to L; the backward scatters the samples' E adjoints,
// adds to the pixel's a, m and n_s adjoints and sums each hit's material adjoint in its record.
template <bool BWD>
__device__ __forceinline__ void ind_pairs(const ShadeArgs& A, const EnvView& env, size_t si, uint32_t rem, int c,
                                          int jb, int jend, int cb, float (*hr)[32], uint16_t* list, float3 g,
                                          float3 sa, float sm, float3& L, float3& ga, float& gm, float3& gns,
                                          uint32_t& c_brdf) {
    const int lane = threadIdx.x & 31;
    const float3 fdx = ((1.0f - sm) * kInvPi) * sa;
    const float invNs = 1.0f / (float)A.Ns;
    const float invW = 1.0f / (float)env.W;
    const uint32_t* sb = A.secbits + si * A.ws;
    const int blo = jb * A.Ns, bhi = jend * A.Ns;
    for (int wbase = blo >> 5; wbase < ((bhi + 31) >> 5); wbase += 32) {
        const int tot = enumerate_bits_in(sb, wbase, (bhi + 31) >> 5, blo, bhi, list);
        for (int t0 = 0; t0 < tot; t0 += 32) {
            const int e = t0 + lane;
            if (e >= tot) continue;
            const int bit = wbase * 32 + list[e];
            const int jj = bit / A.Ns, s = bit - jj * A.Ns;
            const int hl = cb + jj - jb;
            const float wbj = hr[HWB][hl];
            if (wbj == 0.0f) continue;
            const float3 fdyj = f3(hr[HF_X][hl], hr[HF_Y][hl], hr[HF_Z][hl]);
            const float3 nsyj = f3(hr[HN_X][hl], hr[HN_Y][hl], hr[HN_Z][hl]);
            const uint4 h2 = philox(make_uint4(rem, (uint32_t)c, (uint32_t)(jj * A.Ns + s), 2u), A.key);
            // the texel gen_seclight's search picked (a live sample was queued, so it was
            // recorded), its row by one corrected FP32 quotient as for direct samples
            const uint32_t t = A.tsel2[si * A.Nb * A.Ns + bit];
            uint32_t row = (uint32_t)((float)t * invW);
            if (row * (uint32_t)env.W > t) --row;
            else if ((row + 1u) * (uint32_t)env.W <= t) ++row;
            LightSample ls;
            finish_sample(env, h2, row, t - row * (uint32_t)env.W, &ls);
            const float3 wl = normalize(tof(ls.dir));
            const float cs = dot(nsyj, wl);
            if (cs <= 0.0f) continue;
            ++c_brdf;
            const float term = ls.inv_pdf * invNs * cs;
            const float3 ET = term * ls.E;
            if (!BWD) {
                L += wbj * (fdx * (fdyj * ET));
            } else {
                // E of the light sample
                const float3 gE = (wbj * term) * (g * (fdx * fdyj));
                atomicAdd(A.genv + ls.texel, make_float4(gE.x, gE.y, gE.z, 0.0f));
                // f_d(x) and n_s(x) through max(n_s(x).w_j, 0)
                const float3 gfdx = wbj * (g * (fdyj * ET));
                ga += ((1.0f - sm) * kInvPi) * gfdx;
                gm += -dot(gfdx, sa) * kInvPi;
                gns += (hr[HPBS][hl] * dot(g, fdx * (fdyj * ET))) * f3(hr[HJ_X][hl], hr[HJ_Y][hl], hr[HJ_Z][hl]);
                // the material at y (its geometry is a constant of the derivative): the
                // adjoints of f_d(y) and n_s(y), summed per hit
                const float3 gLsec = wbj * (g * fdx);
                const float3 gfdy = gLsec * ET;
                const float3 gnsy = (ls.inv_pdf * invNs * dot(gLsec, fdyj * ls.E)) * wl;
                atomicAdd(&hr[GFD_X][hl], gfdy.x);
                atomicAdd(&hr[GFD_Y][hl], gfdy.y);
                atomicAdd(&hr[GFD_Z][hl], gfdy.z);
                atomicAdd(&hr[GNS_X][hl], gnsy.x);
                atomicAdd(&hr[GNS_Y][hl], gnsy.y);
                atomicAdd(&hr[GNS_Z][hl], gnsy.z);
            }
        }
        __syncwarp();
    }
}

template <typename T, bool BWD, bool COUNT, bool IND>
__global__ void __launch_bounds__(kShadeWarps * 32, shade_min_blocks(BWD, IND)) shade_kernel(ShadeArgs A) {
    __shared__ uint16_t s_list[kShadeWarps][kListMax];
    __shared__ float hit[kShadeWarps][IND ? (BWD ? kHitBwd : kHitFwd) : 1][32];
    const int lane = threadIdx.x & 31;
    const int hw = threadIdx.x >> 5;
    uint16_t* list = s_list[hw];
    float (*hr)[32] = hit[hw];
    const uint32_t total = *A.count;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    EnvView env = A.env;
    env.Q = *A.env.Qp;
    unsigned long long my_samples = 0;
    uint32_t c_brdf = 0;
    const uint32_t end = min(A.shade_end, total);
    const bool ind = IND && A.Nb > 0 && A.lambda != 0.0f;
    // A warp takes PB consecutive pixels at a time.  With N_b <= 16 secondary rays per pixel it
    // first evaluates the hit records of all PB = 32 / N_b pixels, one lane per (pixel, ray),
    // so that the lanes are not idle for 32 - N_b of the 32 columns; with more it takes one
    // pixel and evaluates its records 32 rays at a time inside the pixel's loop.
    const int PB = (ind && A.Nb <= 16) ? 32 / A.Nb : 1;
    const bool grouped = ind && A.Nb <= 16;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint32_t i0 = A.shade_begin + warp * (uint32_t)PB; i0 < end; i0 += nwarps * (uint32_t)PB) {
        const uint32_t i_end = min(i0 + (uint32_t)PB, end);
        if (IND && grouped) {
            // ---- the hit records of the group: lane l takes ray l mod N_b of pixel i0 + l / N_b
            const int p = lane / A.Nb, j = lane - p * A.Nb;
            const uint32_t ip = i0 + (uint32_t)p;
            bool live = p < PB && ip < i_end;
            uint32_t rem = 0;
            int c = 0;
            if (live) {
                const uint32_t pid = A.pixels[ip];
                int px, py;
                pixel_of(A, pid, &c, &px, &py, &rem);
                if (BWD) {
                    const float3 g = ld3(A.grad_rgb + 3 * (size_t)pid);
                    live = !(g.x == 0.0f && g.y == 0.0f && g.z == 0.0f);  // a pixel the backward skips
                }
            }
            if (live) {
                const float4* R = A.prec + kPrec * (size_t)ip;
                const float4 r3 = R[3], r4 = R[4], r6 = R[6];
                ind_record<T, BWD>(A, (size_t)(ip - A.state_base), rem, c, j, s3(r3.x, r3.y, r3.z),
                                   s3(r3.w, r4.x, r4.y), f3(r6.y, r6.z, r6.w), hr, lane);
            } else {
                hr[HWB][lane] = 0.0f;
            }
            __syncwarp();
        }
        for (uint32_t i = i0; i < i_end; ++i) {
            const uint32_t pid = A.pixels[i];
            const size_t si = (size_t)(i - A.state_base);  // the pixel's row of the per-sample state
            int c, px, py;
            uint32_t rem;
            pixel_of(A, pid, &c, &px, &py, &rem);
            float3 g = f3(0.f, 0.f, 0.f);
            if (BWD) {
                g = ld3(A.grad_rgb + 3 * (size_t)pid);
                if (g.x == 0.0f && g.y == 0.0f && g.z == 0.0f) continue;
            }
            const float4* R = A.prec + kPrec * (size_t)i;
            // shading state at x (Eqs. 10-11) from the pixel's record
            const float4 r1 = R[1], r5 = R[5], r6 = R[6];
            const float3 wo = f3(r1.x, r1.y, r1.z);
            const float3 sa = f3(r5.x, r5.y, r5.z), sns = f3(r6.y, r6.z, r6.w);
            const float sr = r5.w, sm = r6.x;
            float3 L = f3(0.f, 0.f, 0.f);
            float3 gns = f3(0.f, 0.f, 0.f), gwo = f3(0.f, 0.f, 0.f), ga = f3(0.f, 0.f, 0.f);
            float gr = 0.f, gm = 0.f;
            // ---- direct light (Eq. 17): the pixel's unoccluded samples, one per lane
            const float invNd = 1.0f / (float)A.Nd;
            const float invW = 1.0f / (float)env.W;
            const uint32_t* vb = A.visbits + si * A.wd;
            for (int wbase = 0; wbase < A.wd; wbase += 32) {
                const int tot = enumerate_bits(vb, wbase, A.wd, list);
                for (int t0 = 0; t0 < tot; t0 += 32) {
                    const int e = t0 + lane;
                    if (e < tot) {
                        const int k = wbase * 32 + list[e];
                        const uint4 h = philox(make_uint4(rem, (uint32_t)c, (uint32_t)k, 0u), A.key);
                        // the texel gen_direct's search picked for this sample (a live sample was
                        // queued, so it was recorded); t < 2^22 is exact in FP32, and one step
                        // corrects the rounded quotient
                        const uint32_t t = A.tsel[si * A.Nd + k];
                        uint32_t row = (uint32_t)((float)t * invW);
                        if (row * (uint32_t)env.W > t) --row;
                        else if ((row + 1u) * (uint32_t)env.W <= t) ++row;
                        LightSample ls;
                        finish_sample(env, h, row, t - row * (uint32_t)env.W, &ls);
                        const float3 wi = normalize(tof(ls.dir));
                        const float w = ls.inv_pdf * invNd;
                        ++c_brdf;
                        if (!BWD) {
                            L += w * (ls.E * brdf_cos(sns, wi, wo, sa, sr, sm));
                        } else {
                            const float3 fc =
                                brdf_cos_adjoint(sns, wi, wo, sa, sr, sm, w * (g * ls.E), gns, gwo, ga, gr, gm);
                            const float3 gE = w * (g * fc);
                            atomicAdd(A.genv + ls.texel, make_float4(gE.x, gE.y, gE.z, 0.0f));
                        }
                    }
                }
                __syncwarp();
            }
            if (!BWD && lane == 0) my_samples += (unsigned long long)A.Nd;
            // ---- one-bounce indirect (Eqs. 18-19): the live (j, s) pairs of the pixel's rays
            // (named by the visibility bits), against the hit records of those rays
            if (IND && ind) {
                if (!BWD) {
                    int valid = 0;
                    for (int j0 = 0; j0 < A.Nb; j0 += 32) {
                        const int j = j0 + lane;
                        valid += __popc(__ballot_sync(0xffffffffu, j < A.Nb && A.hits[si * A.Nb + j] >= 0));
                    }
                    if (lane == 0) my_samples += (unsigned long long)A.Nb + (unsigned long long)valid * A.Ns;
                }
                // a ray whose record has wb = 0 adds nothing, so a pixel (or batch) whose rays all
                // have it skips the listing of its light samples
                if (grouped) {
                    const int cb = (int)(i - i0) * A.Nb;
                    if (__any_sync(0xffffffffu, lane < A.Nb && hr[HWB][cb + lane] != 0.0f))
                        ind_pairs<BWD>(A, env, si, rem, c, 0, A.Nb, cb, hr, list, g, sa, sm, L, ga, gm, gns, c_brdf);
                } else {
                    const float4 r3 = R[3], r4 = R[4];
                    const S3 org = s3(r3.x, r3.y, r3.z), ngs = s3(r3.w, r4.x, r4.y);
                    for (int jb = 0; jb < A.Nb; jb += 32) {
                        const int j = jb + lane;
                        if (j < A.Nb) ind_record<T, BWD>(A, si, rem, c, j, org, ngs, sns, hr, lane);
                        else hr[HWB][lane] = 0.0f;
                        __syncwarp();
                        if (__any_sync(0xffffffffu, hr[HWB][lane] != 0.0f))
                            ind_pairs<BWD>(A, env, si, rem, c, jb, min(jb + 32, A.Nb), 0, hr, list, g, sa, sm, L, ga,
                                           gm, gns, c_brdf);
                        // backward: each hit's summed material adjoint to its map footprint, once
                        if (BWD && A.gmaps && A.sec_material && hr[HWB][lane] != 0.0f) ind_scatter(A, hr, lane);
                        __syncwarp();
                    }
                }
            }
            if (!BWD) {
                float v[4] = {L.x, L.y, L.z, 0.0f};
                const float t = warp_sum_spread<4>(v);  // lanes 0, 8, 16: L.x, L.y, L.z
                if ((lane & 7) == 0 && lane < 24) A.out[3 * (size_t)pid + (lane >> 3)] = t;
                continue;
            }
            // ---- the pixel's sums of the sample adjoints, for the epilogue
            float v[16] = {gns.x, gns.y, gns.z, gwo.x, gwo.y, gwo.z, ga.x, ga.y, ga.z, gr, gm, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float t = warp_sum_spread<16>(v);  // lanes 2q and 2q + 1: value q
            if ((lane & 1) == 0 && lane < 22) A.pacc[12 * (size_t)i + (lane >> 1)] = t;
        }
        if (IND && grouped) {
            // backward: each hit's summed material adjoint to its map footprint, once
            __syncwarp();
            if (BWD && A.gmaps && A.sec_material && hr[HWB][lane] != 0.0f) ind_scatter(A, hr, lane);
            __syncwarp();
        }
    }
    if (!BWD) {
        if (lane == 0 && my_samples) atomicAdd(A.samples, my_samples);
    }
    if (COUNT) {
        for (int ofs = 16; ofs > 0; ofs >>= 1) c_brdf += __shfl_xor_sync(0xffffffffu, c_brdf, ofs);
        if (lane == 0) atomicAdd(A.work + 2, (unsigned long long)c_brdf);
    }
}

// Adjoint of the attribute query at x (Eqs. 10-11), one thread per pixel: from the sums of
// the sample adjoints of n_s, w_o, a, r and m to the map texels of the bilinear footprint
// and, when vertex gradients are asked for, through the tangent frame, the UV and the
// camera-ray barycentrics to the vertices, their normals and the UV-vertex tangents.
template <typename T>
__global__ void __launch_bounds__(256) shade_epilogue_kernel(ShadeArgs A) {
    const uint32_t total = *A.count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t pid = A.pixels[i];
        const float3 g = ld3(A.grad_rgb + 3 * (size_t)pid);
        if (g.x == 0.0f && g.y == 0.0f && g.z == 0.0f) continue;  // the sample kernel skipped it
        int c, px, py;
        uint32_t rem;
        pixel_of(A, pid, &c, &px, &py, &rem);
        const Cam& cam = A.cams[c];
        const float4* q = reinterpret_cast<const float4*>(A.pacc + 12 * (size_t)i);
        const float4 q0 = q[0], q1 = q[1], q2 = q[2];
        const float acc[11] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z};
        const float3 gns = f3(acc[0], acc[1], acc[2]);
        const float3 gwo = f3(acc[3], acc[4], acc[5]);
        const int f = (int)(uint32_t)(A.visbuf[pid] & 0xffffffffull);
        PixelShade E;
        pixel_shade<T>(A, i, f, true, E);
        const Surface& su = E.su;
        const int i0 = E.i0, i1 = E.i1, i2 = E.i2, u0 = E.u0, u1 = E.u1, u2 = E.u2;
        const float3 P0 = E.P0, P1 = E.P1, P2 = E.P2;
        const float3 N0 = E.N0, N1 = E.N1, N2 = E.N2, T0 = E.T0, T1 = E.T1, T2 = E.T2;
        const float3 ni = E.ni, ti = E.ti;
        const float2 uv0 = E.uv0, uv1 = E.uv1, uv2 = E.uv2;
        const Footprint fp = E.fp;
        const float* b = E.b;
        const float* dfs = E.dfs;
        const float* dft = E.dft;
        const float vol = E.vol;
        const float3 wo2 = E.wo;
        // camera-ray direction (FP32 suffices for the barycentric adjoint)
        const float dxf = ((float)px + 0.5f - cam.cx) / cam.kx, dyf = (cam.cy - ((float)py + 0.5f)) / cam.ky;
        const float3 dvv = f3(cam.fwd[0] + dxf * cam.right[0] + dyf * cam.up[0],
                              cam.fwd[1] + dxf * cam.right[1] + dyf * cam.up[1],
                              cam.fwd[2] + dxf * cam.right[2] + dyf * cam.up[2]);
        S3 o = s3(cam.eye[0], cam.eye[1], cam.eye[2]);
        float gatt[8];
        gatt[0] = acc[6]; gatt[1] = acc[7]; gatt[2] = acc[8];
        gatt[3] = acc[9];
        gatt[4] = A.metallic ? acc[10] : 0.0f;
        // n_s = T nt.x + B nt.y + n nt.z;  B = s (n x T);  nt = q / |q|
        const float3 gnt = f3(dot(su.T, gns), dot(su.B, gns), dot(su.n, gns));
        const float3 gq = (1.0f / su.ql) * (gnt - dot(gnt, su.nt) * su.nt);
        gatt[5] = gq.x; gatt[6] = gq.y; gatt[7] = gq.z;
        if (A.gmaps) {
            const float wt[4] = {(1.f - fp.fs) * (1.f - fp.ft), fp.fs * (1.f - fp.ft), (1.f - fp.fs) * fp.ft, fp.fs * fp.ft};
            float4* gm = reinterpret_cast<float4*>(A.gmaps);
#pragma unroll
            for (int tap = 0; tap < 4; ++tap) {
                const float w = wt[tap];
                atomicAdd(gm + 2 * (size_t)fp.t[tap], make_float4(w * gatt[0], w * gatt[1], w * gatt[2], w * gatt[3]));
                atomicAdd(gm + 2 * (size_t)fp.t[tap] + 1, make_float4(w * gatt[4], w * gatt[5], w * gatt[6], w * gatt[7]));
            }
        }
        if (A.gV == nullptr) continue;
        const float3 gB = su.nt.y * gns;
        float3 gT = su.nt.x * gns + su.s * cross(gB, su.n);
        float3 gn = su.nt.z * gns + su.s * cross(su.T, gB);
        // T = u / |u|, u = ti - (n.ti) n
        const float ul = sqrtf(dot(su.u, su.u));
        const float3 gu = (1.0f / ul) * (gT - dot(gT, su.T) * su.T);
        const float nti = dot(su.n, ti);
        const float3 gti = gu - dot(gu, su.n) * su.n;
        gn = gn - (nti * gu + dot(gu, su.n) * ti);
        const float nl = sqrtf(dot(ni, ni));
        const float3 gni = (1.0f / nl) * (gn - dot(gn, su.n) * su.n);
        float gb[3];
        gb[0] = dot(N0, gni) + dot(T0, gti);
        gb[1] = dot(N1, gni) + dot(T1, gti);
        gb[2] = dot(N2, gni) + dot(T2, gti);
        // uv
        float gfs = 0.f, gft = 0.f;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) { gfs += gatt[ch] * dfs[ch]; gft += gatt[ch] * dft[ch]; }
        const float gu_ = gfs * (float)A.map.W, gv_ = gft * (float)A.map.H;
        gb[0] += uv0.x * gu_ + uv0.y * gv_;
        gb[1] += uv1.x * gu_ + uv1.y * gv_;
        gb[2] += uv2.x * gu_ + uv2.y * gv_;
        // x through w_o = (eye - x) / |eye - x|
        const float3 gx = (-1.0f / vol) * (gwo - dot(gwo, wo2) * wo2);
        gb[0] += dot(P0, gx); gb[1] += dot(P1, gx); gb[2] += dot(P2, gx);
        float3 gP0 = b[0] * gx, gP1 = b[1] * gx, gP2 = b[2] * gx;
        // barycentrics of the camera ray (Moller-Trumbore) w.r.t. the vertices
        {
            const float3 dv = dvv, oo = tof(o);
            const float3 e1 = P1 - P0, e2 = P2 - P0, sv = oo - P0;
            const float3 pv = cross(dv, e2);
            const float det = dot(e1, pv);
            const float b1 = b[1], b2 = b[2];
            const float g1 = gb[1] - gb[0], g2 = gb[2] - gb[0];
            const float gn1 = g1 / det, gn2 = g2 / det, gdet = -(g1 * b1 + g2 * b2) / det;
            float3 gs = gn1 * pv;
            const float3 gp = gn1 * sv + gdet * e1;
            const float3 gqv = gn2 * dv;
            float3 ge1 = gdet * pv;
            gs += cross(e1, gqv);
            ge1 += cross(gqv, sv);
            const float3 ge2 = cross(gp, dv);
            gP0 += f3(0.f, 0.f, 0.f) - gs - ge1 - ge2;
            gP1 += ge1;
            gP2 += ge2;
        }
        const int vi[3] = {i0, i1, i2}, ui[3] = {u0, u1, u2};
        const float3 gP[3] = {gP0, gP1, gP2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicAdd(A.gV + 3 * vi[k], gP[k].x);
            atomicAdd(A.gV + 3 * vi[k] + 1, gP[k].y);
            atomicAdd(A.gV + 3 * vi[k] + 2, gP[k].z);
            const float3 a1 = b[k] * gni, a2 = b[k] * gti;
            atomicAdd(A.gnrm + vi[k], make_float4(a1.x, a1.y, a1.z, 0.0f));
            atomicAdd(A.gtan + ui[k], make_float4(a2.x, a2.y, a2.z, 0.0f));
        }
    }
}

__global__ void env_grad_finish_kernel(const float4* __restrict__ genv, int n, float* grad_env) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float4 v = genv[t];
    grad_env[3 * (size_t)t] += v.x;
    grad_env[3 * (size_t)t + 1] += v.y;
    grad_env[3 * (size_t)t + 2] += v.z;
}

}  // namespace exm

using namespace exm;

static ShadeArgs make_args(exm_ctx* ctx, const exm_mesh* m, const void* maps, int mapW, int mapH, const exm_env* e,
                           exm_frame* f, const exm_params* p) {
    ShadeArgs A{};
    A.V = m->V; A.F = m->F; A.UV = m->UV; A.Fuv = m->Fuv;
    A.nrm = m->nrm; A.tan = m->tan; A.fsign = m->fsign;
    A.bvh.tris = m->layout == EXM_BVH_8Q ? m->tris8 : m->tris;
    A.bvh.nodes4 = m->nodes4;
    A.bvh.nodes8 = m->nodes8;
    A.bvh.nodesq = m->nodesq;
    A.bvh.sphere = m->sphere;
    A.bvh_layout = m->layout;
    A.map.data = maps; A.map.W = mapW; A.map.H = mapH; A.map.wrap_u = (p->flags & EXM_FLAG_WRAP_U) != 0;
    A.env.texel = e->texel; A.env.cdf = e->cdf; A.env.rguide = e->rguide; A.env.cguide = e->cguide;
    A.env.rowpre = e->rowpre; A.env.rowsum = e->rowsum;
    A.env.srowend = nullptr; A.env.srguide = nullptr;
    A.env_smem = env_rows_shared_bytes(e->H, e->rbits, kEnvSharedMax);
    A.env.W = e->W; A.env.H = e->H;
    A.env.rbits = e->rbits; A.env.cbits = e->cbits;
    A.env.Qp = e->total;
    A.cams = (const Cam*)f->cams;
    A.visbuf = (const unsigned long long*)f->visbuf;
    A.pixels = f->pixels;
    A.count = f->counters;
    A.W = f->W; A.H = f->H;
    A.Nd = p->n_direct; A.Nb = p->n_bounce; A.Ns = p->n_bounce > 0 ? p->n_light : 0;
    A.wd = (p->n_direct + 31) / 32;
    A.ws = (p->n_bounce > 0 && p->lambda_ind != 0.0f) ? (p->n_bounce * p->n_light + 31) / 32 : 0;
    strata2((uint32_t)A.Nd, &A.nxd, &A.nyd);
    strata2((uint32_t)(A.Ns > 0 ? A.Ns : 1), &A.nxs, &A.nys);
    A.lambda = p->lambda_ind;
    A.metallic = (p->flags & EXM_FLAG_NO_METALLIC) == 0;
    A.sec_material = (p->flags & EXM_FLAG_NO_SECONDARY_MATERIAL) == 0;
    A.key = make_uint2((uint32_t)p->seed, (uint32_t)(p->seed >> 32));
    A.samples = f->samples;
    A.work = f->work;
    A.status = ctx->d_status;
    const size_t P = (size_t)f->views * f->W * f->H;
    A.prec = f->prec;
    A.pacc = f->pacc;
    A.tsel = f->tsel;
    A.tsel2 = f->tsel2;
    A.visbits = f->bits;
    A.secbits = f->bits ? f->bits + P * A.wd : nullptr;
    A.hits = f->hits;
    A.rays = f->rays;
    return A;
}

// Kernel timing (EXM_FLAG_TIME_KERNELS): events around each launch of the four main kernels.
static void time_begin(exm_frame* f, const exm_params* p, int which, cudaStream_t s) {
    if (!(p->flags & EXM_FLAG_TIME_KERNELS)) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    f->timers.push_back({which, a, b});
}
static void time_end(exm_frame* f, const exm_params* p, cudaStream_t s) {
    if (!(p->flags & EXM_FLAG_TIME_KERNELS) || f->timers.empty()) return;
    cudaEventRecord(f->timers.back().end, s);
}

// One resident wave: the grid-stride loop then gives every warp the same share of pixels
// and no block waits for a second wave.
template <typename T, bool BWD, bool COUNT, bool IND>
static void launch_shade_one(const ShadeArgs& A, int num_sms, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, shade_kernel<T, BWD, COUNT, IND>, kShadeWarps * 32, 0) !=
                cudaSuccess || n < 1)
            n = 1;
        per_sm = n;
    }
    shade_kernel<T, BWD, COUNT, IND><<<num_sms * per_sm, kShadeWarps * 32, 0, s>>>(A);
}

template <bool BWD, bool COUNT, bool IND>
static void launch_shade_t(const ShadeArgs& A, exm_dtype dt, int num_sms, cudaStream_t s) {
    switch (dt) {
        case EXM_F32: launch_shade_one<float, BWD, COUNT, IND>(A, num_sms, s); break;
        case EXM_BF16: launch_shade_one<__nv_bfloat16, BWD, COUNT, IND>(A, num_sms, s); break;
        default: launch_shade_one<__half, BWD, COUNT, IND>(A, num_sms, s); break;
    }
}

// The thread-per-pixel kernels around the sample loops: the surface records before them, and
// after the backward's, its epilogue.
template <typename T>
static void launch_pixel_kernels(const ShadeArgs& A, bool epilogue, int num_sms, cudaStream_t s) {
    if (epilogue) shade_epilogue_kernel<T><<<num_sms * 8, 256, 0, s>>>(A);
    else pixel_surface_kernel<T><<<num_sms * 8, 256, 0, s>>>(A);
}
static void launch_pixel_kernels(const ShadeArgs& A, exm_dtype dt, bool epilogue, int num_sms, cudaStream_t s) {
    switch (dt) {
        case EXM_F32: launch_pixel_kernels<float>(A, epilogue, num_sms, s); break;
        case EXM_BF16: launch_pixel_kernels<__nv_bfloat16>(A, epilogue, num_sms, s); break;
        default: launch_pixel_kernels<__half>(A, epilogue, num_sms, s); break;
    }
}

// The thread-per-pixel surface records (material and n_s) from the maps of the pass.
static void launch_surface(exm_ctx* ctx, exm_frame* f, const exm_params* p, const ShadeArgs& A, exm_dtype dt,
                           bool bwd, cudaStream_t s) {
    time_begin(f, p, bwd ? 3 : 2, s);
    launch_pixel_kernels(A, dt, false, ctx->num_sms, s);
    time_end(f, p, s);
    ctx->launches += 1;
}

// The warp-per-pixel sample loops over covered pixels [A.shade_begin, A.shade_end).
template <bool BWD>
static void launch_samples(exm_ctx* ctx, exm_frame* f, const exm_params* p, const ShadeArgs& A, exm_dtype dt,
                           cudaStream_t s) {
    const int sms = ctx->num_sms;
    time_begin(f, p, BWD ? 3 : 2, s);
    const bool ind = A.Nb > 0 && A.lambda != 0.0f;
    const bool count = (p->flags & EXM_FLAG_COUNT_WORK) != 0;
    if (ind) {
        if (count) launch_shade_t<BWD, true, true>(A, dt, sms, s);
        else launch_shade_t<BWD, false, true>(A, dt, sms, s);
    } else {
        if (count) launch_shade_t<BWD, true, false>(A, dt, sms, s);
        else launch_shade_t<BWD, false, false>(A, dt, sms, s);
    }
    time_end(f, p, s);
    ctx->launches += 1;
}

template <bool CLOSEST>
static void launch_trace(exm_ctx* ctx, exm_frame* f, const exm_params* p, const ShadeArgs& A, cudaStream_t s) {
    const int blocks = ctx->num_sms * kTraceBlocksPerSM;
    time_begin(f, p, CLOSEST ? 1 : 0, s);
    const bool count = (p->flags & EXM_FLAG_COUNT_WORK) != 0;
    if (A.bvh_layout == EXM_BVH_8Q) {
        if (count) trace_kernel<CLOSEST, true, EXM_BVH_8Q><<<blocks, kTraceThreads, 0, s>>>(A);
        else trace_kernel<CLOSEST, false, EXM_BVH_8Q><<<blocks, kTraceThreads, 0, s>>>(A);
    } else if (A.bvh_layout == EXM_BVH_4Q) {
        if (count) trace_kernel<CLOSEST, true, EXM_BVH_4Q><<<blocks, kTraceThreads, 0, s>>>(A);
        else trace_kernel<CLOSEST, false, EXM_BVH_4Q><<<blocks, kTraceThreads, 0, s>>>(A);
    } else {
        if (count) trace_kernel<CLOSEST, true, EXM_BVH_4><<<blocks, kTraceThreads, 0, s>>>(A);
        else trace_kernel<CLOSEST, false, EXM_BVH_4><<<blocks, kTraceThreads, 0, s>>>(A);
    }
    time_end(f, p, s);
    ctx->launches += 1;
}

// Per-sample state a frame keeps for the whole frame at most (the texel each direct sample
// picked, the visibility bits and the secondary hit ids); above it the state lives one chunk
// at a time and the backward pass recomputes it chunk by chunk.
constexpr uint64_t kSavedBudgetDefault = 16ull << 30;

// How a pass splits the frame's pixels into chunks: the rays of a chunk fit one queue and,
// when the per-sample state is recomputed, the chunk's state fits the budget.
struct ChunkPlan {
    size_t P = 0;            // frame pixels (views * W * H): the covered ones are a prefix of the list
    int wd = 0, ws = 0;      // visibility words per pixel: direct, secondary light samples
    int nb = 0;              // secondary rays per pixel with an active indirect term, else 0
    bool indirect = false;
    uint32_t Pc = 0;         // pixels per chunk (a multiple of 32)
    uint32_t ray_cap = 0;    // queue entries per chunk
    size_t nchunks = 0;
    bool recompute = false;  // per-sample state per chunk, recomputed by the backward pass
    size_t Ps = 0;           // pixels whose per-sample state is resident at once
    size_t state_per_px = 0; // bytes of per-sample state per pixel
};

static ChunkPlan plan_chunks(const exm_frame* f, const exm_params* p) {
    ChunkPlan c;
    c.P = (size_t)f->views * f->W * f->H;
    c.wd = (p->n_direct + 31) / 32;
    c.indirect = p->n_bounce > 0 && p->lambda_ind != 0.0f;
    c.ws = c.indirect ? (int)(((int64_t)p->n_bounce * p->n_light + 31) / 32) : 0;
    c.nb = c.indirect ? p->n_bounce : 0;
    const size_t cap_max = f->ray_cap ? f->ray_cap : kRayCapDefault;
    // rays a pixel queues at most: one per direct sample, secondary ray and secondary light sample
    const size_t per_pixel = std::max((size_t)c.wd * 32 + (size_t)c.ws * 32, (size_t)std::max(c.nb, 1));
    const size_t P32 = (c.P + 31) & ~(size_t)31;
    size_t Pc = std::max((size_t)32, std::min(P32, (cap_max / per_pixel) & ~(size_t)31));
    c.state_per_px = std::max((size_t)1, 4 * (size_t)p->n_direct + 4 * (size_t)(c.wd + c.ws) + 4 * (size_t)c.nb +
                                             (c.indirect ? 4 * (size_t)p->n_bounce * p->n_light : 0));
    const uint64_t budget = f->saved_budget ? f->saved_budget : kSavedBudgetDefault;
    c.recompute = (p->flags & EXM_FLAG_RECOMPUTE) != 0 || (uint64_t)c.P * c.state_per_px > budget;
    if (c.recompute) Pc = std::max((size_t)32, std::min(Pc, (size_t)(budget / c.state_per_px) & ~(size_t)31));
    c.Pc = (uint32_t)Pc;
    c.ray_cap = (uint32_t)std::min(cap_max, Pc * per_pixel);
    c.nchunks = (c.P + Pc - 1) / Pc;
    c.Ps = c.recompute ? Pc : c.P;
    return c;
}

// Ray generation and tracing of chunk `ch`: secondary rays and their closest hits, then the
// shadow rays of the direct samples and of the secondary hits' light samples, as bits.
static void trace_chunk(exm_ctx* ctx, exm_frame* f, const exm_params* p, const ChunkPlan& c, ShadeArgs& A,
                        size_t ch, cudaStream_t s) {
    ExmRange range("chunk: ray generation and tracing");
    A.chunk_begin = (uint32_t)(ch * c.Pc);
    A.chunk_pixels = c.Pc;
    A.ctr = f->ctr + 4 * ch;
    A.state_base = c.recompute ? A.chunk_begin : 0;
    if (c.recompute) {  // this chunk's state starts empty
        cudaMemsetAsync(f->bits, 0, c.Ps * (size_t)(c.wd + c.ws) * sizeof(uint32_t), s);
        if (c.indirect) cudaMemsetAsync(f->hits, 0xff, c.Ps * (size_t)c.nb * sizeof(int32_t), s);
    }
    if (c.indirect) {
        gen_secondary_kernel<<<exm_blocks((size_t)c.Pc, 256), 256, 0, s>>>(A);
        ctx->launches += 1;
        launch_trace<true>(ctx, f, p, A, s);
    }
    if (p->n_direct > 0) {  // 0 in the indirect-only half-resolution pass
        const unsigned gb = exm_blocks((size_t)c.Pc * ((p->n_direct + kGenK - 1) / kGenK), kGenThreads);
        if (A.env_smem) gen_direct_kernel<true><<<gb, kGenThreads, A.env_smem, s>>>(A);
        else gen_direct_kernel<false><<<gb, kGenThreads, 0, s>>>(A);
        ctx->launches += 1;
    }
    if (c.indirect) {
        const unsigned sb = exm_blocks((size_t)c.Pc, kGenThreads);
        if (A.env_smem) gen_seclight_kernel<true><<<sb, kGenThreads, A.env_smem, s>>>(A);
        else gen_seclight_kernel<false><<<sb, kGenThreads, 0, s>>>(A);
        ctx->launches += 1;
    }
    launch_trace<false>(ctx, f, p, A, s);
}

exm_status exm_shade_forward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                                  const exm_env* e, exm_frame* f, const exm_params* p, float* out, cudaStream_t s) {
    if (dt != EXM_F32 && dt != EXM_BF16 && dt != EXM_F16) return exm_fail(EXM_ERR_ARG, "map dtype");
    const ChunkPlan c = plan_chunks(f, p);
    const size_t P = c.P;
    f->last_nd = -1;  // no valid saved state until this pass is enqueued
    if (!ensure(&f->prec, &f->prec_cap, P * (size_t)kPrec) || !ensure(&f->pacc, &f->pacc_cap, P * (size_t)12) ||
        (p->n_direct > 0 && !ensure(&f->tsel, &f->tsel_cap, c.Ps * (size_t)p->n_direct)) ||
        (c.indirect && !ensure(&f->tsel2, &f->tsel2_cap, c.Ps * (size_t)p->n_bounce * p->n_light)) ||
        !ensure(&f->bits, &f->bits_cap, c.Ps * (size_t)(c.wd + c.ws)) ||
        !ensure(&f->rays, &f->rays_cap, (size_t)c.ray_cap * 2) ||
        (c.indirect && !ensure(&f->hits, &f->hits_cap, c.Ps * (size_t)c.nb)))
        return exm_fail(EXM_ERR_OOM, "wavefront buffers");
    if (!ensure(&f->ctr, &f->ctr_cap, c.nchunks * 4)) return exm_fail(EXM_ERR_OOM, "chunk counters");
    ShadeArgs A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.secbits = f->bits + c.Ps * (size_t)c.wd;
    A.ray_cap = c.ray_cap;
    A.out = out;
    pixel_prep_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(A);
    ctx->launches += 1;
    cudaMemsetAsync(f->samples, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(out, 0, P * 3 * sizeof(float), s);
    cudaMemsetAsync(f->ctr, 0, c.nchunks * 4 * sizeof(uint32_t), s);
    if (!c.recompute) {
        cudaMemsetAsync(f->bits, 0, P * (size_t)(c.wd + c.ws) * sizeof(uint32_t), s);
        if (c.indirect) cudaMemsetAsync(f->hits, 0xff, P * (size_t)c.nb * sizeof(int32_t), s);
    }
    if (p->flags & EXM_FLAG_COUNT_WORK) cudaMemsetAsync(f->work, 0, 4 * sizeof(unsigned long long), s);
    {
        ExmRange r("pixel records");
        launch_surface(ctx, f, p, A, dt, false, s);
    }
    for (size_t ch = 0; ch < c.nchunks; ++ch) {
        trace_chunk(ctx, f, p, c, A, ch, s);
        if (c.recompute) {  // shade the chunk while its state is resident
            ExmRange r("shade");
            A.shade_begin = A.chunk_begin;
            A.shade_end = A.chunk_begin + c.Pc;
            launch_samples<false>(ctx, f, p, A, dt, s);
        }
    }
    if (!c.recompute) {
        ExmRange r("shade");
        A.state_base = 0;
        A.shade_begin = 0;
        A.shade_end = 0xffffffffu;
        launch_samples<false>(ctx, f, p, A, dt, s);
    }
    exm_status st = exm_cuda_check(cudaGetLastError(), "forward launch");
    if (st != EXM_OK) return st;
    f->last_wd = c.wd;
    f->last_ws = c.ws;
    f->last_nb = c.nb;
    f->last_ns = c.indirect ? p->n_light : 0;
    f->last_nd = p->n_direct;
    f->fwd_mesh_stamp = m->stamp;
    f->fwd_env_stamp = e->stamp;
    f->fwd_env_W = e->W;
    f->fwd_env_H = e->H;
    f->fwd_mapW = mapW;
    f->fwd_mapH = mapH;
    f->fwd_seed = p->seed;
    f->fwd_recompute = c.recompute;
    f->fwd_chunk = c.Pc;
    f->fwd_ray_cap = c.ray_cap;
    return EXM_OK;
}

// ---------------------------------------------------------------------------------------
// Batched relight forward (relight serving, exm_serve.cu): one request's forward pass split at
// its two tracer launches, which the server makes once for a whole batch of requests
// (trace_batch_kernel).  A request's rays must fit one queue chunk.

struct exm_relight_pass {
    ShadeArgs A;
    ChunkPlan c;
    exm_params p;
    exm_dtype dt;
};

exm_status relight_pass_begin(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                              const exm_env* e, exm_frame* f, const exm_params* p, float* out, cudaStream_t s,
                              exm_relight_pass** out_pass) {
    *out_pass = nullptr;
    if (dt != EXM_F32 && dt != EXM_BF16 && dt != EXM_F16) return exm_fail(EXM_ERR_ARG, "map dtype");
    const ChunkPlan c = plan_chunks(f, p);
    if (c.nchunks != 1 || c.recompute)
        return exm_fail(EXM_ERR_ARG, "relight batch: the request's rays exceed one queue chunk");
    f->last_nd = -1;
    if (!ensure(&f->prec, &f->prec_cap, c.P * (size_t)kPrec) || !ensure(&f->pacc, &f->pacc_cap, c.P * (size_t)12) ||
        (p->n_direct > 0 && !ensure(&f->tsel, &f->tsel_cap, c.Ps * (size_t)p->n_direct)) ||
        (c.indirect && !ensure(&f->tsel2, &f->tsel2_cap, c.Ps * (size_t)p->n_bounce * p->n_light)) ||
        !ensure(&f->bits, &f->bits_cap, c.Ps * (size_t)(c.wd + c.ws)) ||
        !ensure(&f->rays, &f->rays_cap, (size_t)c.ray_cap * 2) ||
        (c.indirect && !ensure(&f->hits, &f->hits_cap, c.Ps * (size_t)c.nb)) || !ensure(&f->ctr, &f->ctr_cap, 4))
        return exm_fail(EXM_ERR_OOM, "relight batch: wavefront buffers");
    exm_relight_pass* rp = new (std::nothrow) exm_relight_pass();
    if (!rp) return exm_fail(EXM_ERR_OOM, "relight batch: host allocation");
    rp->c = c;
    rp->p = *p;
    rp->dt = dt;
    ShadeArgs& A = rp->A;
    A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.secbits = f->bits + c.Ps * (size_t)c.wd;
    A.ray_cap = c.ray_cap;
    A.out = out;
    A.chunk_begin = 0;
    A.chunk_pixels = c.Pc;
    A.ctr = f->ctr;
    A.state_base = 0;
    A.shade_begin = 0;
    A.shade_end = 0xffffffffu;
    pixel_prep_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(A);
    ctx->launches += 1;
    cudaMemsetAsync(f->samples, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(out, 0, c.P * 3 * sizeof(float), s);
    cudaMemsetAsync(f->ctr, 0, 4 * sizeof(uint32_t), s);
    cudaMemsetAsync(f->bits, 0, c.P * (size_t)(c.wd + c.ws) * sizeof(uint32_t), s);
    launch_surface(ctx, f, p, A, dt, false, s);
    if (c.indirect) {
        cudaMemsetAsync(f->hits, 0xff, c.P * (size_t)c.nb * sizeof(int32_t), s);
        gen_secondary_kernel<<<exm_blocks((size_t)c.Pc, 256), 256, 0, s>>>(A);
        ctx->launches += 1;
    }
    *out_pass = rp;
    return exm_cuda_check(cudaGetLastError(), "relight batch: setup");
}

bool relight_pass_indirect(const exm_relight_pass* rp) { return rp->c.indirect; }

void relight_pass_shadow_rays(exm_ctx* ctx, exm_relight_pass* rp, cudaStream_t s) {
    const ShadeArgs& A = rp->A;
    if (rp->p.n_direct > 0) {
        const unsigned gb = exm_blocks((size_t)rp->c.Pc * ((rp->p.n_direct + kGenK - 1) / kGenK), kGenThreads);
        if (A.env_smem) gen_direct_kernel<true><<<gb, kGenThreads, A.env_smem, s>>>(A);
        else gen_direct_kernel<false><<<gb, kGenThreads, 0, s>>>(A);
        ctx->launches += 1;
    }
    if (rp->c.indirect) {
        if (A.env_smem)
            gen_seclight_kernel<true><<<exm_blocks((size_t)rp->c.Pc, kGenThreads), kGenThreads, A.env_smem, s>>>(A);
        else gen_seclight_kernel<false><<<exm_blocks((size_t)rp->c.Pc, kGenThreads), kGenThreads, 0, s>>>(A);
        ctx->launches += 1;
    }
}

exm_status relight_pass_shade(exm_ctx* ctx, exm_relight_pass* rp, exm_frame* f, cudaStream_t s) {
    launch_samples<false>(ctx, f, &rp->p, rp->A, rp->dt, s);
    const ChunkPlan& c = rp->c;
    f->last_wd = c.wd;
    f->last_ws = c.ws;
    f->last_nb = c.nb;
    f->last_ns = c.indirect ? rp->p.n_light : 0;
    f->last_nd = rp->p.n_direct;
    f->fwd_recompute = false;
    f->fwd_chunk = c.Pc;
    f->fwd_ray_cap = c.ray_cap;
    f->fwd_seed = rp->p.seed;
    return exm_cuda_check(cudaGetLastError(), "relight batch: shade");
}

void relight_pass_free(exm_relight_pass* rp) { delete rp; }

// Rays a request of these sizes queues at most (its one chunk).
uint64_t relight_queue_rays(int views, int W, int H, const exm_params* p) {
    const bool indirect = p->n_bounce > 0 && p->lambda_ind != 0.0f;
    const uint64_t wd = (uint64_t)(p->n_direct + 31) / 32;
    const uint64_t ws = indirect ? ((uint64_t)p->n_bounce * p->n_light + 31) / 32 : 0;
    const uint64_t per_pixel = std::max(wd * 32 + ws * 32, (uint64_t)(indirect ? p->n_bounce : 1));
    const uint64_t P32 = ((uint64_t)views * W * H + 31) & ~(uint64_t)31;
    return P32 * per_pixel;
}

static exm_status relight_trace_batch_layout(exm_ctx* ctx, exm_relight_pass* const* passes, int n, bool closest,
                                             int layout, ExmTraceJob* h_jobs, ExmTraceJob* d_jobs, cudaStream_t s);

exm_status relight_trace_batch(exm_ctx* ctx, exm_relight_pass* const* passes, int n, bool closest,
                               ExmTraceJob* h_jobs, ExmTraceJob* d_jobs, cudaStream_t s) {
    if (n < 1 || n > kMaxBatch) return exm_fail(EXM_ERR_ARG, "relight batch: size");
    // one launch per BVH layout among the batch's assets
    for (int l = 0; l < kJobLayouts; ++l) {
        exm_status st = relight_trace_batch_layout(ctx, passes, n, closest, EXM_BVH_4 + l, h_jobs + l * n,
                                                   d_jobs + l * n, s);
        if (st != EXM_OK) return st;
    }
    return EXM_OK;
}

static exm_status relight_trace_batch_layout(exm_ctx* ctx, exm_relight_pass* const* passes, int n, bool closest,
                                             int layout, ExmTraceJob* h_jobs, ExmTraceJob* d_jobs, cudaStream_t s) {
    int k = 0;
    uint32_t* cursor = nullptr;
    for (int i = 0; i < n; ++i) {
        const ShadeArgs& A = passes[i]->A;
        if (closest && !passes[i]->c.indirect) continue;
        if (A.bvh_layout != layout) continue;
        TraceJob& j = h_jobs[k++];
        j.nodes4 = layout == EXM_BVH_8Q ? A.bvh.nodes8 : (layout == EXM_BVH_4Q ? A.bvh.nodesq : A.bvh.nodes4);
        j.tris = A.bvh.tris;
        j.sphere = A.bvh.sphere;
        j.rays = A.rays;
        j.qcount = A.ctr + (closest ? 0 : 2);
        j.ray_cap = A.ray_cap;
        j.visbits = A.visbits;
        j.secbits = A.secbits;
        j.hits = A.hits;
        if (!cursor) cursor = A.ctr + (closest ? 1 : 3);  // zeroed with the first pass's counters
    }
    if (k == 0) return EXM_OK;
    exm_status st = exm_cuda_check(cudaMemcpyAsync(d_jobs, h_jobs, (size_t)k * sizeof(ExmTraceJob),
                                                   cudaMemcpyHostToDevice, s), "relight batch: job table");
    if (st != EXM_OK) return st;
    ShadeArgs A = passes[0]->A;
    const int blocks = ctx->num_sms * kTraceBatchBlocksPerSM;
    if (layout == EXM_BVH_8Q) {
        if (closest) trace_batch_kernel<true, EXM_BVH_8Q><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
        else trace_batch_kernel<false, EXM_BVH_8Q><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
    } else if (layout == EXM_BVH_4Q) {
        if (closest) trace_batch_kernel<true, EXM_BVH_4Q><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
        else trace_batch_kernel<false, EXM_BVH_4Q><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
    } else {
        if (closest) trace_batch_kernel<true, EXM_BVH_4><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
        else trace_batch_kernel<false, EXM_BVH_4><<<blocks, kTraceThreads, 0, s>>>(A, d_jobs, k, cursor);
    }
    ctx->launches += 1;
    return exm_cuda_check(cudaGetLastError(), "relight batch: trace");
}

// The backward pass reads what the forward pass left in the frame: the pixel records, and the
// recorded texels, visibility bits and hit ids (or, recomputed, their chunks).  They index the
// forward's mesh, environment and maps, so the backward must get the same objects, unchanged.
static exm_status check_saved(const exm_frame* f, const exm_mesh* m, const exm_env* e, int mapW, int mapH,
                              const exm_params* p) {
    const bool indirect = p->n_bounce > 0 && p->lambda_ind != 0.0f;
    if (f->last_nd != p->n_direct || f->last_nb != (indirect ? p->n_bounce : 0) ||
        f->last_ns != (indirect ? p->n_light : 0) || !f->bits || !f->pacc)
        return exm_fail(EXM_ERR_ARG, "backward: the frame holds no forward pass with these sample counts");
    if (f->fwd_mesh_stamp != m->stamp)
        return exm_fail(EXM_ERR_ARG, "backward: the mesh, its vertices or its BVH differ from the forward pass's");
    if (f->fwd_env_stamp != e->stamp || f->fwd_env_W != e->W || f->fwd_env_H != e->H)
        return exm_fail(EXM_ERR_ARG, "backward: the environment differs from the one the forward pass sampled (" +
                                         std::to_string(f->fwd_env_W) + "x" + std::to_string(f->fwd_env_H) +
                                         " prepared before it)");
    if (f->fwd_mapW != mapW || f->fwd_mapH != mapH)
        return exm_fail(EXM_ERR_ARG, "backward: the map size differs from the forward pass's");
    if (f->fwd_seed != p->seed) return exm_fail(EXM_ERR_ARG, "backward: the sample seed differs from the forward pass's");
    return EXM_OK;
}

// True when `cams` are the cameras the frame's last pass uploaded.
static bool cameras_match(const exm_frame* f, const exm_camera* cams, int views) {
    const size_t bytes = (size_t)views * sizeof(exm_camera);
    return f->cams_host.size() == bytes && memcmp(f->cams_host.data(), cams, bytes) == 0;
}

exm_status exm_check_backward(const exm_frame* f, const exm_mesh* m, const exm_env* e, int mapW, int mapH,
                              const exm_camera* cams, int views, const exm_params* p) {
    if (!cameras_match(f, cams, views))
        return exm_fail(EXM_ERR_ARG, "backward: the cameras differ from the forward pass's");
    return check_saved(f, m, e, mapW, mapH, p);
}

// The sample loops and epilogue of the backward pass, with A's gradient outputs set.  With a
// recomputed state, each chunk's rays are generated and traced again (the same decisions: the
// streams are counter-based and the traversal deterministic) before its sample loops.  Uses
// only buffers the frame's forward pass allocated.
static exm_status backward_core(exm_ctx* ctx, exm_frame* f, const exm_params* p, ShadeArgs& A, exm_dtype dt,
                                cudaStream_t s) {
    ExmRange range("adjoint");
    ChunkPlan c = plan_chunks(f, p);
    c.recompute = f->fwd_recompute;  // the forward's split, whatever the limits are now
    c.Pc = f->fwd_chunk;
    c.ray_cap = f->fwd_ray_cap;
    c.nchunks = (c.P + c.Pc - 1) / c.Pc;
    c.Ps = c.recompute ? c.Pc : c.P;
    A.secbits = f->bits + c.Ps * (size_t)c.wd;
    A.ray_cap = c.ray_cap;
    if (p->flags & EXM_FLAG_COUNT_WORK) cudaMemsetAsync(f->work, 0, 4 * sizeof(unsigned long long), s);
    launch_surface(ctx, f, p, A, dt, true, s);
    if (!c.recompute) {
        A.state_base = 0;
        A.shade_begin = 0;
        A.shade_end = 0xffffffffu;
        launch_samples<true>(ctx, f, p, A, dt, s);
    } else {
        cudaMemsetAsync(f->ctr, 0, c.nchunks * 4 * sizeof(uint32_t), s);
        for (size_t ch = 0; ch < c.nchunks; ++ch) {
            trace_chunk(ctx, f, p, c, A, ch, s);
            A.shade_begin = A.chunk_begin;
            A.shade_end = A.chunk_begin + c.Pc;
            launch_samples<true>(ctx, f, p, A, dt, s);
        }
    }
    if (A.gmaps || A.gV) {
        time_begin(f, p, 3, s);
        launch_pixel_kernels(A, dt, true, ctx->num_sms, s);
        time_end(f, p, s);
        ctx->launches += 1;
    }
    return exm_cuda_check(cudaGetLastError(), "backward launch");
}

exm_status exm_shade_backward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                                   const exm_env* e, exm_frame* f, const exm_params* p, const float* grad_rgb,
                                   float* grad_maps, float* grad_env, float* grad_V, cudaStream_t s) {
    if (dt != EXM_F32 && dt != EXM_BF16 && dt != EXM_F16) return exm_fail(EXM_ERR_ARG, "map dtype");
    exm_status st = check_saved(f, m, e, mapW, mapH, p);
    if (st != EXM_OK) return st;
    ShadeArgs A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.grad_rgb = grad_rgb;
    A.gmaps = grad_maps;
    size_t nenv = (size_t)e->W * e->H;
    if (!ensure(&f->genv, &f->genv_capacity, nenv)) return exm_fail(EXM_ERR_OOM, "env gradient");
    size_t nfr = (size_t)(m->nv > m->nuv ? m->nv : m->nuv);
    if (grad_V && (!ensure(&f->gnrm, &f->gframe_capacity, nfr) || !ensure(&f->gtan, &f->gtan_capacity, nfr)))
        return exm_fail(EXM_ERR_OOM, "frame gradient");
    if (p->flags & EXM_FLAG_ZERO_GRADS) {
        if (grad_maps) cudaMemsetAsync(grad_maps, 0, (size_t)mapW * mapH * 8 * sizeof(float), s);
        if (grad_env) cudaMemsetAsync(grad_env, 0, nenv * 3 * sizeof(float), s);
        if (grad_V) cudaMemsetAsync(grad_V, 0, (size_t)m->nv * 3 * sizeof(float), s);
    }
    cudaMemsetAsync(f->genv, 0, nenv * sizeof(float4), s);
    A.genv = f->genv;
    if (grad_V) {
        cudaMemsetAsync(f->gnrm, 0, (size_t)m->nv * sizeof(float4), s);
        cudaMemsetAsync(f->gtan, 0, (size_t)m->nuv * sizeof(float4), s);
        A.gV = grad_V;
        A.gnrm = f->gnrm;
        A.gtan = f->gtan;
    }
    st = backward_core(ctx, f, p, A, dt, s);
    if (st != EXM_OK) return st;
    if (grad_env) {
        env_grad_finish_kernel<<<exm_blocks(nenv, 256), 256, 0, s>>>(f->genv, (int)nenv, grad_env);
        ctx->launches += 1;
    }
    if (grad_V) {
        st = exm_frames_adjoint(const_cast<exm_mesh*>(m), f->gnrm, f->gtan, grad_V, s);
        if (st != EXM_OK) return st;
        ctx->launches += 3;
    }
    return exm_cuda_check(cudaGetLastError(), "backward finish");
}

// ---------------------------------------------------------------------------------------
// Backward pass that allocates nothing.
//
// Some callers cannot call cudaMalloc while they run: for example, a host whose device
// memory is entirely owned by another allocator (a framework's caching allocator or a
// pre-reserved arena that forbids driver allocations), or a latency-critical loop in which
// the implicit device synchronisation of cudaMalloc/cudaFree is unacceptable.  The regular
// exm_render_backward may allocate its environment-gradient accumulator on first use; this
// variant instead keeps that accumulator in the file-scope array below, which every GPU that
// loads the library holds (EXM_STATIC_ENV_MAX_TEXELS x 16 bytes = 4 MiB) until the process
// exits.  It computes the map and environment gradients only (grad_V is not supported here,
// because vertex gradients need per-vertex scratch proportional to the mesh).
//
// The array is shared by every call on a device and keeps the last call's contents: each
// call clears the part it uses before its kernel runs, so calls that overlap on the GPU
// (different streams, or different host threads) race on it and must be serialised by the
// caller.  The first call on a device resolves the array's device address with
// cudaGetSymbolAddress while that device is current; make that first call before any
// stream capture.
#include <mutex>

static __device__ __align__(256) float4 g_env_grad_scratch[EXM_STATIC_ENV_MAX_TEXELS];

namespace {
constexpr int kMaxScratchDevices = 64;
std::mutex g_scratch_mutex;
float4* g_scratch_addr[kMaxScratchDevices] = {};

// Device address of g_env_grad_scratch on `device` (which must be current).
exm_status static_scratch(int device, float4** out) {
    if (device < 0 || device >= kMaxScratchDevices) return exm_fail(EXM_ERR_ARG, "static scratch: device index");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_env_grad_scratch);
        if (e != cudaSuccess) return exm_cuda_check(e, "cudaGetSymbolAddress(env gradient scratch)");
        g_scratch_addr[device] = static_cast<float4*>(p);
    }
    *out = g_scratch_addr[device];
    return EXM_OK;
}
}  // namespace

extern "C" exm_status exm_render_backward_noalloc(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt,
                                                  int mapW, int mapH, const exm_env* e, const exm_camera* cams,
                                                  int views, const exm_params* p, exm_frame* f,
                                                  const float* grad_rgb, float* grad_maps, float* grad_env,
                                                  void* stream) {
    exm_status st = check_render(ctx, m, maps, dt, mapW, mapH, e, cams, views, p, f, "exm_render_backward_noalloc");
    if (st != EXM_OK) return st;
    if (!grad_rgb) return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: grad_rgb is NULL");
    if ((long long)e->W * e->H > EXM_STATIC_ENV_MAX_TEXELS)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: environment has " +
                                         std::to_string((long long)e->W * e->H) + " texels, more than the " +
                                         std::to_string(EXM_STATIC_ENV_MAX_TEXELS) + " the static scratch holds");
    if ((p->flags & EXM_FLAG_HALF_RES_INDIRECT) && p->n_bounce > 0 && p->lambda_ind != 0.0f)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: half-resolution indirect light is not offered");
    DeviceGuard g(ctx->device);
    // every check before anything is enqueued: a rejected call leaves the outputs untouched
    st = exm_check_backward(f, m, e, mapW, mapH, cams, views, p);
    if (st != EXM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4* scratch = nullptr;
    st = static_scratch(ctx->device, &scratch);
    if (st != EXM_OK) return st;
    const size_t nenv = (size_t)e->W * e->H;
    ShadeArgs A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.grad_rgb = grad_rgb;
    A.gmaps = grad_maps;
    A.genv = scratch;
    A.gV = nullptr;
    if (p->flags & EXM_FLAG_ZERO_GRADS) {
        if (grad_maps) cudaMemsetAsync(grad_maps, 0, (size_t)mapW * mapH * 8 * sizeof(float), s);
        if (grad_env) cudaMemsetAsync(grad_env, 0, nenv * 3 * sizeof(float), s);
    }
    cudaMemsetAsync(scratch, 0, nenv * sizeof(float4), s);
    st = backward_core(ctx, f, p, A, dt, s);
    if (st == EXM_OK && grad_env) {
        env_grad_finish_kernel<<<exm_blocks(nenv, 256), 256, 0, s>>>(scratch, (int)nenv, grad_env);
        ctx->launches += 1;
    }
    if (st == EXM_OK) st = exm_cuda_check(cudaGetLastError(), "exm_render_backward_noalloc launch");
    return st;
}

extern "C" exm_status exm_frame_saved_state(exm_frame* f, const uint32_t** pixels, const uint32_t** visbits,
                                            const int32_t** hits, int dims[4]) {
    if (!f || !pixels || !visbits || !hits || !dims) return exm_fail(EXM_ERR_ARG, "exm_frame_saved_state: NULL argument");
    if (f->last_nd < 0 || !f->bits) return exm_fail(EXM_ERR_ARG, "exm_frame_saved_state: no forward pass yet");
    if (f->fwd_recompute)
        return exm_fail(EXM_ERR_ARG, "exm_frame_saved_state: the last forward kept its state one chunk at a time");
    *pixels = f->pixels;
    *visbits = f->bits;
    *hits = f->last_nb > 0 ? f->hits : nullptr;
    dims[0] = f->last_wd;
    dims[1] = f->last_ws;
    dims[2] = f->last_nb;
    dims[3] = f->views * f->W * f->H;
    return EXM_OK;
}
