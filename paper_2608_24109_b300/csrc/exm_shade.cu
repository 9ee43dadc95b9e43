// Shading and its adjoint (Sec. 5.1-5.3, Eqs. 10-20), one thread per covered pixel,
// persistent grid over the tile-ordered covered-pixel list.
//
// Forward, per pixel: barycentrics of the camera ray on the visible face; interpolated
// position, UV, vertex normal and tangent; bilinear 8-channel fetch; n_s from the normal
// map in the interpolated tangent frame (Eqs. 10-11).  Direct light: N_d stratified
// environment samples, each with f_r = f_d + f_s (Eqs. 13-16) and a BVH any-hit shadow
// ray (Eq. 17).  Indirect: N_b cosine-weighted secondary rays about n_g with closest-hit
// traversal; at each valid (front-facing) hit the same attribute query, N_s light samples
// with shadow rays (Eq. 18), weighted by f_d(x) max(n_s(x).w, 0) / p_b (Eq. 19).
// Î = L_dir + lambda_ind L_ind (Eq. 20).
//
// Backward recomputes the same decisions (same counter-based samples, same traversal)
// and scatters dL/d(map texels) (4 bilinear taps x 8 channels, vector float4 atomics),
// dL/dE (padded float4 accumulator per texel) and dL/dV (through barycentrics, position,
// view direction, interpolated normals/tangents and UV; the frame adjoint finishes it).
#include "exm_device.cuh"
#include "exm_internal.h"



namespace exm {

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
    // maps, env, frame
    MapView map;
    EnvView env;
    const Cam* cams;
    const unsigned long long* visbuf;
    const uint32_t* pixels;
    const uint32_t* count;
    int W, H;
    // params
    int Nd, Nb, Ns;
    float lambda;
    bool metallic;
    uint2 key;
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

// (f_d + f_s) * max(n.wi, 0), Eqs. 13-16 (FP32).  The GGX denominator uses
// |n x h|^2 + alpha^2 (n.h)^2, equal to (n.h)^2 (alpha^2 - 1) + 1 for unit vectors.
__device__ __forceinline__ float3 brdf_cos(float3 ns, float3 wi, float3 wo, float3 a, float r, float m) {
    float ci = dot(ns, wi), co = dot(ns, wo);
    if (ci <= 0.0f) return f3(0.f, 0.f, 0.f);
    float om = 1.0f - m;
    float3 res = (om / kPi) * a;
    if (co > 0.0f) {
        float rc = fminf(fmaxf(r, kRMin), 1.0f);
        float al = rc * rc, a2 = al * al;
        float3 hu = wi + wo;
        float3 h = rsqrtf(dot(hu, hu)) * hu;
        float nh = dot(ns, h), vh = dot(wi, h);
        float3 cx = cross(ns, h);
        float k = dot(cx, cx) + a2 * nh * nh;
        float D = a2 / (kPi * k * k);
        float sqi = sqrtf(a2 + (1.0f - a2) * ci * ci), sqo = sqrtf(a2 + (1.0f - a2) * co * co);
        float G = (2.0f * ci / (ci + sqi)) * (2.0f * co / (co + sqo));
        float om5 = 1.0f - vh, w2 = om5 * om5, w5 = w2 * w2 * om5;
        float3 F0 = f3(om * kFDielectric + m * a.x, om * kFDielectric + m * a.y, om * kFDielectric + m * a.z);
        float3 Fr = f3(F0.x + (1.f - F0.x) * w5, F0.y + (1.f - F0.y) * w5, F0.z + (1.f - F0.z) * w5);
        float P = D * G / (4.0f * ci * co + kSpecEps);
        res += P * Fr;
    }
    return ci * res;
}

// Adjoint of brdf_cos for an upstream RGB gradient G3; accumulates into gns, gwo, ga, gr, gm.
__device__ __forceinline__ void brdf_cos_adjoint(float3 ns, float3 wi, float3 wo, float3 a, float r, float m, float3 G3,
                                                 float3& gns, float3& gwo, float3& ga, float& gr, float& gm) {
    float ci = dot(ns, wi), co = dot(ns, wo);
    if (ci <= 0.0f) return;
    float om = 1.0f - m;
    float3 fd = (om / kPi) * a;
    float3 res = fd;
    float gci = 0.0f, gco = 0.0f;
    float3 gres = ci * G3;
    ga += (om / kPi) * gres;
    gm += -dot(gres, a) / kPi;
    if (co > 0.0f) {
        float rc = fminf(fmaxf(r, kRMin), 1.0f);
        float al = rc * rc, a2 = al * al;
        float3 hu = wi + wo;
        float hl = rsqrtf(dot(hu, hu));
        float3 h = hl * hu;
        float nh = dot(ns, h), vh = dot(wi, h);
        float3 cx = cross(ns, h);
        float k = dot(cx, cx) + a2 * nh * nh;
        float D = a2 / (kPi * k * k);
        float sqi = sqrtf(a2 + (1.0f - a2) * ci * ci), sqo = sqrtf(a2 + (1.0f - a2) * co * co);
        float G1i = 2.0f * ci / (ci + sqi), G1o = 2.0f * co / (co + sqo);
        float G = G1i * G1o;
        float om5 = 1.0f - vh, w2 = om5 * om5, w4 = w2 * w2, w5 = w4 * om5;
        float3 F0 = f3(om * kFDielectric + m * a.x, om * kFDielectric + m * a.y, om * kFDielectric + m * a.z);
        float3 Fr = f3(F0.x + (1.f - F0.x) * w5, F0.y + (1.f - F0.y) * w5, F0.z + (1.f - F0.z) * w5);
        float den = 4.0f * ci * co + kSpecEps;
        float P = D * G / den;
        res += P * Fr;
        float S = dot(gres, Fr);
        float3 gF = P * gres;
        float gD = S * G / den, gG = S * D / den, gden = -S * P / den;
        gci += gden * 4.0f * co;
        gco += gden * 4.0f * ci;
        float3 gF0 = f3(gF.x * (1.f - w5), gF.y * (1.f - w5), gF.z * (1.f - w5));
        float gw5 = gF.x * (1.f - F0.x) + gF.y * (1.f - F0.y) + gF.z * (1.f - F0.z);
        float gvh = -5.0f * w4 * gw5;
        gm += gF0.x * (a.x - kFDielectric) + gF0.y * (a.y - kFDielectric) + gF0.z * (a.z - kFDielectric);
        ga += m * gF0;
        float gk = -2.0f * gD * D / k;
        float ga2 = gD / (kPi * k * k) + gk * nh * nh;
        float gnh = gk * 2.0f * nh * (a2 - 1.0f);
        float ci2 = ci + sqi, co2 = co + sqo;
        gci += gG * G1o * (2.0f * a2 / (sqi * ci2 * ci2));
        gco += gG * G1i * (2.0f * a2 / (sqo * co2 * co2));
        ga2 += gG * G1o * (-ci * (1.0f - ci * ci) / (sqi * ci2 * ci2));
        ga2 += gG * G1i * (-co * (1.0f - co * co) / (sqo * co2 * co2));
        if (r >= kRMin && r <= 1.0f) gr += ga2 * 4.0f * rc * rc * rc;
        gns += gnh * h;
        float3 gh = gnh * ns + gvh * wi;
        gwo += hl * (gh - dot(gh, h) * h);
        gns += gco * wo;
        gwo += gco * ns;
    }
    gci += dot(G3, res);
    gns += gci * wi;
}

__device__ __forceinline__ void scatter8(float* gmaps, const Footprint& fp, const float g[8]) {
    float w[4] = {(1.f - fp.fs) * (1.f - fp.ft), fp.fs * (1.f - fp.ft), (1.f - fp.fs) * fp.ft, fp.fs * fp.ft};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4* p = reinterpret_cast<float4*>(gmaps) + 2 * (size_t)fp.t[k];
        atomicAdd(p, make_float4(w[k] * g[0], w[k] * g[1], w[k] * g[2], w[k] * g[3]));
        atomicAdd(p + 1, make_float4(w[k] * g[4], w[k] * g[5], w[k] * g[6], w[k] * g[7]));
    }
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

template <typename T, bool BWD, bool COUNT>
__global__ void __launch_bounds__(128) shade_kernel(ShadeArgs A) {
    const uint32_t total = *A.count;
    const uint32_t per_view = (uint32_t)A.W * (uint32_t)A.H;
    uint32_t err = 0;
    unsigned long long my_samples = 0;
    EnvView env = A.env;
    env.Q = *A.env.Qp;
    uint32_t c_nodes = 0, c_tris = 0, c_brdf = 0, c_rays = 0;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t pid = A.pixels[idx];
        const int c = (int)(pid / per_view);
        const uint32_t rem = pid - (uint32_t)c * per_view;
        const int py = (int)(rem / (uint32_t)A.W), px = (int)(rem - (uint32_t)py * (uint32_t)A.W);
        float3 g = f3(0.f, 0.f, 0.f);
        if (BWD) {
            g = ld3(A.grad_rgb + 3 * (size_t)pid);
            if (g.x == 0.0f && g.y == 0.0f && g.z == 0.0f) continue;
        }
        const int f = (int)(uint32_t)(A.visbuf[pid] & 0xffffffffull);
        const Cam& cam = A.cams[c];
        const int i0 = __ldg(A.F + 3 * f), i1 = __ldg(A.F + 3 * f + 1), i2 = __ldg(A.F + 3 * f + 2);
        const int u0 = __ldg(A.Fuv + 3 * f), u1 = __ldg(A.Fuv + 3 * f + 1), u2 = __ldg(A.Fuv + 3 * f + 2);
        const float3 P0 = ld3(A.V + 3 * i0), P1 = ld3(A.V + 3 * i1), P2 = ld3(A.V + 3 * i2);
        S3 o, d, xs, ngs;
        float bs[3];
        camera_ray(cam, px, py, &o, &d);
        surface_point(o, d, s3(P0.x, P0.y, P0.z), s3(P1.x, P1.y, P1.z), s3(P2.x, P2.y, P2.z), &xs, &ngs, bs);
        const S3 org = offset_origin(xs, ngs);
        // ---- attribute query at x (Eqs. 10-11); shading geometry in FP64
        const D3 eyed = d3(cam.eye[0], cam.eye[1], cam.eye[2]);
        const double dxd = ((double)px + 0.5 - (double)cam.cx) / (double)cam.kx;
        const double dyd = ((double)cam.cy - ((double)py + 0.5)) / (double)cam.ky;
        const D3 dd = d3(cam.fwd[0] + dxd * cam.right[0] + dyd * cam.up[0],
                         cam.fwd[1] + dxd * cam.right[1] + dyd * cam.up[1],
                         cam.fwd[2] + dxd * cam.right[2] + dyd * cam.up[2]);
        double bd[3];
        bary_d(eyed, dd, dof(P0), dof(P1), dof(P2), bd);
        const float b[3] = {(float)bd[0], (float)bd[1], (float)bd[2]};
        const float2 uv0 = make_float2(__ldg(A.UV + 2 * u0), __ldg(A.UV + 2 * u0 + 1));
        const float2 uv1 = make_float2(__ldg(A.UV + 2 * u1), __ldg(A.UV + 2 * u1 + 1));
        const float2 uv2 = make_float2(__ldg(A.UV + 2 * u2), __ldg(A.UV + 2 * u2 + 1));
        const double sd = (bd[0] * uv0.x + bd[1] * uv1.x + bd[2] * uv2.x) * A.map.W - 0.5;
        const double td = (bd[0] * uv0.y + bd[1] * uv1.y + bd[2] * uv2.y) * A.map.H - 0.5;
        const Footprint fp = footprint_d(A.map, sd, td);
        float att[8], dfs[8], dft[8];
        fetch8<T>(A.map, fp, att, BWD ? dfs : nullptr, dft);
        const float3 N0 = ld3(A.nrm + 3 * i0), N1 = ld3(A.nrm + 3 * i1), N2 = ld3(A.nrm + 3 * i2);
        const float3 T0 = ld3(A.tan + 3 * u0), T1 = ld3(A.tan + 3 * u1), T2 = ld3(A.tan + 3 * u2);
        const float3 ni = b[0] * N0 + b[1] * N1 + b[2] * N2;
        const float3 ti = b[0] * T0 + b[1] * T1 + b[2] * T2;
        const float sgn = __ldg(A.fsign + f);
        const Surface su = make_surface(att, ni, ti, sgn, A.metallic);
        const D3 vod = dsub(eyed, d3(bd[0] * P0.x + bd[1] * P1.x + bd[2] * P2.x,
                                     bd[0] * P0.y + bd[1] * P1.y + bd[2] * P2.y,
                                     bd[0] * P0.z + bd[1] * P1.z + bd[2] * P2.z));
        const double vold = sqrt(ddot(vod, vod));
        const float vol = (float)vold;
        const float3 wo = f3((float)(vod.x / vold), (float)(vod.y / vold), (float)(vod.z / vold));
        const uint32_t pixel = rem;
        // adjoint accumulators at x
        float3 gns = f3(0.f, 0.f, 0.f), gwo = f3(0.f, 0.f, 0.f), ga = f3(0.f, 0.f, 0.f);
        float gr = 0.f, gm = 0.f;
        // ---- direct light (Eq. 17)
        float3 L = f3(0.f, 0.f, 0.f);
        const float invNd = 1.0f / (float)A.Nd;
        for (int k = 0; k < A.Nd; ++k) {
            const uint4 h = philox(make_uint4(pixel, (uint32_t)c, (uint32_t)k, 0u), A.key);
            const LightSample ls = light_sample(env, h, (uint32_t)k, (uint32_t)A.Nd);
            const float3 wi = normalize(tof(ls.dir));
            if (dot(su.ns, wi) <= 0.0f) continue;
            if (!(sdot(ngs, ls.dir) > 0.0f)) continue;
            if (ls.E.x == 0.0f && ls.E.y == 0.0f && ls.E.z == 0.0f && !BWD) continue;
            ++c_rays;
            if (any_hit(A.bvh, make_ray(org, ls.dir), &err, c_nodes, c_tris)) continue;
            const float w = ls.inv_pdf * invNd;
            ++c_brdf;
            const float3 fc = brdf_cos(su.ns, wi, wo, su.a, su.r, su.m);
            L += w * (ls.E * fc);
            if (BWD) {
                const float3 gE = w * (g * fc);
                atomicAdd(A.genv + ls.texel, make_float4(gE.x, gE.y, gE.z, 0.0f));
                brdf_cos_adjoint(su.ns, wi, wo, su.a, su.r, su.m, w * (g * ls.E), gns, gwo, ga, gr, gm);
            }
        }
        my_samples += (unsigned long long)A.Nd;
        // ---- one-bounce indirect (Eqs. 18-19)
        if (A.Nb > 0 && A.lambda != 0.0f) {
            const float3 fdx = ((1.0f - su.m) / kPi) * su.a;
            const float scale = A.lambda / (float)A.Nb;
            const float invNs = 1.0f / (float)A.Ns;
            float3 Lind = f3(0.f, 0.f, 0.f);
            for (int j = 0; j < A.Nb; ++j) {
                const uint4 h = philox(make_uint4(pixel, (uint32_t)c, (uint32_t)j, 1u), A.key);
                const float xi1 = smul(__uint2float_rn(stratified32((uint32_t)j, (uint32_t)A.Nb, h.x) >> 8), 0x1p-24f);
                const float xi2 = unit24(h.y);
                const S3 wjs = cosine_dir(ngs, xi1, xi2);
                my_samples += 1ull;
                const float3 wj = normalize(tof(wjs));
                const float cxj = dot(su.ns, wj);
                if (cxj <= 0.0f) continue;
                float thit;
                bool front;
                ++c_rays;
                const int gtri = closest_hit(A.bvh, make_ray(org, wjs), &thit, &front, &err, c_nodes, c_tris);
                if (gtri < 0 || !front) continue;
                my_samples += (unsigned long long)A.Ns;
                const int j0 = __ldg(A.F + 3 * gtri), j1 = __ldg(A.F + 3 * gtri + 1), j2 = __ldg(A.F + 3 * gtri + 2);
                const int v0 = __ldg(A.Fuv + 3 * gtri), v1 = __ldg(A.Fuv + 3 * gtri + 1), v2 = __ldg(A.Fuv + 3 * gtri + 2);
                const float3 Q0 = ld3(A.V + 3 * j0), Q1 = ld3(A.V + 3 * j1), Q2 = ld3(A.V + 3 * j2);
                S3 ys, ngy;
                float bys[3];
                surface_point(org, wjs, s3(Q0.x, Q0.y, Q0.z), s3(Q1.x, Q1.y, Q1.z), s3(Q2.x, Q2.y, Q2.z), &ys, &ngy, bys);
                const S3 yorg = offset_origin(ys, ngy);
                double byd[3];
                bary_d(d3(org.x, org.y, org.z), d3(wjs.x, wjs.y, wjs.z), dof(Q0), dof(Q1), dof(Q2), byd);
                const float by[3] = {(float)byd[0], (float)byd[1], (float)byd[2]};
                const double syd = (byd[0] * __ldg(A.UV + 2 * v0) + byd[1] * __ldg(A.UV + 2 * v1) +
                                    byd[2] * __ldg(A.UV + 2 * v2)) * A.map.W - 0.5;
                const double tyd = (byd[0] * __ldg(A.UV + 2 * v0 + 1) + byd[1] * __ldg(A.UV + 2 * v1 + 1) +
                                    byd[2] * __ldg(A.UV + 2 * v2 + 1)) * A.map.H - 0.5;
                const Footprint fpy = footprint_d(A.map, syd, tyd);
                float atty[8];
                fetch8<T>(A.map, fpy, atty, nullptr, nullptr);
                const float3 niy = by[0] * ld3(A.nrm + 3 * j0) + by[1] * ld3(A.nrm + 3 * j1) + by[2] * ld3(A.nrm + 3 * j2);
                const float3 tiy = by[0] * ld3(A.tan + 3 * v0) + by[1] * ld3(A.tan + 3 * v1) + by[2] * ld3(A.tan + 3 * v2);
                const Surface sy = make_surface(atty, niy, tiy, __ldg(A.fsign + gtri), A.metallic);
                const float3 fdy = ((1.0f - sy.m) / kPi) * sy.a;
                const float wb = scale * kPi * cxj / __fsqrt_rn(ssub(1.0f, xi1));
                const float3 gLsec = wb * (g * fdx);
                float3 Esum = f3(0.f, 0.f, 0.f);
                float3 gnsy = f3(0.f, 0.f, 0.f);
                for (int s = 0; s < A.Ns; ++s) {
                    const uint4 h2 = philox(make_uint4(pixel, (uint32_t)c, (uint32_t)(j * A.Ns + s), 2u), A.key);
                    const LightSample ls = light_sample(env, h2, (uint32_t)s, (uint32_t)A.Ns);
                    const float3 wl = normalize(tof(ls.dir));
                    const float cs = dot(sy.ns, wl);
                    if (cs <= 0.0f) continue;
                    if (!(sdot(ngy, ls.dir) > 0.0f)) continue;
                    ++c_rays;
                    if (any_hit(A.bvh, make_ray(yorg, ls.dir), &err, c_nodes, c_tris)) continue;
                    ++c_brdf;
                    const float wl_ = ls.inv_pdf * invNs * cs;
                    Esum += wl_ * ls.E;
                    if (BWD) {
                        const float3 gE = wl_ * (gLsec * fdy);
                        atomicAdd(A.genv + ls.texel, make_float4(gE.x, gE.y, gE.z, 0.0f));
                        gnsy += (ls.inv_pdf * invNs * dot(gLsec, fdy * ls.E)) * wl;
                    }
                }
                const float3 Lsec = fdy * Esum;
                Lind += wb * (fdx * Lsec);
                if (BWD) {
                    // primary: dL/df_d(x) and dL/dn_s(x) through max(n_s(x).w_j, 0)
                    const float3 gfdx = wb * (g * Lsec);
                    ga += ((1.0f - su.m) / kPi) * gfdx;
                    gm += -dot(gfdx, su.a) / kPi;
                    const float gc = scale * kPi / __fsqrt_rn(ssub(1.0f, xi1)) * dot(g, fdx * Lsec);
                    gns += gc * wj;
                    // secondary material at y (its geometry is a constant of the derivative)
                    const float3 gfdy = gLsec * Esum;
                    float gy[8];
                    const float3 gay = ((1.0f - sy.m) / kPi) * gfdy;
                    gy[0] = gay.x; gy[1] = gay.y; gy[2] = gay.z; gy[3] = 0.0f;
                    gy[4] = A.metallic ? -dot(gfdy, sy.a) / kPi : 0.0f;
                    const float3 gnt = f3(dot(sy.T, gnsy), dot(sy.B, gnsy), dot(sy.n, gnsy));
                    const float3 gq = (1.0f / sy.ql) * (gnt - dot(gnt, sy.nt) * sy.nt);
                    gy[5] = gq.x; gy[6] = gq.y; gy[7] = gq.z;
                    if (A.gmaps) scatter8(A.gmaps, fpy, gy);
                }
            }
            L += Lind;
        }
        if (!BWD) {
            float* out = A.out + 3 * (size_t)pid;
            out[0] = L.x; out[1] = L.y; out[2] = L.z;
            continue;
        }
        // ---- adjoint of the attribute query at x
        float gatt[8];
        gatt[0] = ga.x; gatt[1] = ga.y; gatt[2] = ga.z;
        gatt[3] = gr;
        gatt[4] = A.metallic ? gm : 0.0f;
        // n_s = T nt.x + B nt.y + n nt.z;  B = s (n x T);  nt = q / |q|
        const float3 gnt = f3(dot(su.T, gns), dot(su.B, gns), dot(su.n, gns));
        const float3 gq = (1.0f / su.ql) * (gnt - dot(gnt, su.nt) * su.nt);
        gatt[5] = gq.x; gatt[6] = gq.y; gatt[7] = gq.z;
        if (A.gmaps) scatter8(A.gmaps, fp, gatt);
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
        // scatter to the vertex-normal / UV-vertex-tangent adjoints
        const int vi[3] = {i0, i1, i2}, ui[3] = {u0, u1, u2};
        for (int k = 0; k < 3; ++k) {
            const float3 a1 = b[k] * gni, a2v = b[k] * gti;
            atomicAdd(A.gnrm + vi[k], make_float4(a1.x, a1.y, a1.z, 0.0f));
            atomicAdd(A.gtan + ui[k], make_float4(a2v.x, a2v.y, a2v.z, 0.0f));
        }
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
        const float3 gx = (-1.0f / vol) * (gwo - dot(gwo, wo) * wo);
        gb[0] += dot(P0, gx); gb[1] += dot(P1, gx); gb[2] += dot(P2, gx);
        float3 gP0 = b[0] * gx, gP1 = b[1] * gx, gP2 = b[2] * gx;
        // barycentrics of the camera ray (Moller-Trumbore) w.r.t. the vertices
        {
            const float3 dv = f3((float)dd.x, (float)dd.y, (float)dd.z), oo = tof(o);
            const float3 e1 = P1 - P0, e2 = P2 - P0, sv = oo - P0;
            const float3 pv = cross(dv, e2), qv = cross(sv, e1);
            const float det = dot(e1, pv);
            const float b1 = b[1], b2 = b[2];
            const float g1 = gb[1] - gb[0], g2 = gb[2] - gb[0];
            const float gn1 = g1 / det, gn2 = g2 / det, gdet = -(g1 * b1 + g2 * b2) / det;
            float3 gs = gn1 * pv;
            float3 gp = gn1 * sv + gdet * e1;
            const float3 gqv = gn2 * dv;
            float3 ge1 = gdet * pv;
            gs += cross(e1, gqv);
            ge1 += cross(gqv, sv);
            const float3 ge2 = cross(gp, dv);
            gP0 += f3(0.f, 0.f, 0.f) - gs - ge1 - ge2;
            gP1 += ge1;
            gP2 += ge2;
        }
        const float3 gp3[3] = {gP0, gP1, gP2};
        for (int k = 0; k < 3; ++k) {
            atomicAdd(A.gV + 3 * vi[k], gp3[k].x);
            atomicAdd(A.gV + 3 * vi[k] + 1, gp3[k].y);
            atomicAdd(A.gV + 3 * vi[k] + 2, gp3[k].z);
        }
    }
    if (err) atomicOr(A.status, err);
    if (COUNT) {
        atomicAdd(A.work, (unsigned long long)c_nodes);
        atomicAdd(A.work + 1, (unsigned long long)c_tris);
        atomicAdd(A.work + 2, (unsigned long long)c_brdf);
        atomicAdd(A.work + 3, (unsigned long long)c_rays);
    }
    if (!BWD) {
        for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
        if ((threadIdx.x & 31) == 0 && my_samples) atomicAdd(A.samples, my_samples);
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
    A.bvh.nodes = m->nodes; A.bvh.tris = m->tris;
    A.map.data = maps; A.map.W = mapW; A.map.H = mapH; A.map.wrap_u = (p->flags & EXM_FLAG_WRAP_U) != 0;
    A.env.texel = e->texel; A.env.cdf = e->cdf; A.env.guide = e->guide; A.env.W = e->W; A.env.H = e->H;
    A.env.gbits = e->gbits;
    A.env.Qp = e->total;
    A.cams = (const Cam*)f->cams;
    A.visbuf = (const unsigned long long*)f->visbuf;
    A.pixels = f->pixels;
    A.count = f->counters;
    A.W = f->W; A.H = f->H;
    A.Nd = p->n_direct; A.Nb = p->n_bounce; A.Ns = p->n_light;
    A.lambda = p->lambda_ind;
    A.metallic = (p->flags & EXM_FLAG_NO_METALLIC) == 0;
    A.key = make_uint2((uint32_t)p->seed, (uint32_t)(p->seed >> 32));
    A.samples = f->samples;
    A.work = f->work;
    A.status = ctx->d_status;
    return A;
}

template <bool BWD, bool COUNT>
static exm_status launch_t(const ShadeArgs& A, exm_dtype dt, int blocks, cudaStream_t s) {
    switch (dt) {
        case EXM_F32: shade_kernel<float, BWD, COUNT><<<blocks, 128, 0, s>>>(A); break;
        case EXM_BF16: shade_kernel<__nv_bfloat16, BWD, COUNT><<<blocks, 128, 0, s>>>(A); break;
        case EXM_F16: shade_kernel<__half, BWD, COUNT><<<blocks, 128, 0, s>>>(A); break;
        default: return exm_fail(EXM_ERR_ARG, "map dtype");
    }
    return exm_cuda_check(cudaGetLastError(), "shade launch");
}

template <bool BWD>
static exm_status launch(const ShadeArgs& A, exm_dtype dt, int blocks, cudaStream_t s, bool count) {
    return count ? launch_t<BWD, true>(A, dt, blocks, s) : launch_t<BWD, false>(A, dt, blocks, s);
}

exm_status exm_shade_forward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                                  const exm_env* e, exm_frame* f, const exm_params* p, float* out, cudaStream_t s) {
    ShadeArgs A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.out = out;
    cudaMemsetAsync(f->samples, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(out, 0, (size_t)f->views * f->W * f->H * 3 * sizeof(float), s);
    bool count = (p->flags & EXM_FLAG_COUNT_WORK) != 0;
    if (count) cudaMemsetAsync(f->work, 0, 4 * sizeof(unsigned long long), s);
    return launch<false>(A, dt, ctx->num_sms * 8, s, count);
}

exm_status exm_shade_backward_impl(exm_ctx* ctx, const exm_mesh* m, const void* maps, exm_dtype dt, int mapW, int mapH,
                                   const exm_env* e, exm_frame* f, const exm_params* p, const float* grad_rgb,
                                   float* grad_maps, float* grad_env, float* grad_V, cudaStream_t s) {
    ShadeArgs A = make_args(ctx, m, maps, mapW, mapH, e, f, p);
    A.grad_rgb = grad_rgb;
    A.gmaps = grad_maps;
    size_t nenv = (size_t)e->W * e->H;
    if (nenv > f->genv_capacity) {
        cudaFree(f->genv);
        f->genv = nullptr;
        if (cudaMalloc(&f->genv, nenv * sizeof(float4)) != cudaSuccess) { f->genv_capacity = 0; return exm_fail(EXM_ERR_OOM, "env gradient"); }
        f->genv_capacity = nenv;
    }
    size_t nfr = (size_t)(m->nv > m->nuv ? m->nv : m->nuv);
    if (grad_V && nfr > f->gframe_capacity) {
        cudaFree(f->gnrm);
        cudaFree(f->gtan);
        f->gnrm = f->gtan = nullptr;
        if (cudaMalloc(&f->gnrm, nfr * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&f->gtan, nfr * sizeof(float4)) != cudaSuccess) {
            f->gframe_capacity = 0;
            return exm_fail(EXM_ERR_OOM, "frame gradient");
        }
        f->gframe_capacity = nfr;
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
    bool count = (p->flags & EXM_FLAG_COUNT_WORK) != 0;
    if (count) cudaMemsetAsync(f->work, 0, 4 * sizeof(unsigned long long), s);
    if (p->flags & EXM_FLAG_ZERO_GRADS) {
        if (grad_maps) cudaMemsetAsync(grad_maps, 0, (size_t)mapW * mapH * 8 * sizeof(float), s);
        if (grad_env) cudaMemsetAsync(grad_env, 0, nenv * 3 * sizeof(float), s);
        if (grad_V) cudaMemsetAsync(grad_V, 0, (size_t)m->nv * 3 * sizeof(float), s);
    }
    exm_status st = launch<true>(A, dt, ctx->num_sms * 8, s, count);
    if (st != EXM_OK) return st;
    if (grad_env) env_grad_finish_kernel<<<exm_blocks(nenv, 256), 256, 0, s>>>(f->genv, (int)nenv, grad_env);
    if (grad_V) {
        st = exm_frames_adjoint(const_cast<exm_mesh*>(m), f->gnrm, f->gtan, grad_V, s);
        if (st != EXM_OK) return st;
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
    if (!ctx || !m || !maps || !e || !cams || !p || !f || !grad_rgb)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: NULL argument");
    if ((long long)e->W * e->H > EXM_STATIC_ENV_MAX_TEXELS)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: environment has " +
                                         std::to_string((long long)e->W * e->H) + " texels, more than the " +
                                         std::to_string(EXM_STATIC_ENV_MAX_TEXELS) + " the static scratch holds");
    if (dt != EXM_F32 && dt != EXM_BF16 && dt != EXM_F16)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: map dtype");
    if (mapW < 1 || mapH < 1 || (long long)mapW * mapH > (1ll << 28))
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: map size");
    if (views != f->views) return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: views differ from the frame's");
    if (p->n_direct < 1 || p->n_direct > 65536 || p->n_bounce < 0 || p->n_bounce > 4096 ||
        (p->n_bounce > 0 && (p->n_light < 1 || p->n_light > 4096)))
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: sample counts");
    if (m->ctx != ctx || e->ctx != ctx || f->ctx != ctx)
        return exm_fail(EXM_ERR_ARG, "exm_render_backward_noalloc: objects of another context");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    float4* scratch = nullptr;
    exm_status st = static_scratch(ctx->device, &scratch);
    if (st == EXM_OK)
        st = exm_cuda_check(cudaMemcpyAsync(f->cams, cams, (size_t)views * sizeof(exm_camera), cudaMemcpyHostToDevice, s),
                            "camera upload");
    if (st == EXM_OK) {
        size_t nenv = (size_t)e->W * e->H;
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
        st = launch<true>(A, dt, ctx->num_sms * 8, s, false);
        if (st == EXM_OK && grad_env)
            env_grad_finish_kernel<<<exm_blocks(nenv, 256), 256, 0, s>>>(scratch, (int)nenv, grad_env);
        if (st == EXM_OK) st = exm_cuda_check(cudaGetLastError(), "exm_render_backward_noalloc launch");
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return st;
}
