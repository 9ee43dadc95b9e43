// Device-side building blocks of the Stage-II renderer (sm_103a).
//
// Two kinds of arithmetic live here:
//  * the FP32 decision specification -- every step that decides an integer (coverage,
//    texel choice, shadow-ray visibility, secondary hit id) or builds the rays that feed
//    such a decision is written with explicitly rounded intrinsics (__fadd_rn, __fmul_rn,
//    ...), so the compiler cannot contract it into FMAs and the decision is the one the
//    specification fixes;
//  * shading, which is ordinary FP32 (contraction allowed).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace exm {

// Device error bits latched in the context's status word.
enum : uint32_t { ERRBIT_GUARD = 1u, ERRBIT_TRAVERSAL = 2u, ERRBIT_INDEX = 4u, ERRBIT_QUEUE = 8u };

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kFDielectric = 0.04f;   // F_dielectric of Eq. 16
constexpr float kSpecEps = 1e-6f;       // epsilon of Eq. 15
constexpr float kRMin = 0.08f;          // roughness clamp before alpha = r^2
constexpr int kStackSize4 = 192;  // 3 pushes per level of a tree at most 62 levels deep
constexpr int kEmptyChild = 0x7fffffff;
constexpr int kTraversalCap = 1 << 20;

// ------------------------------------------------------------- spec arithmetic
struct S3 { float x, y, z; };
__device__ __forceinline__ S3 s3(float x, float y, float z) { return S3{x, y, z}; }
__device__ __forceinline__ float sadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ssub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float smul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float sdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ S3 ssub3(S3 a, S3 b) { return s3(ssub(a.x, b.x), ssub(a.y, b.y), ssub(a.z, b.z)); }
__device__ __forceinline__ float sdot(S3 a, S3 b) {
    return sadd(sadd(smul(a.x, b.x), smul(a.y, b.y)), smul(a.z, b.z));
}
__device__ __forceinline__ S3 scross(S3 a, S3 b) {
    return s3(ssub(smul(a.y, b.z), smul(a.z, b.y)), ssub(smul(a.z, b.x), smul(a.x, b.z)),
              ssub(smul(a.x, b.y), smul(a.y, b.x)));
}
__device__ __forceinline__ float scomp(S3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// sin(2 pi s), cos(2 pi s) for s in [0, 1): exact quadrant reduction, Taylor polynomials
// of degree 9 / 10 in Horner form on |a| <= pi/4 (coefficients 1/n! rounded to float).
__device__ __forceinline__ void sincos2pi(float s, float* sn, float* cs) {
    int q = __float2int_rn(smul(s, 4.0f));
    float r = ssub(s, smul((float)q, 0.25f));
    float a = smul(r, 0x1.921fb6p+2f);
    float a2 = smul(a, a);
    float ps = 0x1.71de3ap-19f;
    ps = ssub(smul(ps, a2), 0x1.a01a02p-13f);
    ps = sadd(smul(ps, a2), 0x1.111112p-7f);
    ps = ssub(smul(ps, a2), 0x1.555556p-3f);
    float sa = sadd(a, smul(smul(a, a2), ps));
    float pc = -0x1.27e4fcp-22f;
    pc = sadd(smul(pc, a2), 0x1.a01a02p-16f);
    pc = ssub(smul(pc, a2), 0x1.6c16c2p-10f);
    pc = sadd(smul(pc, a2), 0x1.555556p-5f);
    pc = ssub(smul(pc, a2), 0.5f);
    float ca = sadd(1.0f, smul(a2, pc));
    switch (q & 3) {
        case 0: *sn = sa; *cs = ca; break;
        case 1: *sn = ca; *cs = -sa; break;
        case 2: *sn = -sa; *cs = -ca; break;
        default: *sn = -ca; *cs = sa; break;
    }
}

// ------------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC 2011).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__device__ __forceinline__ float unit24(uint32_t h) { return smul(__uint2float_rn(h >> 8), 0x1p-24f); }
// floor((k * 2^32 + r) / n): stratum k of n as a 32-bit fraction.
__device__ __forceinline__ uint32_t stratified32(uint32_t k, uint32_t n, uint32_t r) {
    uint64_t num = ((uint64_t)k << 32) | (uint64_t)r;
    if ((n & (n - 1)) == 0) return (uint32_t)(num >> (31 - __clz(n)));
    return (uint32_t)(num / n);
}

// ------------------------------------------------------------------- rays (spec)
struct Ray {
    S3 o, d;
    int kx, ky, kz;
    float Sx, Sy, Sz;
    float3 inv;   // 1/d for the (padded, conservative) box test
    float3 oinv;  // -o/d
    int nx, ny, nz;  // 0 when the near plane of that axis is the box's lo, 3 when it is hi
};

// 32-byte read-only load (a 256-bit vector load, sm_100 and later): two float4 from a 32-byte
// aligned address in one instruction.
__device__ __forceinline__ void ldg32(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// 3-input minimum / maximum (PTX min.f32 / max.f32 with three operands; a NaN operand is
// ignored, which keeps the box test conservative for axis-parallel rays).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ Ray make_ray(S3 o, S3 d) {
    Ray r;
    r.o = o; r.d = d;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = ax >= ay ? (ax >= az ? 0 : 2) : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dz = scomp(d, kz);
    if (dz < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = sdiv(scomp(d, kx), dz);
    r.Sy = sdiv(scomp(d, ky), dz);
    r.Sz = sdiv(1.0f, dz);
    r.inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    r.oinv = make_float3(-o.x * r.inv.x, -o.y * r.inv.y, -o.z * r.inv.z);
    r.nx = r.inv.x >= 0.0f ? 0 : 3;
    r.ny = r.inv.y >= 0.0f ? 0 : 3;
    r.nz = r.inv.z >= 0.0f ? 0 : 3;
    return r;
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013).  True on a hit with
// t = T/det > 0; det > 0 when the face's counter-clockwise side faces the ray origin.
__device__ __forceinline__ bool woop(const Ray& r, S3 p0, S3 p1, S3 p2, float* Tout, float* detout) {
    S3 A = ssub3(p0, r.o), B = ssub3(p1, r.o), C = ssub3(p2, r.o);
    float Akz = scomp(A, r.kz), Bkz = scomp(B, r.kz), Ckz = scomp(C, r.kz);
    float Ax = ssub(scomp(A, r.kx), smul(r.Sx, Akz)), Ay = ssub(scomp(A, r.ky), smul(r.Sy, Akz));
    float Bx = ssub(scomp(B, r.kx), smul(r.Sx, Bkz)), By = ssub(scomp(B, r.ky), smul(r.Sy, Bkz));
    float Cx = ssub(scomp(C, r.kx), smul(r.Sx, Ckz)), Cy = ssub(scomp(C, r.ky), smul(r.Sy, Ckz));
    float U = ssub(smul(Cx, By), smul(Cy, Bx));
    float V = ssub(smul(Ax, Cy), smul(Ay, Cx));
    float W = ssub(smul(Bx, Ay), smul(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = __double2float_rn(__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx)));
        V = __double2float_rn(__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx)));
        W = __double2float_rn(__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax)));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    float det = sadd(sadd(U, V), W);
    if (det == 0.0f) return false;
    float Az = smul(r.Sz, Akz), Bz = smul(r.Sz, Bkz), Cz = smul(r.Sz, Ckz);
    float T = sadd(sadd(smul(U, Az), smul(V, Bz)), smul(W, Cz));
    if (!((det > 0.0f && T > 0.0f) || (det < 0.0f && T < 0.0f))) return false;
    *Tout = T;
    *detout = det;
    return true;
}

// Moller-Trumbore barycentrics of o + t d on (p0, p1, p2); x = (b0 p0 + b1 p1) + b2 p2;
// unit geometric normal of the face.
__device__ __forceinline__ void surface_point(S3 o, S3 d, S3 p0, S3 p1, S3 p2, S3* x, S3* ng, float b[3]) {
    S3 e1 = ssub3(p1, p0), e2 = ssub3(p2, p0);
    S3 pv = scross(d, e2);
    float det = sdot(e1, pv);
    float inv = sdiv(1.0f, det);
    S3 s = ssub3(o, p0);
    float b1 = smul(sdot(s, pv), inv);
    S3 qv = scross(s, e1);
    float b2 = smul(sdot(d, qv), inv);
    float b0 = ssub(ssub(1.0f, b1), b2);
    b[0] = b0; b[1] = b1; b[2] = b2;
    *x = s3(sadd(sadd(smul(b0, p0.x), smul(b1, p1.x)), smul(b2, p2.x)),
            sadd(sadd(smul(b0, p0.y), smul(b1, p1.y)), smul(b2, p2.y)),
            sadd(sadd(smul(b0, p0.z), smul(b1, p1.z)), smul(b2, p2.z)));
    S3 c = scross(e1, e2);
    float len = __fsqrt_rn(sdot(c, c));
    *ng = s3(sdiv(c.x, len), sdiv(c.y, len), sdiv(c.z, len));
}

__device__ __forceinline__ S3 offset_origin(S3 x, S3 ng) {
    const float eps = 0x1.a36e2ep-14f;  // 1e-4 scene units
    return s3(sadd(x.x, smul(eps, ng.x)), sadd(x.y, smul(eps, ng.y)), sadd(x.z, smul(eps, ng.z)));
}

struct Cam {  // mirrors exm_camera
    float eye[3], right[3], up[3], fwd[3];
    float kx, ky, cx, cy, near_plane;
    float pad[3];
};

__device__ __forceinline__ void camera_ray(const Cam& c, int px, int py, S3* o, S3* d) {
    float dx = sdiv(ssub(sadd((float)px, 0.5f), c.cx), c.kx);
    float dy = sdiv(ssub(c.cy, sadd((float)py, 0.5f)), c.ky);
    *o = s3(c.eye[0], c.eye[1], c.eye[2]);
    *d = s3(sadd(sadd(c.fwd[0], smul(dx, c.right[0])), smul(dy, c.up[0])),
            sadd(sadd(c.fwd[1], smul(dx, c.right[1])), smul(dy, c.up[1])),
            sadd(sadd(c.fwd[2], smul(dx, c.right[2])), smul(dy, c.up[2])));
}

// Orthonormal basis about n (Duff et al., JCGT 2017) and a cosine-weighted direction.
__device__ __forceinline__ S3 cosine_dir(S3 n, float xi1, float xi2) {
    float sign = copysignf(1.0f, n.z);
    float a = sdiv(-1.0f, sadd(sign, n.z));
    float b = smul(smul(n.x, n.y), a);
    S3 t = s3(sadd(1.0f, smul(smul(smul(sign, n.x), n.x), a)), smul(sign, b), -smul(sign, n.x));
    S3 bb = s3(b, sadd(sign, smul(smul(n.y, n.y), a)), -n.y);
    float r = __fsqrt_rn(xi1);
    float sp, cp;
    sincos2pi(xi2, &sp, &cp);
    float lx = smul(r, cp), ly = smul(r, sp), lz = __fsqrt_rn(ssub(1.0f, xi1));
    return s3(sadd(sadd(smul(t.x, lx), smul(bb.x, ly)), smul(n.x, lz)),
              sadd(sadd(smul(t.y, lx), smul(bb.y, ly)), smul(n.y, lz)),
              sadd(sadd(smul(t.z, lx), smul(bb.z, ly)), smul(n.z, lz)));
}

// Light direction of texel (i, j) = (row, column) jittered by (xu, xv); also sin(theta).
__device__ __forceinline__ S3 light_dir(int i, int j, int W, int H, float xu, float xv, float* sin_theta) {
    float fv = sdiv(sadd((float)i, xv), (float)H);
    float fu = sdiv(sadd((float)j, xu), (float)W);
    float st, ct, sp, cp;
    sincos2pi(smul(fv, 0.5f), &st, &ct);
    sincos2pi(fu, &sp, &cp);
    *sin_theta = st;
    return s3(smul(st, sp), ct, -smul(st, cp));
}

// ------------------------------------------------------------ environment sampling
struct EnvView {
    const float4* texel;     // [H*W]: E.rgb, (q/Q) * W*H / (2 pi^2)
    const uint64_t* cdf;     // [H*W] inclusive prefix of the integer weights (row-major)
    const uint32_t* rguide;  // [Gr+1]: row picked at U1 = g * 2^(32-rbits)
    const uint32_t* cguide;  // [H*(Gc+1)]: column picked in row i at U2 = g * 2^(32-cbits)
    const uint64_t* Qp;      // total of the integer weights (device)
    const uint64_t* rowpre;  // [H] exclusive prefix of the row sums
    const uint64_t* rowsum;  // [H] row sums
    uint64_t Q;              // loaded from Qp once per thread
    int W, H;
    int rbits, cbits;
    // the row phase of a texel pick from shared memory, when a kernel staged it there
    // (env_rows_to_shared): the CDF at each row's end and the row guide; null: from global memory
    const uint64_t* srowend;
    const uint32_t* srguide;
};

// Bytes of shared memory env_rows_to_shared needs, or 0 when they exceed `limit` (the search then
// reads global memory).
__host__ __device__ __forceinline__ size_t env_rows_shared_bytes(int H, int rbits, size_t limit) {
    const size_t b = (size_t)H * 8 + (((size_t)1 << rbits) + 1) * 4;
    return b <= limit ? b : 0;
}

// Stages the row phase of the texel search in shared memory `s` (env_rows_shared_bytes of them,
// 8-byte aligned): the inclusive CDF at the end of each row, rowpre + rowsum (the same integers
// as cdf[row W + W - 1]), then the row guide.  Every thread of the block calls it (it
// synchronises); afterwards pick_texel reads those values there.
__device__ __forceinline__ void env_rows_to_shared(EnvView& e, void* s) {
    uint64_t* rowend = reinterpret_cast<uint64_t*>(s);
    uint32_t* guide = reinterpret_cast<uint32_t*>(rowend + e.H);
    for (int t = threadIdx.x; t < e.H; t += blockDim.x) rowend[t] = __ldg(e.rowpre + t) + __ldg(e.rowsum + t);
    const int G = (1 << e.rbits) + 1;
    for (int t = threadIdx.x; t < G; t += blockDim.x) guide[t] = __ldg(e.rguide + t);
    __syncthreads();
    e.srowend = rowend;
    e.srguide = guide;
}

// The CDF at the end of row r and the row guide entry g: from shared memory when the kernel
// staged them (SR), else from global memory.
template <bool SR>
__device__ __forceinline__ uint64_t env_rowend(const EnvView& e, uint32_t r) {
    if constexpr (SR) return e.srowend[r];
    else return __ldg(e.cdf + (size_t)r * e.W + e.W - 1);
}
template <bool SR>
__device__ __forceinline__ uint32_t env_rguide(const EnvView& e, uint32_t g) {
    if constexpr (SR) return e.srguide[g];
    else return __ldg(e.rguide + g);
}

__device__ __forceinline__ uint64_t scaled_target(uint32_t U, uint64_t X) {
    return (uint64_t)U * (X >> 32) + (((uint64_t)U * (X & 0xffffffffull)) >> 32);
}

// 2D strata of n samples: ny = the largest divisor of n not above sqrt(n), nx = n / ny.
__host__ __device__ __forceinline__ void strata2(uint32_t n, uint32_t* nx, uint32_t* ny) {
    uint32_t best = 1;
    for (uint32_t d = 1; d * d <= n; ++d)
        if (n % d == 0) best = d;
    *ny = best;
    *nx = n / best;
}

// Texel chosen by the row fraction U1 and column fraction U2: the row is the smallest i
// whose inclusive row prefix exceeds floor(U1 Q / 2^32); the column the smallest j of row i
// whose in-row prefix exceeds floor(U2 rowsum_i / 2^32) (guide tables bound both searches).
template <bool SR = false>
__device__ __forceinline__ void pick_texel(const EnvView& e, uint32_t U1, uint32_t U2, uint32_t* row_out,
                                           uint32_t* col_out) {
    const uint64_t tr = scaled_target(U1, e.Q);
    const uint32_t g = U1 >> (32 - e.rbits);
    uint32_t lo = env_rguide<SR>(e, g), hi = env_rguide<SR>(e, g + 1);
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (env_rowend<SR>(e, mid) > tr) hi = mid; else lo = mid + 1;
    }
    const uint32_t row = lo;
    const uint64_t* rc = e.cdf + (size_t)row * e.W;
    const uint64_t pre = row ? env_rowend<SR>(e, row - 1) : 0ull;
    const uint64_t tc = pre + scaled_target(U2, env_rowend<SR>(e, row) - pre);
    const uint32_t* cg = e.cguide + (size_t)row * ((1u << e.cbits) + 1);
    const uint32_t g2 = U2 >> (32 - e.cbits);
    lo = __ldg(cg + g2);
    hi = __ldg(cg + g2 + 1);
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(rc + mid) > tc) hi = mid; else lo = mid + 1;
    }
    *row_out = row;
    *col_out = lo;
}

// Two texel picks in lockstep: the same arithmetic as pick_texel for each, with the loads of
// both searches issued together so that their latencies overlap.
template <bool SR = false>
__device__ __forceinline__ void pick_texel2(const EnvView& e, uint32_t U1a, uint32_t U2a, uint32_t U1b,
                                            uint32_t U2b, uint32_t* ra, uint32_t* ca, uint32_t* rb,
                                            uint32_t* cb) {
    const uint64_t tra = scaled_target(U1a, e.Q), trb = scaled_target(U1b, e.Q);
    const uint32_t ga = U1a >> (32 - e.rbits), gb = U1b >> (32 - e.rbits);
    uint32_t loa = env_rguide<SR>(e, ga), hia = env_rguide<SR>(e, ga + 1);
    uint32_t lob = env_rguide<SR>(e, gb), hib = env_rguide<SR>(e, gb + 1);
    while (loa < hia || lob < hib) {
        const bool aa = loa < hia, ab = lob < hib;
        const uint32_t ma = loa + ((hia - loa) >> 1), mb = lob + ((hib - lob) >> 1);
        const uint64_t va = aa ? env_rowend<SR>(e, ma) : 0ull;
        const uint64_t vb = ab ? env_rowend<SR>(e, mb) : 0ull;
        if (aa) { if (va > tra) hia = ma; else loa = ma + 1; }
        if (ab) { if (vb > trb) hib = mb; else lob = mb + 1; }
    }
    const uint32_t rowa = loa, rowb = lob;
    const uint64_t* rca = e.cdf + (size_t)rowa * e.W;
    const uint64_t* rcb = e.cdf + (size_t)rowb * e.W;
    const uint64_t prea = rowa ? env_rowend<SR>(e, rowa - 1) : 0ull, preb = rowb ? env_rowend<SR>(e, rowb - 1) : 0ull;
    const uint64_t enda = env_rowend<SR>(e, rowa), endb = env_rowend<SR>(e, rowb);
    const uint64_t tca = prea + scaled_target(U2a, enda - prea), tcb = preb + scaled_target(U2b, endb - preb);
    const uint32_t stride = (1u << e.cbits) + 1;
    const uint32_t g2a = U2a >> (32 - e.cbits), g2b = U2b >> (32 - e.cbits);
    loa = __ldg(e.cguide + (size_t)rowa * stride + g2a);
    hia = __ldg(e.cguide + (size_t)rowa * stride + g2a + 1);
    lob = __ldg(e.cguide + (size_t)rowb * stride + g2b);
    hib = __ldg(e.cguide + (size_t)rowb * stride + g2b + 1);
    while (loa < hia || lob < hib) {
        const bool aa = loa < hia, ab = lob < hib;
        const uint32_t ma = loa + ((hia - loa) >> 1), mb = lob + ((hib - lob) >> 1);
        const uint64_t va = aa ? __ldg(rca + ma) : 0ull, vb = ab ? __ldg(rcb + mb) : 0ull;
        if (aa) { if (va > tca) hia = ma; else loa = ma + 1; }
        if (ab) { if (vb > tcb) hib = mb; else lob = mb + 1; }
    }
    *ra = rowa; *ca = loa; *rb = rowb; *cb = lob;
}

struct LightSample {
    S3 dir;        // unnormalised spec direction
    float inv_pdf; // 1 / p_omega
    float3 E;      // environment radiance of the texel
    uint32_t texel;
};

// Light sample k of n = nx * ny (strata2): 2D-stratified, row stratum k / nx and column
// stratum k % nx.
__device__ __forceinline__ void strata_of(uint32_t k, uint32_t nx, uint32_t* kx, uint32_t* ky) {
    if ((nx & (nx - 1)) == 0) {  // the strata of power-of-two sample counts: no integer division
        *kx = k & (nx - 1);
        *ky = k >> (31 - __clz(nx));
    } else {
        *kx = k % nx;
        *ky = k / nx;
    }
}

__device__ __forceinline__ void finish_sample(const EnvView& e, uint4 h, uint32_t i, uint32_t j, LightSample* s) {
    const uint32_t t = i * (uint32_t)e.W + j;
    float st;
    s->dir = light_dir((int)i, (int)j, e.W, e.H, unit24(h.y), unit24(h.z), &st);
    const float4 tx = __ldg(e.texel + t);
    s->E = make_float3(tx.x, tx.y, tx.z);
    s->inv_pdf = __fdividef(st, tx.w);  // an estimator weight, not a decision
    s->texel = t;
}

template <bool SR = false>
__device__ __forceinline__ LightSample light_sample(const EnvView& e, uint4 h, uint32_t k, uint32_t nx, uint32_t ny) {
    LightSample s;
    uint32_t kx, ky, i, j;
    strata_of(k, nx, &kx, &ky);
    pick_texel<SR>(e, stratified32(ky, ny, h.x), stratified32(kx, nx, h.w), &i, &j);
    finish_sample(e, h, i, j, &s);
    return s;
}

// Light samples ka and kb together (pick_texel2): each equal to light_sample's.
template <bool SR = false>
__device__ __forceinline__ void light_sample2(const EnvView& e, uint4 ha, uint32_t ka, uint4 hb, uint32_t kb,
                                              uint32_t nx, uint32_t ny, LightSample* sa, LightSample* sb) {
    uint32_t kxa, kya, kxb, kyb, ia, ja, ib, jb;
    strata_of(ka, nx, &kxa, &kya);
    strata_of(kb, nx, &kxb, &kyb);
    pick_texel2<SR>(e, stratified32(kya, ny, ha.x), stratified32(kxa, nx, ha.w), stratified32(kyb, ny, hb.x),
                stratified32(kxb, nx, hb.w), &ia, &ja, &ib, &jb);
    finish_sample(e, ha, ia, ja, sa);
    finish_sample(e, hb, ib, jb, sb);
}

// ----------------------------------------------------------------------- BVH
// 4-wide BVH, 128-byte nodes (8 float4): the four child boxes as lo.x[4] lo.y[4] lo.z[4]
// hi.x[4] hi.y[4] hi.z[4], then the four child references (>= 0: node, < 0: a leaf of one to
// kMaxLeafTris consecutive triangles in leaf order (encoding below), kEmptyChild: unused slot).  Triangles in leaf order, 64-byte
// records (p0 + original id bits in .w, p1, p2, padding).
//
// Bank skew.  The lanes of a warp read different nodes with the same load instruction.  Were
// chunk j (32 bytes) of every node at the same offset of its 128-byte line, every lane would
// address the same eight of the L1's 32 banks and the lanes would be served one per cycle.  So
// chunk j of node q is stored at chunk position j xor (q mod 4) of the node, and chunk j of
// triangle record k at position j xor (k/2 mod 2) of the record (records sit at offset 0 or 64
// of a line by the parity of k): over the lanes' nodes and records the reads spread across the
// four bank groups.  node4_at / tri_at give the float4 index of element v of a record; the
// traversal forms the same addresses by xor-ing the record's (128- or 64-byte aligned) address,
// one logic operation per chunk (chunk_at).
struct BvhView {
    const float4* tris;
    const float4* nodes4;
    const float4* sphere;  // bounding sphere of the triangles: centre, R^2
    const float4* nodes8;  // 8-wide compressed nodes (exm_bvh.cu), when the mesh uses them
    const float4* nodesq;  // 4-wide nodes with quantised boxes, when the mesh uses them
};
// 4-wide node with quantised child boxes (EXM_BVH_4Q), 64 bytes in two 32-byte chunks (skewed
// like the triangle records: chunk j of node q at position j xor (q/2 mod 2)):
//   chunk 0: p.x p.y p.z step.x | ref[4]
//   chunk 1: qlo.x qlo.y qlo.z qhi.x | qhi.y qhi.z step.y step.z
// The q words hold one byte per child (child c in byte c); child c's box on axis a is
// [p_a + qlo_c step_a, p_a + qhi_c step_a] with power-of-two steps.  An empty slot has qlo 255,
// qhi 0 and ref kEmptyChild.
constexpr int kNodeQ4 = 4;     // float4 per quantised 4-wide node
// A 4-wide leaf reference ~(k | (c - 1) << kLeafCountShift) names c consecutive triangle records
// from k (c = 1..kMaxLeafTris; k < 2^28).
constexpr int kLeafCountShift = 28;
constexpr int kMaxLeafTris = 4;
constexpr int kNode8 = 5;      // float4 per 8-wide compressed node
constexpr int kTri = 4;        // float4 per triangle record: the vertices (original id in the first .w), padding
constexpr int kStackSize8 = 64;  // node groups on the 8-wide traversal stack: one per level

__host__ __device__ __forceinline__ size_t node4_at(size_t q, unsigned v) {
    return 8 * q + 2 * ((v / 2) ^ ((unsigned)q & 3u)) + (v & 1u);
}
__host__ __device__ __forceinline__ size_t tri_at(size_t k, unsigned v) {
    return (size_t)kTri * k + 2 * ((v / 2) ^ ((unsigned)(k >> 1) & 1u)) + (v & 1u);
}
// float4 v (0..3) of quantised 4-wide node q (layout below): skewed like a triangle record.
__host__ __device__ __forceinline__ size_t nodeq_at(size_t q, unsigned v) {
    return 4 * q + 2 * ((v / 2) ^ ((unsigned)(q >> 1) & 1u)) + (v & 1u);
}
// The chunk at byte offset `x` (a multiple of 32 below the record's alignment) of an aligned
// record: no carry can occur, so the xor stays in the address's low word.
__device__ __forceinline__ const float4* chunk_at(const float4* rec, unsigned x) {
    return reinterpret_cast<const float4*>(reinterpret_cast<uintptr_t>(rec) ^ (uintptr_t)x);
}

// Ray parameter beyond which o + t d lies outside the bounding sphere `sp` (centre, R^2), where
// no triangle can be hit, plus a margin (0.1% relative and 1e-4 R absolute) far above the
// rounding of this computation; 0 when the ray does not meet the sphere ahead of its origin.
// A traversal clipped to it visits fewer boxes and reaches every triangle it would hit.
__device__ __forceinline__ float sphere_exit(S3 o, S3 d, float4 sp) {
    const float ox = o.x - sp.x, oy = o.y - sp.y, oz = o.z - sp.z;
    const float a = d.x * d.x + d.y * d.y + d.z * d.z;
    const float b = ox * d.x + oy * d.y + oz * d.z;
    const float c = ox * ox + oy * oy + oz * oz - sp.w;
    const float disc = b * b - a * c;
    if (!(disc > 0.0f) || !(a > 0.0f)) return 0.0f;
    const float t = (sqrtf(disc) - b) / a;
    return t > 0.0f ? t * 1.001f + 1e-4f * sqrtf(sp.w / a) : 0.0f;
}

__device__ __forceinline__ bool tri_test(const BvhView& b, int k, const Ray& r, float* T, float* det, int* id) {
    float4 a, c;
    const float4* rec = b.tris + kTri * (size_t)k;
    const unsigned x = ((unsigned)k & 2u) << 4;  // 32 when bit 1 of k is set
    ldg32(chunk_at(rec, x), a, c);
    const float4 d = __ldg(chunk_at(rec, x ^ 32u));
    *id = __float_as_int(a.w);
    return woop(r, s3(a.x, a.y, a.z), s3(c.x, c.y, c.z), s3(d.x, d.y, d.z), T, det);
}

// ----------------------------------------------------------------- map texels
template <typename T> struct MapLoad;
template <> struct MapLoad<float> {
    __device__ static __forceinline__ void load(const void* base, size_t texel, float v[8]) {
        const float4* p = reinterpret_cast<const float4*>(base) + 2 * texel;
        float4 a = __ldg(p), b = __ldg(p + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};
template <> struct MapLoad<__nv_bfloat16> {
    __device__ static __forceinline__ void load(const void* base, size_t texel, float v[8]) {
        uint4 a = __ldg(reinterpret_cast<const uint4*>(base) + texel);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
        for (int k = 0; k < 4; ++k) { float2 f = __bfloat1622float2(h[k]); v[2 * k] = f.x; v[2 * k + 1] = f.y; }
    }
};
template <> struct MapLoad<__half> {
    __device__ static __forceinline__ void load(const void* base, size_t texel, float v[8]) {
        uint4 a = __ldg(reinterpret_cast<const uint4*>(base) + texel);
        const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
        for (int k = 0; k < 4; ++k) { float2 f = __half22float2(h[k]); v[2 * k] = f.x; v[2 * k + 1] = f.y; }
    }
};

struct MapView {
    const void* data;
    int W, H;
    bool wrap_u;
};

// Bilinear footprint: 4 texel indices and weights, plus d(weights)/d(fs, ft) data.
struct Footprint {
    uint32_t t[4];
    float fs, ft;
};

__device__ __forceinline__ Footprint footprint(const MapView& m, float u, float v) {
    Footprint f;
    float s = u * (float)m.W - 0.5f, t = v * (float)m.H - 0.5f;
    float i0f = floorf(s), j0f = floorf(t);
    f.fs = s - i0f;
    f.ft = t - j0f;
    int i0 = (int)i0f, j0 = (int)j0f;
    int c0, c1;
    if (m.wrap_u) {
        c0 = i0 % m.W; if (c0 < 0) c0 += m.W;
        c1 = c0 + 1 == m.W ? 0 : c0 + 1;
    } else {
        c0 = min(max(i0, 0), m.W - 1);
        c1 = min(max(i0 + 1, 0), m.W - 1);
    }
    int r0 = min(max(j0, 0), m.H - 1), r1 = min(max(j0 + 1, 0), m.H - 1);
    f.t[0] = (uint32_t)r0 * m.W + c0;
    f.t[1] = (uint32_t)r0 * m.W + c1;
    f.t[2] = (uint32_t)r1 * m.W + c0;
    f.t[3] = (uint32_t)r1 * m.W + c1;
    return f;
}

// ------------------------------------------- float-float shading geometry (accuracy only)
// The barycentrics of a shading point must be accurate to ~1e-7 relative: narrow GGX lobes
// amplify their error ~50x into radiance.  In plain FP32 they are not -- the ray origin lies
// |o - p0| ~ 3 units from a triangle whose edges are ~0.004 units, and the triple products of
// Moller-Trumbore cancel ~1000-fold -- so they are evaluated in float-float ("double-word")
// arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, and the operations are the
// error-free transformations TwoSum (Knuth) and TwoProd (one FMA) composed as in Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 2017): relative errors of a few 2^-48.  No decision
// depends on these values.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff(float a) { return FF{a, 0.0f}; }
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {  // exponent of a >= exponent of b
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return FF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
// sum of two double-words (the accurate algorithm, relative error <= 3 u^2)
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.hi, b.hi);
    const FF t = ff_two_sum(a.lo, b.lo);
    const FF v = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return ff_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }
// product of two double-words (relative error <= 5 u^2)
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const FF c = ff_two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
    return ff_fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}
// double-word times float (relative error <= 2 u^2)
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
    const FF c = ff_two_prod(a.hi, b);
    return ff_fast_two_sum(c.hi, __fmaf_rn(a.lo, b, c.lo));
}
// quotient of two double-words (one correction of the float quotient)
__device__ __forceinline__ FF ff_div(FF a, FF b) {
    const float th = __fdiv_rn(a.hi, b.hi);
    const FF r = ff_mul_f(b, th);
    const float d = __fadd_rn(__fsub_rn(a.hi, r.hi), __fsub_rn(a.lo, r.lo));
    return ff_fast_two_sum(th, __fdiv_rn(d, b.hi));
}
__device__ __forceinline__ float ff_f(FF a) { return __fadd_rn(a.hi, a.lo); }

struct FF3 { FF x, y, z; };
__device__ __forceinline__ FF3 ff3_sub(float3 a, float3 b) {  // exact
    return FF3{ff_two_sum(a.x, -b.x), ff_two_sum(a.y, -b.y), ff_two_sum(a.z, -b.z)};
}
__device__ __forceinline__ FF3 ff3_cross(FF3 a, FF3 b) {
    return FF3{ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)), ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
               ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
__device__ __forceinline__ FF ff3_dot(FF3 a, FF3 b) {
    return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}

// Moller-Trumbore barycentrics of the ray o + t d on (p0, p1, p2): b1 = (s . (d x e2)) / det,
// b2 = (d . (s x e1)) / det with s = o - p0, e1 = p1 - p0, e2 = p2 - p0, det = e1 . (d x e2);
// b0 = 1 - b1 - b2.  The differences of float inputs are exact double-words.
__device__ __forceinline__ void bary_ff(FF3 s, FF3 d, float3 p0, float3 p1, float3 p2, FF b[3]) {
    const FF3 e1 = ff3_sub(p1, p0), e2 = ff3_sub(p2, p0);
    const FF3 pv = ff3_cross(d, e2);
    const FF det = ff3_dot(e1, pv);
    b[1] = ff_div(ff3_dot(s, pv), det);
    b[2] = ff_div(ff3_dot(d, ff3_cross(s, e1)), det);
    b[0] = ff_sub(ff_sub(ff(1.0f), b[1]), b[2]);
}

// Texel-space coordinate (b0 c0 + b1 c1 + b2 c2) * n - 1/2 of a UV component c at double-word
// barycentrics, split into floor and fraction (the fraction to ~1e-7 of a texel on 4096^2
// maps, where a float coordinate would keep only 5e-4).
__device__ __forceinline__ void texel_coord(const FF b[3], float c0, float c1, float c2, int n, int* i0, float* frac) {
    FF x = ff_add(ff_add(ff_mul_f(b[0], c0), ff_mul_f(b[1], c1)), ff_mul_f(b[2], c2));
    x = ff_add(ff_mul_f(x, (float)n), ff(-0.5f));
    float fl = floorf(x.hi);
    float fr = __fadd_rn(__fsub_rn(x.hi, fl), x.lo);  // x.hi - fl is exact
    if (fr < 0.0f) {  // x.hi an integer and x.lo < 0
        fl = __fsub_rn(fl, 1.0f);
        fr = __fadd_rn(fr, 1.0f);
    }
    if (fr >= 1.0f) {
        fl = __fadd_rn(fl, 1.0f);
        fr = 0.0f;
    }
    *i0 = (int)fmaxf(fminf(fl, 1e9f), -1e9f);
    *frac = fr;
}

template <typename T>
__device__ __forceinline__ void fetch8(const MapView& m, const Footprint& f, float out[8], float dfs[8], float dft[8]) {
    float a[8], b[8], c[8], d[8];
    MapLoad<T>::load(m.data, f.t[0], a);
    MapLoad<T>::load(m.data, f.t[1], b);
    MapLoad<T>::load(m.data, f.t[2], c);
    MapLoad<T>::load(m.data, f.t[3], d);
    float w0 = (1.f - f.fs) * (1.f - f.ft), w1 = f.fs * (1.f - f.ft), w2 = (1.f - f.fs) * f.ft, w3 = f.fs * f.ft;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        out[k] = w0 * a[k] + w1 * b[k] + w2 * c[k] + w3 * d[k];
        if (dfs) {
            dfs[k] = (1.f - f.ft) * (b[k] - a[k]) + f.ft * (d[k] - c[k]);
            dft[k] = (1.f - f.fs) * (c[k] - a[k]) + f.fs * (d[k] - b[k]);
        }
    }
}

// Bilinear footprint from an integer texel position and its fractions (wrap / clamp rules of
// footprint_d).
__device__ __forceinline__ Footprint footprint_i(const MapView& m, int i0, int j0, float fs, float ft) {
    Footprint f;
    f.fs = fs;
    f.ft = ft;
    int c0, c1;
    if (m.wrap_u) {
        c0 = i0 % m.W;
        if (c0 < 0) c0 += m.W;
        c1 = c0 + 1 == m.W ? 0 : c0 + 1;
    } else {
        c0 = min(max(i0, 0), m.W - 1);
        c1 = min(max(i0 + 1, 0), m.W - 1);
    }
    const int r0 = min(max(j0, 0), m.H - 1), r1 = min(max(j0 + 1, 0), m.H - 1);
    f.t[0] = (uint32_t)r0 * m.W + c0;
    f.t[1] = (uint32_t)r0 * m.W + c1;
    f.t[2] = (uint32_t)r1 * m.W + c0;
    f.t[3] = (uint32_t)r1 * m.W + c1;
    return f;
}

// Adds the 8-channel gradient g to the four texels of a footprint, bilinearly weighted.
__device__ __forceinline__ void scatter8(float* gmaps, const Footprint& fp, const float g[8]) {
    float w[4] = {(1.f - fp.fs) * (1.f - fp.ft), fp.fs * (1.f - fp.ft), (1.f - fp.fs) * fp.ft, fp.fs * fp.ft};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4* p = reinterpret_cast<float4*>(gmaps) + 2 * (size_t)fp.t[k];
        atomicAdd(p, make_float4(w[k] * g[0], w[k] * g[1], w[k] * g[2], w[k] * g[3]));
        atomicAdd(p + 1, make_float4(w[k] * g[4], w[k] * g[5], w[k] * g[6], w[k] * g[7]));
    }
}

// ------------------------------------------------------------------ small vectors
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ float3 tof(S3 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 ld3(const float* p) { return f3(__ldg(p), __ldg(p + 1), __ldg(p + 2)); }

}  // namespace exm
