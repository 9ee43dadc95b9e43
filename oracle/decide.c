/*
 * Oracle, part 1: the discrete decisions of the Stage-II renderer, brute force, on the CPU.
 *
 * TEST INFRASTRUCTURE.  This file is the checker, not the product: only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header or table with the CUDA library.
 *
 * The renderer of Sec. 5 makes four kinds of discrete decision: which triangle a pixel
 * sees (primary visibility, Sec. 5.1), which environment texel a light sample picks
 * (importance sampling by brightness x spherical area, Sec. 5.2), whether a shadow ray
 * is blocked (Vis of Eq. 12 / Eq. 17 / Eq. 18) and which front-facing triangle a
 * secondary ray hits (Sec. 5.3).  Each is decided here exactly as the specification
 * written for this project fixes it:
 *
 *   - primary visibility: 8-subpixel-bit fixed-point edge functions, top-left fill
 *     rule, back faces culled, depth interpolated in integers, nearest depth wins and
 *     equal depths go to the lower triangle id;
 *   - texel choice: integer importance weights, exact 64-bit prefix sums, stratified
 *     32-bit targets from a counter-based generator (Philox4x32-10, Salmon et al. 2011);
 *   - rays: built by a fixed FP32 operation sequence and tested against every triangle
 *     with the watertight ray/triangle test of Woop, Benthin and Wald (JCGT 2013).
 *
 * Every floating-point step that feeds a decision is single precision with one rounding
 * per operation (this file is compiled with -ffp-contract=off), so the decision is the
 * one the FP32 specification defines.  Radiance itself is evaluated in FP64 elsewhere
 * (oracle/shade.py); nothing here is accelerated: every ray is tested against every
 * triangle and every pixel against every triangle.
 */
#pragma STDC FP_CONTRACT OFF
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_GUARDBAND (-4)

/* ------------------------------------------------------------------ Philox4x32-10 */
/* Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC 2011): ten rounds of two 32x32->64 multiplications, with
 * a Weyl-sequence key schedule. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* A 24-bit uniform in [0,1): exact in FP32 and FP64. */
static float unit24(uint32_t h) { return (float)(h >> 8) * 0x1p-24f; }

/* Stratum k of n, jittered by the 32-bit word r: floor((k * 2^32 + r) / n), a 32-bit
 * fixed-point fraction in [k/n, (k+1)/n). */
static uint32_t stratified32(uint32_t k, uint32_t n, uint32_t r) {
    uint64_t num = ((uint64_t)k << 32) | (uint64_t)r;
    return (uint32_t)(num / (uint64_t)n);
}

/* --------------------------------------------------------------- FP32 sin / cos */
/* sin(2 pi s), cos(2 pi s) for s in [0, 1): quadrant reduction (exact), then Taylor
 * polynomials of degree 9 (sin) and 10 (cos) on |a| <= pi/4. */
void orc_sincos2pi(float s, float* sn, float* cs) {
    int q = (int)rintf(s * 4.0f);
    float r = s - (float)q * 0.25f;
    float a = r * 0x1.921fb6p+2f;
    float a2 = a * a;
    float ps = 0x1.71de3ap-19f;           /* 1/9! */
    ps = ps * a2 - 0x1.a01a02p-13f;       /* 1/7! */
    ps = ps * a2 + 0x1.111112p-7f;        /* 1/5! */
    ps = ps * a2 - 0x1.555556p-3f;        /* 1/3! */
    float sa = a + (a * a2) * ps;
    float pc = -0x1.27e4fcp-22f;          /* 1/10! */
    pc = pc * a2 + 0x1.a01a02p-16f;       /* 1/8! */
    pc = pc * a2 - 0x1.6c16c2p-10f;       /* 1/6! */
    pc = pc * a2 + 0x1.555556p-5f;        /* 1/4! */
    pc = pc * a2 - 0.5f;                  /* 1/2! */
    float ca = 1.0f + a2 * pc;
    switch (q & 3) {
        case 0: *sn = sa; *cs = ca; break;
        case 1: *sn = ca; *cs = -sa; break;
        case 2: *sn = -sa; *cs = -ca; break;
        default: *sn = -ca; *cs = sa; break;
    }
}

void orc_sincos2pi_many(const float* s, int n, float* sn, float* cs) {
    for (int i = 0; i < n; ++i) orc_sincos2pi(s[i], &sn[i], &cs[i]);
}

/* ------------------------------------------------------------------- FP32 vectors */
typedef struct { float x, y, z; } f3;
static f3 mk(float x, float y, float z) { f3 r = {x, y, z}; return r; }
static f3 ld3(const float* p) { return mk(p[0], p[1], p[2]); }
static f3 sub3(f3 a, f3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static float dot3(f3 a, f3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static f3 cross3(f3 a, f3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static float comp(f3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ----------------------------------------------------------- vertex snap (per view) */
/* Camera record: eye(3) right(3) up(3) fwd(3) kx ky cx cy near pad(3). */
int orc_snap(const float* V, int nv, const float* cam, int32_t* XY, uint32_t* Zq) {
    f3 eye = ld3(cam), rt = ld3(cam + 3), up = ld3(cam + 6), fw = ld3(cam + 9);
    float kx = cam[12], ky = cam[13], cx = cam[14], cy = cam[15], nearp = cam[16];
    int status = ORC_OK;
    for (int v = 0; v < nv; ++v) {
        f3 d = sub3(ld3(V + 3 * v), eye);
        float xc = dot3(d, rt), yc = dot3(d, up), w = dot3(d, fw);
        if (!(w >= nearp)) { status = ORC_ERR_GUARDBAND; XY[2 * v] = XY[2 * v + 1] = 0; Zq[v] = 0; continue; }
        float sx = cx + kx * (xc / w);
        float sy = cy - ky * (yc / w);
        if (!(fabsf(sx) < 16384.0f && fabsf(sy) < 16384.0f)) {
            status = ORC_ERR_GUARDBAND; XY[2 * v] = XY[2 * v + 1] = 0; Zq[v] = 0; continue;
        }
        XY[2 * v] = (int32_t)rintf(sx * 256.0f);
        XY[2 * v + 1] = (int32_t)rintf(sy * 256.0f);
        float z = 1.0f - nearp / w;
        if (z < 0.0f) z = 0.0f;
        if (z > 1.0f) z = 1.0f;
        Zq[v] = (uint32_t)rintf(z * 16777215.0f);
    }
    return status;
}

/* --------------------------------------------------------------------- raster */
/* Inside test of one pixel centre against one triangle (vertices already oriented so
 * that a visible face has a positive doubled area).  Returns 1 and the interpolated
 * integer depth when the centre is covered under the top-left rule. */
static int edge_incl(int64_t dx, int64_t dy) { return dy > 0 || (dy == 0 && dx < 0); }

static int cover(int64_t X0, int64_t Y0, int64_t X1, int64_t Y1, int64_t X2, int64_t Y2,
                 uint32_t Z0, uint32_t Z1, uint32_t Z2, int64_t Px, int64_t Py,
                 int64_t A2, uint32_t* depth) {
    int64_t E0 = (Y1 - Py) * (X2 - Px) - (X1 - Px) * (Y2 - Py);
    int64_t E1 = (Y2 - Py) * (X0 - Px) - (X2 - Px) * (Y0 - Py);
    int64_t E2 = (Y0 - Py) * (X1 - Px) - (X0 - Px) * (Y1 - Py);
    if (!(E0 > 0 || (E0 == 0 && edge_incl(X2 - X1, Y2 - Y1)))) return 0;
    if (!(E1 > 0 || (E1 == 0 && edge_incl(X0 - X2, Y0 - Y2)))) return 0;
    if (!(E2 > 0 || (E2 == 0 && edge_incl(X1 - X0, Y1 - Y0)))) return 0;
    int64_t num = E0 * (int64_t)Z0 + E1 * (int64_t)Z1 + E2 * (int64_t)Z2;
    *depth = (uint32_t)(num / A2);
    return 1;
}

static int64_t area2(int64_t X0, int64_t Y0, int64_t X1, int64_t Y1, int64_t X2, int64_t Y2) {
    return (Y1 - Y0) * (X2 - X0) - (X1 - X0) * (Y2 - Y0);
}

#define A2_LIMIT (((int64_t)1) << 38)

/* Per-pixel brute force over every triangle.  pix: npix triples (view, py, px);
 * keys: one (depth << 32 | tri) per listed pixel, all ones where nothing is visible. */
int orc_raster_pixels(const float* V, int nv, const int32_t* F, int nf, const float* cams,
                      int views, int W, int H, const int32_t* pix, int npix, uint64_t* keys) {
    int32_t* XY = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)nv * views);
    uint32_t* Zq = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nv * views);
    int status = ORC_OK;
    for (int c = 0; c < views; ++c)
        if (orc_snap(V, nv, cams + 20 * c, XY + 2 * (size_t)nv * c, Zq + (size_t)nv * c) != ORC_OK)
            status = ORC_ERR_GUARDBAND;
    int guard = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : guard)
    for (int p = 0; p < npix; ++p) {
        int c = pix[3 * p], py = pix[3 * p + 1], px = pix[3 * p + 2];
        const int32_t* xy = XY + 2 * (size_t)nv * c;
        const uint32_t* zq = Zq + (size_t)nv * c;
        int64_t Px = (int64_t)px * 256 + 128, Py = (int64_t)py * 256 + 128;
        uint64_t best = ~(uint64_t)0;
        (void)W; (void)H;
        for (int f = 0; f < nf; ++f) {
            int a = F[3 * f], b = F[3 * f + 1], d = F[3 * f + 2];
            int64_t X0 = xy[2 * a], Y0 = xy[2 * a + 1], X1 = xy[2 * b], Y1 = xy[2 * b + 1];
            int64_t X2 = xy[2 * d], Y2 = xy[2 * d + 1];
            int64_t A2 = area2(X0, Y0, X1, Y1, X2, Y2);
            if (A2 <= 0) continue;
            if (A2 >= A2_LIMIT) { guard = 1; continue; }
            uint32_t z;
            if (cover(X0, Y0, X1, Y1, X2, Y2, zq[a], zq[b], zq[d], Px, Py, A2, &z)) {
                uint64_t key = ((uint64_t)z << 32) | (uint32_t)f;
                if (key < best) best = key;
            }
        }
        keys[p] = best;
    }
    free(XY);
    free(Zq);
    if (guard) status = ORC_ERR_GUARDBAND;
    return status;
}

/* Triangle-major form of the same definition: every front face visits the pixel
 * centres of its bounding box.  keys: [views, H, W]. */
int orc_raster_full(const float* V, int nv, const int32_t* F, int nf, const float* cams,
                    int views, int W, int H, uint64_t* keys) {
    int32_t* XY = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)nv);
    uint32_t* Zq = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nv);
    int status = ORC_OK;
    memset(keys, 0xff, sizeof(uint64_t) * (size_t)views * W * H);
    for (int c = 0; c < views; ++c) {
        if (orc_snap(V, nv, cams + 20 * c, XY, Zq) != ORC_OK) status = ORC_ERR_GUARDBAND;
        uint64_t* kv = keys + (size_t)c * W * H;
        for (int f = 0; f < nf; ++f) {
            int a = F[3 * f], b = F[3 * f + 1], d = F[3 * f + 2];
            int64_t X0 = XY[2 * a], Y0 = XY[2 * a + 1], X1 = XY[2 * b], Y1 = XY[2 * b + 1];
            int64_t X2 = XY[2 * d], Y2 = XY[2 * d + 1];
            int64_t A2 = area2(X0, Y0, X1, Y1, X2, Y2);
            if (A2 <= 0) continue;
            if (A2 >= A2_LIMIT) { status = ORC_ERR_GUARDBAND; continue; }
            int64_t mnx = X0 < X1 ? (X0 < X2 ? X0 : X2) : (X1 < X2 ? X1 : X2);
            int64_t mxx = X0 > X1 ? (X0 > X2 ? X0 : X2) : (X1 > X2 ? X1 : X2);
            int64_t mny = Y0 < Y1 ? (Y0 < Y2 ? Y0 : Y2) : (Y1 < Y2 ? Y1 : Y2);
            int64_t mxy = Y0 > Y1 ? (Y0 > Y2 ? Y0 : Y2) : (Y1 > Y2 ? Y1 : Y2);
            /* pixel px has centre 256 px + 128: the covered range of centres */
            int64_t x0 = mnx - 128 <= 0 ? 0 : (mnx - 128 + 255) / 256;
            int64_t x1 = mxx - 128 < 0 ? -1 : (mxx - 128) / 256;
            int64_t y0 = mny - 128 <= 0 ? 0 : (mny - 128 + 255) / 256;
            int64_t y1 = mxy - 128 < 0 ? -1 : (mxy - 128) / 256;
            if (x1 > W - 1) x1 = W - 1;
            if (y1 > H - 1) y1 = H - 1;
            for (int64_t py = y0; py <= y1; ++py)
                for (int64_t px = x0; px <= x1; ++px) {
                    uint32_t z;
                    if (cover(X0, Y0, X1, Y1, X2, Y2, Zq[a], Zq[b], Zq[d], px * 256 + 128,
                              py * 256 + 128, A2, &z)) {
                        uint64_t key = ((uint64_t)z << 32) | (uint32_t)f;
                        uint64_t* slot = kv + py * W + px;
                        if (key < *slot) *slot = key;
                    }
                }
        }
    }
    free(XY);
    free(Zq);
    return status;
}

/* Coverage counts with culling off (a test of the fill rule): for each pixel centre of
 * view 0, how many front faces and how many back faces contain it.  A back face is
 * tested with its winding reversed. */
int orc_coverage_counts(const float* V, int nv, const int32_t* F, int nf, const float* cam,
                        int W, int H, int32_t* front, int32_t* back) {
    int32_t* XY = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)nv);
    uint32_t* Zq = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nv);
    int status = orc_snap(V, nv, cam, XY, Zq);
    memset(front, 0, sizeof(int32_t) * (size_t)W * H);
    memset(back, 0, sizeof(int32_t) * (size_t)W * H);
    for (int f = 0; f < nf; ++f) {
        int a = F[3 * f], b = F[3 * f + 1], d = F[3 * f + 2];
        int64_t A2 = area2(XY[2 * a], XY[2 * a + 1], XY[2 * b], XY[2 * b + 1], XY[2 * d], XY[2 * d + 1]);
        if (A2 == 0) continue;
        int isback = A2 < 0;
        if (isback) { int t = b; b = d; d = t; A2 = -A2; }
        int64_t X0 = XY[2 * a], Y0 = XY[2 * a + 1], X1 = XY[2 * b], Y1 = XY[2 * b + 1];
        int64_t X2 = XY[2 * d], Y2 = XY[2 * d + 1];
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < W; ++px) {
                uint32_t z;
                if (A2 < A2_LIMIT &&
                    cover(X0, Y0, X1, Y1, X2, Y2, Zq[a], Zq[b], Zq[d], (int64_t)px * 256 + 128,
                          (int64_t)py * 256 + 128, A2, &z)) {
                    if (isback) back[py * W + px]++; else front[py * W + px]++;
                }
            }
    }
    free(XY);
    free(Zq);
    return status;
}

/* ------------------------------------------------------- environment distribution */
/* Importance weight of texel (i, j): Rec. 709 luminance times sin(theta) at the row
 * centre, quantised to 24 bits of the largest weight, plus one so every direction keeps
 * a positive density.  q: [H*W] integer weights; cdf: inclusive prefix sums (row-major).
 * Returns the total Q = cdf[H*W-1]. */
uint64_t orc_env_table(const float* E, int W, int H, uint32_t* q, uint64_t* cdf) {
    size_t n = (size_t)W * H;
    float* w = (float*)malloc(sizeof(float) * n);
    float wmax = 0.0f;
    for (int i = 0; i < H; ++i) {
        float sn, cs;
        orc_sincos2pi((float)(2 * i + 1) / (float)(4 * H), &sn, &cs);
        for (int j = 0; j < W; ++j) {
            const float* e = E + 3 * ((size_t)i * W + j);
            float lum = (0x1.b367a0p-3f * e[0] + 0x1.6e2eb2p-1f * e[1]) + 0x1.27bb30p-4f * e[2];
            float wt = lum * sn;
            if (!(wt > 0.0f)) wt = 0.0f;
            w[(size_t)i * W + j] = wt;
            if (wt > wmax) wmax = wt;
        }
    }
    float scale = 0.0f;
    if (wmax > 0.0f) {
        scale = 16777216.0f / wmax;
        if (!(scale <= 3.4028235e38f)) scale = 3.4028235e38f;
    }
    uint64_t acc = 0;
    for (size_t t = 0; t < n; ++t) {
        uint32_t qq = 1;
        if (w[t] > 0.0f) {
            float v = w[t] * scale;
            if (!(v < 16777216.0f)) v = 16777216.0f;
            qq = 1u + (uint32_t)v;
        }
        q[t] = qq;
        acc += qq;
        cdf[t] = acc;
    }
    free(w);
    return acc;
}

/* Smallest texel index whose inclusive prefix exceeds the target (binary search). */
static uint32_t pick_texel(const uint64_t* cdf, uint32_t n, uint64_t target) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static uint64_t scaled_target(uint32_t U, uint64_t Q) {
    return (uint64_t)(((unsigned __int128)U * Q) >> 32);
}

/* 2D strata of n samples: ny = the largest divisor of n not above sqrt(n), nx = n / ny. */
void orc_strata2(uint32_t n, uint32_t* nx, uint32_t* ny) {
    uint32_t best = 1;
    for (uint32_t d = 1; (uint64_t)d * d <= n; ++d)
        if (n % d == 0) best = d;
    *ny = best;
    *nx = n / best;
}

/* Texel choice and in-texel jitter for light sample k of n (2D-stratified inversion of the
 * marginal row distribution, then of the chosen row's conditional column distribution).
 * Sample k lies in row stratum k / nx and column stratum k % nx.  cdf is the row-major
 * inclusive prefix; row i ends at cdf[i*W + W - 1].  Returns the texel index. */
static uint32_t light_sample(const uint64_t* cdf, int W, int H, uint64_t Q, uint32_t k, uint32_t n,
                             const uint32_t h[4], float* xu, float* xv) {
    uint32_t nx, ny;
    orc_strata2(n, &nx, &ny);
    uint32_t kx = k % nx, ky = k / nx;
    uint64_t tr = scaled_target(stratified32(ky, ny, h[0]), Q);
    int lo = 0, hi = H - 1;
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (cdf[(size_t)mid * W + W - 1] > tr) hi = mid; else lo = mid + 1;
    }
    int row = lo;
    uint64_t pre = row ? cdf[(size_t)row * W - 1] : 0;
    uint64_t rsum = cdf[(size_t)row * W + W - 1] - pre;
    uint64_t tc = pre + scaled_target(stratified32(kx, nx, h[3]), rsum);
    uint32_t col = pick_texel(cdf + (size_t)row * W, (uint32_t)W, tc);
    *xu = unit24(h[1]);
    *xv = unit24(h[2]);
    return (uint32_t)row * (uint32_t)W + col;
}

/* Direction of a light sample: theta = pi (i + xv) / H from +y, phi = 2 pi (j + xu) / W
 * from -z towards +x: d = (sin t sin p, cos t, -sin t cos p). */
static f3 light_dir(uint32_t t, int W, int H, float xu, float xv) {
    int i = (int)(t / (uint32_t)W), j = (int)(t % (uint32_t)W);
    float fv = ((float)i + xv) / (float)H;
    float fu = ((float)j + xu) / (float)W;
    float st, ct, sp, cp;
    orc_sincos2pi(fv * 0.5f, &st, &ct);
    orc_sincos2pi(fu, &sp, &cp);
    return mk(st * sp, ct, -(st * cp));
}

void orc_light_dirs(const uint32_t* t, const float* xi, int n, int W, int H, float* out) {
    for (int k = 0; k < n; ++k) {
        f3 d = light_dir(t[k], W, H, xi[2 * k], xi[2 * k + 1]);
        out[3 * k] = d.x; out[3 * k + 1] = d.y; out[3 * k + 2] = d.z;
    }
}

/* ------------------------------------------------------ ray / triangle (watertight) */
typedef struct { f3 o, d; int kx, ky, kz; float Sx, Sy, Sz; } ray_t;

static ray_t make_ray(f3 o, f3 d) {
    ray_t r;
    r.o = o; r.d = d;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = ax >= ay ? (ax >= az ? 0 : 2) : (ay >= az ? 1 : 2);
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    if (comp(d, kz) < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = comp(d, kx) / comp(d, kz);
    r.Sy = comp(d, ky) / comp(d, kz);
    r.Sz = 1.0f / comp(d, kz);
    return r;
}

/* Returns 1 on a hit with t > 0; *T and *det give t = T / det, det > 0 for a face whose
 * counter-clockwise side faces the ray origin. */
static int woop(const ray_t* r, f3 p0, f3 p1, f3 p2, float* Tout, float* detout) {
    f3 A = sub3(p0, r->o), B = sub3(p1, r->o), C = sub3(p2, r->o);
    float Akz = comp(A, r->kz), Bkz = comp(B, r->kz), Ckz = comp(C, r->kz);
    float Ax = comp(A, r->kx) - r->Sx * Akz, Ay = comp(A, r->ky) - r->Sy * Akz;
    float Bx = comp(B, r->kx) - r->Sx * Bkz, By = comp(B, r->ky) - r->Sy * Bkz;
    float Cx = comp(C, r->kx) - r->Sx * Ckz, Cy = comp(C, r->ky) - r->Sy * Ckz;
    float U = Cx * By - Cy * Bx;
    float Vv = Ax * Cy - Ay * Cx;
    float Ww = Bx * Ay - By * Ax;
    if (U == 0.0f || Vv == 0.0f || Ww == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        Vv = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        Ww = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || Vv < 0.0f || Ww < 0.0f) && (U > 0.0f || Vv > 0.0f || Ww > 0.0f)) return 0;
    float det = (U + Vv) + Ww;
    if (det == 0.0f) return 0;
    float Az = r->Sz * Akz, Bz = r->Sz * Bkz, Cz = r->Sz * Ckz;
    float T = (U * Az + Vv * Bz) + Ww * Cz;
    if (!((det > 0.0f && T > 0.0f) || (det < 0.0f && T < 0.0f))) return 0;
    *Tout = T;
    *detout = det;
    return 1;
}

static f3 vtx(const float* V, const int32_t* F, int f, int k) { return ld3(V + 3 * F[3 * f + k]); }

static int any_hit(const float* V, const int32_t* F, int nf, f3 o, f3 d) {
    ray_t r = make_ray(o, d);
    for (int f = 0; f < nf; ++f) {
        float T, det;
        if (woop(&r, vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), &T, &det)) return 1;
    }
    return 0;
}

/* Closest hit (smallest t = T/det, ties to the lower id).  Returns the triangle or -1;
 * *front = det > 0; *gap = second-smallest t minus smallest t (inf if one hit). */
static int closest_hit(const float* V, const int32_t* F, int nf, f3 o, f3 d, float* tbest,
                       int* front, float* gap) {
    ray_t r = make_ray(o, d);
    int best = -1;
    float bt = INFINITY, second = INFINITY, bdet = 0.0f;
    for (int f = 0; f < nf; ++f) {
        float T, det;
        if (!woop(&r, vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), &T, &det)) continue;
        float t = T / det;
        if (t < bt) { second = bt; bt = t; best = f; bdet = det; }
        else if (t < second) second = t;
    }
    *tbest = bt;
    *front = bdet > 0.0f;
    *gap = second - bt;
    return best;
}

/* Batched ray queries for tests: mode 0 any-hit (out_tri = 1/0), mode 1 closest. */
void orc_trace(const float* V, const int32_t* F, int nf, const float* O, const float* D, int n,
               int mode, int32_t* out_tri, float* out_t, int32_t* out_front) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        f3 o = ld3(O + 3 * i), d = ld3(D + 3 * i);
        if (mode == 0) {
            out_tri[i] = any_hit(V, F, nf, o, d);
        } else {
            float t, gap;
            int front;
            out_tri[i] = closest_hit(V, F, nf, o, d, &t, &front, &gap);
            out_t[i] = t;
            out_front[i] = front;
        }
    }
}

/* ------------------------------------------------------ surface point (FP32 spec) */
/* Barycentrics of the ray o + t d on triangle (p0, p1, p2) by the Moller-Trumbore
 * formulas; the point x = b0 p0 + b1 p1 + b2 p2 and the unit geometric normal. */
static void surface_point(f3 o, f3 d, f3 p0, f3 p1, f3 p2, f3* x, f3* ng, float b[3]) {
    f3 e1 = sub3(p1, p0), e2 = sub3(p2, p0);
    f3 pv = cross3(d, e2);
    float det = dot3(e1, pv);
    float inv = 1.0f / det;
    f3 s = sub3(o, p0);
    float b1 = dot3(s, pv) * inv;
    f3 qv = cross3(s, e1);
    float b2 = dot3(d, qv) * inv;
    float b0 = (1.0f - b1) - b2;
    b[0] = b0; b[1] = b1; b[2] = b2;
    *x = mk((b0 * p0.x + b1 * p1.x) + b2 * p2.x, (b0 * p0.y + b1 * p1.y) + b2 * p2.y,
            (b0 * p0.z + b1 * p1.z) + b2 * p2.z);
    f3 c = cross3(e1, e2);
    float len = sqrtf(dot3(c, c));
    *ng = mk(c.x / len, c.y / len, c.z / len);
}

static f3 offset_origin(f3 x, f3 ng) {
    const float eps = 0x1.a36e2ep-14f; /* 1e-4 scene units */
    return mk(x.x + eps * ng.x, x.y + eps * ng.y, x.z + eps * ng.z);
}

/* Camera ray through the centre of pixel (px, py). */
static void camera_ray(const float* cam, int px, int py, f3* o, f3* d) {
    f3 rt = ld3(cam + 3), up = ld3(cam + 6), fw = ld3(cam + 9);
    float kx = cam[12], ky = cam[13], cx = cam[14], cy = cam[15];
    float dx = (((float)px + 0.5f) - cx) / kx;
    float dy = (cy - ((float)py + 0.5f)) / ky;
    *o = ld3(cam);
    *d = mk((fw.x + dx * rt.x) + dy * up.x, (fw.y + dx * rt.y) + dy * up.y, (fw.z + dx * rt.z) + dy * up.z);
}

/* Orthonormal basis about n (Duff, Burgess, Christensen, Hery, Kensler, Liani,
 * Villemin, "Building an Orthonormal Basis, Revisited", JCGT 2017). */
static void onb(f3 n, f3* b1, f3* b2) {
    float sign = copysignf(1.0f, n.z);
    float a = -1.0f / (sign + n.z);
    float b = (n.x * n.y) * a;
    *b1 = mk(1.0f + ((sign * n.x) * n.x) * a, sign * b, -(sign * n.x));
    *b2 = mk(b, sign + (n.y * n.y) * a, -n.y);
}

/* Cosine-weighted direction about n from (xi1, xi2). */
static f3 cosine_dir(f3 n, float xi1, float xi2) {
    f3 t, b;
    onb(n, &t, &b);
    float r = sqrtf(xi1);
    float sp, cp;
    orc_sincos2pi(xi2, &sp, &cp);
    float lx = r * cp, ly = r * sp, lz = sqrtf(1.0f - xi1);
    return mk((t.x * lx + b.x * ly) + n.x * lz, (t.y * lx + b.y * ly) + n.y * lz,
              (t.z * lx + b.z * ly) + n.z * lz);
}

/* --------------------------------------------------------- per-pixel decisions */
/* For each listed pixel (view, py, px) whose key names a triangle: the light-sample
 * texels and jitters, the shadow-ray visibility bits, the secondary closest hits (with
 * FP64 barycentrics of the traced ray), and at each valid secondary hit its light-sample
 * texels, jitters and visibility.  Layouts (P pixels):
 *   dtex [P,Nd] i32, dxi [P,Nd,2] f32, dvis [P,Nd] u8,
 *   stri [P,Nb] i32 (-1: no valid hit), sb [P,Nb,3] f64, sdir [P,Nb,3] f32, sxi1 [P,Nb] f32,
 *   sgap [P,Nb] f32, ltex [P,Nb,Ns] i32, lxi [P,Nb,Ns,2] f32, lvis [P,Nb,Ns] u8.
 * seed: 64-bit sample-set seed (Philox key).  Counters: (pixel = py*W+px, view, k, stream)
 * with stream 0 = direct light samples, 1 = secondary directions, 2 = light samples at
 * secondary hits (k = j*Ns + s). */
int orc_decide(const float* V, const int32_t* F, int nf, const float* cams, int W, int H,
               const uint64_t* cdf, int envW, int envH, uint64_t seed,
               int Nd, int Nb, int Ns, const int32_t* pix, const uint64_t* keys, int npix,
               int32_t* dtex, float* dxi, uint8_t* dvis,
               int32_t* stri, double* sb, float* sdir, float* sxi1, float* sgap,
               int32_t* ltex, float* lxi, uint8_t* lvis) {
    uint32_t ntex = (uint32_t)envW * (uint32_t)envH;
    uint64_t Q = cdf[ntex - 1];
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    (void)H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npix; ++p) {
        int c = pix[3 * p], py = pix[3 * p + 1], px = pix[3 * p + 2];
        uint32_t tri = (uint32_t)(keys[p] & 0xffffffffu);
        for (int k = 0; k < Nd; ++k) { dtex[(size_t)p * Nd + k] = -1; dvis[(size_t)p * Nd + k] = 0; }
        for (int j = 0; j < Nb; ++j) {
            stri[(size_t)p * Nb + j] = -1;
            for (int s = 0; s < Ns; ++s) {
                ltex[((size_t)p * Nb + j) * Ns + s] = -1;
                lvis[((size_t)p * Nb + j) * Ns + s] = 0;
            }
        }
        if (tri == 0xffffffffu) continue;
        const float* cam = cams + 20 * c;
        f3 o, d, x, ng;
        float b[3];
        camera_ray(cam, px, py, &o, &d);
        surface_point(o, d, vtx(V, F, tri, 0), vtx(V, F, tri, 1), vtx(V, F, tri, 2), &x, &ng, b);
        f3 org = offset_origin(x, ng);
        uint32_t pixel = (uint32_t)py * (uint32_t)W + (uint32_t)px;
        for (int k = 0; k < Nd; ++k) {
            uint32_t ctr[4] = {pixel, (uint32_t)c, (uint32_t)k, 0u}, h[4];
            orc_philox(ctr, key, h);
            float xu, xv;
            uint32_t t = light_sample(cdf, envW, envH, Q, (uint32_t)k, (uint32_t)Nd, h, &xu, &xv);
            f3 wi = light_dir(t, envW, envH, xu, xv);
            int vis = dot3(ng, wi) > 0.0f && !any_hit(V, F, nf, org, wi);
            dtex[(size_t)p * Nd + k] = (int32_t)t;
            dxi[2 * ((size_t)p * Nd + k)] = xu;
            dxi[2 * ((size_t)p * Nd + k) + 1] = xv;
            dvis[(size_t)p * Nd + k] = (uint8_t)vis;
        }
        for (int j = 0; j < Nb; ++j) {
            size_t pj = (size_t)p * Nb + j;
            uint32_t ctr[4] = {pixel, (uint32_t)c, (uint32_t)j, 1u}, h[4];
            orc_philox(ctr, key, h);
            float xi1 = (float)(stratified32((uint32_t)j, (uint32_t)Nb, h[0]) >> 8) * 0x1p-24f;
            float xi2 = unit24(h[1]);
            f3 wj = cosine_dir(ng, xi1, xi2);
            sdir[3 * pj] = wj.x; sdir[3 * pj + 1] = wj.y; sdir[3 * pj + 2] = wj.z;
            sxi1[pj] = xi1;
            float t, gap;
            int front;
            int g = closest_hit(V, F, nf, org, wj, &t, &front, &gap);
            sgap[pj] = gap;
            if (g < 0 || !front) continue;
            stri[pj] = g;
            f3 p0 = vtx(V, F, g, 0), p1 = vtx(V, F, g, 1), p2 = vtx(V, F, g, 2);
            /* FP64 barycentrics of the traced ray, for shading */
            {
                double O[3] = {org.x, org.y, org.z}, Dd[3] = {wj.x, wj.y, wj.z};
                double P0[3] = {p0.x, p0.y, p0.z}, P1[3] = {p1.x, p1.y, p1.z}, P2[3] = {p2.x, p2.y, p2.z};
                double e1[3], e2[3], s[3], pv[3], qv[3];
                for (int a = 0; a < 3; ++a) { e1[a] = P1[a] - P0[a]; e2[a] = P2[a] - P0[a]; s[a] = O[a] - P0[a]; }
                pv[0] = Dd[1] * e2[2] - Dd[2] * e2[1]; pv[1] = Dd[2] * e2[0] - Dd[0] * e2[2]; pv[2] = Dd[0] * e2[1] - Dd[1] * e2[0];
                double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
                double b1 = (s[0] * pv[0] + s[1] * pv[1] + s[2] * pv[2]) / det;
                qv[0] = s[1] * e1[2] - s[2] * e1[1]; qv[1] = s[2] * e1[0] - s[0] * e1[2]; qv[2] = s[0] * e1[1] - s[1] * e1[0];
                double b2 = (Dd[0] * qv[0] + Dd[1] * qv[1] + Dd[2] * qv[2]) / det;
                sb[3 * pj] = 1.0 - b1 - b2; sb[3 * pj + 1] = b1; sb[3 * pj + 2] = b2;
            }
            f3 y, ngy;
            float by[3];
            surface_point(org, wj, p0, p1, p2, &y, &ngy, by);
            f3 yorg = offset_origin(y, ngy);
            for (int s = 0; s < Ns; ++s) {
                size_t pjs = pj * Ns + s;
                uint32_t ctr2[4] = {pixel, (uint32_t)c, (uint32_t)(j * Ns + s), 2u}, h2[4];
                orc_philox(ctr2, key, h2);
                float xu, xv;
                uint32_t tt = light_sample(cdf, envW, envH, Q, (uint32_t)s, (uint32_t)Ns, h2, &xu, &xv);
                f3 wl = light_dir(tt, envW, envH, xu, xv);
                int vis = dot3(ngy, wl) > 0.0f && !any_hit(V, F, nf, yorg, wl);
                ltex[pjs] = (int32_t)tt;
                lxi[2 * pjs] = xu;
                lxi[2 * pjs + 1] = xv;
                lvis[pjs] = (uint8_t)vis;
            }
        }
    }
    return ORC_OK;
}
