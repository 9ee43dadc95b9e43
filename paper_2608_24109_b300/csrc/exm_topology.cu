// One Stage-I topology round (Sec. 4.1-4.3, Eqs. 1-6) on the device.
//
//   G_v <- beta_g G_v + (1 - beta_g) |grad_v|                              (Eq. 1)
//   K_f  = mean over edge-adjacent faces of arccos(n_f . n_f')             (Eq. 2)
//   S_f  = w_g mean(G of the corners) + w_k K_f                            (Eq. 3)
//   D_f  = Area / l_max^2                                                  (Eq. 4)
//
// Splits: faces with area >= the lower median are ranked by S_f (descending, ties by index)
// and the first ceil(split_percent % of the faces) are tried.  Each takes the edge with the
// largest l / mean valence, the new vertex at the mean of the projections of the opposite
// vertices (the midpoint on a boundary edge), and is discarded when mu = |v_s - v_a| / |e| is
// outside [0.25, 0.75].  Merges, on the mesh after the splits: unmodified faces with
// C_rend = 0 or D_f < tau_degen and area <= the lower median, ranked by D_f ascending; the
// collapse edge is the shortest boundary edge, else the shortest edge, and the lower-valence
// endpoint merges into the other (ties: the higher index goes).
//
// "Skipped if a face to be modified was already modified in the round" is read as a greedy
// pass in rank order.  Here it runs in parallel rounds: every undecided candidate writes its
// rank into the faces it would modify (atomicMin); a candidate holding all of its faces is
// accepted (no lower-ranked undecided candidate shares one) and takes them; a candidate that
// meets a taken face is rejected.  The result is exactly the sequential greedy one.
// Accepted splits are applied in rank order while the face count fits the budget.
//
// Every floating-point value that decides something is computed in FP32 in a fixed order
// (no contraction), arccos by Abramowitz and Stegun 4.4.46, so the round is reproducible
// bit for bit.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <climits>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

// ------------------------------------------------------------------ FP32 helpers (no fusion)
__device__ __forceinline__ float tdot(const float* a, const float* b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}
__device__ __forceinline__ void tsub(const float* a, const float* b, float* o) {
    o[0] = __fsub_rn(a[0], b[0]);
    o[1] = __fsub_rn(a[1], b[1]);
    o[2] = __fsub_rn(a[2], b[2]);
}
__device__ __forceinline__ float tlen(const float* a) { return __fsqrt_rn(tdot(a, a)); }
__device__ __forceinline__ void tload(const float* V, int v, float* o) {
    o[0] = V[3 * (size_t)v];
    o[1] = V[3 * (size_t)v + 1];
    o[2] = V[3 * (size_t)v + 2];
}

// Abramowitz and Stegun 4.4.46: arccos x = sqrt(1 - x) (a0 + ... + a7 x^7) on [0, 1],
// |error| <= 2e-8; arccos(-x) = pi - arccos(x).
__device__ __forceinline__ float acos_as(float x) {
    const float ax = fabsf(x);
    float p = -0.0012624911f;
    p = __fadd_rn(__fmul_rn(p, ax), 0.0066700901f);
    p = __fadd_rn(__fmul_rn(p, ax), -0.0170881256f);
    p = __fadd_rn(__fmul_rn(p, ax), 0.0308918810f);
    p = __fadd_rn(__fmul_rn(p, ax), -0.0501743046f);
    p = __fadd_rn(__fmul_rn(p, ax), 0.0889789874f);
    p = __fadd_rn(__fmul_rn(p, ax), -0.2145988016f);
    p = __fadd_rn(__fmul_rn(p, ax), 1.5707963050f);
    const float r = __fmul_rn(__fsqrt_rn(__fsub_rn(1.0f, ax)), p);
    return x < 0.0f ? __fsub_rn(3.14159265358979f, r) : r;
}

__device__ __forceinline__ uint32_t ord_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

#define TOPO_LOOP(i, n) for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)(n); \
                             i += (size_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ scores
__global__ void ema_kernel(int nv, const float* __restrict__ G0, const float* __restrict__ grad, float beta,
                           float* G) {
    TOPO_LOOP(v, nv) {
        float g[3];
        tload(grad, (int)v, g);
        const float gn = tlen(g);
        G[v] = __fadd_rn(__fmul_rn(beta, G0[v]), __fmul_rn(__fsub_rn(1.0f, beta), gn));
    }
}

__global__ void face_geom_kernel(int nf, const float* __restrict__ V, const int32_t* __restrict__ F, float* nrm,
                                 float* area, float* elen, float* degen) {
    TOPO_LOOP(f, nf) {
        float p[3][3];
        for (int k = 0; k < 3; ++k) tload(V, F[3 * f + k], p[k]);
        float e1[3], e2[3];
        tsub(p[1], p[0], e1);
        tsub(p[2], p[0], e2);
        const float c[3] = {__fsub_rn(__fmul_rn(e1[1], e2[2]), __fmul_rn(e1[2], e2[1])),
                            __fsub_rn(__fmul_rn(e1[2], e2[0]), __fmul_rn(e1[0], e2[2])),
                            __fsub_rn(__fmul_rn(e1[0], e2[1]), __fmul_rn(e1[1], e2[0]))};
        const float ln = tlen(c);
        for (int i = 0; i < 3; ++i) nrm[3 * f + i] = ln > 0.0f ? __fdiv_rn(c[i], ln) : 0.0f;
        const float a = __fmul_rn(0.5f, ln);
        area[f] = a;
        float lm = 0.0f;
        for (int k = 0; k < 3; ++k) {
            float d[3];
            tsub(p[(k + 1) % 3], p[k], d);
            const float l = tlen(d);
            elen[3 * f + k] = l;
            lm = k == 0 ? l : fmaxf(lm, l);
        }
        degen[f] = lm > 0.0f ? __fdiv_rn(a, __fmul_rn(lm, lm)) : 0.0f;
    }
}

__global__ void edge_keys_kernel(int nf, const int32_t* __restrict__ F, unsigned long long* keys, uint32_t* vals) {
    TOPO_LOOP(e, 3 * (size_t)nf) {
        const size_t f = e / 3;
        const int k = (int)(e - 3 * f);
        const uint32_t a = (uint32_t)F[3 * f + k], b = (uint32_t)F[3 * f + (k + 1) % 3];
        keys[e] = ((unsigned long long)min(a, b) << 32) | max(a, b);
        vals[e] = (uint32_t)e;
    }
}

// Runs of equal edge keys: neighbour across an edge used by exactly two faces; valences.
__global__ void edge_runs_kernel(size_t n, const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
                                 int32_t* nb, int32_t* deg) {
    TOPO_LOOP(i, n) {
        const unsigned long long key = keys[i];
        if (i > 0 && keys[i - 1] == key) continue;
        size_t j = i + 1;
        while (j < n && keys[j] == key) ++j;
        atomicAdd(deg + (uint32_t)(key >> 32), 1);
        atomicAdd(deg + (uint32_t)(key & 0xffffffffu), 1);
        if (j - i == 2) {
            nb[vals[i]] = (int32_t)vals[i + 1];
            nb[vals[i + 1]] = (int32_t)vals[i];
        }
    }
}

__global__ void curvature_score_kernel(int nf, const int32_t* __restrict__ F, const float* __restrict__ nrm,
                                       const int32_t* __restrict__ nb, const float* __restrict__ G, float wg,
                                       float wk, float* S) {
    TOPO_LOOP(f, nf) {
        float s = 0.0f;
        int cnt = 0;
        for (int k = 0; k < 3; ++k) {
            const int e = nb[3 * f + k];
            if (e < 0) continue;
            const int g = e / 3;
            float d = tdot(nrm + 3 * f, nrm + 3 * (size_t)g);
            d = fminf(fmaxf(d, -1.0f), 1.0f);
            s = __fadd_rn(s, acos_as(d));
            ++cnt;
        }
        const float K = cnt ? __fdiv_rn(s, (float)cnt) : 0.0f;
        const float Gf = __fdiv_rn(__fadd_rn(__fadd_rn(G[F[3 * f]], G[F[3 * f + 1]]), G[F[3 * f + 2]]), 3.0f);
        S[f] = __fadd_rn(__fmul_rn(wg, Gf), __fmul_rn(wk, K));
    }
}

__global__ void copy_kernel(size_t n, const float* __restrict__ a, float* b) { TOPO_LOOP(i, n) b[i] = a[i]; }

// Candidates first (key < 0xffffffff), ranked by key, ties by index (stable sort).
__global__ void split_keys_kernel(int nf, const float* __restrict__ area, const float* __restrict__ sorted_area,
                                  const float* __restrict__ S, uint32_t* keys, uint32_t* vals, uint32_t* ncand) {
    const float amed = sorted_area[(nf - 1) / 2];
    TOPO_LOOP(f, nf) {
        const bool c = area[f] >= amed;
        keys[f] = c ? ord_f32(-S[f]) : 0xffffffffu;
        vals[f] = (uint32_t)f;
        if (c) atomicAdd(ncand, 1u);
    }
}

struct SplitCand {
    int f, k, g, kg;
    float vs[3];
    float mu;
    int state;  // 0 undecided, 1 accepted, 2 rejected
};

__global__ void split_prep_kernel(int n, const uint32_t* __restrict__ order, const float* __restrict__ V,
                                  const int32_t* __restrict__ F, const float* __restrict__ elen,
                                  const int32_t* __restrict__ deg, const int32_t* __restrict__ nb, SplitCand* cand) {
    TOPO_LOOP(i, n) {
        const int f = (int)order[i];
        float sc[3];
        for (int k = 0; k < 3; ++k) {
            const int a = F[3 * f + k], b = F[3 * f + (k + 1) % 3];
            sc[k] = __fdiv_rn(elen[3 * f + k], __fmul_rn((float)(deg[a] + deg[b]), 0.5f));
        }
        int k = 0;
        for (int c = 1; c < 3; ++c)
            if (sc[c] > sc[k]) k = c;
        const int e = nb[3 * f + k];
        const int g = e >= 0 ? e / 3 : -1, kg = e >= 0 ? e - 3 * g : -1;
        float va[3], vb[3], ed[3];
        tload(V, F[3 * f + k], va);
        tload(V, F[3 * f + (k + 1) % 3], vb);
        tsub(vb, va, ed);
        const float ee = tdot(ed, ed);
        float vs[3];
        if (g < 0) {
            for (int i2 = 0; i2 < 3; ++i2) vs[i2] = __fmul_rn(__fadd_rn(va[i2], vb[i2]), 0.5f);
        } else {
            float pc[3], pd[3], tc[3], td[3], q[3];
            tload(V, F[3 * f + (k + 2) % 3], pc);
            tload(V, F[3 * g + (kg + 2) % 3], pd);
            tsub(pc, va, q);
            const float t1 = __fdiv_rn(tdot(q, ed), ee);
            tsub(pd, va, q);
            const float t2 = __fdiv_rn(tdot(q, ed), ee);
            for (int i2 = 0; i2 < 3; ++i2) {
                tc[i2] = __fadd_rn(va[i2], __fmul_rn(t1, ed[i2]));
                td[i2] = __fadd_rn(va[i2], __fmul_rn(t2, ed[i2]));
                vs[i2] = __fmul_rn(__fadd_rn(tc[i2], td[i2]), 0.5f);
            }
        }
        float dv[3];
        tsub(vs, va, dv);
        const float mu = __fdiv_rn(tlen(dv), __fsqrt_rn(ee));
        SplitCand c;
        c.f = f; c.k = k; c.g = g; c.kg = kg;
        c.vs[0] = vs[0]; c.vs[1] = vs[1]; c.vs[2] = vs[2];
        c.mu = mu;
        c.state = (mu >= 0.25f && mu <= 0.75f) ? 0 : 2;  // NaN fails both
        cand[i] = c;
    }
}

// ------------------------------------------------------------------ greedy selection rounds
__global__ void split_claim_kernel(int n, const SplitCand* __restrict__ c, int32_t* owner) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        atomicMin(owner + c[i].f, (int)i);
        if (c[i].g >= 0) atomicMin(owner + c[i].g, (int)i);
    }
}
__global__ void split_accept_kernel(int n, SplitCand* c, const int32_t* __restrict__ owner, uint8_t* taken) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        if (owner[c[i].f] == (int)i && (c[i].g < 0 || owner[c[i].g] == (int)i)) {
            c[i].state = 1;
            taken[c[i].f] = 1;
            if (c[i].g >= 0) taken[c[i].g] = 1;
        }
    }
}
__global__ void split_reject_kernel(int n, SplitCand* c, const uint8_t* __restrict__ taken, uint32_t* undecided) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        if (taken[c[i].f] || (c[i].g >= 0 && taken[c[i].g])) c[i].state = 2;
        else atomicAdd(undecided, 1u);
    }
}

// accepted splits in rank order with their face and UV counts
__global__ void split_flags_kernel(int n, const SplitCand* __restrict__ c, uint32_t* acc) {
    TOPO_LOOP(i, n) acc[i] = c[i].state == 1 ? 1u : 0u;
}
__global__ void split_list_kernel(int n, const SplitCand* __restrict__ c, const uint32_t* __restrict__ pos,
                                  uint32_t* list, uint32_t* adds) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 1) continue;
        list[pos[i]] = (uint32_t)i;
        adds[pos[i]] = c[i].g >= 0 ? 2u : 1u;
    }
}
// number of accepted splits whose inclusive face count fits the budget
__global__ void budget_kernel(int m, const uint32_t* __restrict__ adds_incl, long long room, uint32_t* applied) {
    TOPO_LOOP(j, m) {
        if ((long long)adds_incl[j] > room) atomicMin(applied, (uint32_t)j);
    }
}

__device__ __forceinline__ int corner_of(const int32_t* F, int face, int v) {
    return F[3 * face] == v ? 0 : (F[3 * face + 1] == v ? 1 : 2);
}

// UV candidates of an applied split and its UV count (1 shared or boundary, 2 across a seam).
__global__ void split_uv_kernel(int m, const uint32_t* __restrict__ list, const SplitCand* __restrict__ c,
                                const int32_t* __restrict__ F, const float* __restrict__ UV,
                                const int32_t* __restrict__ Fuv, float tau_uv, float* u, uint32_t* uvn) {
    TOPO_LOOP(j, m) {
        const SplitCand s = c[list[j]];
        const int va = F[3 * s.f + s.k], vb = F[3 * s.f + (s.k + 1) % 3];
        const float om = __fsub_rn(1.0f, s.mu);
        float u1[2], u2[2];
        {
            const int ua = Fuv[3 * s.f + corner_of(F, s.f, va)], ub = Fuv[3 * s.f + corner_of(F, s.f, vb)];
            for (int i = 0; i < 2; ++i)
                u1[i] = __fadd_rn(__fmul_rn(om, UV[2 * (size_t)ua + i]), __fmul_rn(s.mu, UV[2 * (size_t)ub + i]));
        }
        uint32_t cnt = 1;
        float w[4] = {u1[0], u1[1], 0.f, 0.f};
        if (s.g >= 0) {
            const int ua = Fuv[3 * s.g + corner_of(F, s.g, va)], ub = Fuv[3 * s.g + corner_of(F, s.g, vb)];
            for (int i = 0; i < 2; ++i)
                u2[i] = __fadd_rn(__fmul_rn(om, UV[2 * (size_t)ua + i]), __fmul_rn(s.mu, UV[2 * (size_t)ub + i]));
            const float d0 = __fsub_rn(u1[0], u2[0]), d1 = __fsub_rn(u1[1], u2[1]);
            if (__fsqrt_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1))) < tau_uv) {
                w[0] = __fmul_rn(__fadd_rn(u1[0], u2[0]), 0.5f);
                w[1] = __fmul_rn(__fadd_rn(u1[1], u2[1]), 0.5f);
            } else {
                w[2] = u2[0];
                w[3] = u2[1];
                cnt = 2;
            }
        }
        for (int i = 0; i < 4; ++i) u[4 * j + i] = w[i];
        uvn[j] = cnt;
    }
}

struct Mesh1 {
    float* V; int32_t* F; float* UV; int32_t* Fuv; float* G; uint8_t* touched;
    int nv0, nf0, nuv0;
};

__global__ void split_apply_kernel(int m, const uint32_t* __restrict__ list, const SplitCand* __restrict__ c,
                                   const uint32_t* __restrict__ face_off, const uint32_t* __restrict__ uv_off,
                                   const uint32_t* __restrict__ uvn, const float* __restrict__ u,
                                   const int32_t* __restrict__ F0, const int32_t* __restrict__ Fuv0, Mesh1 o) {
    TOPO_LOOP(j, m) {
        const SplitCand s = c[list[j]];
        const int sidx = o.nv0 + (int)j;
        const int va = F0[3 * s.f + s.k], vb = F0[3 * s.f + (s.k + 1) % 3];
        for (int i = 0; i < 3; ++i) o.V[3 * (size_t)sidx + i] = s.vs[i];
        o.G[sidx] = __fmul_rn(__fadd_rn(o.G[va], o.G[vb]), 0.5f);
        const int ub = o.nuv0 + (int)uv_off[j];
        o.UV[2 * (size_t)ub] = u[4 * j];
        o.UV[2 * (size_t)ub + 1] = u[4 * j + 1];
        if (uvn[j] == 2) {
            o.UV[2 * (size_t)ub + 2] = u[4 * j + 2];
            o.UV[2 * (size_t)ub + 3] = u[4 * j + 3];
        }
        const int faces[2] = {s.f, s.g};
        const int ks[2] = {s.k, s.kg};
        const int uvs[2] = {ub, uvn[j] == 2 ? ub + 1 : ub};
        for (int h = 0; h < (s.g >= 0 ? 2 : 1); ++h) {
            const int face = faces[h], kk = ks[h];
            const int x0 = F0[3 * face + kk], x1 = F0[3 * face + (kk + 1) % 3], x2 = F0[3 * face + (kk + 2) % 3];
            const int t0 = Fuv0[3 * face + kk], t1 = Fuv0[3 * face + (kk + 1) % 3], t2 = Fuv0[3 * face + (kk + 2) % 3];
            o.F[3 * (size_t)face] = x0; o.F[3 * (size_t)face + 1] = sidx; o.F[3 * (size_t)face + 2] = x2;
            o.Fuv[3 * (size_t)face] = t0; o.Fuv[3 * (size_t)face + 1] = uvs[h]; o.Fuv[3 * (size_t)face + 2] = t2;
            const size_t nfc = (size_t)o.nf0 + face_off[j] + h;
            o.F[3 * nfc] = sidx; o.F[3 * nfc + 1] = x1; o.F[3 * nfc + 2] = x2;
            o.Fuv[3 * nfc] = uvs[h]; o.Fuv[3 * nfc + 1] = t1; o.Fuv[3 * nfc + 2] = t2;
            o.touched[face] = 1;
            o.touched[nfc] = 1;
        }
    }
}

// ------------------------------------------------------------------ merges
__global__ void merge_keys_kernel(int nf, int nf_orig, const float* __restrict__ area,
                                  const float* __restrict__ sorted_area, const float* __restrict__ degen,
                                  const uint8_t* __restrict__ touched, const uint32_t* __restrict__ counts,
                                  float tau, uint32_t* keys, uint32_t* vals, uint32_t* ncand) {
    const float amed = sorted_area[(nf - 1) / 2];
    TOPO_LOOP(f, nf) {
        const uint32_t cr = f < (size_t)nf_orig ? counts[f] : 0u;
        const bool c = !touched[f] && area[f] <= amed && (cr == 0u || degen[f] < tau);
        keys[f] = c ? ord_f32(degen[f]) : 0xffffffffu;
        vals[f] = (uint32_t)f;
        if (c) atomicAdd(ncand, 1u);
    }
}

struct MergeCand {
    int vr, vs;
    int state;
};

__global__ void merge_prep_kernel(int n, const uint32_t* __restrict__ order, const int32_t* __restrict__ F,
                                  const float* __restrict__ elen, const int32_t* __restrict__ nb,
                                  const int32_t* __restrict__ deg, MergeCand* cand) {
    TOPO_LOOP(i, n) {
        const int f = (int)order[i];
        int ks[3], nk = 0;
        for (int k = 0; k < 3; ++k)
            if (nb[3 * f + k] < 0) ks[nk++] = k;
        if (nk == 0) { ks[0] = 0; ks[1] = 1; ks[2] = 2; nk = 3; }
        int k = ks[0];
        for (int c = 1; c < nk; ++c)
            if (elen[3 * f + ks[c]] < elen[3 * f + k]) k = ks[c];
        const int a = F[3 * f + k], b = F[3 * f + (k + 1) % 3];
        MergeCand m;
        if (deg[a] < deg[b] || (deg[a] == deg[b] && a > b)) { m.vr = a; m.vs = b; }
        else { m.vr = b; m.vs = a; }
        m.state = 0;
        cand[i] = m;
    }
}

// vertex -> incident faces (sorted corner list)
__global__ void corner_keys_kernel(int nf, const int32_t* __restrict__ F, uint32_t* keys, uint32_t* vals) {
    TOPO_LOOP(e, 3 * (size_t)nf) {
        keys[e] = (uint32_t)F[e];
        vals[e] = (uint32_t)(e / 3);
    }
}
__global__ void star_ranges_kernel(size_t n, const uint32_t* __restrict__ keys, uint32_t* first, uint32_t* last) {
    TOPO_LOOP(i, n) {
        const uint32_t v = keys[i];
        if (i == 0 || keys[i - 1] != v) first[v] = (uint32_t)i;
        if (i + 1 == n || keys[i + 1] != v) last[v] = (uint32_t)(i + 1);
    }
}

__global__ void merge_claim_kernel(int n, const MergeCand* __restrict__ c, const uint32_t* __restrict__ first,
                                   const uint32_t* __restrict__ last, const uint32_t* __restrict__ star,
                                   int32_t* owner) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        for (uint32_t s = first[c[i].vr]; s < last[c[i].vr]; ++s) atomicMin(owner + star[s], (int)i);
    }
}
__global__ void merge_accept_kernel(int n, MergeCand* c, const uint32_t* __restrict__ first,
                                    const uint32_t* __restrict__ last, const uint32_t* __restrict__ star,
                                    const int32_t* __restrict__ owner, uint8_t* taken) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        bool mine = true;
        for (uint32_t s = first[c[i].vr]; s < last[c[i].vr]; ++s) mine = mine && owner[star[s]] == (int)i;
        if (!mine) continue;
        c[i].state = 1;
        for (uint32_t s = first[c[i].vr]; s < last[c[i].vr]; ++s) taken[star[s]] = 1;
    }
}
__global__ void merge_reject_kernel(int n, MergeCand* c, const uint32_t* __restrict__ first,
                                    const uint32_t* __restrict__ last, const uint32_t* __restrict__ star,
                                    const uint8_t* __restrict__ taken, uint32_t* undecided) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 0) continue;
        bool hit = false;
        for (uint32_t s = first[c[i].vr]; s < last[c[i].vr]; ++s) hit = hit || taken[star[s]];
        if (hit) c[i].state = 2;
        else atomicAdd(undecided, 1u);
    }
}

__global__ void vmap_init_kernel(int nv, int32_t* vmap, uint32_t* alive) {
    TOPO_LOOP(v, nv) {
        vmap[v] = (int32_t)v;
        alive[v] = 1u;
    }
}
__global__ void vmap_apply_kernel(int n, const MergeCand* __restrict__ c, int32_t* vmap, uint32_t* alive,
                                  uint32_t* merges) {
    TOPO_LOOP(i, n) {
        if (c[i].state != 1) continue;
        vmap[c[i].vr] = c[i].vs;
        alive[c[i].vr] = 0u;
        atomicAdd(merges, 1u);
    }
}
// faces after the merges: remapped vertices; kept unless a vertex repeats
__global__ void face_keep_kernel(int nf, int32_t* F, const int32_t* __restrict__ vmap, uint32_t* keep) {
    TOPO_LOOP(f, nf) {
        const int a = vmap[F[3 * f]], b = vmap[F[3 * f + 1]], c = vmap[F[3 * f + 2]];
        F[3 * f] = a; F[3 * f + 1] = b; F[3 * f + 2] = c;
        keep[f] = (a != b && b != c && c != a) ? 1u : 0u;
    }
}
__global__ void uv_used_kernel(int nf, const int32_t* __restrict__ Fuv, const uint32_t* __restrict__ keep,
                               uint32_t* used) {
    TOPO_LOOP(f, nf) {
        if (!keep[f]) continue;
        used[Fuv[3 * f]] = 1u;
        used[Fuv[3 * f + 1]] = 1u;
        used[Fuv[3 * f + 2]] = 1u;
    }
}
__global__ void compact_faces_kernel(int nf, const int32_t* __restrict__ F, const int32_t* __restrict__ Fuv,
                                     const uint32_t* __restrict__ keep, const uint32_t* __restrict__ fpos,
                                     const uint32_t* __restrict__ vpos, const uint32_t* __restrict__ upos,
                                     int32_t* Fo, int32_t* Fuvo) {
    TOPO_LOOP(f, nf) {
        if (!keep[f]) continue;
        const uint32_t o = fpos[f];
        for (int k = 0; k < 3; ++k) {
            Fo[3 * (size_t)o + k] = (int32_t)vpos[F[3 * f + k]];
            Fuvo[3 * (size_t)o + k] = (int32_t)upos[Fuv[3 * f + k]];
        }
    }
}
__global__ void compact_verts_kernel(int nv, const float* __restrict__ V, const float* __restrict__ G,
                                     const uint32_t* __restrict__ alive, const uint32_t* __restrict__ vpos,
                                     float* Vo, float* Go) {
    TOPO_LOOP(v, nv) {
        if (!alive[v]) continue;
        const uint32_t o = vpos[v];
        Vo[3 * (size_t)o] = V[3 * v];
        Vo[3 * (size_t)o + 1] = V[3 * v + 1];
        Vo[3 * (size_t)o + 2] = V[3 * v + 2];
        Go[o] = G[v];
    }
}
__global__ void compact_uvs_kernel(int nuv, const float* __restrict__ UV, const uint32_t* __restrict__ used,
                                   const uint32_t* __restrict__ upos, float* UVo) {
    TOPO_LOOP(t, nuv) {
        if (!used[t]) continue;
        UVo[2 * (size_t)upos[t]] = UV[2 * t];
        UVo[2 * (size_t)upos[t] + 1] = UV[2 * t + 1];
    }
}

__global__ void render_count_kernel(size_t n, const unsigned long long* __restrict__ visbuf, int nf, uint32_t* counts) {
    TOPO_LOOP(p, n) {
        const unsigned long long key = visbuf[p];
        if (key == ~0ull) continue;
        const uint32_t tri = (uint32_t)(key & 0xffffffffull);
        if (tri < (uint32_t)nf) atomicAdd(counts + tri, 1u);
    }
}

#undef TOPO_LOOP

}  // namespace exm

using namespace exm;

// ------------------------------------------------------------------ host side

struct exm_topology {
    exm_ctx* ctx = nullptr;
    // result
    float* V = nullptr; int32_t* F = nullptr; float* UV = nullptr; int32_t* Fuv = nullptr; float* G = nullptr;
    size_t cV = 0, cF = 0, cUV = 0, cFuv = 0, cG = 0;
    int nv = 0, nf = 0, nuv = 0;
    int stats[3] = {0, 0, 0};
    // scratch
    std::vector<std::pair<void*, size_t>> bufs;
    void* tmp = nullptr;
    size_t tmp_cap = 0;
};

// selection rounds launched between two read-backs of the undecided count
constexpr int kSelectBatch = 4;

namespace {

// named scratch slots of a topology object (grown on demand, contents not kept)
template <typename T>
T* scratch(exm_topology* t, int slot, size_t n) {
    if ((int)t->bufs.size() <= slot) t->bufs.resize(slot + 1, {nullptr, 0});
    auto& b = t->bufs[slot];
    const size_t bytes = (n ? n : 1) * sizeof(T);
    if (b.second < bytes) {
        cudaFree(b.first);
        b.first = nullptr;
        b.second = 0;
        if (exm_malloc((void**)&b.first, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        b.second = bytes;
    }
    return (T*)b.first;
}

bool ensure_tmp(exm_topology* t, size_t bytes) {
    if (t->tmp_cap >= bytes && t->tmp) return true;
    cudaFree(t->tmp);
    t->tmp = nullptr;
    t->tmp_cap = 0;
    if (exm_malloc((void**)&t->tmp, bytes ? bytes : 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    t->tmp_cap = bytes;
    return true;
}

int grid(exm_ctx* c, size_t n) {
    const size_t want = (n + 255) / 256, cap = (size_t)c->num_sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

template <typename K>
exm_status sort_pairs(exm_topology* t, K* kin, K* kout, uint32_t* vin, uint32_t* vout, size_t n, int bits,
                      cudaStream_t s) {
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, vout, (int)n, 0, bits, s);
    if (!ensure_tmp(t, bytes)) return exm_fail(EXM_ERR_OOM, "topology sort scratch");
    cub::DeviceRadixSort::SortPairs(t->tmp, bytes, kin, kout, vin, vout, (int)n, 0, bits, s);
    return EXM_OK;
}

exm_status excl_scan(exm_topology* t, uint32_t* in, uint32_t* out, size_t n, cudaStream_t s) {
    size_t bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)n, s);
    if (!ensure_tmp(t, bytes)) return exm_fail(EXM_ERR_OOM, "topology scan scratch");
    cub::DeviceScan::ExclusiveSum(t->tmp, bytes, in, out, (int)n, s);
    return EXM_OK;
}

exm_status incl_scan(exm_topology* t, uint32_t* in, uint32_t* out, size_t n, cudaStream_t s) {
    size_t bytes = 0;
    cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out, (int)n, s);
    if (!ensure_tmp(t, bytes)) return exm_fail(EXM_ERR_OOM, "topology scan scratch");
    cub::DeviceScan::InclusiveSum(t->tmp, bytes, in, out, (int)n, s);
    return EXM_OK;
}

exm_status read_u32(const uint32_t* d, uint32_t* h, cudaStream_t s) {
    if (cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return exm_cuda_check(cudaGetLastError(), "topology read-back");
    return EXM_OK;
}

// Face geometry, edge table (neighbours across two-face edges) and valences of a mesh.
struct Adjacency {
    float *nrm, *area, *elen, *degen, *sorted_area;
    int32_t *nb, *deg;
};

exm_status adjacency(exm_topology* t, int base, const float* V, int nv, const int32_t* F, int nf, Adjacency* A,
                     cudaStream_t s) {
    exm_ctx* c = t->ctx;
    A->nrm = scratch<float>(t, base + 0, 3 * (size_t)nf);
    A->area = scratch<float>(t, base + 1, nf);
    A->elen = scratch<float>(t, base + 2, 3 * (size_t)nf);
    A->degen = scratch<float>(t, base + 3, nf);
    A->sorted_area = scratch<float>(t, base + 4, nf);
    A->nb = scratch<int32_t>(t, base + 5, 3 * (size_t)nf);
    A->deg = scratch<int32_t>(t, base + 6, nv);
    float* area_copy = scratch<float>(t, base + 7, nf);
    unsigned long long* k0 = scratch<unsigned long long>(t, base + 8, 3 * (size_t)nf);
    unsigned long long* k1 = scratch<unsigned long long>(t, base + 9, 3 * (size_t)nf);
    uint32_t* v0 = scratch<uint32_t>(t, base + 10, 3 * (size_t)nf);
    uint32_t* v1 = scratch<uint32_t>(t, base + 11, 3 * (size_t)nf);
    uint32_t* ia = scratch<uint32_t>(t, base + 12, nf);
    uint32_t* ib = scratch<uint32_t>(t, base + 13, nf);
    if (!A->nrm || !A->area || !A->elen || !A->degen || !A->sorted_area || !A->nb || !A->deg || !area_copy || !k0 ||
        !k1 || !v0 || !v1 || !ia || !ib)
        return exm_fail(EXM_ERR_OOM, "topology adjacency buffers");
    face_geom_kernel<<<grid(c, nf), 256, 0, s>>>(nf, V, F, A->nrm, A->area, A->elen, A->degen);
    edge_keys_kernel<<<grid(c, 3 * (size_t)nf), 256, 0, s>>>(nf, F, k0, v0);
    exm_status st = sort_pairs(t, k0, k1, v0, v1, 3 * (size_t)nf, 64, s);
    if (st != EXM_OK) return st;
    cudaMemsetAsync(A->nb, 0xff, 3 * (size_t)nf * sizeof(int32_t), s);
    cudaMemsetAsync(A->deg, 0, (size_t)nv * sizeof(int32_t), s);
    edge_runs_kernel<<<grid(c, 3 * (size_t)nf), 256, 0, s>>>(3 * (size_t)nf, k1, v1, A->nb, A->deg);
    // lower median of the areas: sort a copy (ascending; positive floats order as their bits)
    copy_kernel<<<grid(c, nf), 256, 0, s>>>(nf, A->area, area_copy);
    st = sort_pairs(t, (uint32_t*)area_copy, (uint32_t*)A->sorted_area, ia, ib, nf, 32, s);
    c->launches += 5;
    return st;
}

}  // namespace

extern "C" {

exm_status exm_topology_create(exm_ctx* c, exm_topology** out) {
    if (!c || !out) return exm_fail(EXM_ERR_ARG, "exm_topology_create: NULL argument");
    *out = nullptr;
    exm_topology* t = new (std::nothrow) exm_topology();
    if (!t) return exm_fail(EXM_ERR_OOM, "exm_topology_create: host allocation");
    t->ctx = c;
    *out = t;
    return EXM_OK;
}

void exm_topology_destroy(exm_topology* t) {
    if (!t) return;
    {
        DeviceGuard guard(t->ctx->device);
        for (auto& b : t->bufs) cudaFree(b.first);
        cudaFree(t->tmp);
        cudaFree(t->V); cudaFree(t->F); cudaFree(t->UV); cudaFree(t->Fuv); cudaFree(t->G);
    }
    delete t;
}

exm_status exm_face_render_counts(exm_frame* f, int nf, uint32_t* counts, void* stream) {
    if (!f || !counts || nf < 1) return exm_fail(EXM_ERR_ARG, "exm_face_render_counts: bad argument");
    DeviceGuard guard(f->ctx->device);
    const size_t P = (size_t)f->views * f->W * f->H;
    render_count_kernel<<<grid(f->ctx, P), 256, 0, (cudaStream_t)stream>>>(P, (const unsigned long long*)f->visbuf,
                                                                          nf, counts);
    f->ctx->launches += 1;
    return exm_cuda_check(cudaGetLastError(), "exm_face_render_counts launch");
}

exm_status exm_topology_round(exm_topology* t, const float* V, int nv, const int32_t* F, int nf, const float* UV,
                              int nuv, const int32_t* Fuv, const float* ema, const float* grad_V,
                              const uint32_t* render_counts, const exm_topology_params* p, void* stream) {
    ExmRange range("exm_topology_round");
    if (!t || !V || !F || !UV || !Fuv || !ema || !grad_V || !render_counts || !p || nv < 3 || nf < 1 || nuv < 1)
        return exm_fail(EXM_ERR_ARG, "exm_topology_round: bad argument");
    if (p->split_percent < 0 || p->split_percent > 100 || p->max_faces < 1 || (long long)nf * 3 >= INT_MAX / 2)
        return exm_fail(EXM_ERR_ARG, "exm_topology_round: parameters");
    exm_ctx* c = t->ctx;
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    exm_status st = EXM_OK;
    uint32_t* cnt = scratch<uint32_t>(t, 0, 8);
    float* G = scratch<float>(t, 1, nv);
    if (!cnt || !G) return exm_fail(EXM_ERR_OOM, "topology buffers");
    // ---- 1-4: EMA, geometry, adjacency, curvature and split scores on the input mesh
    ema_kernel<<<grid(c, nv), 256, 0, s>>>(nv, ema, grad_V, p->beta_g, G);
    Adjacency A0;
    st = adjacency(t, 10, V, nv, F, nf, &A0, s);
    if (st != EXM_OK) return st;
    float* S = scratch<float>(t, 2, nf);
    uint32_t* sk0 = scratch<uint32_t>(t, 3, nf);
    uint32_t* sk1 = scratch<uint32_t>(t, 4, nf);
    uint32_t* sv0 = scratch<uint32_t>(t, 5, nf);
    uint32_t* sv1 = scratch<uint32_t>(t, 6, nf);
    if (!S || !sk0 || !sk1 || !sv0 || !sv1) return exm_fail(EXM_ERR_OOM, "topology buffers");
    curvature_score_kernel<<<grid(c, nf), 256, 0, s>>>(nf, F, A0.nrm, A0.nb, G, p->w_g, p->w_k, S);
    cudaMemsetAsync(cnt, 0, 8 * sizeof(uint32_t), s);
    split_keys_kernel<<<grid(c, nf), 256, 0, s>>>(nf, A0.area, A0.sorted_area, S, sk0, sv0, cnt);
    st = sort_pairs(t, sk0, sk1, sv0, sv1, nf, 32, s);
    if (st != EXM_OK) return st;
    uint32_t ncand = 0;
    st = read_u32(cnt, &ncand, s);
    if (st != EXM_OK) return st;
    const int K = (int)std::min<long long>(ncand, ((long long)nf * p->split_percent + 99) / 100);
    // ---- 5: split candidates and the greedy selection
    SplitCand* cand = scratch<SplitCand>(t, 7, K);
    int32_t* owner = scratch<int32_t>(t, 8, nf);
    uint8_t* taken = scratch<uint8_t>(t, 9, nf);
    if (!cand || !owner || !taken) return exm_fail(EXM_ERR_OOM, "topology buffers");
    cudaMemsetAsync(taken, 0, nf, s);
    int applied = 0;
    uint32_t* list = scratch<uint32_t>(t, 30, K);
    uint32_t* adds = scratch<uint32_t>(t, 31, K);
    uint32_t* pos = scratch<uint32_t>(t, 32, K);
    uint32_t* incl = scratch<uint32_t>(t, 33, K);
    if (!list || !adds || !pos || !incl) return exm_fail(EXM_ERR_OOM, "topology buffers");
    if (K > 0) {
        split_prep_kernel<<<grid(c, K), 256, 0, s>>>(K, sv1, V, F, A0.elen, A0.deg, A0.nb, cand);
        // kSelectBatch rounds between read-backs of the undecided count: the kernels skip
        // decided candidates, so rounds after the last decision change nothing
        for (int it = 0;; it += kSelectBatch) {
            if (it > K + 1) return exm_fail(EXM_ERR_CUDA, "topology split selection did not converge");
            for (int b = 0; b < kSelectBatch; ++b) {
                cudaMemsetAsync(owner, 0x7f, (size_t)nf * sizeof(int32_t), s);
                split_claim_kernel<<<grid(c, K), 256, 0, s>>>(K, cand, owner);
                split_accept_kernel<<<grid(c, K), 256, 0, s>>>(K, cand, owner, taken);
                cudaMemsetAsync(cnt + 1, 0, 4, s);
                split_reject_kernel<<<grid(c, K), 256, 0, s>>>(K, cand, taken, cnt + 1);
                c->launches += 3;
            }
            uint32_t und = 0;
            st = read_u32(cnt + 1, &und, s);
            if (st != EXM_OK) return st;
            if (und == 0) break;
        }
        // accepted splits in rank order, then the face budget
        split_flags_kernel<<<grid(c, K), 256, 0, s>>>(K, cand, adds);
        st = excl_scan(t, adds, pos, K, s);
        if (st != EXM_OK) return st;
        split_list_kernel<<<grid(c, K), 256, 0, s>>>(K, cand, pos, list, incl);
        uint32_t last_pos = 0, last_flag = 0;
        st = read_u32(pos + (K - 1), &last_pos, s);
        if (st == EXM_OK) st = read_u32(adds + (K - 1), &last_flag, s);
        if (st != EXM_OK) return st;
        const int m = (int)(last_pos + last_flag);
        if (m > 0) {
            st = incl_scan(t, incl, adds, m, s);  // adds <- inclusive face counts
            if (st != EXM_OK) return st;
            cudaMemcpyAsync(cnt + 2, &m, 4, cudaMemcpyHostToDevice, s);
            budget_kernel<<<grid(c, m), 256, 0, s>>>(m, adds, (long long)p->max_faces - nf, cnt + 2);
            uint32_t ap = 0;
            st = read_u32(cnt + 2, &ap, s);
            if (st != EXM_OK) return st;
            applied = (int)ap;
        }
        c->launches += 4;
    }
    // ---- 6: apply the splits into the intermediate mesh
    uint32_t* face_off = scratch<uint32_t>(t, 34, applied);
    uint32_t* uvn = scratch<uint32_t>(t, 35, applied);
    uint32_t* uv_off = scratch<uint32_t>(t, 36, applied);
    float* uvc = scratch<float>(t, 37, 4 * (size_t)applied);
    if (!face_off || !uvn || !uv_off || !uvc) return exm_fail(EXM_ERR_OOM, "topology buffers");
    int add_faces = 0, add_uvs = 0;
    if (applied > 0) {
        // per-split face counts in `incl` (list order); exclusive offsets
        st = excl_scan(t, incl, face_off, applied, s);
        if (st != EXM_OK) return st;
        split_uv_kernel<<<grid(c, applied), 256, 0, s>>>(applied, list, cand, F, UV, Fuv, p->tau_uv, uvc, uvn);
        st = excl_scan(t, uvn, uv_off, applied, s);
        if (st != EXM_OK) return st;
        uint32_t fo = 0, fl = 0, uo = 0, ul = 0;
        st = read_u32(face_off + applied - 1, &fo, s);
        if (st == EXM_OK) st = read_u32(incl + applied - 1, &fl, s);
        if (st == EXM_OK) st = read_u32(uv_off + applied - 1, &uo, s);
        if (st == EXM_OK) st = read_u32(uvn + applied - 1, &ul, s);
        if (st != EXM_OK) return st;
        add_faces = (int)(fo + fl);
        add_uvs = (int)(uo + ul);
    }
    const int nv1 = nv + applied, nf1 = nf + add_faces, nuv1 = nuv + add_uvs;
    Mesh1 m1;
    m1.V = scratch<float>(t, 40, 3 * (size_t)nv1);
    m1.F = scratch<int32_t>(t, 41, 3 * (size_t)nf1);
    m1.UV = scratch<float>(t, 42, 2 * (size_t)nuv1);
    m1.Fuv = scratch<int32_t>(t, 43, 3 * (size_t)nf1);
    m1.G = scratch<float>(t, 44, nv1);
    m1.touched = scratch<uint8_t>(t, 45, nf1);
    m1.nv0 = nv; m1.nf0 = nf; m1.nuv0 = nuv;
    if (!m1.V || !m1.F || !m1.UV || !m1.Fuv || !m1.G || !m1.touched) return exm_fail(EXM_ERR_OOM, "topology buffers");
    cudaMemcpyAsync(m1.V, V, 3 * (size_t)nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m1.F, F, 3 * (size_t)nf * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m1.UV, UV, 2 * (size_t)nuv * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m1.Fuv, Fuv, 3 * (size_t)nf * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m1.G, G, (size_t)nv * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(m1.touched, 0, nf1, s);
    if (applied > 0) {
        split_apply_kernel<<<grid(c, applied), 256, 0, s>>>(applied, list, cand, face_off, uv_off, uvn, uvc, F, Fuv,
                                                            m1);
        c->launches += 2;
    }
    // ---- 7: merges on the intermediate mesh
    Adjacency A1;
    st = adjacency(t, 50, m1.V, nv1, m1.F, nf1, &A1, s);
    if (st != EXM_OK) return st;
    uint32_t* mk0 = scratch<uint32_t>(t, 70, nf1);
    uint32_t* mk1 = scratch<uint32_t>(t, 71, nf1);
    uint32_t* mv0 = scratch<uint32_t>(t, 72, nf1);
    uint32_t* mv1 = scratch<uint32_t>(t, 73, nf1);
    if (!mk0 || !mk1 || !mv0 || !mv1) return exm_fail(EXM_ERR_OOM, "topology buffers");
    cudaMemsetAsync(cnt + 3, 0, 4, s);
    merge_keys_kernel<<<grid(c, nf1), 256, 0, s>>>(nf1, nf, A1.area, A1.sorted_area, A1.degen, m1.touched,
                                                   render_counts, p->tau_degen, mk0, mv0, cnt + 3);
    st = sort_pairs(t, mk0, mk1, mv0, mv1, nf1, 32, s);
    if (st != EXM_OK) return st;
    uint32_t nmc = 0;
    st = read_u32(cnt + 3, &nmc, s);
    if (st != EXM_OK) return st;
    const int MC = (int)nmc;
    MergeCand* mc = scratch<MergeCand>(t, 74, MC);
    uint32_t* ck0 = scratch<uint32_t>(t, 75, 3 * (size_t)nf1);
    uint32_t* ck1 = scratch<uint32_t>(t, 76, 3 * (size_t)nf1);
    uint32_t* cv0 = scratch<uint32_t>(t, 77, 3 * (size_t)nf1);
    uint32_t* star = scratch<uint32_t>(t, 78, 3 * (size_t)nf1);
    uint32_t* first = scratch<uint32_t>(t, 79, nv1);
    uint32_t* last = scratch<uint32_t>(t, 80, nv1);
    int32_t* owner1 = scratch<int32_t>(t, 81, nf1);
    uint8_t* taken1 = scratch<uint8_t>(t, 82, nf1);
    int32_t* vmap = scratch<int32_t>(t, 83, nv1);
    uint32_t* alive = scratch<uint32_t>(t, 84, nv1);
    if (!mc || !ck0 || !ck1 || !cv0 || !star || !first || !last || !owner1 || !taken1 || !vmap || !alive)
        return exm_fail(EXM_ERR_OOM, "topology buffers");
    vmap_init_kernel<<<grid(c, nv1), 256, 0, s>>>(nv1, vmap, alive);
    cudaMemsetAsync(cnt + 5, 0, 4, s);
    if (MC > 0) {
        merge_prep_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mv1, m1.F, A1.elen, A1.nb, A1.deg, mc);
        corner_keys_kernel<<<grid(c, 3 * (size_t)nf1), 256, 0, s>>>(nf1, m1.F, ck0, cv0);
        st = sort_pairs(t, ck0, ck1, cv0, star, 3 * (size_t)nf1, 32, s);
        if (st != EXM_OK) return st;
        cudaMemsetAsync(first, 0, (size_t)nv1 * 4, s);
        cudaMemsetAsync(last, 0, (size_t)nv1 * 4, s);
        star_ranges_kernel<<<grid(c, 3 * (size_t)nf1), 256, 0, s>>>(3 * (size_t)nf1, ck1, first, last);
        // faces modified by the splits are taken from the start
        cudaMemcpyAsync(taken1, m1.touched, nf1, cudaMemcpyDeviceToDevice, s);
        // rounds of reject, claim, accept, kSelectBatch at a time, then a reject whose count
        // of undecided candidates is read back (rounds after the last decision change nothing)
        for (int it = 0;; it += kSelectBatch) {
            if (it > MC + 1) return exm_fail(EXM_ERR_CUDA, "topology merge selection did not converge");
            cudaMemsetAsync(cnt + 4, 0, 4, s);
            merge_reject_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mc, first, last, star, taken1, cnt + 4);
            uint32_t und = 0;
            st = read_u32(cnt + 4, &und, s);
            if (st != EXM_OK) return st;
            if (und == 0) break;
            for (int b = 0; b < kSelectBatch; ++b) {
                cudaMemsetAsync(owner1, 0x7f, (size_t)nf1 * sizeof(int32_t), s);
                merge_claim_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mc, first, last, star, owner1);
                merge_accept_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mc, first, last, star, owner1, taken1);
                c->launches += 2;
                if (b + 1 < kSelectBatch) {
                    merge_reject_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mc, first, last, star, taken1, cnt + 4);
                    c->launches += 1;
                }
            }
            c->launches += 1;
        }
        vmap_apply_kernel<<<grid(c, MC), 256, 0, s>>>(MC, mc, vmap, alive, cnt + 5);
        c->launches += 4;
    }
    // ---- 8: delete, compact
    uint32_t* keep = scratch<uint32_t>(t, 85, nf1);
    uint32_t* fpos = scratch<uint32_t>(t, 86, nf1);
    uint32_t* vpos = scratch<uint32_t>(t, 87, nv1);
    uint32_t* used = scratch<uint32_t>(t, 88, nuv1);
    uint32_t* upos = scratch<uint32_t>(t, 89, nuv1);
    if (!keep || !fpos || !vpos || !used || !upos) return exm_fail(EXM_ERR_OOM, "topology buffers");
    face_keep_kernel<<<grid(c, nf1), 256, 0, s>>>(nf1, m1.F, vmap, keep);
    cudaMemsetAsync(used, 0, (size_t)nuv1 * 4, s);
    uv_used_kernel<<<grid(c, nf1), 256, 0, s>>>(nf1, m1.Fuv, keep, used);
    st = excl_scan(t, keep, fpos, nf1, s);
    if (st == EXM_OK) st = excl_scan(t, alive, vpos, nv1, s);
    if (st == EXM_OK) st = excl_scan(t, used, upos, nuv1, s);
    if (st != EXM_OK) return st;
    uint32_t h[6];
    st = read_u32(fpos + nf1 - 1, h, s);
    if (st == EXM_OK) st = read_u32(keep + nf1 - 1, h + 1, s);
    if (st == EXM_OK) st = read_u32(vpos + nv1 - 1, h + 2, s);
    if (st == EXM_OK) st = read_u32(alive + nv1 - 1, h + 3, s);
    if (st == EXM_OK) st = read_u32(upos + nuv1 - 1, h + 4, s);
    if (st == EXM_OK) st = read_u32(used + nuv1 - 1, h + 5, s);
    uint32_t merges = 0;
    if (st == EXM_OK) st = read_u32(cnt + 5, &merges, s);
    if (st != EXM_OK) return st;
    const int nf2 = (int)(h[0] + h[1]), nv2 = (int)(h[2] + h[3]), nuv2 = (int)(h[4] + h[5]);
    if (!ensure(&t->V, &t->cV, 3 * (size_t)nv2) || !ensure(&t->F, &t->cF, 3 * (size_t)nf2) ||
        !ensure(&t->UV, &t->cUV, 2 * (size_t)nuv2) || !ensure(&t->Fuv, &t->cFuv, 3 * (size_t)nf2) ||
        !ensure(&t->G, &t->cG, (size_t)nv2))
        return exm_fail(EXM_ERR_OOM, "topology result");
    compact_faces_kernel<<<grid(c, nf1), 256, 0, s>>>(nf1, m1.F, m1.Fuv, keep, fpos, vpos, upos, t->F, t->Fuv);
    compact_verts_kernel<<<grid(c, nv1), 256, 0, s>>>(nv1, m1.V, m1.G, alive, vpos, t->V, t->G);
    compact_uvs_kernel<<<grid(c, nuv1), 256, 0, s>>>(nuv1, m1.UV, used, upos, t->UV);
    c->launches += 7;
    st = exm_cuda_check(cudaStreamSynchronize(s), "topology round");
    if (st != EXM_OK) return st;
    t->nv = nv2;
    t->nf = nf2;
    t->nuv = nuv2;
    t->stats[0] = applied;
    t->stats[1] = (int)merges;
    t->stats[2] = nf1 - nf2;
    return EXM_OK;
}

exm_status exm_topology_result(exm_topology* t, int* nv, int* nf, int* nuv, const float** V, const int32_t** F,
                               const float** UV, const int32_t** Fuv, const float** ema, int stats[3]) {
    if (!t) return exm_fail(EXM_ERR_ARG, "exm_topology_result: NULL topology");
    if (nv) *nv = t->nv;
    if (nf) *nf = t->nf;
    if (nuv) *nuv = t->nuv;
    if (V) *V = t->V;
    if (F) *F = t->F;
    if (UV) *UV = t->UV;
    if (Fuv) *Fuv = t->Fuv;
    if (ema) *ema = t->G;
    if (stats) for (int k = 0; k < 3; ++k) stats[k] = t->stats[k];
    return EXM_OK;
}

}  // extern "C"
