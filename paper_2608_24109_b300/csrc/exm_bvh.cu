// Shadow-ray / secondary-ray acceleration structure (ray tracing of Sec. 5.2-5.3), built on
// the device: triangle centroids -> 30-bit Morton codes -> radix sort -> padded leaf boxes
// (so that the box test is conservative with respect to the watertight triangle test) ->
// binary hierarchy by locally-ordered clustering -> 4-wide nodes by a surface-area-greedy
// collapse.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cfloat>
#include <utility>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

__device__ __forceinline__ uint32_t f2o(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__global__ void centroid_bounds_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int nf, int nv,
                                       uint32_t* box, uint32_t* status) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {INFINITY, INFINITY, INFINITY};
    float cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (f < nf) {
        int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
            atomicOr(status, ERRBIT_INDEX);
        } else {
            for (int k = 0; k < 3; ++k) {
                float v = (V[3 * i0 + k] + V[3 * i1 + k] + V[3 * i2 + k]) * (1.0f / 3.0f);
                c[k] = v;
                cmax[k] = v;
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        float lo = c[k], hi = cmax[k];
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0 && lo <= hi) {
            atomicMin(box + k, f2o(lo));
            atomicMax(box + 3 + k, f2o(hi));
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void morton_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int nf, int nv,
                              const uint32_t* __restrict__ box, uint32_t* codes, uint32_t* ids) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    uint32_t code = 0;
    if (i0 >= 0 && i1 >= 0 && i2 >= 0 && i0 < nv && i1 < nv && i2 < nv) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float lo = o2f(box[k]), hi = o2f(box[3 + k]);
            float v = (V[3 * i0 + k] + V[3 * i1 + k] + V[3 * i2 + k]) * (1.0f / 3.0f);
            float ext = hi - lo;
            float u = ext > 0.0f ? (v - lo) / ext : 0.5f;
            q[k] = (uint32_t)fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);
        }
        code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    }
    codes[f] = code;
    ids[f] = (uint32_t)f;
}

__device__ __forceinline__ float pad_of(float lo, float hi) {
    return 2e-5f * (1.0f + fmaxf(fabsf(lo), fabsf(hi)));
}

__global__ void init_box_kernel(uint32_t* box) {
    int k = threadIdx.x;
    if (k < 3) box[k] = 0xffffffffu;
    else if (k < 6) box[k] = 0u;
}


// ---- Binary hierarchy by locally-ordered clustering (PLOC: Meister and Bittner, "Parallel
// locally-ordered clustering for bounding volume hierarchy construction", TVCG 2018).
// Clusters start as the leaves in Morton order.  Each round every cluster finds, among the
// kPlocR clusters on either side, the one whose merged box has the smallest surface
// (ties: the lower index); mutual nearest neighbours merge into a new internal node at
// the lower position and the cluster array is compacted.  Node ids are handed out from
// n-2 downwards in scan order, so the last merge, the root, is node 0.
constexpr int kDefaultLayout = EXM_BVH_4;  // the BVH layout of EXM_BVH_AUTO
constexpr int kDefaultCollapse = EXM_BVH_COLLAPSE_SAH;  // the 4-wide collapse of EXM_BVH_COLLAPSE_AUTO
constexpr int kPlocR = 16;
constexpr int kPlocBlock = 256;
constexpr int kPlocMaxRounds = 4096;

__device__ __forceinline__ float merged_half_area(const float* a, const float* b) {
    const float dx = fmaxf(a[3], b[3]) - fminf(a[0], b[0]);
    const float dy = fmaxf(a[4], b[4]) - fminf(a[1], b[1]);
    const float dz = fmaxf(a[5], b[5]) - fminf(a[2], b[2]);
    return dx * dy + dy * dz + dz * dx;
}

// Padded leaf boxes and triangle records in Morton order; the initial clusters (leaf ~k).
__global__ void leaf_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int n, int nv,
                            const uint32_t* __restrict__ ids_sorted, float* bounds, float4* tris, int32_t* clusters) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t f = ids_sorted[k];
    int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    i0 = min(max(i0, 0), nv - 1); i1 = min(max(i1, 0), nv - 1); i2 = min(max(i2, 0), nv - 1);
    float p[3][3];
    for (int c = 0; c < 3; ++c) { p[0][c] = V[3 * i0 + c]; p[1][c] = V[3 * i1 + c]; p[2][c] = V[3 * i2 + c]; }
    tris[tri_at(k, 0)] = make_float4(p[0][0], p[0][1], p[0][2], __int_as_float((int)f));
    tris[tri_at(k, 1)] = make_float4(p[1][0], p[1][1], p[1][2], 0.0f);
    tris[tri_at(k, 2)] = make_float4(p[2][0], p[2][1], p[2][2], 0.0f);
    tris[tri_at(k, 3)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float* b = bounds + 6 * (size_t)(n - 1 + k);
    for (int c = 0; c < 3; ++c) {
        const float lo = fminf(p[0][c], fminf(p[1][c], p[2][c])), hi = fmaxf(p[0][c], fmaxf(p[1][c], p[2][c]));
        const float pd = pad_of(lo, hi);
        b[c] = lo - pd;
        b[3 + c] = hi + pd;
    }
    clusters[k] = ~k;
}

__global__ void __launch_bounds__(kPlocBlock) ploc_nearest_kernel(int n, int m, const int32_t* __restrict__ C,
                                                                  const float* __restrict__ bounds, int32_t* nn) {
    __shared__ float box[(kPlocBlock + 2 * kPlocR) * 6];
    const int base = blockIdx.x * kPlocBlock - kPlocR;
    for (int t = threadIdx.x; t < kPlocBlock + 2 * kPlocR; t += blockDim.x) {
        const int g = base + t;
        if (g >= 0 && g < m) {
            const int c = C[g];
            const float* b = bounds + 6 * (size_t)(c < 0 ? n - 1 + ~c : c);
            for (int a = 0; a < 6; ++a) box[6 * t + a] = b[a];
        }
    }
    __syncthreads();
    const int i = blockIdx.x * kPlocBlock + threadIdx.x;
    if (i >= m) return;
    const float* bi = box + 6 * (threadIdx.x + kPlocR);
    float best = INFINITY;
    int bj = -1;
    for (int o = -kPlocR; o <= kPlocR; ++o) {
        const int j = i + o;
        if (o == 0 || j < 0 || j >= m) continue;
        const float a = fminf(merged_half_area(bi, box + 6 * (threadIdx.x + kPlocR + o)), FLT_MAX);  // NaN, inf -> FLT_MAX
        if (a < best) { best = a; bj = j; }  // ascending j: a tie keeps the lower index
    }
    nn[i] = bj;
}

// flag = merges << 32 | keeps: the lower cluster of a mutual pair merges, the upper one goes.
__global__ void ploc_flag_kernel(int m, const int32_t* __restrict__ nn, unsigned long long* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    flag[i] = ((unsigned long long)(mutual && i < j) << 32) | (unsigned long long)!(mutual && i > j);
}

__global__ void ploc_merge_kernel(int n, int m, int id_top, const int32_t* __restrict__ C,
                                  const int32_t* __restrict__ nn, const unsigned long long* __restrict__ flag,
                                  const unsigned long long* __restrict__ scan, int32_t* Cout, int32_t* child,
                                  float* bounds, uint32_t* totals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const unsigned long long f = flag[i], s = scan[i];
    if (i == m - 1) {
        totals[0] = (uint32_t)(s + f);
        totals[1] = (uint32_t)((s + f) >> 32);
    }
    if (!(f & 1ull)) return;
    int cl = C[i];
    if (f >> 32) {
        const int a = cl, b = C[nn[i]];
        const int id = id_top - (int)(s >> 32);
        child[2 * id] = a;
        child[2 * id + 1] = b;
        const int ia = a < 0 ? n - 1 + ~a : a, ib = b < 0 ? n - 1 + ~b : b;
        const float* ba = bounds + 6 * (size_t)ia;
        const float* bb = bounds + 6 * (size_t)ib;
        float* bn = bounds + 6 * (size_t)id;
        for (int c = 0; c < 3; ++c) {
            bn[c] = fminf(ba[c], bb[c]);
            bn[3 + c] = fmaxf(ba[3 + c], bb[3 + c]);
        }
        cl = id;
    }
    Cout[(uint32_t)s] = cl;
}

// ---- 4-wide collapse.  A 4-wide node starts from the two children of a binary node and
// opens the internal candidate with the largest box surface until it holds four (a node
// whose candidates are all leaves keeps fewer).  128-byte node: child boxes as lo.x[4] lo.y[4] lo.z[4] hi.x[4] hi.y[4] hi.z[4],
// then the four child references (>= 0: node, < 0: leaf ~k, kEmpty: unused slot).
constexpr int kEmpty4 = 0x7fffffff;
constexpr uint32_t kSahLeafBit = 1u << 9;  // sah_code: the binary node is cut as one leaf

__device__ __forceinline__ int bounds_index(int n, int c) { return c < 0 ? n - 1 + ~c : c; }

// Writes 4-wide node q with the given slots (binary nodes >= 0 or leaves ~k, in slot order);
// each internal slot becomes a new node, queued on the next frontier, unless the SAH collapse
// made it a leaf of several triangles (`leaf_span` non-null: its first record and count).
__device__ void emit4_node(int n, const int32_t* slots, int ns, const float* __restrict__ bounds, int q, int2* out,
                           uint32_t* n_out, uint32_t* n_nodes, float4* nodes4, const uint32_t* __restrict__ code = nullptr,
                           const int2* __restrict__ leaf_span = nullptr) {
    float v[6][4];
    int refs[4];
    for (int k = 0; k < 4; ++k) {
        if (k < ns) {
            const float* bb = bounds + 6 * (size_t)bounds_index(n, slots[k]);
            for (int a = 0; a < 6; ++a) v[a][k] = bb[a];
            if (slots[k] < 0) refs[k] = slots[k];
            else if (leaf_span && (code[slots[k]] & kSahLeafBit)) {
                const int2 sp = leaf_span[slots[k]];  // first triangle record, triangles
                refs[k] = ~(sp.x | ((sp.y - 1) << kLeafCountShift));
            } else {
                const uint32_t idx = atomicAdd(n_nodes, 1u);
                refs[k] = (int)idx;
                const uint32_t o = atomicAdd(n_out, 1u);
                out[o] = make_int2(slots[k], (int)idx);
            }
        } else {
            for (int a = 0; a < 3; ++a) { v[a][k] = 0.0f; v[3 + a][k] = 0.0f; }
            refs[k] = kEmpty4;
        }
    }
    for (int a = 0; a < 6; ++a) nodes4[node4_at(q, a)] = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
    nodes4[node4_at(q, 6)] = make_float4(__int_as_float(refs[0]), __int_as_float(refs[1]), __int_as_float(refs[2]),
                                         __int_as_float(refs[3]));
    nodes4[node4_at(q, 7)] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void collapse4_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                 const int2* __restrict__ in, const uint32_t* __restrict__ n_in, int2* out,
                                 uint32_t* n_out, uint32_t* n_nodes, float4* nodes4) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *n_in) return;
    const int b = in[t].x, q = in[t].y;
    int slots[4];
    int ns = 2;
    slots[0] = child[2 * b];
    slots[1] = child[2 * b + 1];
    while (ns < 4) {
        int pick = -1;
        float best = -1.0f;
        for (int k = 0; k < ns; ++k) {
            if (slots[k] < 0) continue;
            const float* bb = bounds + 6 * (size_t)slots[k];
            const float dx = bb[3] - bb[0], dy = bb[4] - bb[1], dz = bb[5] - bb[2];
            const float a = dx * dy + dy * dz + dz * dx;
            if (a > best) { best = a; pick = k; }
        }
        if (pick < 0) break;
        const int c = slots[pick];
        slots[pick] = child[2 * c];
        slots[ns++] = child[2 * c + 1];
    }
    emit4_node(n, slots, ns, bounds, q, out, n_out, n_nodes, nodes4);
}

// ---- SAH collapse (EXM_BVH_COLLAPSE=sah): the binary tree cut into 4-wide nodes by dynamic
// programming over slot counts (the collapse of Ylitie, Karras and Laine, HPG 2017, restated for
// four slots).  C(x, i) is the least expected cost of the subtree of x when it may take up to i
// slots of its parent node, with A(x) the surface area of x's box:
//   leaf x:      C(x, i) = c_tri A(x)
//   internal x:  D(x, k) = min over j = 1..k-1 of C(l, j) + C(r, k - j)   (l, r: its children)
//                C(x, 1) = c_node A(x) + D(x, 4)                          (x becomes a 4-wide node)
//                C(x, i) = min(C(x, 1), D(x, i)) for i = 2..4
// The costs are evaluated bottom-up: a thread per leaf climbs towards the root, and of the two
// threads that reach a binary node the second evaluates it.  The nodes are then emitted
// top-down, level by level, each 4-wide node's slots read back from the recorded choices.
// A binary node may also be cut as one leaf of its n <= kMaxLeafTris triangles when their records
// are consecutive, at c_tri n A(x) (sah_cost_kernel).  c_tri / c_node = 0.6 is the tracer's cost
// of a triangle test against a node visit (0.45 and 0.8 traced within 0.5% of it).
constexpr float kSahNode = 1.0f, kSahTri = 0.6f;

__device__ __forceinline__ float box_area(const float* bb) {
    const float dx = bb[3] - bb[0], dy = bb[4] - bb[1], dz = bb[5] - bb[2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void parents_kernel(int n, const int32_t* __restrict__ child, int32_t* parent_int, int32_t* parent_leaf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n - 1) return;
    if (b == 0) parent_int[0] = -1;
    for (int e = 0; e < 2; ++e) {
        const int c = child[2 * b + e];
        if (c >= 0) parent_int[c] = b;
        else parent_leaf[~c] = b;
    }
}

// C(c, i) of a child: a leaf's from its box, an internal node's from the table (written by
// another thread before its release; read through L2).
__device__ __forceinline__ float child_cost(int n, int c, int i, const float* __restrict__ bounds, const float4* cost) {
    if (c < 0) return kSahTri * box_area(bounds + 6 * (size_t)(n - 1 + ~c));
    const float4 v = __ldcg(cost + c);
    return i == 1 ? v.x : (i == 2 ? v.y : (i == 3 ? v.z : v.w));
}

// code[x]: bits 2(k-2)..2(k-2)+1 hold j - 1 of the best split of D(x, k), k = 2..4; bit 6 + i - 2
// is set when C(x, i) = C(x, 1) (x kept as one slot with i slots available), i = 2..4; bit 9
// (kSahLeafBit) when that one slot is a leaf of x's triangles rather than a 4-wide node.
// span[x]: x's first leaf (its triangle record, in leaf order) and leaf count, -1 for the first
// when x's leaves are not consecutive records.  A leaf of several triangles costs c_tri n A(x):
// all its triangles are tested when its box is hit.  It is allowed for up to kMaxLeafTris
// consecutive records, not at the root.
__global__ void sah_cost_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                const int32_t* __restrict__ parent_int, const int32_t* __restrict__ parent_leaf,
                                uint32_t* cnt, float4* cost, uint32_t* code, int2* span) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int b = parent_leaf[k];
    while (b >= 0) {
        __threadfence();                                  // release this thread's last node
        if (atomicAdd(cnt + b, 1u) == 0u) return;         // the other child is not evaluated yet
        __threadfence();                                  // acquire the other child's
        const int l = child[2 * b], r = child[2 * b + 1];
        float cl[5], cr[5];
        for (int i = 1; i <= 4; ++i) {
            cl[i] = child_cost(n, l, i, bounds, cost);
            cr[i] = child_cost(n, r, i, bounds, cost);
        }
        const int2 sl = l < 0 ? make_int2(~l, 1) : __ldcg(span + l);
        const int2 sr = r < 0 ? make_int2(~r, 1) : __ldcg(span + r);
        // consecutive records when both halves are and they abut (in either order)
        int first = -1;
        if (sl.x >= 0 && sr.x >= 0) {
            if (sl.x + sl.y == sr.x) first = sl.x;
            else if (sr.x + sr.y == sl.x) first = sr.x;
        }
        const int leaves = sl.y + sr.y;
        float D[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        int J[5] = {1, 1, 1, 1, 1};
        for (int kk = 2; kk <= 4; ++kk) {
            D[kk] = INFINITY;
            for (int j = 1; j < kk; ++j) {
                const float v = cl[j] + cr[kk - j];
                if (v < D[kk]) { D[kk] = v; J[kk] = j; }
            }
        }
        const float A = box_area(bounds + 6 * (size_t)b);
        float c1 = kSahNode * A + D[4];
        uint32_t cd = (uint32_t)(J[2] - 1) | ((uint32_t)(J[3] - 1) << 2) | ((uint32_t)(J[4] - 1) << 4);
        if (b != 0 && first >= 0 && leaves <= kMaxLeafTris) {
            const float cleaf = kSahTri * (float)leaves * A;
            if (cleaf < c1) { c1 = cleaf; cd |= kSahLeafBit; }
        }
        float C[5];
        C[1] = c1;
        for (int i = 2; i <= 4; ++i) {
            if (c1 <= D[i]) { C[i] = c1; cd |= 1u << (6 + i - 2); }
            else C[i] = D[i];
        }
        cost[b] = make_float4(C[1], C[2], C[3], C[4]);
        code[b] = cd;
        span[b] = make_int2(first, leaves);
        b = parent_int[b];
    }
}

__global__ void collapse4_sah_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                     const uint32_t* __restrict__ code, const int2* __restrict__ span,
                                     const int2* __restrict__ in, const uint32_t* __restrict__ n_in, int2* out,
                                     uint32_t* n_out, uint32_t* n_nodes, float4* nodes4) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *n_in) return;
    const int b = in[t].x, q = in[t].y;
    // the slots of D(b, 4): a stack of (subtree, slots it may take), at most 4 entries since
    // every entry takes at least one of the 4 slots
    int sx[4], si[4], sp = 0;
    const int j4 = (int)((code[b] >> 4) & 3u) + 1;
    sx[sp] = child[2 * b + 1]; si[sp++] = 4 - j4;
    sx[sp] = child[2 * b];     si[sp++] = j4;
    int slots[4];
    int ns = 0;
    while (sp > 0 && ns < 4) {
        --sp;
        const int x = sx[sp], i = si[sp];
        if (x < 0 || i == 1 || ((code[x] >> (6 + i - 2)) & 1u)) { slots[ns++] = x; continue; }
        const int j = (int)((code[x] >> (2 * (i - 2))) & 3u) + 1;
        sx[sp] = child[2 * x + 1]; si[sp++] = i - j;
        sx[sp] = child[2 * x];     si[sp++] = j;
    }
    emit4_node(n, slots, ns, bounds, q, out, n_out, n_nodes, nodes4, code, span);
}

// ---- 8-wide compressed nodes (the node format of Ylitie, Karras and Laine, "Efficient
// incoherent ray traversal on GPUs through compressed wide BVHs", HPG 2017).  A node holds up
// to eight children: its box origin p and per-axis power-of-two steps 2^e, and each child's box
// quantised to 8 bits per plane on that grid, rounded outwards (lo down, hi up), so a decoded
// box contains the child's (padded) box.  Internal children come first, in slots 0..ni-1, and
// are the consecutive nodes child_base + c; the triangle children follow, in slots ni..ni+nt-1,
// and are the consecutive triangle records tri_base + (c - ni).  80 bytes (5 x 16):
//   [0] p.x p.y p.z, ex | ey << 8 | ez << 16 (biased exponents of the steps)
//   [1] child_base, tri_base, ni | nt << 8, 0
//   [2] qlo.x[8] qlo.y[8]   [3] qlo.z[8] qhi.x[8]   [4] qhi.y[8] qhi.z[8]
// An empty slot has qlo = 255 and qhi = 0.

// Biased exponent e with 2^(e - 127) * div >= ext (ext > 0), within 1..253 (so that 2^-(e-127)
// is a normal float too).
__device__ __forceinline__ uint32_t step_exponent(float ext, float div = 255.0f) {
    const float x = __fdiv_ru(ext, div);
    const uint32_t b = __float_as_uint(x);
    uint32_t e = (b >> 23) & 0xffu;
    if (b & 0x7fffffu) ++e;
    return min(max(e, 1u), 253u);
}

__global__ void collapse8_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                 const int2* __restrict__ in, const uint32_t* __restrict__ n_in, int2* out,
                                 uint32_t* n_out, uint32_t* n_nodes, uint32_t* n_tris, const float4* __restrict__ tris_in,
                                 float4* tris_out, float4* nodes8) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *n_in) return;
    const int b = in[t].x, q = in[t].y;
    int slots[8];
    int ns = 2;
    slots[0] = child[2 * b];
    slots[1] = child[2 * b + 1];
    while (ns < 8) {
        int pick = -1;
        float best = -1.0f;
        for (int k = 0; k < ns; ++k) {
            if (slots[k] < 0) continue;
            const float* bb = bounds + 6 * (size_t)slots[k];
            const float dx = bb[3] - bb[0], dy = bb[4] - bb[1], dz = bb[5] - bb[2];
            const float a = dx * dy + dy * dz + dz * dx;
            if (a > best) { best = a; pick = k; }
        }
        if (pick < 0) break;
        const int c = slots[pick];
        slots[pick] = child[2 * c];
        slots[ns++] = child[2 * c + 1];
    }
    // internal children first, then the triangles
    int order[8], ni = 0, nt = 0;
    for (int k = 0; k < ns; ++k)
        if (slots[k] >= 0) order[ni++] = slots[k];
    for (int k = 0; k < ns; ++k)
        if (slots[k] < 0) order[ni + nt++] = slots[k];
    const uint32_t cbase = ni ? atomicAdd(n_nodes, (uint32_t)ni) : 0u;
    const uint32_t tbase = nt ? atomicAdd(n_tris, (uint32_t)nt) : 0u;
    for (int k = 0; k < ni; ++k) out[atomicAdd(n_out, 1u)] = make_int2(order[k], (int)(cbase + k));
    for (int k = 0; k < nt; ++k) {
        const int leaf = ~order[ni + k];
        for (int v = 0; v < kTri; ++v) tris_out[tri_at(tbase + k, v)] = tris_in[tri_at(leaf, v)];
    }
    // the node's grid: origin at its box's low corner, steps covering its extent in 255
    const float* nb = bounds + 6 * (size_t)b;
    uint32_t e[3];
    float inv_step[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = step_exponent(fmaxf(__fsub_ru(nb[3 + a], nb[a]), 1e-30f));
        inv_step[a] = __uint_as_float((254u - e[a]) << 23);  // 2^-(e - 127)
    }
    uint32_t qlo[3][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}}, qhi[3][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}};
    for (int k = 0; k < 8; ++k) {
        for (int a = 0; a < 3; ++a) {
            uint32_t lo = 255u, hi = 0u;
            if (k < ns) {
                const float* cb = bounds + 6 * (size_t)bounds_index(n, order[k]);
                const float l = floorf(__fmul_rd(__fsub_rd(cb[a], nb[a]), inv_step[a]));
                const float h = ceilf(__fmul_ru(__fsub_ru(cb[3 + a], nb[a]), inv_step[a]));
                lo = (uint32_t)fminf(fmaxf(l, 0.0f), 255.0f);
                hi = (uint32_t)fminf(fmaxf(h, 0.0f), 255.0f);
            }
            qlo[a][k >> 2] |= lo << (8 * (k & 3));
            qhi[a][k >> 2] |= hi << (8 * (k & 3));
        }
    }
    float4* N = nodes8 + kNode8 * (size_t)q;
    N[0] = make_float4(nb[0], nb[1], nb[2], __uint_as_float(e[0] | (e[1] << 8) | (e[2] << 16)));
    N[1] = make_float4(__uint_as_float(cbase), __uint_as_float(tbase), __uint_as_float((uint32_t)ni | ((uint32_t)nt << 8)),
                       0.0f);
    N[2] = make_float4(__uint_as_float(qlo[0][0]), __uint_as_float(qlo[0][1]), __uint_as_float(qlo[1][0]),
                       __uint_as_float(qlo[1][1]));
    N[3] = make_float4(__uint_as_float(qlo[2][0]), __uint_as_float(qlo[2][1]), __uint_as_float(qhi[0][0]),
                       __uint_as_float(qhi[0][1]));
    N[4] = make_float4(__uint_as_float(qhi[1][0]), __uint_as_float(qhi[1][1]), __uint_as_float(qhi[2][0]),
                       __uint_as_float(qhi[2][1]));
}

// A one-triangle mesh: a single 8-wide node holding triangle 0.
__global__ void single8_kernel(const float* __restrict__ bounds, const float4* __restrict__ tris_in, float4* tris_out,
                               float4* nodes8) {
    for (int v = 0; v < kTri; ++v) tris_out[v] = tris_in[v];
    uint32_t e[3];
    for (int a = 0; a < 3; ++a) e[a] = step_exponent(fmaxf(__fsub_ru(bounds[3 + a], bounds[a]), 1e-30f));
    // the child's box is the node's box: planes 0 and 255 contain it
    const uint32_t lo = 0x000000u | 0xffffff00u, hi = 0x000000ffu;
    float4* N = nodes8;
    N[0] = make_float4(bounds[0], bounds[1], bounds[2], __uint_as_float(e[0] | (e[1] << 8) | (e[2] << 16)));
    N[1] = make_float4(__uint_as_float(0u), __uint_as_float(0u), __uint_as_float(1u << 8), 0.0f);
    N[2] = make_float4(__uint_as_float(lo), __uint_as_float(0xffffffffu), __uint_as_float(lo), __uint_as_float(0xffffffffu));
    N[3] = make_float4(__uint_as_float(lo), __uint_as_float(0xffffffffu), __uint_as_float(hi), 0.0f);
    N[4] = make_float4(__uint_as_float(hi), 0.0f, __uint_as_float(hi), 0.0f);
}

__global__ void seed8_kernel(int2* in, uint32_t* n_in, uint32_t* n_nodes, uint32_t* n_tris) {
    in[0] = make_int2(0, 0);
    *n_in = 1;
    *n_nodes = 1;
    *n_tris = 0;
}

// A one-triangle mesh: a single 4-wide node holding leaf 0 (node 0: no skew).
__global__ void single4_kernel(const float* __restrict__ bounds, float4* nodes4) {
    for (int a = 0; a < 6; ++a) nodes4[node4_at(0, a)] = make_float4(bounds[a], 0.f, 0.f, 0.f);
    nodes4[node4_at(0, 6)] =
        make_float4(__int_as_float(~0), __int_as_float(kEmpty4), __int_as_float(kEmpty4), __int_as_float(kEmpty4));
    nodes4[node4_at(0, 7)] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Bounding sphere of the leaf triangles, for clipping rays: the centre is the middle of the
// root node's box, the radius the largest distance from it to a triangle vertex.  The stored
// R^2 is inflated by 2e-4 relative (far above the FP32 rounding of the distances), so that
// every point of every triangle lies inside the stored sphere.
__global__ void sphere_centre_kernel(const float4* __restrict__ nodes4, float4* sphere) {
    const float4* N = nodes4;  // the root, node 0
    const float* lo[3] = {&N[node4_at(0, 0)].x, &N[node4_at(0, 1)].x, &N[node4_at(0, 2)].x};
    const float* hi[3] = {&N[node4_at(0, 3)].x, &N[node4_at(0, 4)].x, &N[node4_at(0, 5)].x};
    const int* ref = reinterpret_cast<const int*>(&N[node4_at(0, 6)].x);
    float c[3];
    for (int a = 0; a < 3; ++a) {
        float l = INFINITY, h = -INFINITY;
        for (int k = 0; k < 4; ++k)
            if (ref[k] != kEmpty4) { l = fminf(l, lo[a][k]); h = fmaxf(h, hi[a][k]); }
        c[a] = 0.5f * (l + h);
    }
    *sphere = make_float4(c[0], c[1], c[2], 0.0f);
}

// ---- 4-wide nodes with quantised child boxes (EXM_BVH_4Q): the 4-wide tree above, each node
// re-encoded in 64 bytes (layout in exm_device.cuh).  Per node and axis the grid step is the
// smallest power of two with 250 steps covering the node's box (the union of its children's),
// raised while the box's top lies above 252 steps, and the origin p lies at least one step
// below the box (p = lo - step rounded down).  Each child plane is quantised outwards and
// widened by one more step: qlo = floor((lo - p) / step) - 1, qhi = ceil((hi - p) / step) + 1
// with the subtractions rounded down and up respectively, so that qlo >= 0, qhi <= 254 and the
// decoded box contains the child's FP32 box with a margin of one step on every side.  The
// traversal's folded plane evaluation (exm_shade.cu) is exact to half a step, so its box tests
// are conservative: they keep every box the FP32 node's test keeps.
__global__ void quant4_kernel(const float4* __restrict__ nodes4, uint32_t n_nodes, float4* __restrict__ nodesq) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_nodes) return;
    float pl[6][4];
    for (int a = 0; a < 6; ++a) {
        const float4 v = nodes4[node4_at(q, a)];
        pl[a][0] = v.x; pl[a][1] = v.y; pl[a][2] = v.z; pl[a][3] = v.w;
    }
    const float4 rv = nodes4[node4_at(q, 6)];
    const int ref[4] = {__float_as_int(rv.x), __float_as_int(rv.y), __float_as_int(rv.z), __float_as_int(rv.w)};
    float p[3], step[3];
    uint32_t qlo[3], qhi[3];
    for (int a = 0; a < 3; ++a) {
        float L = INFINITY, H = -INFINITY;
        for (int c = 0; c < 4; ++c)
            if (ref[c] != kEmpty4) { L = fminf(L, pl[a][c]); H = fmaxf(H, pl[3 + a][c]); }
        if (!(L <= H)) L = H = 0.0f;
        uint32_t e = step_exponent(fmaxf(__fsub_ru(H, L), 1e-30f), 250.0f);
        float st = __uint_as_float(e << 23), inv = __uint_as_float((254u - e) << 23), o = __fsub_rd(L, st);
        while (e < 253u && __fmul_ru(__fsub_ru(H, o), inv) > 252.0f) {
            ++e;
            st = __uint_as_float(e << 23);
            inv = __uint_as_float((254u - e) << 23);
            o = __fsub_rd(L, st);
        }
        p[a] = o;
        step[a] = st;
        qlo[a] = qhi[a] = 0u;
        for (int c = 0; c < 4; ++c) {
            uint32_t bl = 255u, bh = 0u;
            if (ref[c] != kEmpty4) {
                const float fl = floorf(__fmul_rd(__fsub_rd(pl[a][c], o), inv)) - 1.0f;
                const float fh = ceilf(__fmul_ru(__fsub_ru(pl[3 + a][c], o), inv)) + 1.0f;
                bl = (uint32_t)fminf(fmaxf(fl, 0.0f), 255.0f);
                bh = (uint32_t)fminf(fmaxf(fh, 0.0f), 255.0f);
            }
            qlo[a] |= bl << (8 * c);
            qhi[a] |= bh << (8 * c);
        }
    }
    nodesq[nodeq_at(q, 0)] = make_float4(p[0], p[1], p[2], step[0]);
    nodesq[nodeq_at(q, 1)] = rv;
    nodesq[nodeq_at(q, 2)] = make_float4(__uint_as_float(qlo[0]), __uint_as_float(qlo[1]), __uint_as_float(qlo[2]),
                                         __uint_as_float(qhi[0]));
    nodesq[nodeq_at(q, 3)] = make_float4(__uint_as_float(qhi[1]), __uint_as_float(qhi[2]), step[1], step[2]);
}

// The same centre from the binary root's box (the 8-wide build).
__global__ void sphere8_centre_kernel(const float* __restrict__ bounds, int n, float4* sphere) {
    const float* b = bounds + 6 * (size_t)(n > 1 ? 0 : n - 1);
    *sphere = make_float4(0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5]), 0.0f);
}

__global__ void sphere_radius_kernel(const float4* __restrict__ tris, int nf, float4* sphere) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 c = *sphere;
    float r2 = 0.0f;
    if (k < nf) {
        for (int v = 0; v < 3; ++v) {
            const float4 p = tris[tri_at(k, v)];
            const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        }
        r2 = r2 * 1.0002f + 1e-30f;
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if ((threadIdx.x & 31) == 0 && r2 > 0.0f) atomicMax(reinterpret_cast<unsigned int*>(&sphere->w), __float_as_uint(r2));
}

__global__ void seed4_kernel(int2* in, uint32_t* n_in, uint32_t* n_nodes) {
    in[0] = make_int2(0, 0);
    *n_in = 1;
    *n_nodes = 1;
}

}  // namespace exm

using namespace exm;

exm_status exm_bvh_build_impl(exm_mesh* m, cudaStream_t s) {
    ExmRange range("BVH build");
    int n = m->nf;
    if (!m->codes) {
        size_t nn = (size_t)n;
        size_t internal = (size_t)(n > 1 ? n - 1 : 1);
        bool ok = exm_malloc((void**)&m->codes, nn * 4) == cudaSuccess && exm_malloc((void**)&m->codes_sorted, nn * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->ids, nn * 4) == cudaSuccess && exm_malloc((void**)&m->ids_sorted, nn * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->child, 2 * internal * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->bounds, (2 * nn) * 6 * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->scene_box, 6 * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->tris, nn * kTri * sizeof(float4)) == cudaSuccess &&
                  exm_malloc((void**)&m->nodes4, internal * 8 * sizeof(float4)) == cudaSuccess &&
                  exm_malloc((void**)&m->sphere, sizeof(float4)) == cudaSuccess &&
                  exm_malloc((void**)&m->frontier, 2 * nn * sizeof(int2)) == cudaSuccess &&
                  exm_malloc((void**)&m->frontier_cnt, 4 * sizeof(uint32_t)) == cudaSuccess &&
                  exm_malloc((void**)&m->ploc_c, 2 * nn * 4) == cudaSuccess && exm_malloc((void**)&m->ploc_nn, nn * 4) == cudaSuccess &&
                  exm_malloc((void**)&m->ploc_flag, nn * 8) == cudaSuccess && exm_malloc((void**)&m->ploc_scan, nn * 8) == cudaSuccess;
        if (!ok) return exm_fail(EXM_ERR_OOM, "BVH buffers");
        size_t bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, bytes, m->codes, m->codes_sorted, m->ids, m->ids_sorted, n, 0, 30, s);
        if (exm_malloc((void**)&m->sort_tmp, bytes) != cudaSuccess) return exm_fail(EXM_ERR_OOM, "BVH sort scratch");
        m->sort_tmp_bytes = bytes;
        bytes = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, bytes, m->ploc_flag, m->ploc_scan, n, s);
        if (exm_malloc((void**)&m->scan_tmp, bytes) != cudaSuccess) return exm_fail(EXM_ERR_OOM, "BVH scan scratch");
        m->scan_tmp_bytes = bytes;
    }
    uint32_t* box = (uint32_t*)m->scene_box;
    init_box_kernel<<<1, 32, 0, s>>>(box);
    centroid_bounds_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, box, m->ctx->d_status);
    morton_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, box, m->codes, m->ids);
    size_t bytes = m->sort_tmp_bytes;
    cub::DeviceRadixSort::SortPairs(m->sort_tmp, bytes, m->codes, m->codes_sorted, m->ids, m->ids_sorted, n, 0, 30, s);
    leaf_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, m->ids_sorted, m->bounds, m->tris, m->ploc_c);
    if (n > 1) {
        int32_t* cin = m->ploc_c;
        int32_t* cout = m->ploc_c + n;
        uint32_t* tot = m->frontier_cnt;
        int mcl = n, merged = 0;
        for (int round = 0; mcl > 1; ++round) {
            if (round >= kPlocMaxRounds) return exm_fail(EXM_ERR_ARG, "BVH clustering did not converge");
            ploc_nearest_kernel<<<(mcl + kPlocBlock - 1) / kPlocBlock, kPlocBlock, 0, s>>>(n, mcl, cin, m->bounds,
                                                                                         m->ploc_nn);
            ploc_flag_kernel<<<exm_blocks(mcl, 256), 256, 0, s>>>(mcl, m->ploc_nn, m->ploc_flag);
            size_t sb = m->scan_tmp_bytes;
            cub::DeviceScan::ExclusiveSum(m->scan_tmp, sb, m->ploc_flag, m->ploc_scan, mcl, s);
            ploc_merge_kernel<<<exm_blocks(mcl, 256), 256, 0, s>>>(n, mcl, n - 2 - merged, cin, m->ploc_nn, m->ploc_flag,
                                                                   m->ploc_scan, cout, m->child, m->bounds, tot);
            uint32_t h[2] = {0u, 0u};
            if (cudaMemcpyAsync(h, tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return exm_cuda_check(cudaGetLastError(), "BVH clustering");
            if (h[1] == 0 || (int)h[1] > mcl / 2) return exm_fail(EXM_ERR_CUDA, "BVH clustering made no progress");
            merged += (int)h[1];
            mcl = (int)h[0];
            std::swap(cin, cout);
        }
    }
    // the node layout: 8-wide compressed nodes when asked for, else 4-wide ones (FP32 or quantised
    // boxes).  Measured on the three blob workloads (99K, 499K, 2M triangles), the 8-wide tree
    // visits 32% fewer nodes but its eight quantised boxes cost more instructions per visit: its
    // tracer took 20%, 8% and 1% longer than the FP32 4-wide tree.  The quantised 4-wide nodes
    // halve the node loads (L1 data-pipe use 74% -> 49% on the 2M-triangle tree) for 17% more
    // instructions, and the tracer, then issue-bound, took 8%, 6% and 4% longer.
    int layout = m->ctx->bvh_layout ? m->ctx->bvh_layout : kDefaultLayout;
    if (layout == EXM_BVH_8Q && (size_t)n >= (1u << 27)) layout = EXM_BVH_4Q;  // 8-wide stack entries: 24-bit node indices
    m->layout = layout;
    if (layout == EXM_BVH_8Q) {
        if (!m->nodes8) {
            const size_t nn = (size_t)n;
            if (exm_malloc((void**)&m->nodes8, nn * kNode8 * sizeof(float4)) != cudaSuccess ||
                exm_malloc((void**)&m->tris8, nn * kTri * sizeof(float4)) != cudaSuccess ||
                exm_malloc((void**)&m->n_tris8, 4) != cudaSuccess)
                return exm_fail(EXM_ERR_OOM, "BVH buffers (8-wide)");
        }
        if (n == 1) {
            single8_kernel<<<1, 1, 0, s>>>(m->bounds, m->tris, m->tris8, m->nodes8);
            m->n_nodes = 1;
        } else {
            int2* fin = m->frontier;
            int2* fout = m->frontier + n;
            uint32_t* cnt = m->frontier_cnt;  // [0] in, [1] out, [2] nodes
            seed8_kernel<<<1, 1, 0, s>>>(fin, cnt, cnt + 2, m->n_tris8);
            uint32_t n_in = 1;
            for (int level = 0; n_in > 0; ++level) {
                if (level + 1 > kStackSize8)
                    return exm_fail(EXM_ERR_TRAVERSAL_LIMIT, "BVH deeper than the traversal stack allows");
                cudaMemsetAsync(cnt + 1, 0, 4, s);
                collapse8_kernel<<<exm_blocks(n_in, 128), 128, 0, s>>>(n, m->child, m->bounds, fin, cnt, fout, cnt + 1,
                                                                      cnt + 2, m->n_tris8, m->tris, m->tris8, m->nodes8);
                cudaMemcpyAsync(cnt, cnt + 1, 4, cudaMemcpyDeviceToDevice, s);
                if (cudaMemcpyAsync(&n_in, cnt + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return exm_cuda_check(cudaGetLastError(), "BVH collapse");
                std::swap(fin, fout);
            }
            if (cudaMemcpyAsync(&m->n_nodes, cnt + 2, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return exm_cuda_check(cudaGetLastError(), "BVH node count");
        }
        sphere8_centre_kernel<<<1, 1, 0, s>>>(m->bounds, n, m->sphere);
        sphere_radius_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->tris, n, m->sphere);
        return exm_cuda_check(cudaGetLastError(), "BVH build launch");
    }
    // collapse to 4-wide nodes, level by level (the frontier size is read back per level): by the
    // SAH dynamic programme or by opening the largest child box (EXM_BVH_COLLAPSE)
    const bool sah = (m->ctx->bvh_collapse ? m->ctx->bvh_collapse : kDefaultCollapse) == EXM_BVH_COLLAPSE_SAH;
    if (sah && n > 1) {
        if (!m->sah_cost && (exm_malloc((void**)&m->sah_cost, (size_t)(n - 1) * sizeof(float4)) != cudaSuccess ||
                             exm_malloc((void**)&m->sah_code, (size_t)(n - 1) * sizeof(uint32_t)) != cudaSuccess ||
                             exm_malloc((void**)&m->sah_span, (size_t)(n - 1) * sizeof(int2)) != cudaSuccess))
            return exm_fail(EXM_ERR_OOM, "BVH buffers (SAH collapse)");
        // the clustering's scratch is free now: parents of internal nodes and leaves, and one
        // arrival counter per internal node
        int32_t* parent_int = m->ploc_c;
        uint32_t* arrivals = reinterpret_cast<uint32_t*>(m->ploc_c + n);
        int32_t* parent_leaf = m->ploc_nn;
        parents_kernel<<<exm_blocks(n - 1, 256), 256, 0, s>>>(n, m->child, parent_int, parent_leaf);
        cudaMemsetAsync(arrivals, 0, (size_t)(n - 1) * sizeof(uint32_t), s);
        sah_cost_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(n, m->child, m->bounds, parent_int, parent_leaf, arrivals,
                                                           m->sah_cost, m->sah_code, m->sah_span);
    }
    if (n == 1) {
        single4_kernel<<<1, 1, 0, s>>>(m->bounds, m->nodes4);
    } else {
        int2* fin = m->frontier;
        int2* fout = m->frontier + n;
        uint32_t* cnt = m->frontier_cnt;  // [0] in, [1] out, [2] nodes
        seed4_kernel<<<1, 1, 0, s>>>(fin, cnt, cnt + 2);
        uint32_t n_in = 1;
        int level = 0;
        for (; n_in > 0; ++level) {
            // the traversal stack holds at most 3 entries per level of the current path
            if (3 * (level + 1) > kStackSize4)
                return exm_fail(EXM_ERR_TRAVERSAL_LIMIT, "BVH deeper than the traversal stack allows");
            cudaMemsetAsync(cnt + 1, 0, 4, s);
            if (sah)
                collapse4_sah_kernel<<<exm_blocks(n_in, 128), 128, 0, s>>>(n, m->child, m->bounds, m->sah_code,
                                                                          m->sah_span, fin, cnt, fout, cnt + 1,
                                                                          cnt + 2, m->nodes4);
            else
                collapse4_kernel<<<exm_blocks(n_in, 128), 128, 0, s>>>(n, m->child, m->bounds, fin, cnt, fout, cnt + 1,
                                                                      cnt + 2, m->nodes4);
            cudaMemcpyAsync(cnt, cnt + 1, 4, cudaMemcpyDeviceToDevice, s);
            if (cudaMemcpyAsync(&n_in, cnt + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return exm_cuda_check(cudaGetLastError(), "BVH collapse");
            int2* tmp = fin;
            fin = fout;
            fout = tmp;
        }
    }
    if (n == 1) {
        m->n_nodes = 1;
    } else if (cudaMemcpyAsync(&m->n_nodes, m->frontier_cnt + 2, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        return exm_cuda_check(cudaGetLastError(), "BVH node count");
    }
    sphere_centre_kernel<<<1, 1, 0, s>>>(m->nodes4, m->sphere);
    sphere_radius_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->tris, n, m->sphere);
    if (layout == EXM_BVH_4Q) {
        if (!m->nodesq && exm_malloc((void**)&m->nodesq, (size_t)(n > 1 ? n - 1 : 1) * kNodeQ4 * sizeof(float4)) !=
                              cudaSuccess) {
            m->nodesq = nullptr;
            return exm_fail(EXM_ERR_OOM, "BVH buffers (quantised 4-wide)");
        }
        quant4_kernel<<<exm_blocks(m->n_nodes, 256), 256, 0, s>>>(m->nodes4, m->n_nodes, m->nodesq);
    }
    return exm_cuda_check(cudaGetLastError(), "BVH build launch");
}
