// Shadow-ray / secondary-ray acceleration structure (ray tracing of Sec. 5.2-5.3): a linear
// BVH built on the device.  Triangle centroids -> 30-bit Morton codes -> radix sort ->
// binary hierarchy from the sorted codes (Karras, "Maximizing parallelism in the
// construction of BVHs, octrees and k-d trees", HPG 2012) -> bottom-up box refit ->
// 64-byte traversal nodes holding both child boxes, padded so that the box test is
// conservative with respect to the watertight triangle test.
#include <cub/device/device_radix_sort.cuh>

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

__device__ __forceinline__ int delta(const uint32_t* codes, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint32_t a = codes[i], b = codes[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

// Internal node i of n-1: its key range and split (Karras 2012).  Children: >= 0 internal,
// < 0 leaf ~k (k = sorted position).
__global__ void hierarchy_kernel(const uint32_t* __restrict__ codes, int n, int32_t* child, int32_t* parent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(codes, n, i, i - d);
    int lmax = 2;
    while (delta(codes, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(codes, n, i, j);
    int s = 0;
    int div = 2;
    int t;
    do {
        t = (l + div - 1) / div;
        if (delta(codes, n, i, i + (s + t) * d) > dnode) s += t;
        div <<= 1;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int left = (min(i, j) == gamma) ? ~gamma : gamma;
    int right = (max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    child[2 * i] = left;
    child[2 * i + 1] = right;
    // parent array: internal nodes 0..n-2, leaves at n-1+k
    parent[left < 0 ? (n - 1 + ~left) : left] = i;
    parent[right < 0 ? (n - 1 + ~right) : right] = i;
}

__device__ __forceinline__ float pad_of(float lo, float hi) {
    return 2e-5f * (1.0f + fmaxf(fabsf(lo), fabsf(hi)));
}

// Leaf boxes, triangle records in leaf order, then the bottom-up refit: the second thread
// to reach an internal node merges its children's boxes and continues upwards.
__global__ void refit_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, int n, int nv,
                             const uint32_t* __restrict__ ids_sorted, const int32_t* __restrict__ child,
                             const int32_t* __restrict__ parent, uint32_t* flags, float* bounds, float4* tris,
                             uint32_t* status) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t f = ids_sorted[k];
    int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    i0 = min(max(i0, 0), nv - 1); i1 = min(max(i1, 0), nv - 1); i2 = min(max(i2, 0), nv - 1);
    float p[3][3];
    for (int c = 0; c < 3; ++c) { p[0][c] = V[3 * i0 + c]; p[1][c] = V[3 * i1 + c]; p[2][c] = V[3 * i2 + c]; }
    tris[3 * k] = make_float4(p[0][0], p[0][1], p[0][2], __int_as_float((int)f));
    tris[3 * k + 1] = make_float4(p[1][0], p[1][1], p[1][2], 0.0f);
    tris[3 * k + 2] = make_float4(p[2][0], p[2][1], p[2][2], 0.0f);
    int leaf = n - 1 + k;
    float* b = bounds + 6 * (size_t)leaf;
    for (int c = 0; c < 3; ++c) {
        float lo = fminf(p[0][c], fminf(p[1][c], p[2][c])), hi = fmaxf(p[0][c], fmaxf(p[1][c], p[2][c]));
        float pd = pad_of(lo, hi);
        b[c] = lo - pd;
        b[3 + c] = hi + pd;
    }
    if (n == 1) return;
    int node = parent[leaf];
    for (int guard = 0; node >= 0; ++guard) {
        if (guard > 256) { atomicOr(status, ERRBIT_TRAVERSAL); return; }
        __threadfence();
        if (atomicAdd(flags + node, 1u) == 0) return;
        __threadfence();
        int l = child[2 * node], r = child[2 * node + 1];
        const volatile float* bl = bounds + 6 * (size_t)(l < 0 ? n - 1 + ~l : l);
        const volatile float* br = bounds + 6 * (size_t)(r < 0 ? n - 1 + ~r : r);
        volatile float* bn = bounds + 6 * (size_t)node;
        for (int c = 0; c < 3; ++c) {
            bn[c] = fminf(bl[c], br[c]);
            bn[3 + c] = fmaxf(bl[3 + c], br[3 + c]);
        }
        node = node == 0 ? -1 : parent[node];
    }
}

__global__ void write_nodes_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                   float4* nodes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int l = child[2 * i], r = child[2 * i + 1];
    const float* bl = bounds + 6 * (size_t)(l < 0 ? n - 1 + ~l : l);
    const float* br = bounds + 6 * (size_t)(r < 0 ? n - 1 + ~r : r);
    nodes[4 * i] = make_float4(bl[0], bl[1], bl[2], bl[3]);
    nodes[4 * i + 1] = make_float4(bl[4], bl[5], br[0], br[1]);
    nodes[4 * i + 2] = make_float4(br[2], br[3], br[4], br[5]);
    nodes[4 * i + 3] = make_float4(__int_as_float(l), __int_as_float(r), 0.0f, 0.0f);
}

// A one-triangle mesh: a single node whose two children are both leaf 0.
__global__ void single_node_kernel(const float* __restrict__ bounds, float4* nodes) {
    const float* b = bounds;
    nodes[0] = make_float4(b[0], b[1], b[2], b[3]);
    nodes[1] = make_float4(b[4], b[5], b[0], b[1]);
    nodes[2] = make_float4(b[2], b[3], b[4], b[5]);
    nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), 0.0f, 0.0f);
}

__global__ void init_box_kernel(uint32_t* box) {
    int k = threadIdx.x;
    if (k < 3) box[k] = 0xffffffffu;
    else if (k < 6) box[k] = 0u;
}


// ---- 4-wide collapse.  A 4-wide node takes the grandchildren of a binary node (a leaf child
// stays a leaf).  128-byte node: child boxes as lo.x[4] lo.y[4] lo.z[4] hi.x[4] hi.y[4] hi.z[4],
// then the four child references (>= 0: node, < 0: leaf ~k, kEmpty: unused slot).
constexpr int kEmpty4 = 0x7fffffff;

__device__ __forceinline__ int bounds_index(int n, int c) { return c < 0 ? n - 1 + ~c : c; }

__global__ void collapse4_kernel(int n, const int32_t* __restrict__ child, const float* __restrict__ bounds,
                                 const int2* __restrict__ in, const uint32_t* __restrict__ n_in, int2* out,
                                 uint32_t* n_out, uint32_t* n_nodes, float4* nodes4) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *n_in) return;
    const int b = in[t].x, q = in[t].y;
    int slots[4];
    int ns = 0;
    for (int h = 0; h < 2; ++h) {
        const int c = child[2 * b + h];
        if (c < 0) slots[ns++] = c;
        else { slots[ns++] = child[2 * c]; slots[ns++] = child[2 * c + 1]; }
    }
    float v[6][4];
    int refs[4];
    for (int k = 0; k < 4; ++k) {
        if (k < ns) {
            const float* bb = bounds + 6 * (size_t)bounds_index(n, slots[k]);
            for (int a = 0; a < 6; ++a) v[a][k] = bb[a];
            if (slots[k] < 0) refs[k] = slots[k];
            else {
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
    float4* N = nodes4 + 8 * (size_t)q;
    for (int a = 0; a < 6; ++a) N[a] = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
    N[6] = make_float4(__int_as_float(refs[0]), __int_as_float(refs[1]), __int_as_float(refs[2]), __int_as_float(refs[3]));
    N[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// A one-triangle mesh: a single 4-wide node holding leaf 0.
__global__ void single4_kernel(const float* __restrict__ bounds, float4* nodes4) {
    float4* N = nodes4;
    for (int a = 0; a < 6; ++a) N[a] = make_float4(bounds[a], 0.f, 0.f, 0.f);
    N[6] = make_float4(__int_as_float(~0), __int_as_float(kEmpty4), __int_as_float(kEmpty4), __int_as_float(kEmpty4));
    N[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void seed4_kernel(int2* in, uint32_t* n_in, uint32_t* n_nodes) {
    in[0] = make_int2(0, 0);
    *n_in = 1;
    *n_nodes = 1;
}

}  // namespace exm

using namespace exm;

exm_status exm_bvh_build_impl(exm_mesh* m, cudaStream_t s) {
    int n = m->nf;
    if (!m->codes) {
        size_t nn = (size_t)n;
        size_t internal = (size_t)(n > 1 ? n - 1 : 1);
        bool ok = cudaMalloc(&m->codes, nn * 4) == cudaSuccess && cudaMalloc(&m->codes_sorted, nn * 4) == cudaSuccess &&
                  cudaMalloc(&m->ids, nn * 4) == cudaSuccess && cudaMalloc(&m->ids_sorted, nn * 4) == cudaSuccess &&
                  cudaMalloc(&m->parent, (2 * nn) * 4) == cudaSuccess &&
                  cudaMalloc(&m->child, 2 * internal * 4) == cudaSuccess &&
                  cudaMalloc(&m->flags, internal * 4) == cudaSuccess &&
                  cudaMalloc(&m->bounds, (2 * nn) * 6 * 4) == cudaSuccess &&
                  cudaMalloc(&m->scene_box, 6 * 4) == cudaSuccess &&
                  cudaMalloc(&m->nodes, internal * 4 * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&m->tris, nn * 3 * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&m->nodes4, internal * 8 * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&m->frontier, 2 * nn * sizeof(int2)) == cudaSuccess &&
                  cudaMalloc(&m->frontier_cnt, 4 * sizeof(uint32_t)) == cudaSuccess;
        if (!ok) return exm_fail(EXM_ERR_OOM, "BVH buffers");
        size_t bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, bytes, m->codes, m->codes_sorted, m->ids, m->ids_sorted, n, 0, 30, s);
        if (cudaMalloc(&m->sort_tmp, bytes) != cudaSuccess) return exm_fail(EXM_ERR_OOM, "BVH sort scratch");
        m->sort_tmp_bytes = bytes;
    }
    uint32_t* box = (uint32_t*)m->scene_box;
    init_box_kernel<<<1, 32, 0, s>>>(box);
    centroid_bounds_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, box, m->ctx->d_status);
    morton_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, box, m->codes, m->ids);
    size_t bytes = m->sort_tmp_bytes;
    cub::DeviceRadixSort::SortPairs(m->sort_tmp, bytes, m->codes, m->codes_sorted, m->ids, m->ids_sorted, n, 0, 30, s);
    cudaMemsetAsync(m->parent, 0xff, (size_t)2 * n * 4, s);
    if (n > 1) {
        cudaMemsetAsync(m->flags, 0, (size_t)(n - 1) * 4, s);
        hierarchy_kernel<<<exm_blocks(n - 1, 256), 256, 0, s>>>(m->codes_sorted, n, m->child, m->parent);
    }
    refit_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(m->V, m->F, n, m->nv, m->ids_sorted, m->child, m->parent,
                                                   m->flags, m->bounds, m->tris, m->ctx->d_status);
    if (n > 1)
        write_nodes_kernel<<<exm_blocks(n - 1, 256), 256, 0, s>>>(n, m->child, m->bounds, m->nodes);
    else
        single_node_kernel<<<1, 1, 0, s>>>(m->bounds, m->nodes);
    // collapse to 4-wide nodes, level by level (the frontier size is read back per level)
    if (n == 1) {
        single4_kernel<<<1, 1, 0, s>>>(m->bounds, m->nodes4);
    } else {
        int2* fin = m->frontier;
        int2* fout = m->frontier + n;
        uint32_t* cnt = m->frontier_cnt;  // [0] in, [1] out, [2] nodes
        seed4_kernel<<<1, 1, 0, s>>>(fin, cnt, cnt + 2);
        uint32_t n_in = 1;
        for (int level = 0; level < 64 && n_in > 0; ++level) {
            cudaMemsetAsync(cnt + 1, 0, 4, s);
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
    return exm_cuda_check(cudaGetLastError(), "BVH build launch");
}
