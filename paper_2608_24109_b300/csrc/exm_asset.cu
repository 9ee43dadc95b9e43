// Asset export and import: the resident part of a relightable asset -- the mesh-UV carrier
// (V, F, UV, Fuv: the fixed Stage-II carrier) and its ray-tracing BVH -- copied out to caller
// buffers and back in, so that a serving process can reload exported assets without building
// their BVH again.  Imports are checked before use: every index of the mesh and every node
// reference of the BVH must lie in range, so that no kernel reads outside the asset whatever
// the bytes were; a tree with a cycle passes this check, and the traversal's step and stack
// caps then end its rays with EXM_ERR_TRAVERSAL_LIMIT (exm_sync).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "exm_device.cuh"
#include "exm_internal.h"

namespace exm {

constexpr int kEmptyRef = 0x7fffffff;  // an unused child slot of a 4-wide node

// Range checks of an imported asset; bit 0: a mesh index, bit 1: a node reference, bit 2: a
// triangle record's original face id.  `nodes4`: 4-wide nodes (FP32 boxes, or quantised ones
// when `quant`), whose four child references are checked.
__global__ void asset_check_kernel(const int32_t* __restrict__ F, const int32_t* __restrict__ Fuv, int nf, int nv,
                                   int nuv, const float4* __restrict__ nodes4, bool quant, uint32_t n_nodes,
                                   const float4* __restrict__ tris, uint32_t* bad) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t b = 0;
    if (t < (uint32_t)nf) {
        for (int k = 0; k < 3; ++k) {
            const int i = F[3 * t + k], u = Fuv[3 * t + k];
            if (i < 0 || i >= nv || u < 0 || u >= nuv) b |= 1u;
        }
        if (tris) {
            const int id = __float_as_int(tris[tri_at(t, 0)].w);
            if (id < 0 || id >= nf) b |= 4u;
        }
    }
    if (nodes4 && t < n_nodes) {
        const float4 r = nodes4[quant ? nodeq_at(t, 1) : node4_at(t, 6)];
        const int ref[4] = {__float_as_int(r.x), __float_as_int(r.y), __float_as_int(r.z), __float_as_int(r.w)};
        for (int k = 0; k < 4; ++k) {
            const int c = ref[k];
            // a leaf: ~(k | (count - 1) << kLeafCountShift), records k .. k + count - 1
            const uint32_t lt = ~(uint32_t)c;
            const uint32_t k0 = lt & ((1u << kLeafCountShift) - 1u), cntl = (lt >> kLeafCountShift) + 1u;
            const bool ok = c == kEmptyRef || (c >= 0 && (uint32_t)c < n_nodes) ||
                            (c < 0 && cntl <= (uint32_t)kMaxLeafTris && (uint64_t)k0 + cntl <= (uint64_t)nf);
            if (!ok) b |= 2u;
        }
    }
    if (b) atomicOr(bad, b);
}

// The same for 8-wide compressed nodes: a node's node children child_base .. child_base + ni - 1
// and triangle records tri_base .. tri_base + nt - 1 must exist, with ni + nt <= 8.
__global__ void asset_check8_kernel(const float4* __restrict__ nodes8, uint32_t n_nodes, int nf, uint32_t* bad) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    const float4 w1 = nodes8[kNode8 * (size_t)t + 1];
    const uint64_t cb = __float_as_uint(w1.x), tb = __float_as_uint(w1.y);
    const uint32_t ni = __float_as_uint(w1.z) & 0xffu, nt = (__float_as_uint(w1.z) >> 8) & 0xffu;
    if (ni + nt > 8 || (ni && cb + ni > n_nodes) || (nt && tb + nt > (uint64_t)nf)) atomicOr(bad, 2u);
}

// The corrupt-asset injector: a cycle that every index check passes.  4-wide: the root's first
// node child becomes the root; 8-wide: the root becomes its own only child, with the root's box.
__global__ void asset_corrupt_kernel(float4* nodes, int layout) {
    if (layout == EXM_BVH_8Q) {  // the root becomes its own only child, with the root's box
        uint32_t* w = reinterpret_cast<uint32_t*>(nodes);
        w[4] = 0u;          // child_base
        w[6] = 1u;          // one node child, no triangles
        for (int k = 8; k < 14; ++k) w[k] = (k & 1) ? 0xffffffffu : 0xffffff00u;   // qlo: slot 0 at 0
        for (int k = 14; k < 20; ++k) w[k] = (k & 1) ? 0u : 0x000000ffu;          // qhi: slot 0 at 255
        return;
    }
    int* ref = reinterpret_cast<int*>(&nodes[layout == EXM_BVH_4Q ? nodeq_at(0, 1) : node4_at(0, 6)].x);
    for (int k = 0; k < 4; ++k)
        if (ref[k] >= 0 && ref[k] != kEmptyRef) {
            ref[k] = 0;
            return;
        }
}

}  // namespace exm

using namespace exm;

static uint32_t node_bytes_of(int layout) {
    return (layout == EXM_BVH_8Q ? kNode8 : (layout == EXM_BVH_4Q ? kNodeQ4 : 8)) * (uint32_t)sizeof(float4);
}

static float4* nodes_of(const exm_mesh* m) {
    return m->layout == EXM_BVH_8Q ? m->nodes8 : (m->layout == EXM_BVH_4Q ? m->nodesq : m->nodes4);
}

static void asset_sizes(const exm_mesh* m, uint64_t bytes[EXM_ASSET_SECTIONS]) {
    bytes[0] = (uint64_t)m->nv * 12;
    bytes[1] = (uint64_t)m->nf * 12;
    bytes[2] = (uint64_t)m->nuv * 8;
    bytes[3] = (uint64_t)m->nf * 12;
    bytes[4] = (uint64_t)m->n_nodes * node_bytes_of(m->layout);
    bytes[5] = (uint64_t)m->nf * kTri * sizeof(float4);
    bytes[6] = sizeof(float4);
}

extern "C" {

exm_status exm_mesh_export_info(const exm_mesh* m, exm_asset_info* info) {
    if (!m || !info) return exm_fail(EXM_ERR_ARG, "exm_mesh_export_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->version = EXM_ASSET_VERSION;
    info->node_bytes = node_bytes_of(m->layout);
    info->nv = m->nv;
    info->nf = m->nf;
    info->nuv = m->nuv;
    info->n_nodes = m->n_nodes;
    asset_sizes(m, info->bytes);
    return EXM_OK;
}

exm_status exm_mesh_export(const exm_mesh* m, void* const sections[EXM_ASSET_SECTIONS], void* stream) {
    if (!m || !sections) return exm_fail(EXM_ERR_ARG, "exm_mesh_export: NULL argument");
    for (int k = 0; k < EXM_ASSET_SECTIONS; ++k)
        if (!sections[k]) return exm_fail(EXM_ERR_ARG, "exm_mesh_export: NULL section");
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t bytes[EXM_ASSET_SECTIONS];
    asset_sizes(m, bytes);
    const void* src[EXM_ASSET_SECTIONS] = {m->V, m->F, m->UV, m->Fuv, nodes_of(m),
                                           m->layout == EXM_BVH_8Q ? m->tris8 : m->tris, m->sphere};
    for (int k = 0; k < EXM_ASSET_SECTIONS; ++k) {
        exm_status st = exm_cuda_check(cudaMemcpyAsync(sections[k], src[k], bytes[k], cudaMemcpyDefault, s),
                                       "exm_mesh_export copy");
        if (st != EXM_OK) return st;
    }
    return exm_cuda_check(cudaStreamSynchronize(s), "exm_mesh_export");
}

exm_status exm_mesh_import(exm_ctx* c, const exm_asset_info* info, const void* const sections[EXM_ASSET_SECTIONS],
                           void* stream, exm_mesh** out) {
    if (!out) return exm_fail(EXM_ERR_ARG, "exm_mesh_import: out is NULL");
    *out = nullptr;
    if (!c || !info || !sections) return exm_fail(EXM_ERR_ARG, "exm_mesh_import: NULL argument");
    for (int k = 0; k < EXM_ASSET_SECTIONS; ++k)
        if (!sections[k]) return exm_fail(EXM_ERR_ARG, "exm_mesh_import: NULL section");
    int layout = 0;
    for (const int l : {EXM_BVH_4, EXM_BVH_4Q, EXM_BVH_8Q})
        if (info->node_bytes == node_bytes_of(l)) layout = l;
    if (info->version != EXM_ASSET_VERSION || layout == 0)
        return exm_fail(EXM_ERR_ARG, "exm_mesh_import: asset version or node format differs from this library's");
    if (info->nv < 3 || info->nf < 1 || info->nuv < 3 || info->nf > (1 << 28) || info->nv > (1 << 28) ||
        info->nuv > (1 << 28) || info->n_nodes < 1 || info->n_nodes > (uint32_t)info->nf)
        return exm_fail(EXM_ERR_ARG, "exm_mesh_import: sizes");
    // a 4-wide tree over nf leaves has at most max(nf - 1, 1) nodes (the buffers hold that many)
    if (layout != EXM_BVH_8Q && info->n_nodes > (uint32_t)std::max(info->nf - 1, 1))
        return exm_fail(EXM_ERR_ARG, "exm_mesh_import: more 4-wide nodes than a tree over nf leaves has");
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    // staging copies of the carrier on the device, then the regular upload path (frames, BVH
    // buffers), whose BVH is replaced by the imported one
    void* dV = nullptr;
    void* dF = nullptr;
    void* dUV = nullptr;
    void* dFuv = nullptr;
    exm_mesh* m = nullptr;
    exm_status st = EXM_OK;
    const uint64_t nb[4] = {(uint64_t)info->nv * 12, (uint64_t)info->nf * 12, (uint64_t)info->nuv * 8,
                            (uint64_t)info->nf * 12};
    void** stage[4] = {&dV, &dF, &dUV, &dFuv};
    for (int k = 0; k < 4 && st == EXM_OK; ++k) {
        if (info->bytes[k] != nb[k]) st = exm_fail(EXM_ERR_ARG, "exm_mesh_import: section size");
        else if (exm_malloc(stage[k], nb[k]) != cudaSuccess) st = exm_fail(EXM_ERR_OOM, "exm_mesh_import: staging");
        else st = exm_cuda_check(cudaMemcpyAsync(*stage[k], sections[k], nb[k], cudaMemcpyDefault, s), "import copy");
    }
    uint32_t* bad = nullptr;
    if (st == EXM_OK && exm_malloc((void**)&bad, 4) != cudaSuccess) st = exm_fail(EXM_ERR_OOM, "exm_mesh_import");
    if (st == EXM_OK) {
        cudaMemsetAsync(bad, 0, 4, s);
        // the mesh indices first: the upload path's frame and BVH kernels read through them
        const int n = info->nf;
        asset_check_kernel<<<exm_blocks((size_t)n, 256), 256, 0, s>>>((const int32_t*)dF, (const int32_t*)dFuv, n,
                                                                      info->nv, info->nuv, nullptr, false, 0, nullptr,
                                                                      bad);
        uint32_t h = 0;
        st = exm_cuda_check(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s), "import check");
        if (st == EXM_OK) st = exm_cuda_check(cudaStreamSynchronize(s), "import check");
        if (st == EXM_OK && h) st = exm_fail(EXM_ERR_ARG, "exm_mesh_import: a mesh index is out of range");
    }
    if (st == EXM_OK)
        st = exm_mesh_create(c, (const float*)dV, info->nv, (const int32_t*)dF, info->nf, (const float*)dUV,
                             info->nuv, (const int32_t*)dFuv, stream, &m);
    if (st == EXM_OK) {
        uint64_t bytes[EXM_ASSET_SECTIONS];
        m->n_nodes = info->n_nodes;
        m->layout = layout;
        asset_sizes(m, bytes);
        for (int k = 4; k < EXM_ASSET_SECTIONS && st == EXM_OK; ++k)
            if (info->bytes[k] != bytes[k]) st = exm_fail(EXM_ERR_ARG, "exm_mesh_import: BVH section size");
        if (st == EXM_OK && layout == EXM_BVH_8Q && !m->nodes8 &&
            (exm_malloc((void**)&m->nodes8, (size_t)m->nf * kNode8 * sizeof(float4)) != cudaSuccess ||
             exm_malloc((void**)&m->tris8, (size_t)m->nf * kTri * sizeof(float4)) != cudaSuccess))
            st = exm_fail(EXM_ERR_OOM, "exm_mesh_import: BVH buffers");
        if (st == EXM_OK && layout == EXM_BVH_4Q && !m->nodesq &&
            exm_malloc((void**)&m->nodesq, (size_t)std::max(m->nf - 1, 1) * kNodeQ4 * sizeof(float4)) != cudaSuccess)
            st = exm_fail(EXM_ERR_OOM, "exm_mesh_import: BVH buffers");
        if (st == EXM_OK) {
            void* dst[3] = {nodes_of(m), layout == EXM_BVH_8Q ? m->tris8 : m->tris, m->sphere};
            for (int k = 0; k < 3 && st == EXM_OK; ++k)
                st = exm_cuda_check(cudaMemcpyAsync(dst[k], sections[4 + k], bytes[4 + k], cudaMemcpyDefault, s),
                                    "import BVH copy");
        }
        if (st == EXM_OK) {
            cudaMemsetAsync(bad, 0, 4, s);
            const size_t n = (size_t)std::max((uint32_t)m->nf, m->n_nodes);
            asset_check_kernel<<<exm_blocks(n, 256), 256, 0, s>>>(
                m->F, m->Fuv, m->nf, m->nv, m->nuv, layout == EXM_BVH_8Q ? nullptr : nodes_of(m), layout == EXM_BVH_4Q,
                m->n_nodes, layout == EXM_BVH_8Q ? m->tris8 : m->tris, bad);
            if (layout == EXM_BVH_8Q)
                asset_check8_kernel<<<exm_blocks(m->n_nodes, 256), 256, 0, s>>>(m->nodes8, m->n_nodes, m->nf, bad);
            uint32_t h = 0;
            st = exm_cuda_check(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s), "import check");
            if (st == EXM_OK) st = exm_cuda_check(cudaStreamSynchronize(s), "import check");
            if (st == EXM_OK && h)
                st = exm_fail(EXM_ERR_ARG, std::string("exm_mesh_import: ") +
                                               ((h & 2u) ? "a BVH node reference is out of range"
                                                         : "a BVH triangle record names no face"));
        }
        if (st == EXM_OK && exm_fault_take(kFaultCorrupt))
            asset_corrupt_kernel<<<1, 1, 0, s>>>(nodes_of(m), layout);
        if (st == EXM_OK) {
            m->stamp = exm_next_stamp();
            st = exm_cuda_check(cudaStreamSynchronize(s), "exm_mesh_import");
        }
        if (st != EXM_OK) {
            exm_mesh_destroy(m);
            m = nullptr;
        }
    }
    cudaFree(dV);
    cudaFree(dF);
    cudaFree(dUV);
    cudaFree(dFuv);
    cudaFree(bad);
    *out = m;
    return st;
}

}  // extern "C"
