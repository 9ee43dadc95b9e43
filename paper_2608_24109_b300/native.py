"""ctypes binding of libexmesh (include/exmesh.h): argument marshalling only.

Every entry point keeps its C name.  Device buffers are torch CUDA tensors (their
data_ptr() is passed); streams are torch.cuda streams (their cuda_stream handle).  The
library is loaded from this package's directory; if it is missing the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexmesh.so")

EXM_OK = 0
EXM_ERR_ARG = -1
EXM_ERR_OOM = -2
EXM_ERR_CUDA = -3
EXM_ERR_GUARDBAND = -4
EXM_ERR_TRAVERSAL_LIMIT = -5
EXM_ERR_TIMEOUT = -6
EXM_ERR_BUSY = -7
EXM_ERR_QUEUE_OVERFLOW = -8
EXM_ERR_CANCELLED = -9
FAULT_ALLOC, FAULT_ADMIT, FAULT_SLOW, FAULT_CANCEL, FAULT_CORRUPT = 1, 2, 3, 4, 5
ASSET_VERSION = 4
BVH_AUTO, BVH_4, BVH_4Q, BVH_8Q = 0, 1, 2, 3
BVH_COLLAPSE_AUTO, BVH_COLLAPSE_GREEDY, BVH_COLLAPSE_SAH = 0, 1, 2
ASSET_SECTIONS = 7

EXM_F32, EXM_BF16, EXM_F16 = 0, 1, 2
FLAG_WRAP_U = 1
FLAG_NO_METALLIC = 2
FLAG_COUNT_WORK = 4
FLAG_ZERO_GRADS = 8
FLAG_TIME_KERNELS = 16
FLAG_NO_SECONDARY_MATERIAL = 32
FLAG_HALF_RES_INDIRECT = 64
FLAG_RECOMPUTE = 128

EXPORTS = [
    "exm_create", "exm_destroy", "exm_last_error", "exm_sync", "exm_debug_fault", "exm_ctx_set_bvh_width",
    "exm_ctx_set_bvh_layout", "exm_ctx_set_bvh_collapse",
    "exm_mesh_create", "exm_mesh_update_vertices", "exm_bvh_build", "exm_mesh_destroy", "exm_mesh_frames",
    "exm_mesh_export_info", "exm_mesh_export", "exm_mesh_import",
    "exm_env_create", "exm_env_prepare", "exm_env_destroy", "exm_env_total",
    "exm_frame_create", "exm_frame_destroy", "exm_frame_set_limits", "exm_frame_stats", "exm_frame_work", "exm_frame_kernel_ms",
    "exm_launch_count", "exm_frame_visbuf", "exm_frame_saved_state",
    "exm_render_forward", "exm_render_backward", "exm_render_backward_noalloc", "exm_l1_loss",
    "exm_server_create", "exm_server_destroy", "exm_server_add_asset", "exm_relight_submit", "exm_relight_poll",
    "exm_server_progress", "exm_server_stats", "exm_relight_footprint", "exm_relight_cancel", "exm_relight_wait",
    "exm_server_batches",
    "exm_image_loss", "exm_material_tv", "exm_env_regularizers", "exm_adam_step",
    "exm_topology_create", "exm_topology_destroy", "exm_face_render_counts", "exm_topology_round",
    "exm_topology_result",
]


class ExmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libexmesh error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("n_direct", ctypes.c_int32), ("n_bounce", ctypes.c_int32), ("n_light", ctypes.c_int32),
                ("lambda_ind", ctypes.c_float), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class TopologyParams(ctypes.Structure):
    _fields_ = [("beta_g", ctypes.c_float), ("w_g", ctypes.c_float), ("w_k", ctypes.c_float),
                ("tau_degen", ctypes.c_float), ("tau_uv", ctypes.c_float), ("split_percent", ctypes.c_int32),
                ("max_faces", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RelightReq(ctypes.Structure):
    _fields_ = [("asset", ctypes.c_int32), ("views", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("env", ctypes.c_void_p), ("env_dtype", ctypes.c_int),
                ("env_w", ctypes.c_int32), ("env_h", ctypes.c_int32), ("cams", ctypes.c_void_p), ("params", Params),
                ("out_rgb", ctypes.c_void_p)]


class AssetInfo(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("node_bytes", ctypes.c_uint32), ("nv", ctypes.c_int32),
                ("nf", ctypes.c_int32), ("nuv", ctypes.c_int32), ("n_nodes", ctypes.c_uint32),
                ("bytes", ctypes.c_uint64 * ASSET_SECTIONS)]


_lib = None


def lib():
    """Loads libexmesh.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libexmesh.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, U64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "exm_create": ([I, PP], I),
        "exm_destroy": ([P], None),
        "exm_last_error": ([], ctypes.c_char_p),
        "exm_sync": ([P, P], I),
        "exm_debug_fault": ([I, ctypes.c_uint32], I),
        "exm_ctx_set_bvh_width": ([P, I], I),
        "exm_ctx_set_bvh_layout": ([P, I], I),
        "exm_ctx_set_bvh_collapse": ([P, I], I),
        "exm_mesh_export_info": ([P, ctypes.POINTER(AssetInfo)], I),
        "exm_mesh_export": ([P, ctypes.POINTER(ctypes.c_void_p * ASSET_SECTIONS), P], I),
        "exm_mesh_import": ([P, ctypes.POINTER(AssetInfo), ctypes.POINTER(ctypes.c_void_p * ASSET_SECTIONS), P, PP], I),
        "exm_relight_cancel": ([P, U64], I),
        "exm_relight_wait": ([P, U64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], I),
        "exm_server_batches": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64)], I),
        "exm_mesh_create": ([P, P, I, P, I, P, I, P, P, PP], I),
        "exm_mesh_update_vertices": ([P, P, P], I),
        "exm_bvh_build": ([P, P], I),
        "exm_mesh_destroy": ([P], None),
        "exm_mesh_frames": ([P, PP, PP], I),
        "exm_env_create": ([P, I, I, PP], I),
        "exm_env_prepare": ([P, P, I, P], I),
        "exm_env_destroy": ([P], None),
        "exm_env_total": ([P, ctypes.POINTER(U64)], I),
        "exm_frame_create": ([P, I, I, I, PP], I),
        "exm_frame_destroy": ([P], None),
        "exm_frame_set_limits": ([P, ctypes.c_uint32, U64], I),
        "exm_frame_stats": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64)], I),
        "exm_frame_work": ([P, ctypes.POINTER(U64 * 4)], I),
        "exm_frame_kernel_ms": ([P, ctypes.POINTER(ctypes.c_float * 4)], I),
        "exm_launch_count": ([P, ctypes.POINTER(U64)], I),
        "exm_frame_visbuf": ([P, PP], I),
        "exm_frame_saved_state": ([P, PP, PP, PP, ctypes.POINTER(I * 4)], I),
        "exm_render_forward": ([P, P, P, I, I, I, P, P, I, ctypes.POINTER(Params), P, P, P], I),
        "exm_render_backward": ([P, P, P, I, I, I, P, P, I, ctypes.POINTER(Params), P, P, P, P, P, P], I),
        "exm_render_backward_noalloc": ([P, P, P, I, I, I, P, P, I, ctypes.POINTER(Params), P, P, P, P, P], I),
        "exm_l1_loss": ([P, P, I64, P, P, P], I),
        "exm_server_create": ([P, U64, I, PP], I),
        "exm_server_destroy": ([P], None),
        "exm_server_add_asset": ([P, P, P, I, I, I, ctypes.POINTER(ctypes.c_int32)], I),
        "exm_relight_submit": ([P, ctypes.POINTER(RelightReq), ctypes.POINTER(U64)], I),
        "exm_relight_poll": ([P, U64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], I),
        "exm_server_progress": ([P], I),
        "exm_server_stats": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64),
                              ctypes.POINTER(U64)], I),
        "exm_relight_footprint": ([P, ctypes.POINTER(RelightReq), ctypes.POINTER(U64)], I),
        "exm_image_loss": ([P, P, P, I, I, I, F, P, P, P], I),
        "exm_material_tv": ([P, P, I, I, I, P, ctypes.c_uint32, F, P, P, P], I),
        "exm_env_regularizers": ([P, P, I, I, F, F, P, P, P], I),
        "exm_adam_step": ([P, P, P, P, P, I64, I, F, F, F, F, I, ctypes.POINTER(F), ctypes.POINTER(F), P], I),
        "exm_topology_create": ([P, PP], I),
        "exm_topology_destroy": ([P], None),
        "exm_face_render_counts": ([P, I, P, P], I),
        "exm_topology_round": ([P, P, I, P, I, P, I, P, P, P, P, ctypes.POINTER(TopologyParams), P], I),
        "exm_topology_result": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), PP, PP, PP, PP, PP,
                                 ctypes.POINTER(I * 3)], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def check(code):
    if code != EXM_OK:
        raise ExmError(code, lib().exm_last_error().decode(errors="replace"))
    return code


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def dtype_code(dt):
    import torch
    return {torch.float32: EXM_F32, torch.bfloat16: EXM_BF16, torch.float16: EXM_F16}[dt]


def _cams(cams):
    a = np.ascontiguousarray(cams, dtype=np.float32)
    assert a.ndim == 2 and a.shape[1] == 20, "cameras: float32 [views, 20]"
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ entry points

def exm_create(device: int = 0):
    h = ctypes.c_void_p()
    check(lib().exm_create(device, ctypes.byref(h)))
    return h


def exm_destroy(ctx):
    lib().exm_destroy(ctx)


def exm_sync(ctx, stream=None):
    return check(lib().exm_sync(ctx, _stream(stream)))


def exm_ctx_set_bvh_width(ctx, width):
    return check(lib().exm_ctx_set_bvh_width(ctx, int(width)))


def exm_ctx_set_bvh_layout(ctx, layout):
    return check(lib().exm_ctx_set_bvh_layout(ctx, int(layout)))


def exm_ctx_set_bvh_collapse(ctx, mode):
    return check(lib().exm_ctx_set_bvh_collapse(ctx, int(mode)))


def exm_debug_fault(kind, count):
    return check(lib().exm_debug_fault(int(kind), int(count)))


def exm_mesh_export_info(mesh):
    info = AssetInfo()
    check(lib().exm_mesh_export_info(mesh, ctypes.byref(info)))
    return info


def exm_mesh_export(mesh, sections, stream=None):
    """Copies the asset's sections into `sections` (ASSET_SECTIONS buffers: numpy arrays or
    torch tensors of info.bytes bytes each)."""
    ptrs = (ctypes.c_void_p * ASSET_SECTIONS)(*[_addr(x) for x in sections])
    return check(lib().exm_mesh_export(mesh, ctypes.byref(ptrs), _stream(stream)))


def exm_mesh_import(ctx, info: AssetInfo, sections, stream=None):
    ptrs = (ctypes.c_void_p * ASSET_SECTIONS)(*[_addr(x) for x in sections])
    h = ctypes.c_void_p()
    check(lib().exm_mesh_import(ctx, ctypes.byref(info), ctypes.byref(ptrs), _stream(stream), ctypes.byref(h)))
    return h


def _addr(x):
    """Address of a host numpy array or of a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()


def exm_mesh_create(ctx, V, F, UV, Fuv, stream=None):
    for t, n in ((V, "V"), (F, "F"), (UV, "UV"), (Fuv, "Fuv")):
        assert t.is_cuda and t.is_contiguous(), f"{n} must be a contiguous CUDA tensor"
    h = ctypes.c_void_p()
    check(lib().exm_mesh_create(ctx, _ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(UV), UV.shape[0], _ptr(Fuv),
                                _stream(stream), ctypes.byref(h)))
    return h


def exm_mesh_update_vertices(mesh, V, stream=None):
    return check(lib().exm_mesh_update_vertices(mesh, _ptr(V), _stream(stream)))


def exm_bvh_build(mesh, stream=None):
    return check(lib().exm_bvh_build(mesh, _stream(stream)))


def exm_mesh_destroy(mesh):
    lib().exm_mesh_destroy(mesh)


def exm_mesh_frames(mesh):
    n, t = ctypes.c_void_p(), ctypes.c_void_p()
    check(lib().exm_mesh_frames(mesh, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def exm_env_create(ctx, W, H):
    h = ctypes.c_void_p()
    check(lib().exm_env_create(ctx, W, H, ctypes.byref(h)))
    return h


def exm_env_prepare(env, E, stream=None):
    assert E.is_cuda and E.is_contiguous()
    return check(lib().exm_env_prepare(env, _ptr(E), dtype_code(E.dtype), _stream(stream)))


def exm_env_destroy(env):
    lib().exm_env_destroy(env)


def exm_env_total(env):
    q = ctypes.c_uint64()
    check(lib().exm_env_total(env, ctypes.byref(q)))
    return q.value


def exm_frame_create(ctx, views, W, H):
    h = ctypes.c_void_p()
    check(lib().exm_frame_create(ctx, views, W, H, ctypes.byref(h)))
    return h


def exm_frame_destroy(frame):
    lib().exm_frame_destroy(frame)


def exm_frame_set_limits(frame, ray_cap=0, saved_budget_bytes=0):
    return check(lib().exm_frame_set_limits(frame, int(ray_cap), int(saved_budget_bytes)))


def exm_frame_stats(frame):
    c, s = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().exm_frame_stats(frame, ctypes.byref(c), ctypes.byref(s)))
    return c.value, s.value


def exm_frame_work(frame):
    c = (ctypes.c_uint64 * 4)()
    check(lib().exm_frame_work(frame, ctypes.byref(c)))
    return list(c)


def exm_frame_kernel_ms(frame):
    ms = (ctypes.c_float * 4)()
    check(lib().exm_frame_kernel_ms(frame, ctypes.byref(ms)))
    return list(ms)


def exm_launch_count(ctx):
    n = ctypes.c_uint64()
    check(lib().exm_launch_count(ctx, ctypes.byref(n)))
    return n.value


def exm_frame_visbuf(frame):
    p = ctypes.c_void_p()
    check(lib().exm_frame_visbuf(frame, ctypes.byref(p)))
    return p.value


def exm_frame_saved_state(frame):
    """(pixels, visbits, hits) DEVICE addresses and dims (direct words, secondary words, N_b, rows)."""
    ptrs = [ctypes.c_void_p() for _ in range(3)]
    dims = (ctypes.c_int * 4)()
    check(lib().exm_frame_saved_state(frame, *[ctypes.byref(p) for p in ptrs], ctypes.byref(dims)))
    return [p.value for p in ptrs], list(dims)


def exm_render_forward(ctx, mesh, maps, env, cams, params: Params, frame, out, stream=None):
    a, cp = _cams(cams)
    assert maps.is_cuda and maps.is_contiguous() and maps.shape[-1] == 8
    return check(lib().exm_render_forward(ctx, mesh, _ptr(maps), dtype_code(maps.dtype), maps.shape[1], maps.shape[0],
                                          env, cp, a.shape[0], ctypes.byref(params), frame, _ptr(out),
                                          _stream(stream)))


def exm_render_backward(ctx, mesh, maps, env, cams, params: Params, frame, grad_rgb, grad_maps=None, grad_env=None,
                        grad_V=None, stream=None):
    a, cp = _cams(cams)
    return check(lib().exm_render_backward(ctx, mesh, _ptr(maps), dtype_code(maps.dtype), maps.shape[1],
                                           maps.shape[0], env, cp, a.shape[0], ctypes.byref(params), frame,
                                           _ptr(grad_rgb), _ptr(grad_maps), _ptr(grad_env), _ptr(grad_V),
                                           _stream(stream)))


def exm_render_backward_noalloc(ctx, mesh, maps, env, cams, params: Params, frame, grad_rgb, grad_maps=None,
                                grad_env=None, stream=None):
    """Backward into maps and environment gradients using the library's static scratch
    array instead of any device allocation (see include/exmesh.h)."""
    a, cp = _cams(cams)
    return check(lib().exm_render_backward_noalloc(ctx, mesh, _ptr(maps), dtype_code(maps.dtype), maps.shape[1],
                                                   maps.shape[0], env, cp, a.shape[0], ctypes.byref(params), frame,
                                                   _ptr(grad_rgb), _ptr(grad_maps), _ptr(grad_env),
                                                   _stream(stream)))


def exm_l1_loss(pred, target, loss, grad, stream=None):
    return check(lib().exm_l1_loss(_ptr(pred), _ptr(target), pred.numel(), _ptr(loss), _ptr(grad), _stream(stream)))


def exm_server_create(ctx, hbm_budget_bytes, max_slots):
    h = ctypes.c_void_p()
    check(lib().exm_server_create(ctx, int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
    return h


def exm_server_destroy(server):
    lib().exm_server_destroy(server)


def exm_server_add_asset(server, mesh, maps):
    aid = ctypes.c_int32()
    check(lib().exm_server_add_asset(server, mesh, _ptr(maps), dtype_code(maps.dtype), maps.shape[1], maps.shape[0],
                                     ctypes.byref(aid)))
    return aid.value


def exm_relight_submit(server, req: RelightReq):
    t = ctypes.c_uint64()
    check(lib().exm_relight_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def exm_relight_poll(server, ticket):
    done = ctypes.c_int()
    lat = ctypes.c_double()
    check(lib().exm_relight_poll(server, ticket, ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), lat.value


def exm_relight_cancel(server, ticket):
    return check(lib().exm_relight_cancel(server, int(ticket)))


def exm_relight_wait(server, ticket, timeout_ms):
    lat = ctypes.c_double()
    check(lib().exm_relight_wait(server, int(ticket), float(timeout_ms), ctypes.byref(lat)))
    return lat.value


def exm_server_batches(server):
    b, r = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().exm_server_batches(server, ctypes.byref(b), ctypes.byref(r)))
    return b.value, r.value


def exm_server_progress(server):
    return check(lib().exm_server_progress(server))


def exm_server_stats(server):
    v = [ctypes.c_uint64() for _ in range(4)]
    check(lib().exm_server_stats(server, *[ctypes.byref(x) for x in v]))
    return {"queued": v[0].value, "in_flight": v[1].value, "bytes_in_use": v[2].value, "completed": v[3].value}


def exm_relight_footprint(server, req: RelightReq):
    b = ctypes.c_uint64()
    check(lib().exm_relight_footprint(server, ctypes.byref(req), ctypes.byref(b)))
    return b.value


# ------------------------------------------------------------------ Stage-II objective

def exm_image_loss(ctx, pred, target, lambda_ssim, loss, grad_rgb, stream=None):
    V, H, W, C = pred.shape
    assert C == 3 and target.shape == pred.shape and loss.numel() >= 3 and grad_rgb.shape == pred.shape
    return check(lib().exm_image_loss(ctx, _ptr(pred), _ptr(target), V, W, H, float(lambda_ssim), _ptr(loss),
                                      _ptr(grad_rgb), _stream(stream)))


def exm_material_tv(ctx, maps, frame, flags, lambda_mat, loss, grad_maps=None, stream=None):
    assert maps.shape[-1] == 8 and loss.numel() >= 1
    return check(lib().exm_material_tv(ctx, _ptr(maps), dtype_code(maps.dtype), maps.shape[1], maps.shape[0], frame,
                                       int(flags), float(lambda_mat), _ptr(loss), _ptr(grad_maps), _stream(stream)))


def exm_env_regularizers(ctx, E, lambda_env, lambda_chroma, loss, grad_env, stream=None):
    assert E.shape[-1] == 3 and loss.numel() >= 2 and grad_env.shape == E.shape
    return check(lib().exm_env_regularizers(ctx, _ptr(E), E.shape[1], E.shape[0], float(lambda_env),
                                            float(lambda_chroma), _ptr(loss), _ptr(grad_env), _stream(stream)))


def exm_adam_step(ctx, param, grad, m, v, lr, step, lo=None, hi=None, beta1=0.9, beta2=0.999, eps=1e-8,
                  stream=None):
    channels = param.shape[-1]
    rows = param.numel() // channels
    F = ctypes.c_float * channels
    lo_a = F(*lo) if lo is not None else None
    hi_a = F(*hi) if hi is not None else None
    return check(lib().exm_adam_step(ctx, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), rows, channels, float(lr),
                                     float(beta1), float(beta2), float(eps), int(step), lo_a, hi_a, _stream(stream)))


# ------------------------------------------------------------------ Stage-I topology round

def exm_topology_create(ctx):
    out = ctypes.c_void_p()
    check(lib().exm_topology_create(ctx, ctypes.byref(out)))
    return out


def exm_topology_destroy(topo):
    lib().exm_topology_destroy(topo)


def exm_face_render_counts(frame, nf, counts, stream=None):
    return check(lib().exm_face_render_counts(frame, int(nf), _ptr(counts), _stream(stream)))


def exm_topology_round(topo, V, F, UV, Fuv, ema, grad_V, render_counts, params: TopologyParams, stream=None):
    return check(lib().exm_topology_round(topo, _ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(UV), UV.shape[0],
                                          _ptr(Fuv), _ptr(ema), _ptr(grad_V), _ptr(render_counts),
                                          ctypes.byref(params), _stream(stream)))


def exm_topology_result(topo):
    """(nv, nf, nuv, pointers (V, F, UV, Fuv, ema), stats)."""
    nv, nf, nuv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ptrs = [ctypes.c_void_p() for _ in range(5)]
    stats = (ctypes.c_int * 3)()
    check(lib().exm_topology_result(topo, ctypes.byref(nv), ctypes.byref(nf), ctypes.byref(nuv),
                                    *[ctypes.byref(p) for p in ptrs], ctypes.byref(stats)))
    return nv.value, nf.value, nuv.value, [p.value for p in ptrs], list(stats)
