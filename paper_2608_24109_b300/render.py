"""PyTorch-facing renderer: resident device objects plus a torch.autograd.Function whose
backward is the library's hand-written adjoint.  PyTorch supplies memory and streams only;
every step runs in libexmesh's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N


class Renderer:
    """A mesh-UV carrier (Sec. 5: V, F, UV, Fuv fixed), an environment table set and a frame
    (visibility buffer) for `views` cameras at width x height, on one CUDA device."""

    def __init__(self, V, F, UV, Fuv, env_w, env_h, cams, width, height, n_direct, n_bounce=0, n_light=0,
                 lambda_ind=1.0, seed=0, wrap_u=False, metallic=True, secondary_material=True,
                 half_res_indirect=False, bvh_width=None, bvh_layout=None, bvh_collapse=None, device=0):
        self.device = torch.device("cuda", device)
        dev = self.device
        self.V = torch.as_tensor(np.asarray(V), dtype=torch.float32, device=dev).contiguous()
        self.F = torch.as_tensor(np.asarray(F), dtype=torch.int32, device=dev).contiguous()
        self.UV = torch.as_tensor(np.asarray(UV), dtype=torch.float32, device=dev).contiguous()
        self.Fuv = torch.as_tensor(np.asarray(Fuv), dtype=torch.int32, device=dev).contiguous()
        self.cams = np.ascontiguousarray(cams, dtype=np.float32)
        self.views, self.width, self.height = self.cams.shape[0], width, height
        self.env_w, self.env_h = env_w, env_h
        self.params = N.Params(n_direct=n_direct, n_bounce=n_bounce, n_light=max(n_light, 1 if n_bounce else 0),
                               lambda_ind=lambda_ind, flags=(N.FLAG_WRAP_U if wrap_u else 0) |
                               (0 if metallic else N.FLAG_NO_METALLIC) |
                               (0 if secondary_material else N.FLAG_NO_SECONDARY_MATERIAL) |
                               (N.FLAG_HALF_RES_INDIRECT if half_res_indirect else 0), reserved=0, seed=seed)
        self.ctx = N.exm_create(device)
        if bvh_width is not None:
            N.exm_ctx_set_bvh_width(self.ctx, bvh_width)
        if bvh_layout is not None:
            N.exm_ctx_set_bvh_layout(self.ctx, bvh_layout)
        if bvh_collapse is not None:
            N.exm_ctx_set_bvh_collapse(self.ctx, bvh_collapse)
        self.mesh = N.exm_mesh_create(self.ctx, self.V, self.F, self.UV, self.Fuv)
        self.env = N.exm_env_create(self.ctx, env_w, env_h)
        self.frame = N.exm_frame_create(self.ctx, self.views, width, height)
        self.generation = 0
        N.exm_sync(self.ctx)

    @classmethod
    def from_scene(cls, sc, device=0, **kw):
        args = dict(n_direct=sc.n_direct, n_bounce=sc.n_bounce, n_light=sc.n_light, lambda_ind=sc.lambda_ind,
                    seed=sc.seed, wrap_u=sc.wrap_u, metallic=sc.metallic,
                    secondary_material=sc.secondary_material, half_res_indirect=sc.half_res_indirect)
        args.update(kw)
        return cls(sc.V, sc.F, sc.UV, sc.Fuv, sc.env.shape[1], sc.env.shape[0], sc.cams, sc.width, sc.height,
                   device=device, **args)

    def set_limits(self, ray_cap=0, saved_budget_bytes=0):
        """Ray-queue entries per chunk and the byte budget of the whole-frame per-sample state
        (0: the library's defaults); see exm_frame_set_limits."""
        N.exm_frame_set_limits(self.frame, ray_cap, saved_budget_bytes)

    def image_shape(self):
        return (self.views, self.height, self.width, 3)

    def prepare_env(self, E, stream=None):
        assert E.shape == (self.env_h, self.env_w, 3)
        N.exm_env_prepare(self.env, E.contiguous(), stream)

    def forward(self, maps, E=None, out=None, stream=None):
        """Forward render into `out` ([views, H, W, 3] float32).  E (if given) is prepared first."""
        if E is not None:
            self.prepare_env(E, stream)
        if out is None:
            out = torch.empty(self.image_shape(), dtype=torch.float32, device=self.device)
        N.exm_render_forward(self.ctx, self.mesh, maps.contiguous(), self.env, self.cams, self.params, self.frame, out,
                             stream)
        self.generation += 1
        return out

    def backward(self, maps, grad_rgb, grad_maps=None, grad_env=None, grad_V=None, stream=None):
        """Accumulates the adjoint of the last forward into the given FP32 buffers."""
        N.exm_render_backward(self.ctx, self.mesh, maps.contiguous(), self.env, self.cams, self.params, self.frame,
                              grad_rgb.contiguous(), grad_maps, grad_env, grad_V, stream)

    def l1_loss(self, pred, target, loss, grad, stream=None):
        N.exm_l1_loss(pred, target, loss, grad, stream)

    def sync(self, stream=None):
        N.exm_sync(self.ctx, stream)

    def stats(self):
        return N.exm_frame_stats(self.frame)

    def visbuf(self):
        """Copy of the visibility buffer as int64 [views, H, W] (u64 key bit patterns)."""
        ptr = N.exm_frame_visbuf(self.frame)
        shape = (self.views, self.height, self.width)

        class _View:
            __cuda_array_interface__ = {"shape": shape, "typestr": "<i8", "data": (ptr, False), "version": 3,
                                        "strides": None}

        return torch.as_tensor(_View(), device=self.device).clone()

    def saved_state(self):
        """Copies of the last forward's per-sample decisions: covered-pixel ids [n] (int64),
        direct visibility words [n, wd], secondary light-sample words [n, ws] (uint32 bit
        patterns in int64) and secondary hits [n, N_b] (int32); see exm_frame_saved_state."""
        (pp, pb, ph), (wd, ws, nb, rows) = N.exm_frame_saved_state(self.frame)
        n, _ = self.stats()

        def grab(ptr, shape, typestr):
            class _View:
                __cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                            "strides": None}
            return torch.as_tensor(_View(), device=self.device).clone()

        pixels = grab(pp, (n,), "<i4").long() & 0xFFFFFFFF
        bits_all = grab(pb, (rows * (wd + ws),), "<i4").long() & 0xFFFFFFFF
        dbits = bits_all[:rows * wd].view(rows, wd)[:n]
        sbits = bits_all[rows * wd:].view(rows, ws)[:n]
        hits = grab(ph, (rows * nb,), "<i4").view(rows, nb)[:n] if nb else None
        return pixels, dbits, sbits, hits

    def update_vertices(self, V):
        self.V.copy_(V)
        N.exm_mesh_update_vertices(self.mesh, self.V)

    def render(self, maps, E, V=None):
        """Differentiable render: gradients flow to maps, E and (if given) V."""
        if V is None:
            V = self.V
        return RenderFunction.apply(maps, E, V, self)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            torch.cuda.synchronize(self.device)
            N.exm_frame_destroy(self.frame)
            N.exm_env_destroy(self.env)
            N.exm_mesh_destroy(self.mesh)
            N.exm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFunction(torch.autograd.Function):
    """Î = render(maps, E; V) with the library's adjoint as backward.  The sampling density
    and every discrete decision are constants of the derivative."""

    @staticmethod
    def forward(ctx, maps, E, V, renderer: Renderer):
        if not torch.equal(V.detach(), renderer.V):
            renderer.update_vertices(V.detach())
        out = renderer.forward(maps.detach(), E.detach())
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.save_for_backward(maps, E, V)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        maps, E, V = ctx.saved_tensors
        r: Renderer = ctx.renderer
        if r.generation != ctx.generation:
            # another forward ran on this renderer since: rebuild this call's frame
            r.forward(maps.detach(), E.detach())
        gm = torch.zeros(maps.shape, dtype=torch.float32, device=maps.device) if ctx.needs_input_grad[0] else None
        gE = torch.zeros(E.shape, dtype=torch.float32, device=E.device) if ctx.needs_input_grad[1] else None
        gV = torch.zeros(V.shape, dtype=torch.float32, device=V.device) if ctx.needs_input_grad[2] else None
        r.backward(maps.detach(), grad_out.contiguous().float(), gm, gE, gV)
        if gm is not None and gm.dtype != maps.dtype:
            gm = gm.to(maps.dtype)
        if gE is not None and gE.dtype != E.dtype:
            gE = gE.to(E.dtype)
        return gm, gE, gV, None
