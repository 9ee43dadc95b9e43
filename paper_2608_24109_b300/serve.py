"""Relight serving over resident assets (thin wrapper of libexmesh's native server).

The server (include/exmesh.h, exm_server_*) keeps assets resident on the device, admits
requests by their device footprint against an HBM budget, and runs the admitted requests in
batches on a few batch streams: each batch traces all its requests' rays in shared persistent
tracer launches (every ray through its own asset's BVH), and requests that arrive while a
batch runs join the next one, so batches overlap on the GPU.  This module only marshals
arguments and keeps the Python-side buffers of in-flight requests alive.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N


class RelightServer:
    def __init__(self, hbm_budget_bytes=8 << 30, max_slots=8, device=0):
        self.device = torch.device("cuda", device)
        self.ctx = N.exm_create(device)
        self.server = N.exm_server_create(self.ctx, hbm_budget_bytes, max_slots)
        self.assets = []    # (mesh handle, tensors kept alive)
        self._inflight = {}  # ticket -> (request struct, env, out, cams)

    def add_asset(self, V, F, UV, Fuv, maps):
        """Registers a resident asset; maps is a device tensor [H, W, 8] (FP32, BF16 or FP16)."""
        dev = self.device
        t = [torch.as_tensor(np.asarray(V), dtype=torch.float32, device=dev).contiguous(),
             torch.as_tensor(np.asarray(F), dtype=torch.int32, device=dev).contiguous(),
             torch.as_tensor(np.asarray(UV), dtype=torch.float32, device=dev).contiguous(),
             torch.as_tensor(np.asarray(Fuv), dtype=torch.int32, device=dev).contiguous()]
        mesh = N.exm_mesh_create(self.ctx, *t)
        N.exm_sync(self.ctx)
        maps = maps.to(dev).contiguous()
        aid = N.exm_server_add_asset(self.server, mesh, maps)
        self.assets.append((mesh, t, maps))
        return aid

    def request(self, asset, env, cams, width, height, n_direct, n_bounce=0, n_light=0, lambda_ind=1.0, seed=0,
                wrap_u=False, metallic=True, secondary_material=True, out=None):
        cams = np.ascontiguousarray(cams, dtype=np.float32)
        if out is None:
            out = torch.empty((cams.shape[0], height, width, 3), dtype=torch.float32, device=self.device)
        env = env.contiguous()
        p = N.Params(n_direct=n_direct, n_bounce=n_bounce, n_light=n_light if n_bounce else 0, lambda_ind=lambda_ind,
                     flags=(N.FLAG_WRAP_U if wrap_u else 0) | (0 if metallic else N.FLAG_NO_METALLIC) |
                     (0 if secondary_material else N.FLAG_NO_SECONDARY_MATERIAL), reserved=0,
                     seed=seed)
        req = N.RelightReq(asset=asset, views=cams.shape[0], width=width, height=height, env=env.data_ptr(),
                           env_dtype=N.dtype_code(env.dtype), env_w=env.shape[1], env_h=env.shape[0],
                           cams=cams.ctypes.data, params=p, out_rgb=out.data_ptr())
        return req, (env, out, cams)

    def submit(self, req_and_buffers):
        req, keep = req_and_buffers
        ticket = N.exm_relight_submit(self.server, req)
        self._inflight[ticket] = keep
        return ticket

    def poll(self, ticket):
        try:
            done, lat = N.exm_relight_poll(self.server, ticket)
        except N.ExmError:
            self._inflight.pop(ticket, None)  # done with an error (cancelled, failed)
            raise
        out = None
        if done:
            out = self._inflight.pop(ticket)[1]
        return done, lat, out

    def wait(self, ticket, timeout_ms):
        """(latency ms, output) once the request is done; raises N.ExmError with EXM_ERR_TIMEOUT
        if it is not done within timeout_ms (it stays pending), or the request's own error."""
        try:
            lat = N.exm_relight_wait(self.server, ticket, timeout_ms)
        except N.ExmError as e:
            if e.code != N.EXM_ERR_TIMEOUT:
                self._inflight.pop(ticket, None)
            raise
        return lat, self._inflight.pop(ticket)[1]

    def cancel(self, ticket):
        N.exm_relight_cancel(self.server, ticket)

    def batches(self):
        """(batches launched, requests they held)."""
        return N.exm_server_batches(self.server)

    def add_imported_asset(self, mesh, maps):
        """Registers a mesh handle from exm_mesh_import with its maps; the server frees it on close."""
        maps = maps.to(self.device).contiguous()
        aid = N.exm_server_add_asset(self.server, mesh, maps)
        self.assets.append((mesh, [], maps))
        return aid

    def footprint(self, req_and_buffers):
        return N.exm_relight_footprint(self.server, req_and_buffers[0])

    def progress(self):
        N.exm_server_progress(self.server)

    def stats(self):
        return N.exm_server_stats(self.server)

    def close(self):
        if getattr(self, "server", None) is not None:
            torch.cuda.synchronize(self.device)
            N.exm_server_destroy(self.server)
            self.server = None
            for mesh, _, _ in self.assets:
                N.exm_mesh_destroy(mesh)
            self.assets = []
            N.exm_destroy(self.ctx)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
