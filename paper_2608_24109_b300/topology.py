"""Stage-I topology round on the device (Sec. 4.1-4.3): argument marshalling only; the round
runs in libexmesh's kernels (see exm_topology_round in include/exmesh.h)."""
from __future__ import annotations

import torch

from . import native as N


def _copy(ptr, shape, typestr, dtype, device):
    """A device copy of a library-owned array (shape, element type) at device address ptr."""
    if not ptr or any(d == 0 for d in shape):
        return torch.empty(shape, dtype=dtype, device=device)

    class _View:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False), "version": 3}

    return torch.as_tensor(_View(), device=device).clone()


class TopologyRound:
    """Reusable device state of topology rounds on one context."""

    def __init__(self, ctx, beta_g=0.95, w_g=0.6, w_k=0.4, tau_degen=0.05, tau_uv=1e-4, split_percent=5,
                 max_faces=200000):
        self.ctx = ctx
        self.topo = N.exm_topology_create(ctx)
        self.params = N.TopologyParams(beta_g=beta_g, w_g=w_g, w_k=w_k, tau_degen=tau_degen, tau_uv=tau_uv,
                                       split_percent=split_percent, max_faces=max_faces, reserved=0)

    def __call__(self, V, F, UV, Fuv, ema, grad_V, render_counts, stream=None):
        """Returns new (V, F, UV, Fuv, ema) device tensors and stats {splits, merges, faces_deleted}."""
        args = [V.float().contiguous(), F.int().contiguous(), UV.float().contiguous(), Fuv.int().contiguous(),
                ema.float().contiguous(), grad_V.float().contiguous(), render_counts.int().contiguous()]
        N.exm_topology_round(self.topo, *args, self.params, stream)
        nv, nf, nuv, ptrs, stats = N.exm_topology_result(self.topo)
        dev = V.device
        out = (_copy(ptrs[0], (nv, 3), "<f4", torch.float32, dev), _copy(ptrs[1], (nf, 3), "<i4", torch.int32, dev),
               _copy(ptrs[2], (nuv, 2), "<f4", torch.float32, dev), _copy(ptrs[3], (nf, 3), "<i4", torch.int32, dev),
               _copy(ptrs[4], (nv,), "<f4", torch.float32, dev))
        return out, dict(splits=stats[0], merges=stats[1], faces_deleted=stats[2])

    def close(self):
        if self.topo is not None:
            N.exm_topology_destroy(self.topo)
            self.topo = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
