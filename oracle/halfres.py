"""Oracle, part 4: indirect light at half resolution (the paper's implementation details,
Sec. 6.1: secondary rays evaluated at half resolution in both image dimensions, the indirect
component upsampled to full resolution).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading where the paper is silent:
* The half-resolution pass renders the same cameras with every intrinsic (kx, ky, cx, cy)
  halved, at W' = ceil(W/2) x H' = ceil(H/2): its pixel (i, j) is centred on the full-
  resolution point (2i + 1, 2j + 1).  It evaluates lambda_ind L_ind (Eqs. 18-19) at its own
  primary hits, with no direct samples, and is 0 where it sees no surface.
* Upsampling is bilinear with half-pixel centres: full pixel x reads the half image at
  x' = (x + 1/2)/2 - 1/2 from taps floor(x') and floor(x') + 1 clamped to [0, W'-1] (the
  same in y) -- for even sizes, PyTorch's bilinear interpolation with align_corners=False.
* I = L_dir (full resolution, direct only) + the upsampled term, on covered full-resolution
  pixels; background pixels stay 0.
"""
from __future__ import annotations

import copy
import math

import numpy as np
import torch

from . import Decisions, EnvTable, covered_pixels, raster_full
from .shade import DT, shade


def half_scene(scene):
    h = copy.copy(scene)
    cams = np.array(scene.cams, dtype=np.float32, copy=True)
    cams[:, 12:16] *= 0.5
    h.cams = cams
    h.width = (scene.width + 1) // 2
    h.height = (scene.height + 1) // 2
    h.n_direct = 0
    return h


def direct_scene(scene):
    d = copy.copy(scene)
    d.n_bounce = 0
    d.n_light = 0
    return d


def upsample(img, W, H):
    """[V, H', W', C] -> [V, H, W, C] bilinear with half-pixel centres, clamped taps."""
    Vn, Hh, Wh, C = img.shape

    def taps(n_out, n_in):
        src = (torch.arange(n_out, dtype=DT) + 0.5) * 0.5 - 0.5
        i0 = torch.floor(src)
        f = src - i0
        i0 = i0.long()
        return i0.clamp(0, n_in - 1), (i0 + 1).clamp(0, n_in - 1), f

    x0, x1, fx = taps(W, Wh)
    y0, y1, fy = taps(H, Hh)
    fx = fx[None, None, :, None]
    fy = fy[None, :, None, None]
    top = (1 - fx) * img[:, y0][:, :, x0] + fx * img[:, y0][:, :, x1]
    bot = (1 - fx) * img[:, y1][:, :, x0] + fx * img[:, y1][:, :, x1]
    return (1 - fy) * top + fy * bot


def _image(scene, table, V, maps, env):
    st, keys = raster_full(scene.V, scene.F, scene.cams, scene.width, scene.height)
    pix = covered_pixels(keys)
    dec = Decisions(scene, table, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    # chunked like render_image, but keeping the autograd graph when the inputs require grad
    rad = torch.cat([shade(scene, table, dec, V, maps, env, rows=slice(s, s + 4096))
                     for s in range(0, dec.pix.shape[0], 4096)])
    img = torch.zeros((scene.views, scene.height, scene.width, 3), dtype=DT)
    p = torch.as_tensor(pix, dtype=torch.long)
    img = img.index_put((p[:, 0], p[:, 1], p[:, 2]), rad)
    mask = torch.zeros((scene.views, scene.height, scene.width), dtype=torch.bool)
    mask[p[:, 0], p[:, 1], p[:, 2]] = True
    return img, mask, dec


def render_halfres(scene, table: EnvTable, V, maps, env):
    """Full-resolution image [V, H, W, 3] of the half-resolution-indirect estimator (a
    differentiable function of V, maps and env for fixed decisions) and the half pass's
    decisions."""
    direct, mask, _ = _image(direct_scene(scene), table, V, maps, env)
    hs = half_scene(scene)
    half, _, hdec = _image(hs, table, V, maps, env)
    up = upsample(half, scene.width, scene.height)
    return direct + up * mask[..., None], hdec
