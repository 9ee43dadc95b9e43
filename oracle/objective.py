"""Oracle, part 3: the Stage-II objective (Sec. 5.4, Eqs. 21-24) and the Adam step that
follows it, in FP64 with plain PyTorch CPU operations.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Eq. 21: L_img = lambda_log |log(1 + I^) - log(1 + I)|_1 + lambda_ssim D-SSIM(G(I^), G(I)),
  G the linear-to-sRGB transfer.
* Eq. 22: L_II = L_img + lambda_mat L_mat + lambda_env L_env + lambda_chroma(t) L_chroma.
* Eq. 23: L_mat = sum over P in {A, R, N} (and M with metallic) of TV(P^), P^ the material map
  projected to the screen (its bilinear fetch at each pixel's primary hit); L_env = TV(E).
* Eq. 24: L_chroma = |E_mean - mu_E 1|^2 with E_mean the per-channel mean of E and mu_E the mean
  of its three entries; lambda_chroma(t) = lambda_chroma0 (1 - t / T).

Readings where the paper is silent (each listed with the design):
* lambda_log = 1 - lambda_ssim; the L1 norm is a mean over pixels and channels.
* D-SSIM = 1 - SSIM, SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5), zero
  padding to the image size, C1 = 0.01^2, C2 = 0.03^2, averaged over views, pixels, channels.
* G(x) = 12.92 x for x <= 0.0031308, else 1.055 x^(1/2.4) - 0.055 (the sRGB transfer).
* TV(X) = mean |X(p) - X(p + x)| over horizontal neighbour pairs + the same over vertical
  pairs, each mean over pairs and the channels of X.  Screen-space pairs count only when both
  pixels see the surface; the environment wraps in longitude (texel W-1 neighbours texel 0).
* Adam with PyTorch's defaults (beta1 0.9, beta2 0.999, eps 1e-8), bias-corrected, then each
  parameter is clamped to its range (base colour, roughness, metallic in [0, 1]; the normal
  map is free; E >= 0).
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as Fn

from .shade import DT, _t, bilinear, camera_rays, ray_barycentrics

SSIM_WIN = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2

# channel groups of the 8-channel material map: base colour, roughness, metallic, normal
MAT_GROUPS = {"A": (0, 3), "R": (3, 4), "M": (4, 5), "N": (5, 8)}


def srgb(x):
    """Linear RGB -> sRGB transfer curve."""
    lo = 12.92 * x
    hi = 1.055 * torch.clamp(x, min=0.0031308) ** (1.0 / 2.4) - 0.055
    return torch.where(x <= 0.0031308, lo, hi)


def gaussian_window(n=SSIM_WIN, sigma=SSIM_SIGMA):
    k = torch.arange(n, dtype=DT) - (n - 1) / 2
    g = torch.exp(-(k * k) / (2 * sigma * sigma))
    return g / g.sum()


def ssim(x, y):
    """Mean SSIM of [V, H, W, C] images: Gaussian local statistics per channel, zero padding."""
    g = gaussian_window()
    w2 = (g[:, None] * g[None, :])[None, None]
    C = x.shape[-1]
    xc = x.permute(0, 3, 1, 2).reshape(-1, 1, x.shape[1], x.shape[2])
    yc = y.permute(0, 3, 1, 2).reshape(-1, 1, y.shape[1], y.shape[2])
    pad = SSIM_WIN // 2
    mx = Fn.conv2d(xc, w2, padding=pad)
    my = Fn.conv2d(yc, w2, padding=pad)
    sxx = Fn.conv2d(xc * xc, w2, padding=pad) - mx * mx
    syy = Fn.conv2d(yc * yc, w2, padding=pad) - my * my
    sxy = Fn.conv2d(xc * yc, w2, padding=pad) - mx * my
    s = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))
    return s.mean()


def image_loss(pred, target, lambda_ssim=0.2):
    """Eq. 21 with lambda_log = 1 - lambda_ssim; returns (total, log-L1 term, D-SSIM term)."""
    log_l1 = (torch.log1p(pred) - torch.log1p(target)).abs().mean()
    dssim = 1.0 - ssim(srgb(pred), srgb(target))
    return (1.0 - lambda_ssim) * log_l1 + lambda_ssim * dssim, log_l1, dssim


def screen_tv(img, mask):
    """TV of a [V, H, W, C] screen image over neighbour pairs whose two pixels are both set in
    mask [V, H, W]."""
    C = img.shape[-1]
    mx = mask[:, :, 1:] & mask[:, :, :-1]
    my = mask[:, 1:, :] & mask[:, :-1, :]
    dx = (img[:, :, 1:] - img[:, :, :-1]).abs()[mx]
    dy = (img[:, 1:, :] - img[:, :-1, :]).abs()[my]
    tx = dx.sum() / (mx.sum() * C) if mx.any() else img.sum() * 0
    ty = dy.sum() / (my.sum() * C) if my.any() else img.sum() * 0
    return tx + ty


def env_tv(E):
    """TV of an [H, W, 3] lat-long map, wrapping in longitude."""
    dx = (torch.roll(E, -1, dims=1) - E).abs().mean()
    dy = (E[1:] - E[:-1]).abs().mean() if E.shape[0] > 1 else E.sum() * 0
    return dx + dy


def chroma(E):
    """Eq. 24: squared distance of the mean colour from its grey."""
    m = E.reshape(-1, 3).mean(0)
    return ((m - m.mean()) ** 2).sum()


def primary_material(scene, dec, maps):
    """Screen-space material image [V, H, W, 8] and coverage mask: the bilinear fetch at each
    covered pixel's primary hit (the attribute query of Eqs. 10-11)."""
    V = _t(scene.V)
    F = torch.as_tensor(np.asarray(scene.F), dtype=torch.long)
    Fuv = torch.as_tensor(np.asarray(scene.Fuv), dtype=torch.long)
    UV = _t(scene.UV)
    img = torch.zeros((scene.views, scene.height, scene.width, maps.shape[-1]), dtype=DT)
    mask = torch.zeros((scene.views, scene.height, scene.width), dtype=torch.bool)
    idx = np.nonzero(dec.covered)[0]
    if idx.size == 0:
        return img, mask
    pix = dec.pix[idx]
    tri = torch.as_tensor(dec.tri[idx], dtype=torch.long)
    o, d = camera_rays(scene.cams, pix)
    fv, fuv = F[tri], Fuv[tri]
    b = ray_barycentrics(o, d, V[fv[:, 0]], V[fv[:, 1]], V[fv[:, 2]])
    uv = (b[:, :, None] * UV[fuv]).sum(1)
    att = bilinear(maps, uv, scene.wrap_u)
    p = torch.as_tensor(pix, dtype=torch.long)
    img = img.index_put((p[:, 0], p[:, 1], p[:, 2]), att)
    mask[p[:, 0], p[:, 1], p[:, 2]] = True
    return img, mask


def material_tv(scene, dec, maps, metallic=True):
    """Eq. 23, L_mat: the TV of each projected map of {A, R, N} (and M with metallic)."""
    img, mask = primary_material(scene, dec, maps)
    groups = ["A", "R", "N"] + (["M"] if metallic else [])
    total = maps.sum() * 0
    for gname in groups:
        a, b = MAT_GROUPS[gname]
        total = total + screen_tv(img[..., a:b], mask)
    return total


def stage2_objective(pred, target, scene, dec, maps, env, t=0, T=10000, lambda_ssim=0.2, lambda_mat=0.1,
                     lambda_env=0.1, lambda_chroma0=0.1, metallic=True):
    """Eq. 22 and its terms."""
    l_img, l_log, l_dssim = image_loss(pred, target, lambda_ssim)
    l_mat = material_tv(scene, dec, maps, metallic)
    l_env = env_tv(env)
    l_chr = chroma(env)
    lam_c = lambda_chroma0 * (1.0 - t / T)
    total = l_img + lambda_mat * l_mat + lambda_env * l_env + lam_c * l_chr
    return total, dict(img=l_img, log_l1=l_log, dssim=l_dssim, mat=l_mat, env=l_env, chroma=l_chr)


def adam_step(theta, grad, m, v, step, lr, lo=None, hi=None, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), then a clamp to [lo, hi] per channel (last axis).
    Returns the new (theta, m, v) without modifying the inputs."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * mh / (torch.sqrt(vh) + eps)
    if lo is not None:
        theta = torch.maximum(theta, torch.as_tensor(lo, dtype=theta.dtype))
    if hi is not None:
        theta = torch.minimum(theta, torch.as_tensor(hi, dtype=theta.dtype))
    return theta, m, v


# per-channel ranges of the 8-channel material map and of E
MAP_LO = [0.0, 0.0, 0.0, 0.0, 0.0, -math.inf, -math.inf, -math.inf]
MAP_HI = [1.0, 1.0, 1.0, 1.0, 1.0, math.inf, math.inf, math.inf]
ENV_LO = [0.0, 0.0, 0.0]
ENV_HI = [math.inf, math.inf, math.inf]
