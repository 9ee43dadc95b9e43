"""Oracle, part 2: the Stage-II estimator in FP64 with plain PyTorch CPU operations.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Given the discrete decisions of decide.c (visible triangle, light-sample texels and
jitters, shadow-ray visibility, secondary hits), this module evaluates, per pixel:

* Sec. 5.1, Eq. 10-11: barycentrics of the camera ray on the visible face, interpolated
  position, UV, vertex normal and tangent; bilinear fetch of A, R, M, N; the tangent-space
  normal taken to world space in the interpolated tangent frame -> n_s.
* Sec. 5.2, Eq. 13-17: f_r = f_d + f_s with f_d = (1 - m) a / pi (Eq. 14), the microfacet
  lobe D G F / (4 max(n.wi,0) max(n.wo,0) + eps) (Eq. 15) with GGX D, separable Smith-GGX G
  and Schlick F, F0 = (1 - m) F_dielectric + m a (Eq. 16); the direct estimator
  (1/N_d) sum_k E Vis f_r max(n_s.wi,0) / p (Eq. 17).
* Sec. 5.3, Eq. 18-19: at each valid secondary hit y, L_sec = (1/N_s) sum_s E Vis f_d(y)
  max(n_s(y).w,0) / p; L_ind = (1/N_b) sum_j 1_hit f_d(x) L_sec(y_j) max(n_s(x).w_j,0) / p_b.
* Eq. 20: I = L_dir + lambda_ind L_ind.  Background pixels are 0.
* The No Secondary Material ablation (Sec. 6.4, scene.secondary_material False): no map is
  read at y; y takes albedo 0.5, roughness 0.5, metallic 0 and a flat tangent-space normal.

Readings where the paper is silent (each documented with the design): alpha = r^2 with r
clamped to [0.08, 1]; F_dielectric = 0.04; eps = 1e-6; f_s = 0 unless n_s.wi > 0 and
n_s.wo > 0; the environment is looked up at the sampled texel (piecewise constant); the
sampling density p and every discrete decision are constants of the derivative; the
secondary hit's geometry is a constant too (only its material values carry gradients).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F_DIELECTRIC = 0.04
SPEC_EPS = 1e-6
R_MIN = 0.08
DT = torch.float64


def _t(a, dtype=DT):
    return torch.as_tensor(np.asarray(a), dtype=dtype)


def _normalize(v):
    return v / torch.linalg.vector_norm(v, dim=-1, keepdim=True)


def _dot(a, b):
    return (a * b).sum(-1)


def face_uv_sign(UV, Fuv):
    """Handedness of each face's UV chart: the sign of the UV-space doubled area, decided
    in FP32 (du1*dv2 - du2*dv1, one rounding per operation); +1 when it is zero."""
    uv = np.asarray(UV, np.float32)
    f = np.asarray(Fuv)
    du1 = uv[f[:, 1], 0] - uv[f[:, 0], 0]
    dv1 = uv[f[:, 1], 1] - uv[f[:, 0], 1]
    du2 = uv[f[:, 2], 0] - uv[f[:, 0], 0]
    dv2 = uv[f[:, 2], 1] - uv[f[:, 0], 1]
    det = du1 * dv2 - du2 * dv1
    return np.where(det < 0, -1.0, 1.0)


def vertex_frames(V, F, UV, Fuv, nuv, sgn):
    """Per-vertex unit normals (sum of the incident faces' cross products) and per-UV-vertex
    unit tangents (sum of the incident faces' dP/du directions, UV-area weighted)."""
    F = torch.as_tensor(np.asarray(F), dtype=torch.long)
    Fuv = torch.as_tensor(np.asarray(Fuv), dtype=torch.long)
    UV = _t(UV)
    P0, P1, P2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = P1 - P0, P2 - P0
    fn = torch.linalg.cross(e1, e2)
    nacc = torch.zeros_like(V)
    for k in range(3):
        nacc = nacc.index_add(0, F[:, k], fn)
    nv = _normalize(nacc)
    uv0, uv1, uv2 = UV[Fuv[:, 0]], UV[Fuv[:, 1]], UV[Fuv[:, 2]]
    dv1 = (uv1[:, 1] - uv0[:, 1])[:, None]
    dv2 = (uv2[:, 1] - uv0[:, 1])[:, None]
    tf = (e1 * dv2 - e2 * dv1) * _t(sgn)[:, None]
    tacc = torch.zeros((nuv, 3), dtype=DT)
    for k in range(3):
        tacc = tacc.index_add(0, Fuv[:, k], tf)
    return nv, _normalize(tacc)


def bilinear(maps, uv, wrap_u: bool):
    """Bilinear sample of an [H, W, C] map at uv (texel centres at (i + 1/2)/W); u wraps
    or clamps, v clamps."""
    Hm, Wm = maps.shape[0], maps.shape[1]
    s = uv[..., 0] * Wm - 0.5
    t = uv[..., 1] * Hm - 0.5
    i0f = torch.floor(s).detach()
    j0f = torch.floor(t).detach()
    fs = (s - i0f)[..., None]
    ft = (t - j0f)[..., None]
    i0 = i0f.long()
    j0 = j0f.long()
    if wrap_u:
        c0, c1 = torch.remainder(i0, Wm), torch.remainder(i0 + 1, Wm)
    else:
        c0, c1 = i0.clamp(0, Wm - 1), (i0 + 1).clamp(0, Wm - 1)
    r0, r1 = j0.clamp(0, Hm - 1), (j0 + 1).clamp(0, Hm - 1)
    return ((1 - fs) * (1 - ft) * maps[r0, c0] + fs * (1 - ft) * maps[r0, c1]
            + (1 - fs) * ft * maps[r1, c0] + fs * ft * maps[r1, c1])


def camera_rays(cams, pix):
    """FP64 camera rays through pixel centres: origin eye, direction
    fwd + ((px + 1/2 - cx)/kx) right + ((cy - py - 1/2)/ky) up."""
    c = _t(cams)[torch.as_tensor(pix[:, 0], dtype=torch.long)]
    px = _t(pix[:, 2])
    py = _t(pix[:, 1])
    dx = (px + 0.5 - c[:, 14]) / c[:, 12]
    dy = (c[:, 15] - (py + 0.5)) / c[:, 13]
    d = c[:, 9:12] + dx[:, None] * c[:, 3:6] + dy[:, None] * c[:, 6:9]
    return c[:, 0:3], d


def ray_barycentrics(o, d, P0, P1, P2):
    """Barycentrics (b0, b1, b2) of the ray o + t d on the plane of (P0, P1, P2)."""
    e1, e2 = P1 - P0, P2 - P0
    pv = torch.linalg.cross(d, e2)
    det = _dot(e1, pv)
    s = o - P0
    b1 = _dot(s, pv) / det
    qv = torch.linalg.cross(s, e1)
    b2 = _dot(d, qv) / det
    return torch.stack([1 - b1 - b2, b1, b2], -1)


def light_directions(tex, xi, W, H, table_q, Q):
    """Direction and solid-angle density of light samples (texel + in-texel jitter):
    theta = pi (i + xv)/H, phi = 2 pi (j + xu)/W, w = (sin t sin p, cos t, -sin t cos p),
    p = (q/Q) * W H / (2 pi^2 sin theta)."""
    tex = torch.as_tensor(np.asarray(tex), dtype=torch.long)
    xi = _t(xi)
    i = torch.div(tex, W, rounding_mode="floor")
    j = tex - i * W
    th = math.pi * (i.to(DT) + xi[..., 1]) / H
    ph = 2 * math.pi * (j.to(DT) + xi[..., 0]) / W
    st, ct = torch.sin(th), torch.cos(th)
    w = torch.stack([st * torch.sin(ph), ct, -st * torch.cos(ph)], -1)
    q = _t(table_q.astype(np.float64))[tex]
    pdf = (q / float(Q)) * (W * H) / (2 * math.pi ** 2 * st)
    return w, pdf, i, j


def brdf_cos(ns, wi, wo, a, r, m, specular=True):
    """(f_d + f_s) * max(n_s . wi, 0), RGB, FP64 (Eqs. 13-16)."""
    ci = _dot(ns, wi)
    co = _dot(ns, wo)
    fd = (1 - m)[..., None] * a / math.pi
    out = fd
    if specular:
        on = (ci > 0) & (co > 0)
        ci_s = torch.where(on, ci, torch.ones_like(ci))
        co_s = torch.where(on, co, torch.ones_like(co))
        wi_s = torch.where(on[..., None], wi, ns)
        wo_s = torch.where(on[..., None], wo, ns)
        alpha = r.clamp(R_MIN, 1.0) ** 2
        a2 = alpha * alpha
        h = _normalize(wi_s + wo_s)
        nh = _dot(ns, h)
        vh = _dot(wi_s, h)
        D = a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)

        def G1(c):
            return 2 * c / (c + torch.sqrt(a2 + (1 - a2) * c * c))

        G = G1(ci_s) * G1(co_s)
        F0 = (1 - m)[..., None] * F_DIELECTRIC + m[..., None] * a
        Fr = F0 + (1 - F0) * ((1 - vh) ** 5)[..., None]
        fs = (D * G)[..., None] * Fr / (4 * ci_s * co_s + SPEC_EPS)[..., None]
        out = fd + torch.where(on[..., None], fs, torch.zeros_like(fs))
    return out * ci.clamp(min=0)[..., None]


class Params:
    def __init__(self, V, maps, env):
        self.V = V
        self.maps = maps
        self.env = env


def shade(scene, table, dec, V, maps, env, rows=None, specular=True, metallic=None):
    """Radiance [P, 3] of the pixels of `dec` (rows selects a sub-range), FP64.

    V [Nv,3], maps [Hm,Wm,8], env [He,We,3]: FP64 tensors (leaves for autograd)."""
    metallic = scene.metallic if metallic is None else metallic
    sl = slice(None) if rows is None else rows
    pix = dec.pix[sl]
    cov = dec.covered[sl]
    P = pix.shape[0]
    out = torch.zeros((P, 3), dtype=DT)
    idx = np.nonzero(cov)[0]
    if idx.size == 0:
        return out
    pixc = pix[idx]
    tri = torch.as_tensor(dec.tri[sl][idx], dtype=torch.long)
    F = torch.as_tensor(np.asarray(scene.F), dtype=torch.long)
    Fuv = torch.as_tensor(np.asarray(scene.Fuv), dtype=torch.long)
    UV = _t(scene.UV)
    sgn = face_uv_sign(scene.UV, scene.Fuv)
    nv, tuv = vertex_frames(V, scene.F, scene.UV, scene.Fuv, scene.UV.shape[0], sgn)
    sg = _t(sgn)
    # --- primary attribute query (Sec. 5.1)
    o, d = camera_rays(scene.cams, pixc)
    fv = F[tri]
    fuv = Fuv[tri]
    b = ray_barycentrics(o, d, V[fv[:, 0]], V[fv[:, 1]], V[fv[:, 2]])
    x = (b[:, :, None] * V[fv]).sum(1)
    uv = (b[:, :, None] * UV[fuv]).sum(1)
    att = bilinear(maps, uv, scene.wrap_u)
    ns, a, r, m = _material(att, b, nv[fv], tuv[fuv], sg[tri], metallic)
    wo = _normalize(o - x)
    # --- direct light (Sec. 5.2, Eq. 17)
    Nd = dec.dtex.shape[1]
    dtex = dec.dtex[sl][idx]
    wi, pdf, ei, ej = light_directions(dtex, dec.dxi[sl][idx], table.W, table.H, table.q, table.Q)
    E = env[ei, ej]
    vis = _t(dec.dvis[sl][idx].astype(np.float64))
    fcos = brdf_cos(ns[:, None, :].expand(-1, Nd, -1), wi, wo[:, None, :].expand(-1, Nd, -1),
                    a[:, None, :].expand(-1, Nd, -1), r[:, None].expand(-1, Nd), m[:, None].expand(-1, Nd),
                    specular=specular)
    # an empty sample set (the indirect-only half-resolution pass) has no direct term
    Ldir = (vis[..., None] * E * fcos / pdf[..., None]).sum(1) / Nd if Nd > 0 else torch.zeros((idx.size, 3), dtype=DT)
    total = Ldir
    # --- one-bounce indirect (Sec. 5.3, Eqs. 18-19)
    Nb = dec.stri.shape[1]
    if Nb > 0 and scene.lambda_ind != 0.0:
        Ns = dec.ltex.shape[2]
        stri = dec.stri[sl][idx]
        valid = stri >= 0
        pj = np.nonzero(valid)
        Lind = torch.zeros((idx.size, 3), dtype=DT)
        if pj[0].size > 0:
            g = torch.as_tensor(stri[pj], dtype=torch.long)
            by = _t(dec.sb[sl][idx][pj])
            gv, guv = F[g], Fuv[g]
            uvy = (by[:, :, None] * UV[guv]).sum(1)
            if scene.secondary_material:
                atty = bilinear(maps, uvy, scene.wrap_u)
            else:
                # No Secondary Material ablation (Sec. 6.4): no map read at y; a constant grey
                # diffuse material with a flat tangent-space normal
                atty = torch.tensor([0.5, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 1.0], dtype=DT).expand(uvy.shape[0], 8)
            nsy, ay, _, my = _material(atty, by, nv.detach()[gv], tuv.detach()[guv], sg[g], metallic)
            fdy = (1 - my)[:, None] * ay / math.pi
            ltex = dec.ltex[sl][idx][pj]
            wl, pl, li, lj = light_directions(ltex, dec.lxi[sl][idx][pj], table.W, table.H, table.q, table.Q)
            El = env[li, lj]
            lvis = _t(dec.lvis[sl][idx][pj].astype(np.float64))
            cosl = _dot(nsy[:, None, :], wl).clamp(min=0)
            Lsec = (lvis[..., None] * El * fdy[:, None, :] * cosl[..., None] / pl[..., None]).sum(1) / Ns
            p_i = torch.as_tensor(pj[0], dtype=torch.long)
            wj = _normalize(_t(dec.sdir[sl][idx][pj].astype(np.float64)))
            pb = torch.sqrt(1 - _t(dec.sxi1[sl][idx][pj].astype(np.float64))) / math.pi
            fdx = (1 - m)[p_i][:, None] * a[p_i] / math.pi
            cosx = _dot(ns[p_i], wj).clamp(min=0)
            contrib = fdx * Lsec * (cosx / pb)[:, None]
            Lind = Lind.index_add(0, p_i, contrib)
        total = total + scene.lambda_ind * Lind / Nb
    out = out.index_put((torch.as_tensor(idx, dtype=torch.long),), total)
    return out


def _material(att, b, nvert, tvert, sgn_f, metallic):
    """Material values and the world-space shading normal n_s (Eq. 10-11)."""
    a = att[..., 0:3]
    r = att[..., 3]
    m = att[..., 4] if metallic else torch.zeros_like(att[..., 4])
    q = att[..., 5:8]
    n = _normalize((b[..., None] * nvert).sum(-2))
    ti = (b[..., None] * tvert).sum(-2)
    T = _normalize(ti - _dot(n, ti)[..., None] * n)
    B = sgn_f[..., None] * torch.linalg.cross(n, T)
    nt = _normalize(q)
    ns = T * nt[..., 0:1] + B * nt[..., 1:2] + n * nt[..., 2:3]
    return ns, a, r, m


def render_image(scene, table, dec, V, maps, env, chunk=4096, **kw):
    """Radiance of every pixel of `dec` in chunks (no graph kept)."""
    outs = []
    with torch.no_grad():
        for s in range(0, dec.pix.shape[0], chunk):
            outs.append(shade(scene, table, dec, V, maps, env, rows=slice(s, s + chunk), **kw))
    return torch.cat(outs)


def backward(scene, table, dec, V, maps, env, grad_rgb, chunk=2048, **kw):
    """Gradients of sum(grad_rgb * I) w.r.t. V, maps and env (torch.autograd), chunked."""
    Vl = V.detach().clone().requires_grad_(True)
    Ml = maps.detach().clone().requires_grad_(True)
    El = env.detach().clone().requires_grad_(True)
    g = _t(grad_rgb)
    for s in range(0, dec.pix.shape[0], chunk):
        I = shade(scene, table, dec, Vl, Ml, El, rows=slice(s, s + chunk), **kw)
        (I * g[s:s + chunk]).sum().backward()
    return Vl.grad, Ml.grad, El.grad


def scene_tensors(scene):
    return _t(scene.V.astype(np.float64)), _t(scene.maps.astype(np.float64)), _t(scene.env.astype(np.float64))
