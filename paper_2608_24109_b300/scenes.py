"""Seeded synthetic inputs: meshes with UV atlases, PBR maps, environment maps, cameras.

This module only *makes inputs*.  It holds none of the shading method's arithmetic,
so both the CUDA path and the CPU oracle draw their inputs from it.

Asset conventions (the Stage-II carrier of Sec. 5: fixed vertices V, faces F, UV
coordinates U and the face-corner to UV map Phi; parameters Theta = {A, R, M, N, E}):

* ``V``   float32 [Nv, 3]  vertex positions
* ``F``   int32   [Nf, 3]  position indices, counter-clockwise seen from outside
* ``UV``  float32 [Nuv, 2] texture coordinates, u to the right, v downwards (row 0 at v = 0)
* ``Fuv`` int32   [Nf, 3]  UV index of each face corner
* ``maps`` float32 [Hm, Wm, 8] texel-interleaved material map:
  base colour A (3), roughness R (1), metallic M (1), tangent-space normal N (3)
* ``env`` float32 [He, We, 3] lat-long RGB environment, row 0 = +y (theta = 0)
* ``cams`` float32 [views, 20]: eye(3) right(3) up(3) fwd(3) kx ky cx cy near pad(3);
  a camera-space point (x, y, w) maps to pixel (cx + kx*x/w, cy - ky*y/w)

Workloads follow the shapes and value distributions of the paper's Stage-II setting
(Sec. 5, Sec. 6.1): a closed object mesh, 8-channel PBR maps in a UV atlas, an HDR
lat-long environment and a ring or sphere of cameras.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CAM_FLOATS = 20
MAP_CHANNELS = 8


# --------------------------------------------------------------------------- meshes

def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv faces, outward counter-clockwise winding."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = list(faces)
    for _ in range(subdiv):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    V = np.array(V)
    F = np.array(F, dtype=np.int64)
    return V, _orient_outward_faces(V, F)


def _orient_outward_faces(V, F):
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    c = V[F].mean(axis=1)
    flip = np.einsum("ij,ij->i", n, c) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def sphere_uv(V, F):
    """Per-corner spherical UV (u = phi / 2pi, v = theta / pi) with the seam handled.

    Corners of faces that straddle the u = 0/1 seam are shifted by +1 in u (the sampler
    wraps in u).  A corner at a pole takes the mean u of the face's other two corners.
    UV vertices are shared between faces wherever (vertex, u) agree.
    """
    d = V / np.linalg.norm(V, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 1], -1.0, 1.0))
    phi = np.mod(np.arctan2(d[:, 0], -d[:, 2]), 2.0 * np.pi)
    u = phi / (2.0 * np.pi)
    v = theta / np.pi
    pole = (np.abs(d[:, 1]) > 1.0 - 1e-9)
    corner_u = u[F].copy()
    corner_v = v[F].copy()
    for f in range(F.shape[0]):
        cu = corner_u[f]
        nonpole = [k for k in range(3) if not pole[F[f, k]]]
        vals = cu[nonpole]
        if vals.max() - vals.min() > 0.5:
            for k in nonpole:
                if cu[k] < 0.5:
                    cu[k] += 1.0
        for k in range(3):
            if pole[F[f, k]]:
                cu[k] = np.mean(cu[nonpole])
        corner_u[f] = cu
    keys = {}
    UV = []
    Fuv = np.zeros_like(F)
    for f in range(F.shape[0]):
        for k in range(3):
            key = (int(F[f, k]), round(float(corner_u[f, k]), 9))
            if key not in keys:
                keys[key] = len(UV)
                UV.append((corner_u[f, k], corner_v[f, k]))
            Fuv[f, k] = keys[key]
    return np.array(UV, dtype=np.float64), Fuv


def _real_sh(l, m, theta, phi):
    from scipy.special import lpmv
    x = np.cos(theta)
    p = lpmv(abs(m), l, x)
    if m > 0:
        return p * np.cos(m * phi)
    if m < 0:
        return p * np.sin(-m * phi)
    return p


def sh_displacement(rng, n_terms=8, lmax=6, amplitude=0.05):
    """Radius function r(w) = 1 + amplitude * sum_k c_k * Yhat_{l_k m_k}(w), max|Yhat| = 1."""
    terms = []
    tg = np.linspace(0, np.pi, 257)
    pg = np.linspace(0, 2 * np.pi, 513)
    TT, PP = np.meshgrid(tg, pg, indexing="ij")
    for _ in range(n_terms):
        l = int(rng.integers(0, lmax + 1))
        m = int(rng.integers(-l, l + 1))
        c = float(rng.uniform(-1.0, 1.0))
        ymax = np.abs(_real_sh(l, m, TT, PP)).max()
        terms.append((l, m, c, ymax))

    def radius(d):
        theta = np.arccos(np.clip(d[:, 1], -1.0, 1.0))
        phi = np.arctan2(d[:, 0], -d[:, 2])
        r = np.ones(d.shape[0])
        for l, m, c, ymax in terms:
            r += amplitude * c * _real_sh(l, m, theta, phi) / ymax
        return r

    return radius


def cube_sphere(n: int, map_res: int, rng, dents: int = 0, gutter_texels: int = 4):
    """Closed cube-sphere: 6 grid charts of n x n quads (6*2*n*n triangles).

    Radially displaced by 8 random real spherical harmonics (amplitude 0.05); with
    ``dents`` > 0, spherical dents (balls of radius 0.5 centred at 1.2*d, d uniform on
    the sphere) push the surface inwards to the ball's near side (depth 0.3 at the
    dent centre).  Charts are packed 3 x 2 in the UV atlas with ``gutter_texels`` of
    margin at ``map_res``.
    """
    radius = sh_displacement(rng)
    centres = []
    for _ in range(dents):
        d = rng.normal(size=3)
        centres.append(1.2 * d / np.linalg.norm(d))
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    keys, tris, uvs, ftri_uv = [], [], [], []
    gu = gutter_texels / (map_res / 3.0)
    gv = gutter_texels / (map_res / 2.0)
    q = np.arange(n)
    qi, qj = np.meshgrid(q, q, indexing="ij")
    qi = qi.ravel()
    qj = qj.ravel()
    for chart in range(6):
        a, s = chart // 2, (1 if chart % 2 == 0 else -1)
        b, c = (a + 1) % 3, (a + 2) % 3
        k = np.zeros((ii.size, 3), dtype=np.int64)
        k[:, a] = s * n
        k[:, b] = 2 * ii - n
        k[:, c] = 2 * jj - n
        keys.append(k)
        col, row = chart % 3, chart // 3
        u = (col + gu + (1 - 2 * gu) * ii / n) / 3.0
        v = (row + gv + (1 - 2 * gv) * jj / n) / 2.0
        uvs.append(np.stack([u, v], axis=1))
        base = chart * (n + 1) ** 2
        v00 = base + qi * (n + 1) + qj
        v10 = v00 + (n + 1)
        v11 = v10 + 1
        v01 = v00 + 1
        t = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
        tris.append(t)
    keys = np.concatenate(keys)
    local_F = np.concatenate(tris)
    UV = np.concatenate(uvs)
    uniq, inverse = np.unique(keys, axis=0, return_inverse=True)
    inverse = inverse.ravel()
    F = inverse[local_F]
    Fuv = local_F.copy()
    d = uniq.astype(np.float64) / n
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius(d)
    for cc in centres:
        wc = d @ cc
        disc = wc * wc - cc @ cc + 0.25
        inside = disc > 0
        s_in = wc - np.sqrt(np.maximum(disc, 0.0))
        hit = inside & (s_in < r) & (s_in > 0)
        r = np.where(hit, s_in, r)
    V = d * r[:, None]
    nrm = np.cross(d[F[:, 1]] - d[F[:, 0]], d[F[:, 2]] - d[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, d[F].mean(axis=1)) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    Fuv[flip] = Fuv[flip][:, [0, 2, 1]]
    return V, F, UV, Fuv


# --------------------------------------------------------------------------- parameters

def material_maps(rng, res: int) -> np.ndarray:
    """A ~ U[0.1,0.9]^3, R ~ U[0.2,0.9], M ~ Bernoulli(0.3), N = +z + N(0, 0.1)^3."""
    m = np.empty((res, res, MAP_CHANNELS), dtype=np.float32)
    m[..., 0:3] = rng.uniform(0.1, 0.9, (res, res, 3))
    m[..., 3] = rng.uniform(0.2, 0.9, (res, res))
    m[..., 4] = (rng.uniform(0.0, 1.0, (res, res)) < 0.3).astype(np.float32)
    m[..., 5:8] = np.array([0.0, 0.0, 1.0]) + rng.normal(0.0, 0.1, (res, res, 3))
    return m


def env_map(rng, width: int, height: int, sigma: float) -> np.ndarray:
    """Lat-long RGB environment, i.i.d. log-normal(0, sigma) per channel, [H, W, 3]."""
    return np.exp(rng.normal(0.0, sigma, (height, width, 3))).astype(np.float32)


def look_at_camera(eye, width, height, fovy_deg=45.0, near=0.25, target=(0.0, 0.0, 0.0)):
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up_hint = np.array([0.0, 1.0, 0.0])
    if abs(fwd @ up_hint) > 0.99:
        up_hint = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up_hint)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    k = 0.5 * height / math.tan(math.radians(fovy_deg) / 2.0)
    cam = np.zeros(CAM_FLOATS, dtype=np.float32)
    cam[0:3], cam[3:6], cam[6:9], cam[9:12] = eye, right, up, fwd
    cam[12], cam[13], cam[14], cam[15], cam[16] = k, k, width / 2.0, height / 2.0, near
    return cam


def ring_cameras(count, distance, width, height):
    cams = []
    for i in range(count):
        az = 2.0 * math.pi * i / count
        cams.append(look_at_camera((distance * math.sin(az), 0.0, distance * math.cos(az)), width, height))
    return np.stack(cams)


def fibonacci_cameras(count, distance, width, height):
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(count):
        y = 1.0 - 2.0 * (i + 0.5) / count
        r = math.sqrt(max(0.0, 1.0 - y * y))
        ph = golden * i
        cams.append(look_at_camera((distance * r * math.cos(ph), distance * y, distance * r * math.sin(ph)),
                                   width, height))
    return np.stack(cams)


# --------------------------------------------------------------------------- scenes

@dataclasses.dataclass
class Scene:
    name: str
    V: np.ndarray
    F: np.ndarray
    UV: np.ndarray
    Fuv: np.ndarray
    maps: np.ndarray
    maps_target: np.ndarray
    env: np.ndarray
    cams: np.ndarray
    width: int
    height: int
    n_direct: int
    n_bounce: int = 0
    n_light: int = 0
    lambda_ind: float = 1.0
    seed: int = 0
    wrap_u: bool = False
    metallic: bool = True
    secondary_material: bool = True  # False: the No Secondary Material ablation
    half_res_indirect: bool = False  # indirect light at half resolution, then upsampled

    @property
    def views(self):
        return self.cams.shape[0]


def _finish(name, V, F, UV, Fuv, maps, maps_t, env, cams, W, H, **kw):
    return Scene(name=name, V=np.ascontiguousarray(V, np.float32), F=np.ascontiguousarray(F, np.int32),
                 UV=np.ascontiguousarray(UV, np.float32), Fuv=np.ascontiguousarray(Fuv, np.int32),
                 maps=maps, maps_target=maps_t, env=env, cams=np.ascontiguousarray(cams, np.float32),
                 width=W, height=H, **kw)


def icosphere_scene(res=256, views=4, map_res=256, env_w=64, env_h=32, n_direct=64, seed=0,
                    n_bounce=0, n_light=0):
    """Plain method, tiny: icosphere (subdiv 3, 1280 tris, r = 1), 256^2 maps, 64x32 env,
    4 ring cameras at distance 3, 64 stratified env samples per pixel, no indirect."""
    rng = np.random.default_rng(seed)
    V, F = icosphere(3)
    UV, Fuv = sphere_uv(V, F)
    maps = material_maps(rng, map_res)
    env = env_map(rng, env_w, env_h, 1.0)
    maps_t = material_maps(np.random.default_rng(seed + 1000), map_res)
    cams = ring_cameras(views, 3.0, res, res)
    return _finish("icosphere1280", V, F, UV, Fuv, maps, maps_t, env, cams, res, res,
                   n_direct=n_direct, n_bounce=n_bounce, n_light=n_light, seed=seed, wrap_u=True)


def blob_scene(n=91, map_res=1024, env_w=256, env_h=128, env_sigma=1.5, views=16, res=512,
               n_direct=256, n_bounce=0, n_light=0, dents=0, seed=2, ring=False):
    """Displaced cube-sphere blob (optionally with spherical cavities) in a 3x2 UV atlas."""
    rng = np.random.default_rng(seed)
    V, F, UV, Fuv = cube_sphere(n, map_res, rng, dents=dents)
    maps = material_maps(rng, map_res)
    env = env_map(rng, env_w, env_h, env_sigma)
    maps_t = material_maps(np.random.default_rng(seed + 1000), map_res)
    cams = (ring_cameras if ring else fibonacci_cameras)(views, 3.0, res, res)
    name = f"blob{6 * 2 * n * n}" + (f"_dents{dents}" if dents else "")
    return _finish(name, V, F, UV, Fuv, maps, maps_t, env, cams, res, res, n_direct=n_direct,
                   n_bounce=n_bounce, n_light=n_light, seed=seed)


def config(name: str, **overrides) -> Scene:
    """Named workloads.

    * ``tiny``      icosphere 1280 tris, maps 256^2, env 64x32, 4 x 256^2, 64 spp, direct only
    * ``geometry``  blob 99,372 tris, maps 1024^2, env 256x128, 16 x 512^2, 256 spp, direct only
    * ``indirect``  blob 499,392 tris with 3 cavities, maps 2048^2, env 512x256, 8 x 800^2,
                    128 direct + 8 secondary rays x 4 light samples
    * ``precision`` blob 1,997,568 tris with 3 cavities, maps 4096^2 (stored BF16/FP16 by the
                    caller), env 1024x512, 8 x 1024^2, 64 direct + 4 secondary rays x 4 light samples
    """
    if name == "tiny":
        kw = dict()
        kw.update(overrides)
        return icosphere_scene(**kw)
    if name == "geometry":
        kw = dict(n=91, map_res=1024, env_w=256, env_h=128, env_sigma=1.5, views=16, res=512,
                  n_direct=256, seed=2)
        kw.update(overrides)
        return blob_scene(**kw)
    if name == "indirect":
        kw = dict(n=204, map_res=2048, env_w=512, env_h=256, env_sigma=1.5, views=8, res=800,
                  n_direct=128, n_bounce=8, n_light=4, dents=3, seed=3)
        kw.update(overrides)
        return blob_scene(**kw)
    if name == "precision":
        kw = dict(n=408, map_res=4096, env_w=1024, env_h=512, env_sigma=1.5, views=8, res=1024,
                  n_direct=64, n_bounce=4, n_light=4, dents=3, seed=4)
        kw.update(overrides)
        return blob_scene(**kw)
    raise KeyError(name)
