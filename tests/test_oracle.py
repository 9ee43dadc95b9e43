"""Pins of the CPU oracle against facts fixed independently of it.

Each test compares the oracle with something other than itself: published known-answer
vectors, closed forms, FP64 ray casting, quadratures, Monte Carlo convergence to exact
integrals, and finite differences.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import shade
from paper_2608_24109_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def fp64_closest_front(o, d, V, F):
    """FP64 Moller-Trumbore of rays (o [R,3], d [R,3]) against every triangle.
    Returns (tri, bary margin of the hit, depth gap to the next front hit); tri = -1 if none."""
    P0, P1, P2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = P1 - P0, P2 - P0
    nrm = np.cross(e1, e2)
    out_t, out_m, out_g = [], [], []
    for r in range(o.shape[0]):
        pv = np.cross(d[r], e2)
        det = np.einsum("ij,ij->i", e1, pv)
        s = o[r] - P0
        b1 = np.einsum("ij,ij->i", s, pv) / det
        qv = np.cross(s, e1)
        b2 = (qv @ d[r]) / det
        t = np.einsum("ij,ij->i", e2, qv) / det
        b0 = 1 - b1 - b2
        margin = np.minimum(np.minimum(b0, b1), b2)
        front = (nrm @ d[r]) < 0
        ok = (margin > -1e-9) & front & (t > 0)
        if not ok.any():
            out_t.append(-1)
            out_m.append(-np.max(np.where(front & (t > 0), margin, -1.0)) if (front & (t > 0)).any() else 1.0)
            out_g.append(np.inf)
            continue
        ts = np.where(ok, t, np.inf)
        k = int(np.argmin(ts))
        srt = np.sort(ts)
        out_t.append(k)
        out_m.append(margin[k])
        out_g.append(srt[1] - srt[0] if srt.size > 1 else np.inf)
    return np.array(out_t), np.array(out_m), np.array(out_g)


def pixel_rays(cam, W, H, rows):
    py, px = np.meshgrid(rows, np.arange(W), indexing="ij")
    py, px = py.ravel(), px.ravel()
    c = cam.astype(np.float64)
    dx = (px + 0.5 - c[14]) / c[12]
    dy = (c[15] - (py + 0.5)) / c[13]
    d = c[9:12][None] + dx[:, None] * c[3:6][None] + dy[:, None] * c[6:9][None]
    o = np.repeat(c[0:3][None], d.shape[0], 0)
    return o, d, py, px


def faceted(V, F):
    """Un-welded copy: each face gets its own three vertices (flat vertex normals)."""
    V2 = V[F].reshape(-1, 3)
    F2 = np.arange(V2.shape[0]).reshape(-1, 3)
    return V2, F2


def constant_scene(V, F, albedo, env_rgb, res=128, views=1, n_direct=64, env_w=32, env_h=16,
                   n_bounce=0, n_light=0):
    UV, Fuv = scenes.sphere_uv(V, F)
    maps = np.zeros((64, 64, 8), np.float32)
    maps[..., 0:3] = albedo
    maps[..., 3] = 0.5
    maps[..., 4] = 0.0
    maps[..., 7] = 1.0
    env = np.ones((env_h, env_w, 3), np.float32) * np.asarray(env_rgb, np.float32)
    cams = scenes.ring_cameras(views, 3.0, res, res)
    return scenes._finish("const", V, F, UV, Fuv, maps, maps, env, cams, res, res, n_direct=n_direct,
                          n_bounce=n_bounce, n_light=n_light, seed=7, wrap_u=True)


def full_decisions(sc):
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    assert st == 0
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    return keys, tab, dec


# ----------------------------------------------------------------- generators

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_sincos_against_libm():
    s = np.random.default_rng(0).random(2_000_000).astype(np.float32)
    s = np.concatenate([s, np.float32([0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 0.99999994])])
    sn, cs = oracle.sincos2pi(s)
    ang = 2 * np.pi * s.astype(np.float64)
    assert np.abs(sn - np.sin(ang)).max() < 2.5e-7
    assert np.abs(cs - np.cos(ang)).max() < 2.5e-7


# ----------------------------------------------------------------- raster

def test_raster_triangle_major_equals_pixel_brute_force():
    sc = scenes.config("tiny", res=96, views=2)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, 96, 96)
    allpix = np.argwhere(np.ones((2, 96, 96))).astype(np.int32)
    st2, k2 = oracle.raster_pixels(sc.V, sc.F, sc.cams, 96, 96, allpix)
    assert st == 0 and st2 == 0
    assert np.array_equal(k2, keys.reshape(-1))


def test_fill_rule_is_watertight_on_closed_mesh():
    # culling off: every pixel centre is inside exactly as many front as back faces,
    # at most one of each, for a closed convex mesh; and no hole inside the silhouette
    for res in (64, 97, 256):
        sc = scenes.config("tiny", res=res, views=4)
        for v in range(4):
            st, fr, bk = oracle.coverage_counts(sc.V, sc.F, sc.cams[v], res, res)
            assert st == 0
            assert fr.max() <= 1 and bk.max() <= 1
            assert np.array_equal(fr, bk)
            inner = fr[1:-1, 1:-1]
            nb = fr[:-2, 1:-1] & fr[2:, 1:-1] & fr[1:-1, :-2] & fr[1:-1, 2:]
            assert not np.any((nb == 1) & (inner == 0))


@pytest.mark.parametrize("which", ["sphere", "occluded"])
def test_raster_matches_fp64_ray_casting(which):
    V, F = scenes.icosphere(3)
    if which == "occluded":
        V2, F2 = scenes.icosphere(2)
        V = np.concatenate([V, 0.5 * V2 + np.array([0.1, 0.05, 1.2])])
        F = np.concatenate([F, F2 + 642])
    W = H = 80
    cam = scenes.look_at_camera((0.0, 0.0, 3.0), W, H)
    st, keys = oracle.raster_full(V.astype(np.float32), F.astype(np.int32), cam[None], W, H)
    assert st == 0
    o, d, py, px = pixel_rays(cam, W, H, np.arange(H))
    tri, margin, gap = fp64_closest_front(o, d, V.astype(np.float32).astype(np.float64), F)
    got = (keys[0, py, px] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    got[got == 0xFFFFFFFF] = -1
    clear = (margin > 2e-3) & (gap > 1e-3)
    assert clear.sum() > 0.3 * W * H
    assert np.array_equal(got[clear], tri[clear])
    if which == "occluded":
        assert np.any(got[clear] >= 1280)  # the front sphere is seen
        assert np.any((got[clear] < 1280) & (got[clear] >= 0))


def test_guard_band_reported():
    sc = scenes.config("tiny", res=64, views=1)
    cam = sc.cams.copy()
    cam[0, 0:3] = [0.0, 0.0, 0.9]  # eye inside the sphere's bounds: vertices behind the near plane
    st, _ = oracle.raster_full(sc.V, sc.F, cam, 64, 64)
    assert st == oracle.GUARDBAND


# ----------------------------------------------------------------- rays

def test_watertight_rays_through_vertices_and_edges():
    V, F = scenes.icosphere(3)
    V = V.astype(np.float32)
    edges = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    mids = (V[edges[:, 0]] + V[edges[:, 1]]) * np.float32(0.5)
    targets = np.concatenate([V, mids]).astype(np.float32)
    O = np.zeros_like(targets)
    assert oracle.trace(V, F, O, targets, closest=False).all()
    tri, t, front = oracle.trace(V, F, O, targets, closest=True)
    assert (tri >= 0).all() and not front.any()  # seen from inside: back faces
    O2 = (targets * np.float32(3.0)).astype(np.float32)
    D2 = (-targets).astype(np.float32)
    tri2, t2, front2 = oracle.trace(V, F, O2, D2, closest=True)
    assert (tri2 >= 0).all() and front2.all()
    assert np.allclose(t2, 2.0, atol=1e-3)  # from 3p towards the origin, hit near p (|p| ~ 1)


def test_closest_hit_matches_fp64():
    V, F = scenes.icosphere(3)
    rng = np.random.default_rng(3)
    o = rng.normal(size=(400, 3))
    o = 2.5 * o / np.linalg.norm(o, axis=1, keepdims=True)
    tgt = rng.normal(size=(400, 3))
    tgt = 0.7 * tgt / np.linalg.norm(tgt, axis=1, keepdims=True)
    d = tgt - o
    Vf = V.astype(np.float32)
    tri, t, front = oracle.trace(Vf, F, o.astype(np.float32), d.astype(np.float32), closest=True)
    ref, margin, gap = fp64_closest_front(o.astype(np.float32).astype(np.float64),
                                          d.astype(np.float32).astype(np.float64), Vf.astype(np.float64), F)
    ok = margin > 1e-4
    assert ok.sum() > 300
    assert np.array_equal(tri[ok], ref[ok])
    assert front[ok].all()


# ----------------------------------------------------------------- environment sampling

def test_light_direction_spec_matches_fp64():
    env = scenes.env_map(np.random.default_rng(0), 64, 32, 1.0)
    tab = oracle.EnvTable(env)
    rng = np.random.default_rng(1)
    tex = rng.integers(0, 64 * 32, 5000).astype(np.uint32)
    xi = (rng.integers(0, 1 << 24, (5000, 2)) * 2.0 ** -24).astype(np.float32)
    d32 = oracle.light_dirs(tex, xi, 64, 32)
    w64, pdf, i, j = shade.light_directions(tex.astype(np.int64), xi, 64, 32, tab.q, tab.Q)
    assert np.abs(d32 - w64.numpy()).max() < 3e-7
    # row 0 is the +y pole
    top = oracle.light_dirs(np.array([5], np.uint32), np.array([[0.5, 0.0]], np.float32), 64, 32)
    assert top[0, 1] > 0.9999


def test_env_importance_estimator_integrates_env():
    """E(w)/p(w) averaged over texels drawn with probability q/Q and uniform in-texel jitter
    converges to the exact integral of the piecewise-constant map over the sphere."""
    W, H = 48, 24
    env = scenes.env_map(np.random.default_rng(5), W, H, 1.5)
    tab = oracle.EnvTable(env)
    rng = np.random.default_rng(6)
    n = 400_000
    tex = rng.choice(W * H, size=n, p=tab.q / tab.Q)
    xi = rng.random((n, 2))
    w, pdf, i, j = shade.light_directions(tex, xi, W, H, tab.q, tab.Q)
    f = env[i.numpy(), j.numpy()].astype(np.float64) / pdf.numpy()[:, None]
    est, sig = f.mean(0), f.std(0) / math.sqrt(n)
    th = np.pi * np.arange(H + 1) / H
    omega = (2 * np.pi / W) * (np.cos(th[:-1]) - np.cos(th[1:]))
    exact = (env.astype(np.float64) * omega[:, None, None]).sum((0, 1))
    assert np.all(np.abs(est - exact) < 5 * sig + 1e-12)


def test_texel_choice_frequencies_follow_weights():
    """The stratified integer-CDF picker of decide.c, fed by the Philox streams, picks texel t
    with frequency q_t / Q (chi-square over all decisions of many pixels)."""
    sc = scenes.config("tiny", res=48, views=1, env_w=16, env_h=8, n_direct=64)
    keys, tab, dec = full_decisions(sc)
    t = dec.dtex[dec.covered].ravel()
    n = t.size
    counts = np.bincount(t, minlength=tab.q.size)
    expect = n * tab.q.astype(np.float64) / tab.Q
    m = expect > 5
    chi2 = ((counts[m] - expect[m]) ** 2 / expect[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    # every pixel's 64 samples are stratified: one sample per 1/64 of the CDF
    assert n > 10000


# ----------------------------------------------------------------- shading pieces

def test_bilinear_ramp_and_wrap():
    H, W = 8, 16
    ramp = np.zeros((H, W, 2))
    ramp[..., 0] = np.arange(W)[None, :]
    ramp[..., 1] = np.arange(H)[:, None]
    M = torch.tensor(ramp)
    uv = torch.tensor([[0.3, 0.6], [0.5, 0.5], [(3 + 0.5) / W, (2 + 0.5) / H]], dtype=torch.float64)
    out = shade.bilinear(M, uv, wrap_u=False)
    assert torch.allclose(out[:, 0], uv[:, 0] * W - 0.5)
    assert torch.allclose(out[:, 1], uv[:, 1] * H - 0.5)
    # wrapping: half way between the last and the first column
    out = shade.bilinear(M, torch.tensor([[0.0, 0.5]], dtype=torch.float64), wrap_u=True)
    assert abs(out[0, 0].item() - 0.5 * (W - 1)) < 1e-12
    out = shade.bilinear(M, torch.tensor([[1.0, 0.5]], dtype=torch.float64), wrap_u=True)
    assert abs(out[0, 0].item() - 0.5 * (W - 1)) < 1e-12


def test_vertex_frames_on_sphere():
    V, F = scenes.icosphere(3)
    UV, Fuv = scenes.sphere_uv(V, F)
    sgn = shade.face_uv_sign(UV.astype(np.float32), Fuv)
    nv, tuv = shade.vertex_frames(torch.tensor(V), F, UV, Fuv, UV.shape[0], sgn)
    assert (torch.einsum("ij,ij->i", nv, torch.tensor(V)) > 0.995).all()
    # tangent = dP/du = direction of increasing phi: (cos phi, 0, sin phi) away from poles
    owner = np.zeros(UV.shape[0], np.int64)
    owner[Fuv.ravel()] = F.ravel()
    P = V[owner]
    phi = 2 * np.pi * UV[:, 0]
    ref = np.stack([np.cos(phi), np.zeros_like(phi), np.sin(phi)], 1)
    away = np.abs(P[:, 1]) < 0.9
    assert (np.einsum("ij,ij->i", tuv.numpy()[away], ref[away]) > 0.95).all()
    assert len(set(sgn.tolist())) == 1


# ---- the tangent-space normal of Eq. 11, pinned by geometry on a flat quad

def _quad_chart(flip_u=False, flip_v=False):
    """A unit square in a tilted plane, P(s, t) = O + s a + t b with a, b orthonormal, two
    counter-clockwise faces seen from a x b, and UVs u = s, v = t, mirrored in u and/or v.  By
    construction dP/du = +-a and dP/dv = +-b."""
    a = np.array([0.6, 0.8, 0.0])
    b = np.array([-0.48, 0.36, 0.8])
    O = np.array([0.2, -0.1, 0.3])
    st = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    V = O + st[:, :1] * a + st[:, 1:] * b
    F = np.array([[0, 1, 2], [0, 2, 3]])
    UV = st.copy()
    if flip_u:
        UV[:, 0] = 1 - UV[:, 0]
    if flip_v:
        UV[:, 1] = 1 - UV[:, 1]
    dPdu = -a if flip_u else a
    dPdv = -b if flip_v else b
    return V, F, UV.astype(np.float32), dPdu, dPdv, np.cross(a, b)


def _oracle_ns(V, F, UV, q, bary=(0.2, 0.3, 0.5), face=0):
    """n_s of the oracle at a point of `face` for a constant normal-map value q, through its own
    chain: UV handedness, vertex frames, bilinear fetch of a constant map, Eq. 11."""
    sgn = shade.face_uv_sign(UV, F)
    nv, tuv = shade.vertex_frames(torch.tensor(V, dtype=torch.float64), F, UV, F, UV.shape[0], sgn)
    att = torch.tensor([[0.5, 0.5, 0.5, 0.5, 0.0, *q]], dtype=torch.float64)
    b = torch.tensor([bary], dtype=torch.float64)
    fv = torch.as_tensor(F[face:face + 1], dtype=torch.long)
    ns, _, _, _ = shade._material(att, b, nv[fv], tuv[fv], torch.tensor(sgn[face:face + 1]), True)
    return ns[0].numpy()


def _normal_map_pins():
    """The tangent frame's meaning, independent of any formula: the map's x axis follows
    increasing u, its y axis increasing v, its z axis the surface normal; a tilted value mixes
    them and is renormalised.  In all four UV orientations (mirrored charts have s_f = -1)."""
    for flip_u in (False, True):
        for flip_v in (False, True):
            V, F, UV, du, dv, n = _quad_chart(flip_u, flip_v)
            for face in (0, 1):
                for q, want in (((1, 0, 0), du), ((0, 1, 0), dv), ((0, 0, 1), n), ((0.6, 0, 0.8), 0.6 * du + 0.8 * n),
                                ((0, -0.6, 0.8), -0.6 * dv + 0.8 * n), ((3, 4, 0), (3 * du + 4 * dv) / 5)):
                    got = _oracle_ns(V, F, UV, q, face=face)
                    assert np.abs(got - want).max() < 1e-12, (flip_u, flip_v, face, q, got, want)


def test_normal_map_axes_follow_u_v_and_the_normal():
    _normal_map_pins()


def _planted(kind):
    def material(att, b, nvert, tvert, sgn_f, metallic):
        a, r = att[..., 0:3], att[..., 3]
        m = att[..., 4] if metallic else torch.zeros_like(att[..., 4])
        n = shade._normalize((b[..., None] * nvert).sum(-2))
        ti = (b[..., None] * tvert).sum(-2)
        T = shade._normalize(ti - shade._dot(n, ti)[..., None] * n)
        s = sgn_f[..., None]
        B = {"swap": s * torch.linalg.cross(n, T), "flip": -s * torch.linalg.cross(n, T),
             "no_sign": torch.linalg.cross(n, T)}[kind]
        nt = shade._normalize(att[..., 5:8])
        if kind == "swap":
            T, B = B, T
        return T * nt[..., 0:1] + B * nt[..., 1:2] + n * nt[..., 2:3], a, r, m
    return material


@pytest.mark.parametrize("kind", ["swap", "flip", "no_sign"])
def test_normal_map_pins_catch_planted_mistakes(kind, monkeypatch):
    """A T/B swap, a flipped B or a dropped handedness sign planted in the oracle's Eq. 11 each
    fails the pins above."""
    monkeypatch.setattr(shade, "_material", _planted(kind))
    with pytest.raises(AssertionError):
        _normal_map_pins()


def _frame(n):
    n = n / np.linalg.norm(n)
    return torch.tensor(n)


def test_brdf_normal_incidence_closed_form():
    n = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64)
    a = torch.tensor([[0.5, 0.25, 0.75]], dtype=torch.float64)
    for r, m in [(0.5, 0.0), (0.3, 1.0), (0.9, 0.4)]:
        rr = torch.tensor([r], dtype=torch.float64)
        mm = torch.tensor([m], dtype=torch.float64)
        got = shade.brdf_cos(n, n, n, a, rr, mm)
        alpha = r * r
        F0 = (1 - m) * 0.04 + m * a
        want = (1 - m) * a / math.pi + F0 / (math.pi * alpha ** 2) / (4 + 1e-6)
        assert torch.allclose(got, want, rtol=1e-12)


def _hemisphere_quadrature(nt=800, npp=400, lobe_scale=None):
    # midpoint rule in (theta, phi) over the upper hemisphere, theta warped towards 0
    u = (np.arange(nt) + 0.5) / nt
    th = (np.pi / 2) * u ** 2
    dth = (np.pi / 2) * 2 * u / nt
    ph = 2 * np.pi * (np.arange(npp) + 0.5) / npp
    T, P = np.meshgrid(th, ph, indexing="ij")
    w = (np.sin(T) * dth[:, None] * (2 * np.pi / npp))
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    return d.reshape(-1, 3), w.ravel()


def test_brdf_diffuse_albedo_and_reciprocity():
    d, w = _hemisphere_quadrature()
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand(d.shape[0], 3)
    wi = torch.tensor(d)
    wo = _frame(np.array([0.3, -0.2, 0.8]))[None].expand_as(wi)
    a = torch.tensor([0.2, 0.5, 0.9], dtype=torch.float64).expand_as(wi)
    m = torch.zeros(d.shape[0], dtype=torch.float64)
    r = torch.full((d.shape[0],), 0.5, dtype=torch.float64)
    diff = shade.brdf_cos(n, wi, wo, a, r, m, specular=False)
    integ = (diff * torch.tensor(w)[:, None]).sum(0)
    assert torch.allclose(integ, torch.tensor([0.2, 0.5, 0.9], dtype=torch.float64), rtol=1e-5)
    # reciprocity of f_r = brdf_cos / cos_i
    rng = np.random.default_rng(2)
    A = rng.normal(size=(200, 3)); A[:, 2] = np.abs(A[:, 2])
    B = rng.normal(size=(200, 3)); B[:, 2] = np.abs(B[:, 2])
    A /= np.linalg.norm(A, axis=1, keepdims=True); B /= np.linalg.norm(B, axis=1, keepdims=True)
    nn = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand(200, 3)
    aa = torch.tensor([0.6, 0.4, 0.2], dtype=torch.float64).expand(200, 3)
    rr = torch.tensor(rng.uniform(0.2, 0.9, 200))
    mm = torch.tensor(rng.uniform(0, 1, 200))
    fab = shade.brdf_cos(nn, torch.tensor(A), torch.tensor(B), aa, rr, mm) / torch.tensor(A[:, 2:3])
    fba = shade.brdf_cos(nn, torch.tensor(B), torch.tensor(A), aa, rr, mm) / torch.tensor(B[:, 2:3])
    assert torch.allclose(fab, fba, rtol=1e-10)


def test_ggx_lobe_normalisation():
    """With F = 1 (metallic, white) and a narrow lobe, the specular term at normal
    viewing integrates to int D (n.h) dw_h = 1 up to the Smith shadowing loss."""
    d, w = _hemisphere_quadrature(nt=2000, npp=64)
    h = torch.tensor(d)
    nvec = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64)
    wo = nvec.expand_as(h)
    wi = 2 * (h @ nvec)[:, None] * h - wo
    keep = (wi @ nvec) > 0
    jac = 4 * (h @ nvec)  # dw_i = 4 (h . w_o) dw_h
    nn = nvec.expand_as(h)
    one = torch.ones(h.shape[0], dtype=torch.float64)
    for r in (0.2236, 0.3):
        spec = shade.brdf_cos(nn, wi, wo, torch.ones_like(h), one * r, one) - 0.0
        val = (spec[:, 0] * jac * torch.tensor(w))[keep].sum().item()
        assert 0.97 < val < 1.0 + 1e-3, val


def test_ggx_white_furnace_and_closed_form_at_alpha_one():
    """Specular lobe with F = 1 (metallic, white base colour) in a white furnace.  Its
    directional albedo E(mu_o) = int f_s cos_i dw_i, integrated over half vectors with
    dw_i = 4 (h.w_o) dw_h, never exceeds 1 (the lobe loses energy to Smith shadowing, it does
    not create any).  At r = 1 (alpha = 1) the GGX distribution is the constant 1/pi and
    G1(c) = 2c / (1 + c), so E(mu_o) = (1/pi) / (1 + mu_o) * int mu_i / (1 + mu_i) dw_i
    = 2 (1 - ln 2) / (1 + mu_o) in closed form: a wrong normalisation of D, a wrong G1, a
    missing 4 in the denominator or a missing cosine each break it."""
    d, w = _hemisphere_quadrature(nt=1500, npp=128)
    h = torch.tensor(d)
    W = torch.tensor(w)
    n = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64).expand_as(h)
    one = torch.ones(h.shape[0], dtype=torch.float64)
    for deg in (0.0, 30.0, 60.0, 80.0, 89.0):
        t = math.radians(deg)
        wo = torch.tensor([math.sin(t), 0.0, math.cos(t)], dtype=torch.float64).expand_as(h)
        hv = (h * wo).sum(1)
        wi = 2 * hv[:, None] * h - wo
        keep = (wi[:, 2] > 0) & (hv > 0)
        for r in (0.08, 0.2, 0.4, 0.7, 1.0):
            f = shade.brdf_cos(n, wi, wo, torch.ones_like(h), one * r, one)[:, 0]
            E = (f * 4 * hv * W)[keep].sum().item()
            assert E <= 1.0 + 2e-3, (deg, r, E)
            if r == 1.0:
                want = 2 * (1 - math.log(2)) / (1 + math.cos(t))
                assert abs(E - want) <= 2e-3 * want, (deg, E, want)


# ----------------------------------------------------------------- estimators

def test_furnace_diffuse_sphere_under_constant_env():
    """Convex faceted sphere (n_s = n_g), Lambertian albedo a, constant environment c:
    the direct estimator is unbiased for L = a * c (Eq. 12 with Vis = 1 above the surface)."""
    V, F = faceted(*scenes.icosphere(3))
    albedo = np.array([0.3, 0.6, 0.9], np.float32)
    c = np.array([0.5, 1.0, 2.0], np.float32)
    sc = constant_scene(V, F, albedo, c, res=96, n_direct=64)
    keys, tab, dec = full_decisions(sc)
    Vt, Mt, Et = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, Vt, Mt, Et, specular=False).numpy()
    ratio = I / (albedo * c)
    mean = ratio.mean(0)
    sig = ratio.std(0) / math.sqrt(ratio.shape[0])
    assert dec.pix.shape[0] > 3000
    assert np.all(np.abs(mean - 1.0) < 5 * sig + 1e-9), (mean, sig)
    # white furnace: albedo 1, E = 1 -> 1
    sc1 = constant_scene(V, F, np.ones(3, np.float32), np.ones(3, np.float32), res=64, n_direct=64)
    keys, tab, dec = full_decisions(sc1)
    Vt, Mt, Et = shade.scene_tensors(sc1)
    I1 = shade.render_image(sc1, tab, dec, Vt, Mt, Et, specular=False).numpy()[:, 0]
    assert abs(I1.mean() - 1.0) < 5 * I1.std() / math.sqrt(I1.size)


def test_linearity_in_env_and_albedo():
    sc = scenes.config("tiny", res=48, views=1)
    keys, tab, dec = full_decisions(sc)
    Vt, Mt, Et = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, Vt, Mt, Et)
    sc2 = scenes.config("tiny", res=48, views=1)
    sc2.env = sc2.env * np.float32(2.0)
    keys2, tab2, dec2 = full_decisions(sc2)
    assert np.array_equal(dec2.dtex, dec.dtex) and np.array_equal(dec2.dvis, dec.dvis)
    I2 = shade.render_image(sc2, tab2, dec2, Vt, Mt, Et * 2)
    assert torch.allclose(I2, 2 * I, rtol=1e-12)


def test_indirect_vanishes_on_convex_mesh():
    sc = scenes.config("tiny", res=48, views=1, n_bounce=4, n_light=2)
    keys, tab, dec = full_decisions(sc)
    assert (dec.stri == -1).all()
    Vt, Mt, Et = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, Vt, Mt, Et)
    sc0 = scenes.config("tiny", res=48, views=1)
    keys0, tab0, dec0 = full_decisions(sc0)
    I0 = shade.render_image(sc0, tab0, dec0, Vt, Mt, Et)
    assert torch.equal(I, I0)


def test_indirect_sees_cavity():
    sc = scenes.config("indirect", n=12, map_res=64, env_w=32, env_h=16, views=1, res=48, n_direct=16,
                       n_bounce=8, n_light=4)
    keys, tab, dec = full_decisions(sc)
    valid = dec.stri >= 0
    assert valid.any()
    # near-ties between the best and second-best hit are reported, not hidden
    assert np.isfinite(dec.sgap[valid]).any()


def test_no_secondary_material_is_the_default_material():
    """The No Secondary Material ablation (Sec. 6.4) equals the full estimator on maps that
    already hold the default material everywhere, and differs from it on textured maps."""
    sc = scenes.config("indirect", n=24, map_res=64, env_w=32, env_h=16, views=2, res=48, n_direct=16,
                       n_bounce=8, n_light=4)
    keys, tab, dec = full_decisions(sc)
    assert (dec.stri >= 0).sum() > 20
    flat = np.zeros_like(sc.maps)
    flat[..., 0:4] = 0.5
    flat[..., 7] = 1.0
    sc.metallic = True
    for maps, same in ((flat, True), (sc.maps, False)):
        sc.maps = maps
        Vt, Mt, Et = shade.scene_tensors(sc)
        sc.secondary_material = True
        I_full = shade.render_image(sc, tab, dec, Vt, Mt, Et)
        sc.secondary_material = False
        I_abl = shade.render_image(sc, tab, dec, Vt, Mt, Et)
        if same:
            assert torch.equal(I_full, I_abl)
        else:
            d = (I_full - I_abl).abs().max().item()
            assert d > 1e-3 * I_full.abs().max().item()
    # no map gradient flows from the secondary hits: the ablation's map gradient lives on the
    # texels of the primary footprints (the support of the direct-only gradient), while the
    # full estimator also reaches texels seen only through secondary hits
    g = np.random.default_rng(2).normal(size=(dec.pix.shape[0], 3))
    Vt, Mt, Et = shade.scene_tensors(sc)
    grads = {}
    for name, lam, mat in (("direct", 0.0, True), ("ablation", 1.0, False), ("full", 1.0, True)):
        sc.lambda_ind, sc.secondary_material = lam, mat
        grads[name] = shade.backward(sc, tab, dec, Vt, Mt, Et, g)[1].abs().sum(-1)
    primary = grads["direct"] > 0
    assert primary.any()
    assert (grads["ablation"][~primary] == 0).all()
    assert (grads["full"][~primary] > 0).any()


# ----------------------------------------------------------------- gradients

def test_autograd_matches_central_differences():
    sc = scenes.config("tiny", res=64, views=1)
    keys, tab, dec = full_decisions(sc)
    rng = np.random.default_rng(11)
    sel = rng.choice(dec.pix.shape[0], 48, replace=False)
    sub = oracle.Decisions(sc, tab, dec.pix[sel], dec.keys[sel])
    Vt, Mt, Et = shade.scene_tensors(sc)
    g = torch.tensor(rng.normal(size=(48, 3)))
    gV, gM, gE = shade.backward(sc, tab, sub, Vt, Mt, Et, g)

    def loss(V, M, E):
        return (shade.shade(sc, tab, sub, V, M, E) * g).sum().item()

    def fd(which, index, h):
        ts = [Vt.clone(), Mt.clone(), Et.clone()]
        ts[which][index] += h
        lp = loss(*ts)
        ts[which][index] -= 2 * h
        lm = loss(*ts)
        return (lp - lm) / (2 * h)

    picks = []
    nzM = torch.nonzero(gM.abs() > 1e-6 * gM.abs().max())
    for k in rng.choice(nzM.shape[0], 8, replace=False):
        picks.append((1, tuple(nzM[k].tolist()), 1e-6, gM))
    nzE = torch.nonzero(gE.abs() > 1e-6 * gE.abs().max())
    for k in rng.choice(nzE.shape[0], 6, replace=False):
        idx = tuple(nzE[k].tolist())
        picks.append((2, idx, 1e-6 * float(Et[idx]), gE))
    nzV = torch.nonzero(gV.abs() > 1e-6 * gV.abs().max())
    for k in rng.choice(nzV.shape[0], 8, replace=False):
        picks.append((0, tuple(nzV[k].tolist()), 1e-7, gV))
    for which, idx, h, G in picks:
        num = fd(which, idx, h)
        ana = G[idx].item()
        assert abs(num - ana) <= 1e-5 * max(abs(ana), 1e-3 * G.abs().max().item()), (which, idx, num, ana)


def _l_scene(n_bounce, n_light, seed, lambda_ind=1.0):
    """Floor quad (y = 0, x in [-1, 0.5], z in [-1, 1], facing +y) and a wall quad (x = 0.5,
    y in [0, 1], z in [-1, 1], facing -x); constant grey Lambertian maps, flat normals."""
    V = np.array([[-1, 0, -1], [-1, 0, 1], [0.5, 0, 1], [0.5, 0, -1],
                  [0.5, 0, -1], [0.5, 0, 1], [0.5, 1, 1], [0.5, 1, -1]], np.float64)
    F = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]])
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert n[0, 1] > 0 and n[2, 0] < 0
    UV = np.array([[0.1, 0.1], [0.1, 0.9], [0.9, 0.9], [0.9, 0.1]] * 2)
    Fuv = F.copy()
    maps = np.zeros((8, 8, 8), np.float32)
    maps[..., 0:3] = 0.5
    maps[..., 3] = 0.5
    maps[..., 7] = 1.0
    env = scenes.env_map(np.random.default_rng(3), 16, 8, 0.5)
    W = 64
    cam = scenes.look_at_camera((-1.2, 1.4, 0.4), W, W, target=(0.0, 0.0, 0.0))
    sc = scenes._finish("L", V, F, UV, Fuv, maps, maps, env, cam[None], W, W, n_direct=16, n_bounce=n_bounce,
                        n_light=n_light, seed=seed, lambda_ind=lambda_ind)
    sc.metallic = False
    return sc


def _floor_pixel(sc):
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    o, d = shade.camera_rays(sc.cams, pix)
    t = -o[:, 1] / d[:, 1]
    x = (o + t[:, None] * d).numpy()
    tri = (keys[pix[:, 0], pix[:, 1], pix[:, 2]] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    on_floor = tri < 2
    k = np.argmin(np.where(on_floor, np.abs(x[:, 0] - 0.1) + np.abs(x[:, 2]), np.inf))
    return pix[k:k + 1], keys[pix[k, 0], pix[k, 1], pix[k, 2]:pix[k, 2] + 1].copy(), x[k]


def _indirect_by_quadrature(sc, x):
    """L_ind(x) = int f_d(x) L_sec(y(w)) cos(w) dw over the floor's upper hemisphere (Eq. 19 in
    the limit), L_sec(y) = int E Vis f_d(y) max(n.w', 0) dw' (Eq. 18), by midpoint quadrature
    with analytic ray/plane visibility; the environment is piecewise constant per texel."""
    fd = 0.5 / math.pi
    env = sc.env.astype(np.float64)
    He, We = env.shape[:2]
    sub = 6
    th = math.pi * (np.arange(He * sub) + 0.5) / (He * sub)
    ph = 2 * math.pi * (np.arange(We * sub) + 0.5) / (We * sub)
    T, P = np.meshgrid(th, ph, indexing="ij")
    dl = np.stack([np.sin(T) * np.sin(P), np.cos(T), -np.sin(T) * np.cos(P)], -1).reshape(-1, 3)
    dw_l = (np.sin(T) * (math.pi / (He * sub)) * (2 * math.pi / (We * sub))).ravel()
    El = env[(np.arange(He * sub) // sub)[:, None].repeat(We * sub, 1).ravel(),
             (np.arange(We * sub) // sub)[None, :].repeat(He * sub, 0).ravel()]
    nw = np.array([-1.0, 0.0, 0.0])

    def l_sec(y):
        cos = dl @ nw
        ok = cos > 0
        # blocked when the ray y + t w' meets the floor rectangle
        with np.errstate(divide="ignore", invalid="ignore"):
            t = -y[1] / dl[:, 1]
            px, pz = y[0] + t * dl[:, 0], y[2] + t * dl[:, 2]
        blocked = (dl[:, 1] < 0) & (t > 0) & (px >= -1) & (px <= 0.5) & (pz >= -1) & (pz <= 1)
        w = np.where(ok & ~blocked, cos * dw_l, 0.0)
        return fd * (El * w[:, None]).sum(0)

    nt, npp = 96, 192
    u = (np.arange(nt) + 0.5) / nt
    tt = (math.pi / 2) * u
    pp = 2 * math.pi * (np.arange(npp) + 0.5) / npp
    TT, PP = np.meshgrid(tt, pp, indexing="ij")
    dirs = np.stack([np.sin(TT) * np.cos(PP), np.cos(TT), np.sin(TT) * np.sin(PP)], -1).reshape(-1, 3)
    dw = (np.sin(TT) * (math.pi / 2 / nt) * (2 * math.pi / npp)).ravel()
    total = np.zeros(3)
    for w, a in zip(dirs, dw):
        if w[0] <= 0:
            continue
        t = (0.5 - x[0]) / w[0]
        y = x + t * w
        if not (0 <= y[1] <= 1 and -1 <= y[2] <= 1):
            continue
        total += fd * l_sec(y) * w[1] * a
    return total


def test_indirect_estimator_converges_to_quadrature():
    """Eq. 19 with Eq. 18: the one-bounce estimator on a floor point in front of a wall
    converges to the double integral (independent FP64 quadrature with analytic visibility)."""
    ests = []
    for seed in range(4):
        sc = _l_scene(1024, 64, seed)
        pix, keys, x = _floor_pixel(sc)
        tab = oracle.EnvTable(sc.env)
        dec = oracle.Decisions(sc, tab, pix, keys)
        assert (dec.stri >= 0).sum() > 100
        V, M, E = shade.scene_tensors(sc)
        full = shade.render_image(sc, tab, dec, V, M, E).numpy()[0]
        sc0 = _l_scene(1024, 64, seed, lambda_ind=0.0)
        dec0 = oracle.Decisions(sc0, tab, pix, keys)
        direct = shade.render_image(sc0, tab, dec0, V, M, E).numpy()[0]
        ests.append(full - direct)
    ests = np.array(ests)
    est, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    ref = _indirect_by_quadrature(sc, x)
    assert np.all(ref > 0)
    assert np.all(np.abs(est - ref) <= 4 * se + 0.02 * ref), (est, se, ref)
