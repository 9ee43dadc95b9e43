"""GPU path (libexmesh through its C ABI) against the CPU oracle, element by element.

Bars (spec tolerances): visibility-buffer keys bit-exact; radiance per pixel
|g - o| <= 1e-4 * max(|o|, 1e-3 * mean(o)); gradients ||g - o|| / ||o|| <= 1e-3 per tensor.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

RAD_TOL = 1e-4
GRAD_TOL = 1e-3


def _renderer(sc, **kw):
    from paper_2608_24109_b300.render import Renderer
    return Renderer.from_scene(sc, **kw)


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def check_radiance(g, o, what=""):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    mean = np.abs(o).mean()
    tol = RAD_TOL * np.maximum(np.abs(o), 1e-3 * mean)
    err = np.abs(g - o)
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} values outside tolerance; worst rel " \
                          f"{(err / np.maximum(np.abs(o), 1e-3 * mean)).max():.3e}"


def check_grad(g, o, what):
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-30)
    assert rel <= GRAD_TOL, f"{what}: relative L2 error {rel:.3e}"


def keys_u64(t):
    return t.cpu().numpy().view(np.uint64)


def ragged_tiny(W=97, H=61, views=2, n_direct=64, **kw):
    sc = scenes.config("tiny", n_direct=n_direct, **kw)
    cams = np.stack([scenes.look_at_camera(c[0:3], W, H) for c in sc.cams[:views]])
    sc.cams, sc.width, sc.height = cams, W, H
    return sc


def small_cavity(res=64, views=2, n=24, n_direct=16, n_bounce=8, n_light=4):
    sc = scenes.config("indirect", n=n, map_res=128, env_w=64, env_h=32, views=views, res=res, n_direct=n_direct,
                       n_bounce=n_bounce, n_light=n_light)
    return sc


def gpu_forward(sc, maps=None, env=None, **kw):
    r = _renderer(sc, **kw)
    M = _dev(sc.maps if maps is None else maps)
    E = _dev(sc.env if env is None else env)
    out = r.forward(M, E)
    r.sync()
    return r, M, E, out


def oracle_full(sc, maps=None):
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    assert st == 0
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    V, M, E = shade.scene_tensors(sc)
    if maps is not None:
        M = torch.as_tensor(maps, dtype=torch.float64)
    return keys, tab, dec, V, M, E


# ----------------------------------------------------------------- visibility

@pytest.mark.parametrize("size", [(256, 256, 4), (97, 61, 2), (33, 200, 1)])
def test_visibility_buffer_bit_exact(size):
    W, H, views = size
    sc = ragged_tiny(W, H, views)
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, W, H)
    assert st == 0
    got = keys_u64(r.visbuf())
    assert np.array_equal(got, keys)
    cov, samples = r.stats()
    assert cov == int(((keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)).sum())
    assert samples == cov * sc.n_direct


def test_visibility_buffer_bit_exact_blob():
    sc = scenes.config("geometry", views=3, res=160)
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    assert np.array_equal(keys_u64(r.visbuf()), keys)


def _box_pixels(sc):
    """Pixel-box sizes of the front-facing triangles as projected (float64, without snapping)."""
    cam = sc.cams[0].astype(np.float64)
    d = sc.V.astype(np.float64) - cam[0:3]
    w = d @ cam[9:12]
    sx = cam[14] + cam[12] * (d @ cam[3:6]) / w
    sy = cam[15] - cam[13] * (d @ cam[6:9]) / w
    X, Y = sx[sc.F], sy[sc.F]
    area = (Y[:, 1] - Y[:, 0]) * (X[:, 2] - X[:, 0]) - (X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0])
    return ((X.max(1) - X.min(1)) * (Y.max(1) - Y.min(1)))[area > 0]


@pytest.mark.parametrize("eye,size", [((0.0, 0.3, 1.45), (256, 192)), ((0.9, 0.25, 0.95), (97, 61)),
                                      ((0.0, 0.0, 1.3), (640, 480))])
def test_visibility_buffer_bit_exact_close_camera(eye, size):
    """A camera close to the surface: many triangles have pixel boxes of more than 256 pixels,
    which the raster hands to its warp-per-triangle kernel; the keys stay bit-exact."""
    W, H = size
    sc = scenes.config("tiny", n_direct=8)
    sc.cams, sc.width, sc.height = scenes.look_at_camera(eye, W, H)[None], W, H
    assert (_box_pixels(sc) > 400).sum() >= 20
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, W, H)
    assert st == 0
    assert np.array_equal(keys_u64(r.visbuf()), keys)
    r.close()


def test_visibility_buffer_bit_exact_when_the_large_triangle_list_is_full():
    """600,000 front-facing triangles, over 300,000 of them with pixel boxes of several hundred
    pixels: more than the raster's list of 2^18 large triangles holds.  The overflow is
    rasterised by the triangles' own threads, and the keys stay bit-exact with the oracle."""
    rng = np.random.default_rng(21)
    W = H = 64
    K = 600_000
    cam = scenes.look_at_camera((0.0, 0.0, 3.0), W, H)
    c = rng.uniform(-0.9, 0.9, (K, 1, 3)) * np.array([1.0, 1.0, 0.5])
    V = (c + rng.uniform(-0.8, 0.8, (K, 3, 3)) * np.array([1.0, 1.0, 0.2])).reshape(-1, 3)
    F = np.arange(3 * K).reshape(K, 3)
    sc = scenes._finish("overlap", V, F, rng.uniform(0.0, 1.0, (3 * K, 2)), F, scenes.material_maps(rng, 32),
                        scenes.material_maps(rng, 32), scenes.env_map(rng, 32, 16, 1.0), cam[None], W, H, seed=3,
                        n_direct=4)
    # wind every triangle counter-clockwise on screen (y down), so that none is culled
    d = sc.V.astype(np.float64) - cam[0:3]
    w = d @ cam[9:12]
    X = (cam[14] + cam[12] * (d @ cam[3:6]) / w)[sc.F]
    Y = (cam[15] - cam[13] * (d @ cam[6:9]) / w)[sc.F]
    a2 = (Y[:, 1] - Y[:, 0]) * (X[:, 2] - X[:, 0]) - (X[:, 1] - X[:, 0]) * (Y[:, 2] - Y[:, 0])
    flip = a2 < 0
    sc.F[flip] = sc.F[flip][:, [0, 2, 1]]
    box = (np.minimum(X.max(1), W) - np.maximum(X.min(1), 0)) * (np.minimum(Y.max(1), H) - np.maximum(Y.min(1), 0))
    assert (box > 300).sum() > (1 << 18) + 1000
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, W, H)
    assert st == 0
    assert np.array_equal(keys_u64(r.visbuf()), keys)
    r.close()


def test_env_distribution_total_matches():
    from paper_2608_24109_b300 import native as N
    for (w, h, sig) in [(64, 32, 1.0), (256, 128, 1.5), (13, 7, 2.0)]:
        env = scenes.env_map(np.random.default_rng(w), w, h, sig)
        sc = scenes.config("tiny", res=32, views=1, env_w=w, env_h=h)
        sc.env = env
        r = _renderer(sc)
        r.prepare_env(_dev(env))
        r.sync()
        assert N.exm_env_total(r.env) == oracle.EnvTable(env).Q


# ----------------------------------------------------------------- radiance

def test_forward_parity_tiny_ragged_full_frame():
    sc = ragged_tiny(97, 61, 2)
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]]
    check_radiance(g, I, "tiny ragged")
    # background stays exactly zero
    bg = np.ones(g.shape[:0] + out.shape[:3], bool)
    bg[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]] = False
    assert (out.cpu().numpy()[bg] == 0).all()


@pytest.mark.parametrize("env_w,env_h", [(24, 1024), (20, 1100)])
def test_forward_parity_tall_environments(env_w, env_h):
    """The ray-generation kernels stage the row phase of the texel search in shared memory for
    environments of up to 1024 rows and search global memory above: both sides of that limit,
    with indirect light (both kernels), against the oracle."""
    sc = small_cavity(res=40, views=1, n=16, n_direct=24, n_bounce=4, n_light=3)
    sc.env = scenes.env_map(np.random.default_rng(env_h), env_w, env_h, 1.5)
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]]
    check_radiance(g, I, f"env {env_w}x{env_h}")
    r.close()


def test_forward_parity_tiny_full_size_sampled():
    sc = scenes.config("tiny")
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    sel = pix[np.random.default_rng(0).choice(pix.shape[0], 3000, replace=False)]
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, sel, keys[sel[:, 0], sel[:, 1], sel[:, 2]])
    V, Mo, Eo = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[sel[:, 0], sel[:, 1], sel[:, 2]]
    check_radiance(g, I, "tiny full-size sample")


def test_forward_is_deterministic():
    sc = ragged_tiny(64, 64, 2)
    r, M, E, out = gpu_forward(sc)
    out2 = r.forward(M, E)
    r.sync()
    assert torch.equal(out, out2)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_forward_parity_low_precision_maps(dtype):
    sc = ragged_tiny(80, 72, 1)
    Mq = torch.as_tensor(sc.maps).to(dtype)
    r = _renderer(sc)
    out = r.forward(Mq.cuda().contiguous(), _dev(sc.env))
    r.sync()
    keys, tab, dec, V, Mo, Eo = oracle_full(sc, maps=Mq.to(torch.float64).numpy())
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    check_radiance(out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]], I, str(dtype))


def test_forward_parity_indirect_full_frame():
    sc = small_cavity()
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    assert np.array_equal(keys_u64(r.visbuf()), keys)
    assert (dec.stri >= 0).sum() > 100
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]]
    check_radiance(g, I, "cavity indirect")


def test_no_secondary_material_flag():
    sc = small_cavity()
    sc.secondary_material = False
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    assert (dec.stri >= 0).sum() > 100
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]]
    check_radiance(g, I, "no secondary material")


def test_no_metallic_flag():
    sc = ragged_tiny(48, 40, 1)
    sc.metallic = False
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    check_radiance(out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]], I, "dielectric")


# ----------------------------------------------------------------- gradients

def _grad_compare(sc, npix, seed=0, subset=True):
    r, M, E, out = gpu_forward(sc)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    rng = np.random.default_rng(seed)
    sel = pix[rng.choice(pix.shape[0], min(npix, pix.shape[0]), replace=False)] if subset else pix
    g = rng.normal(size=(sel.shape[0], 3))
    grad = np.zeros(out.shape, np.float32)
    grad[sel[:, 0], sel[:, 1], sel[:, 2]] = g
    gm = torch.zeros_like(M)
    gE = torch.zeros_like(E)
    gV = torch.zeros((sc.V.shape[0], 3), dtype=torch.float32, device="cuda")
    r.backward(M, _dev(grad), gm, gE, gV)
    r.sync()
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, sel, keys[sel[:, 0], sel[:, 1], sel[:, 2]])
    V, Mo, Eo = shade.scene_tensors(sc)
    oV, oM, oE = shade.backward(sc, tab, dec, V, Mo, Eo, grad[sel[:, 0], sel[:, 1], sel[:, 2]].astype(np.float64))
    check_grad(gm.cpu().numpy(), oM.numpy(), "dL/dmaps")
    check_grad(gE.cpu().numpy(), oE.numpy(), "dL/dE")
    check_grad(gV.cpu().numpy(), oV.numpy(), "dL/dV")
    return r


def test_backward_parity_tiny():
    _grad_compare(ragged_tiny(96, 80, 2), 4000)


def test_backward_parity_tiny_all_pixels():
    _grad_compare(ragged_tiny(64, 48, 1), 0, subset=False)


def test_backward_parity_indirect():
    _grad_compare(small_cavity(res=48, views=1), 0, subset=False)


def test_backward_parity_no_secondary_material():
    sc = small_cavity(res=48, views=1)
    sc.secondary_material = False
    _grad_compare(sc, 0, subset=False)


def test_autograd_function_matches_direct_backward():
    sc = ragged_tiny(64, 64, 1)
    r = _renderer(sc)
    M = _dev(sc.maps).requires_grad_(True)
    E = _dev(sc.env).requires_grad_(True)
    V = _dev(sc.V).requires_grad_(True)
    img = r.render(M, E, V)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    gm, gE, gV = torch.zeros_like(M), torch.zeros_like(E), torch.zeros_like(V)
    r.forward(M.detach(), E.detach())
    r.backward(M.detach(), w, gm, gE, gV)
    r.sync()
    assert torch.allclose(M.grad, gm, rtol=1e-4, atol=1e-6)
    assert torch.allclose(E.grad, gE, rtol=1e-4, atol=1e-6)
    # the vertex gradients sum contributions of up to ~1e4 by float atomics in either order, so an
    # entry that cancels to near zero carries their rounding: compare against the tensor's scale
    assert float((V.grad - gV).abs().max()) <= 1e-5 * float(gV.abs().max())


def test_l1_loss():
    from paper_2608_24109_b300 import native as N
    a = torch.randn(1000003, device="cuda")
    b = torch.randn(1000003, device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(a)
    N.exm_l1_loss(a, b, loss, grad)
    torch.cuda.synchronize()
    ref = (a - b).abs().double().mean().item()
    assert abs(loss.item() - ref) < 1e-5 * ref
    assert torch.equal(grad, torch.sign(a - b) / a.numel())


# ----------------------------------------------------------------- full-size configs, sampled

def error_table(got, ref):
    """Per-output error: largest absolute error over the largest reference magnitude, and the
    relative L2 error (the gradient bar)."""
    g = np.asarray(got, np.float64).ravel()
    o = np.asarray(ref, np.float64).ravel()
    scale = max(np.abs(o).max(), 1e-30)
    return {"max_rel": float(np.abs(g - o).max() / scale), "l2_rel": float(np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-30))}


def sampled_parity(sc, sel, maps, env, seed, what):
    """Full-size forward and backward on the GPU; the loss gradient is nonzero only on the
    sampled pixels `sel` (a masked loss), so the oracle's brute-force decisions and FP64
    adjoint on those pixels give every output exactly: radiance at the sample, and dL/dmaps,
    dL/dE, dL/dV everywhere.  `maps` / `env` are the stored values (possibly BF16/FP16); the
    oracle reads them widened exactly to FP64.  Returns the per-output error table."""
    r = _renderer(sc)
    Md = maps.cuda().contiguous()
    Ed = env.cuda().contiguous()
    out = r.forward(Md, Ed)
    r.sync()
    vis = keys_u64(r.visbuf())
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, sel)
    assert np.array_equal(keys, vis[sel[:, 0], sel[:, 1], sel[:, 2]])
    rng = np.random.default_rng(seed)
    gs = rng.normal(size=(sel.shape[0], 3)).astype(np.float32)
    grad = torch.zeros(out.shape, dtype=torch.float32, device="cuda")
    grad[torch.as_tensor(sel[:, 0]).long(), torch.as_tensor(sel[:, 1]).long(), torch.as_tensor(sel[:, 2]).long()] = \
        torch.as_tensor(gs, device="cuda")
    gm = torch.zeros(Md.shape, dtype=torch.float32, device="cuda")
    gE = torch.zeros(Ed.shape, dtype=torch.float32, device="cuda")
    gV = torch.zeros((sc.V.shape[0], 3), dtype=torch.float32, device="cuda")
    r.backward(Md, grad, gm, gE, gV)
    r.sync()
    sc.env = env.float().numpy()  # the environment as stored: its distribution and values
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, sel, keys)
    V, _, Eo = shade.scene_tensors(sc)
    Mo = maps.to(torch.float64)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    got = out.cpu().numpy()[sel[:, 0], sel[:, 1], sel[:, 2]]
    check_radiance(got, I, what)
    oV, oM, oE = shade.backward(sc, tab, dec, V, Mo, Eo, gs.astype(np.float64))
    table = {"radiance": error_table(got, I)}
    # compare the gradients on their support (the other entries are zero on both sides)
    gm_c = gm.cpu()
    nz = (gm_c != 0).any(-1) | (oM != 0).any(-1)
    for got_g, ref_g, name in ((gm_c[nz], oM[nz], "dL/dmaps"), (gE.cpu(), oE, "dL/dE"), (gV.cpu(), oV, "dL/dV")):
        check_grad(got_g.numpy(), ref_g.numpy(), f"{what} {name}")
        table[name] = error_table(got_g.numpy(), ref_g.numpy())
    print(what, table)
    r.close()
    return table


def _sample_covered(sc, view_pixels, count, seed, crop=None):
    """`count` covered pixels from the oracle's raster of random candidates (a view and, with
    `crop`, the centre crop of that size)."""
    rng = np.random.default_rng(seed)
    n = 40 * count
    v = rng.integers(0, sc.views if view_pixels is None else 1, n)
    if crop:
        c0 = (sc.width - crop) // 2
        y, x = rng.integers(c0, c0 + crop, n), rng.integers(c0, c0 + crop, n)
    else:
        y, x = rng.integers(0, sc.height, n), rng.integers(0, sc.width, n)
    cand = np.stack([v, y, x], 1).astype(np.int32)
    cand = np.unique(cand, axis=0)
    rng.shuffle(cand)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, cand)
    cov = (keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)
    sel = cand[cov][:count]
    assert sel.shape[0] == count
    return sel


def test_geometry_config_sampled():
    """99K-triangle blob, 16 views of 512^2, N_d = 256: 48 sampled pixels, forward and masked
    backward into maps, environment and vertices."""
    sc = scenes.config("geometry")
    sel = _sample_covered(sc, None, 48, 1)
    sampled_parity(sc, sel, torch.as_tensor(sc.maps), torch.as_tensor(sc.env), 11, "geometry")


def test_indirect_config_sampled():
    """499K-triangle blob with cavities, 8 views of 800^2, N_d = 128, N_b = 8, N_s = 4."""
    sc = scenes.config("indirect")
    sel = _sample_covered(sc, None, 24, 2)
    sampled_parity(sc, sel, torch.as_tensor(sc.maps), torch.as_tensor(sc.env), 12, "indirect")


@pytest.mark.parametrize("mdt", [torch.bfloat16, torch.float16])
def test_precision_form_sampled(mdt):
    """2M-triangle precision workload in the benchmark's configuration (8 views of 1024^2,
    N_d = 64, N_b = 4, N_s = 4), maps stored in BF16 / FP16 and the environment in FP16 with FP32
    shading, accumulation and gradients: 24 pixels of the 256^2 centre crop of view 0, radiance
    and gradients against the FP64 oracle fed the same rounded values (the error left is the
    compute error; the storage rounding is reported separately by the benchmark)."""
    sc = scenes.config("precision")
    sel = _sample_covered(sc, 0, 24, 4, crop=256)
    Mq = torch.as_tensor(sc.maps).to(mdt)
    Eq = torch.as_tensor(sc.env).to(torch.float16)
    sampled_parity(sc, sel, Mq, Eq, 14, f"precision {mdt}")


def test_low_precision_backward_full_frame():
    """BF16 maps and FP16 environment on a small ragged frame: every covered pixel, forward and
    backward, against the oracle fed the same rounded values."""
    sc = ragged_tiny(72, 56, 1)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    sel = oracle.covered_pixels(keys)
    sampled_parity(sc, sel, torch.as_tensor(sc.maps).to(torch.bfloat16),
                   torch.as_tensor(sc.env).to(torch.float16), 15, "tiny bf16/fp16")


# ----------------------------------------------------------------- errors

def test_argument_errors_are_reported():
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(32, 32, 1)
    r = _renderer(sc)
    out = torch.empty(r.image_shape(), device="cuda")
    bad = N.Params(n_direct=0, n_bounce=0, n_light=0, lambda_ind=1.0, flags=0, reserved=0, seed=0)
    with pytest.raises(N.ExmError) as e:
        N.exm_render_forward(r.ctx, r.mesh, _dev(sc.maps), r.env, sc.cams, bad, r.frame, out)
    assert e.value.code == N.EXM_ERR_ARG
    with pytest.raises(N.ExmError):
        N.exm_render_forward(r.ctx, r.mesh, _dev(sc.maps), r.env, np.concatenate([sc.cams, sc.cams]), r.params,
                             r.frame, out)


def test_guard_band_error_from_device():
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(32, 32, 1)
    sc.cams[0, 0:3] = [0.0, 0.0, 0.9]
    r = _renderer(sc)
    r.forward(_dev(sc.maps), _dev(sc.env))
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_GUARDBAND
    r.sync()  # latched error was cleared


@pytest.mark.parametrize("mdt", [torch.bfloat16, torch.float16])
def test_precision_form_one_view_radiance(mdt):
    """2M-triangle precision workload, one view, with maps stored in BF16/FP16 and the environment
    in FP16 (shading and accumulation in FP32): the primary keys and radiance on pixels sampled
    from the 256^2 centre crop against the FP64 oracle fed the same rounded values."""
    sc = scenes.config("precision", views=1)
    Mq = torch.as_tensor(sc.maps).to(mdt)
    Eq = torch.as_tensor(sc.env).to(torch.float16)
    sc.env = Eq.float().numpy()
    r = _renderer(sc)
    out = r.forward(Mq.cuda().contiguous(), Eq.cuda().contiguous())
    r.sync()
    vis = keys_u64(r.visbuf())
    c0 = (sc.width - 256) // 2
    crop = vis[0, c0:c0 + 256, c0:c0 + 256]
    cov = np.argwhere((crop & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF))
    rng = np.random.default_rng(4)
    pick = cov[rng.choice(cov.shape[0], 24, replace=False)]
    sel = np.concatenate([np.zeros((24, 1), np.int64), pick + c0], 1).astype(np.int32)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, sel)
    assert np.array_equal(keys, vis[sel[:, 0], sel[:, 1], sel[:, 2]])
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, sel, keys)
    V, _, Eo = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, V, Mq.to(torch.float64), Eo).numpy()
    check_radiance(out.cpu().numpy()[sel[:, 0], sel[:, 1], sel[:, 2]], I, f"precision form {mdt}")


def test_empty_frame_everywhere():
    """A camera that sees no surface: zero image, zero gradients, zero render counts and a zero
    material TV, with no error latched -- also through the half-resolution indirect pass."""
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300.render import Renderer
    sc = scenes.config("indirect", n=12, map_res=64, env_w=32, env_h=16, views=2, res=40, n_direct=16,
                       n_bounce=4, n_light=2)
    # the mesh is in front of the camera (no guard-band error) but outside its 10-degree view
    sc.cams = np.stack([scenes.look_at_camera((0.0, 0.0, 5.0), 40, 40, fovy_deg=10.0, target=(2.5, 0.0, 0.0))] * 2)
    for half in (False, True):
        sc.half_res_indirect = half
        r = Renderer.from_scene(sc)
        M, E = _dev(sc.maps), _dev(sc.env)
        out = r.forward(M, E)
        r.sync()
        covered, samples = r.stats()
        assert covered == 0 and samples == 0 and float(out.abs().sum()) == 0.0
        gm, gE = torch.zeros_like(M), torch.zeros_like(E)
        gV = torch.zeros((sc.V.shape[0], 3), device="cuda")
        r.backward(M, torch.ones_like(out), gm, gE, gV)
        r.sync()
        assert float(gm.abs().sum() + gE.abs().sum() + gV.abs().sum()) == 0.0
        loss = torch.full((1,), 7.0, device="cuda")
        N.exm_material_tv(r.ctx, M, r.frame, r.params.flags, 0.1, loss, gm)
        counts = torch.zeros(sc.F.shape[0], dtype=torch.int32, device="cuda")
        N.exm_face_render_counts(r.frame, sc.F.shape[0], counts)
        r.sync()
        assert loss.item() == 0.0 and float(gm.abs().sum()) == 0.0 and int(counts.sum()) == 0
        r.close()


# ----------------------------------------------------------------- sample counts off the fast paths

def _forward_and_backward_full(sc, what):
    r, M, E, out = gpu_forward(sc)
    keys, tab, dec, V, Mo, Eo = oracle_full(sc)
    assert np.array_equal(keys_u64(r.visbuf()), keys)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    check_radiance(out.cpu().numpy()[dec.pix[:, 0], dec.pix[:, 1], dec.pix[:, 2]], I, what)
    _grad_compare(sc, 0, subset=False)
    return dec


def test_parity_sample_counts_without_powers_of_two():
    """N_d = 37, N_b = 3, N_s = 3.  The light strata are 37 x 1 and 3 x 1 (the general mapping of
    a sample index to its stratum, not the shift and mask of power-of-two counts); ray
    generation reserves queue slots 8 sample indices at a time, so the direct batches end in
    a tail of 5 (an odd pair) and the secondary light batches hold 3; the visibility words per
    pixel (2 direct, 1 secondary) are partly filled."""
    sc = small_cavity(res=40, views=2, n_direct=37, n_bounce=3, n_light=3)
    dec = _forward_and_backward_full(sc, "N_d 37, N_b 3, N_s 3")
    assert (dec.stri >= 0).sum() > 50


@pytest.mark.parametrize("n_bounce", [5, 16, 17, 40])
def test_parity_secondary_ray_counts_around_the_record_batches(n_bounce):
    """The shade kernels evaluate the secondary hits' records for 32 / N_b pixels at once when
    N_b <= 16 (5: six pixels and two idle lanes; 16: two pixels) and pixel by pixel, 32 rays at a
    time, above (17: one partial batch; 40: a full batch of 32 and a tail of 8); forward and
    backward against the oracle in each case."""
    sc = small_cavity(res=40, views=2, n_direct=16, n_bounce=n_bounce, n_light=2)
    dec = _forward_and_backward_full(sc, f"N_b {n_bounce}")
    assert (dec.stri >= 0).sum() > 50 * n_bounce // 5


def test_parity_more_direct_samples_than_one_list_round():
    """N_d = 1100 takes 35 visibility words per pixel; the shade kernels list a pixel's live
    samples 32 words (1024 samples) at a time, so every pixel needs a second, partial round.
    The strata are 44 x 25."""
    sc = ragged_tiny(26, 22, 1, n_direct=1100)
    _forward_and_backward_full(sc, "N_d 1100")


# ----------------------------------------------------------------- small meshes and occlusion

def _custom_scene(V, F, UV, eye, target, W, H, seed, **kw):
    rng = np.random.default_rng(seed)
    maps = scenes.material_maps(rng, 32)
    env = scenes.env_map(rng, 32, 16, 1.0)
    cam = scenes.look_at_camera(eye, W, H, target=target)
    return scenes._finish("custom", np.asarray(V), np.asarray(F), np.asarray(UV), np.asarray(F), maps, maps, env,
                          cam[None], W, H, seed=seed, **kw)


def test_parity_single_triangle_mesh():
    """A mesh of one triangle: the BVH is one 4-wide node with one child, its bounding sphere
    comes from that child's box, and every shadow ray escapes."""
    V = [[-1.0, -0.8, 0.0], [1.0, -0.8, 0.0], [0.1, 0.9, 0.0]]
    sc = _custom_scene(V, [[0, 1, 2]], [[0.05, 0.05], [0.95, 0.1], [0.5, 0.95]], (0.3, 0.2, 2.5), (0.0, 0.0, 0.0),
                       48, 40, seed=11, n_direct=32)
    dec = _forward_and_backward_full(sc, "one triangle")
    assert dec.pix.shape[0] > 300


def _floor_and_occluder(with_occluder, **kw):
    # floor y = 0 facing +y (x, z in [-1, 1]); occluder quad at y = 0.25 over x, z in [-0.5, 0.5]
    # facing -y, so secondary rays from the floor meet its front face (camera rays from above see
    # its back face, which is culled)
    V = [[-1, 0, -1], [-1, 0, 1], [1, 0, 1], [1, 0, -1]]
    F = [[0, 1, 2], [0, 2, 3]]
    UV = [[0.02, 0.02], [0.02, 0.98], [0.98, 0.98], [0.98, 0.02]]
    if with_occluder:
        V += [[-0.5, 0.25, -0.5], [0.5, 0.25, -0.5], [0.5, 0.25, 0.5], [-0.5, 0.25, 0.5]]
        F += [[4, 5, 6], [4, 6, 7]]
        UV += [[0.3, 0.3], [0.7, 0.3], [0.7, 0.7], [0.3, 0.7]]
    sc = _custom_scene(np.array(V, float), np.array(F), np.array(UV), (-1.3, 1.6, 0.9), (0.0, 0.0, 0.0), 56, 48,
                       seed=5, **kw)
    n = np.cross(sc.V[sc.F[:, 1]] - sc.V[sc.F[:, 0]], sc.V[sc.F[:, 2]] - sc.V[sc.F[:, 0]])
    assert (n[:2, 1] > 0).all() and (not with_occluder or (n[2:, 1] < 0).all())
    return sc


def test_parity_occluder_casts_shadows_direct_and_indirect():
    """A textured floor under a quad that faces it: many of the floor's shadow rays are occluded
    (the any-hit tracer's hit path, which the blob workloads rarely take) and its secondary rays
    find the quad's front face; forward and backward against the oracle."""
    sc = _floor_and_occluder(True, n_direct=64, n_bounce=4, n_light=2)
    dec = _forward_and_backward_full(sc, "occluder")
    bare = _floor_and_occluder(False, n_direct=64)
    st, keys = oracle.raster_full(bare.V, bare.F, bare.cams, bare.width, bare.height)
    pix = oracle.covered_pixels(keys)
    dec_bare = oracle.Decisions(bare, oracle.EnvTable(bare.env), pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    on_floor = dec.tri < 2
    seen = {tuple(p) for p in dec.pix[on_floor]}
    bare_rows = np.array([tuple(p) in seen for p in dec_bare.pix])
    assert bare_rows.sum() == on_floor.sum()
    # the floor's visible direct samples drop by a tenth or more under the occluder
    assert dec.dvis[on_floor].sum() < 0.9 * dec_bare.dvis[bare_rows].sum()
    assert (dec.stri[on_floor] >= 2).sum() > 100
