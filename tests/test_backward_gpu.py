"""Backward pass on the GPU (the adjoint of Eqs. 10-20), beyond the element-wise parity of
test_gpu_parity.py:

* its checks of the frame's saved forward state: a backward handed another environment, a
  re-prepared one, an updated mesh or other cameras is refused before anything is enqueued;
* the per-sample state kept one chunk at a time and recomputed by the backward pass
  (EXM_FLAG_RECOMPUTE, or a saved-state budget the frame would exceed): the same radiance bit
  for bit and the same gradients as the stored state, against the oracle too;
* a ray-queue overflow reported as its own error, with nothing traced out of bounds;
* central differences of the GPU forward on 32 map entries against the gradient of the
  torch.autograd.Function (map texels change no discrete decision, so the derivative of the
  estimator is exactly what the differences approximate);
* the per-sample decisions (visibility bits, secondary hit ids) compared directly with the
  oracle's brute-force ones.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _renderer(sc, **kw):
    from paper_2608_24109_b300.render import Renderer
    return Renderer.from_scene(sc, **kw)


def _rel(a, b):
    a = a.double().cpu().numpy().ravel() if torch.is_tensor(a) else np.asarray(a, np.float64).ravel()
    b = b.double().cpu().numpy().ravel() if torch.is_tensor(b) else np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def ragged_tiny(W=97, H=61, views=2, **kw):
    sc = scenes.config("tiny", **kw)
    sc.cams = np.stack([scenes.look_at_camera(c[0:3], W, H) for c in sc.cams[:views]])
    sc.width, sc.height = W, H
    return sc


def small_cavity(res=48, views=2, n_direct=16, n_bounce=8, n_light=4):
    return scenes.config("indirect", n=24, map_res=128, env_w=64, env_h=32, views=views, res=res,
                         n_direct=n_direct, n_bounce=n_bounce, n_light=n_light)


# ------------------------------------------------------------- saved-state checks

def _expect_refused(fn, what):
    from paper_2608_24109_b300 import native as N
    with pytest.raises(N.ExmError) as e:
        fn()
    assert e.value.code == N.EXM_ERR_ARG, what
    return str(e.value)


def test_backward_refuses_an_environment_other_than_the_forwards():
    """Forward with a 1024 x 512 environment, backward handed a 64 x 32 one: the recorded texel
    indices (up to 2^19) would address far past the smaller environment's gradient.  Both
    backward entry points refuse before any launch and leave the gradient buffers untouched,
    also when asked to zero them."""
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(48, 40, 1, env_w=1024, env_h=512)
    r = _renderer(sc)
    M, E = _dev(sc.maps), _dev(sc.env)
    out = r.forward(M, E)
    r.sync()
    small = N.exm_env_create(r.ctx, 64, 32)
    N.exm_env_prepare(small, _dev(scenes.env_map(np.random.default_rng(1), 64, 32, 1.0)))
    r.sync()
    g = torch.ones_like(out)
    gm = torch.full(M.shape, 7.0, device="cuda")
    gE = torch.full((32, 64, 3), 7.0, device="cuda")
    p = N.Params.from_buffer_copy(r.params)
    p.flags |= N.FLAG_ZERO_GRADS
    launches = N.exm_launch_count(r.ctx)
    msg = _expect_refused(lambda: N.exm_render_backward(r.ctx, r.mesh, M, small, r.cams, p, r.frame, g, gm, gE, None),
                          "exm_render_backward")
    assert "environment" in msg
    _expect_refused(lambda: N.exm_render_backward_noalloc(r.ctx, r.mesh, M, small, r.cams, p, r.frame, g, gm, gE),
                    "exm_render_backward_noalloc")
    r.sync()
    assert N.exm_launch_count(r.ctx) == launches
    assert bool((gm == 7.0).all()) and bool((gE == 7.0).all())
    N.exm_env_destroy(small)
    r.close()


def test_backward_refuses_changed_objects_and_cameras():
    """A re-prepared environment, updated vertices or other cameras between the forward and the
    backward pass are refused; a fresh forward makes the backward valid again."""
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(40, 36, 1)
    r = _renderer(sc)
    M, E = _dev(sc.maps), _dev(sc.env)
    out = r.forward(M, E)
    g = torch.ones_like(out)
    gm = torch.zeros_like(M)
    r.prepare_env(E)
    _expect_refused(lambda: r.backward(M, g, gm), "re-prepared environment")
    r.forward(M, E)
    r.update_vertices(_dev(sc.V) * 1.0001)
    _expect_refused(lambda: r.backward(M, g, gm), "updated mesh")
    r.forward(M, E)
    cams = r.cams.copy()
    cams[0, 12] *= 1.01
    _expect_refused(lambda: N.exm_render_backward(r.ctx, r.mesh, M, r.env, cams, r.params, r.frame, g, gm),
                    "other cameras")
    p = N.Params.from_buffer_copy(r.params)
    p.seed += 1
    _expect_refused(lambda: N.exm_render_backward(r.ctx, r.mesh, M, r.env, r.cams, p, r.frame, g, gm), "other seed")
    r.backward(M, g, gm)
    r.sync()
    assert float(gm.abs().sum()) > 0
    r.close()


# ------------------------------------------------------------- recomputed per-sample state

def _run_fwd_bwd(r, sc, grad_np):
    M, E = _dev(sc.maps), _dev(sc.env)
    out = r.forward(M, E)
    gm, gE = torch.zeros_like(M), torch.zeros_like(E)
    gV = torch.zeros((sc.V.shape[0], 3), device="cuda")
    r.backward(M, _dev(grad_np), gm, gE, gV)
    r.sync()
    return out, gm, gE, gV


@pytest.mark.parametrize("how", ["flag", "budget"])
@pytest.mark.parametrize("scene", ["direct", "indirect"])
def test_recomputed_state_matches_stored_state(how, scene):
    """The state kept per chunk (a 200 KB budget splits these frames into 10-20 chunks; the
    flag alone keeps one chunk) gives the stored state's radiance bit for bit, the same
    gradients up to the order of the atomic sums, and the oracle's gradients."""
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(97, 61, 2, n_direct=64) if scene == "direct" else small_cavity(res=56, views=2)
    rs = _renderer(sc)
    grad = np.random.default_rng(3).normal(size=(sc.views, sc.height, sc.width, 3)).astype(np.float32)
    out_s, gm_s, gE_s, gV_s = _run_fwd_bwd(rs, sc, grad)
    rr = _renderer(sc)
    if how == "flag":
        rr.params.flags |= N.FLAG_RECOMPUTE
    else:
        rr.set_limits(saved_budget_bytes=200_000)
    out_r, gm_r, gE_r, gV_r = _run_fwd_bwd(rr, sc, grad)
    assert torch.equal(out_s, out_r)
    for a, b, what in ((gm_r, gm_s, "maps"), (gE_r, gE_s, "env"), (gV_r, gV_s, "V")):
        assert _rel(a, b) <= 1e-5, what
    # and the oracle
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    V, Mo, Eo = shade.scene_tensors(sc)
    oV, oM, oE = shade.backward(sc, tab, dec, V, Mo, Eo, grad[pix[:, 0], pix[:, 1], pix[:, 2]].astype(np.float64))
    assert _rel(gm_r, oM) <= GRAD_TOL and _rel(gE_r, oE) <= GRAD_TOL and _rel(gV_r, oV) <= GRAD_TOL
    # the frame no longer holds the whole-frame state: its inspection is refused
    with pytest.raises(N.ExmError):
        rr.saved_state()
    rs.close()
    rr.close()


def test_recomputed_state_through_the_allocation_free_backward():
    from paper_2608_24109_b300 import native as N
    sc = small_cavity(res=40, views=1)
    r = _renderer(sc)
    r.set_limits(saved_budget_bytes=100_000)
    M, E = _dev(sc.maps), _dev(sc.env)
    out = r.forward(M, E)
    g = torch.as_tensor(np.random.default_rng(5).normal(size=out.shape), dtype=torch.float32, device="cuda")
    gm, gE = torch.zeros_like(M), torch.zeros_like(E)
    r.backward(M, g, gm, gE)
    gm2, gE2 = torch.zeros_like(M), torch.zeros_like(E)
    N.exm_render_backward_noalloc(r.ctx, r.mesh, M, r.env, r.cams, r.params, r.frame, g, gm2, gE2)
    r.sync()
    assert _rel(gm2, gm) <= 1e-5 and _rel(gE2, gE) <= 1e-5
    r.close()


def test_queue_overflow_is_its_own_error():
    """A queue of 64 rays per chunk cannot hold the 32 x 64 rays of a 32-pixel chunk: the rays
    beyond it are dropped (never traced: the tracer stops at the queue's end) and exm_sync
    reports EXM_ERR_QUEUE_OVERFLOW.  With the default queue the frame renders as before."""
    from paper_2608_24109_b300 import native as N
    sc = ragged_tiny(40, 32, 1, n_direct=64)
    r = _renderer(sc)
    M, E = _dev(sc.maps), _dev(sc.env)
    ref = r.forward(M, E).clone()
    r.sync()
    r.set_limits(ray_cap=64)
    r.forward(M, E)
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_QUEUE_OVERFLOW
    r.set_limits(ray_cap=0)
    out = r.forward(M, E)
    r.sync()
    assert torch.equal(out, ref)
    r.close()


# ------------------------------------------------------------- finite differences

def test_autograd_matches_central_differences_on_32_map_entries():
    """Reduced cavity workload (one bounce of indirect light, so map entries reach the image
    through x and through the secondary hits y).  L = sum(w * I) with a fixed random w, a linear
    loss with no kinks; its gradient comes from the torch.autograd.Function (the library's
    adjoint).  For 32 (texel, channel) entries drawn from those with a gradient above 1% of the
    largest, central differences of the GPU forward with h = 1e-3 agree within 1% of the entry's
    gradient plus 1e-3 of the largest (FP32 rounding of the perturbed pixels' radiance and the
    curvature of the GGX and normal-map terms over +-h)."""
    sc = small_cavity(res=48, views=2)
    r = _renderer(sc)
    M = _dev(sc.maps).requires_grad_(True)
    E = _dev(sc.env)
    img = r.render(M, E)
    w = torch.as_tensor(np.random.default_rng(7).normal(size=img.shape), dtype=torch.float32, device="cuda")
    (img * w).sum().backward()
    grad = M.grad.detach().clone()
    gmax = float(grad.abs().max())
    cand = torch.nonzero(grad.abs().flatten() > 0.01 * gmax).flatten().cpu().numpy()
    assert cand.size > 200
    pick = np.random.default_rng(8).choice(cand, 32, replace=False)
    h = 1e-3
    wd = w.double()
    base = sc.maps.copy()
    fd = []
    for flat in pick:
        vals, moved = [], []
        for sgn in (1.0, -1.0):
            m = base.copy().reshape(-1)
            m[flat] = np.float32(m[flat] + sgn * h)
            moved.append(float(m[flat]))
            out = r.forward(_dev(m.reshape(base.shape)), E)
            vals.append(float((out.double() * wd).sum()))
        fd.append((vals[0] - vals[1]) / (moved[0] - moved[1]))  # the FP32 step actually taken
    r.sync()
    fd = np.array(fd)
    g = grad.flatten()[torch.as_tensor(pick, device="cuda")].double().cpu().numpy()
    err = np.abs(fd - g)
    tol = 1e-2 * np.abs(g) + 1e-3 * gmax
    assert (err <= tol).all(), f"worst entry: fd {fd[err.argmax()]:.6e} grad {g[err.argmax()]:.6e}"
    r.close()


# ------------------------------------------------------------- decisions, directly

def _words_to_bits(words, n):
    w = words.cpu().numpy().astype(np.uint64)
    k = np.arange(n)
    return ((w[:, k // 32] >> (k % 32).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)


def test_visibility_bits_and_hit_ids_equal_the_oracles():
    """The GPU's per-sample decisions -- shadow-ray visibility of every direct sample, the closest
    front-facing hit of every secondary ray and the visibility of every light sample at those
    hits -- equal the brute-force oracle's on every covered pixel of a cavity frame (counted
    apart: secondary hits whose oracle gap between the best and second-best hit distance is
    below 1e-6, where the spec allows either)."""
    sc = small_cavity(res=56, views=2, n_direct=40, n_bounce=6, n_light=3)
    r = _renderer(sc)
    r.forward(_dev(sc.maps), _dev(sc.env))
    r.sync()
    pixels, dbits, sbits, hits = r.saved_state()
    p = pixels.cpu().numpy()
    view = p // (sc.width * sc.height)
    rem = p % (sc.width * sc.height)
    pix = np.stack([view, rem // sc.width, rem % sc.width], 1).astype(np.int32)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, pix)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys)
    assert np.array_equal(_words_to_bits(dbits, sc.n_direct), dec.dvis)
    gh = hits.cpu().numpy()
    tie = (dec.sgap < 1e-6) & (dec.stri >= 0)
    same = (gh == dec.stri) | tie
    assert same.all(), f"{(~same).sum()} secondary hits differ"
    assert (gh >= 0).sum() > 100
    lb = _words_to_bits(sbits, sc.n_bounce * sc.n_light).reshape(-1, sc.n_bounce, sc.n_light)
    ok = (dec.stri >= 0) & ~tie
    assert np.array_equal(lb[ok], dec.lvis[ok])
    assert (lb[gh < 0] == 0).all()
    r.close()
