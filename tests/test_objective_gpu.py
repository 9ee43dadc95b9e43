"""Stage-II objective kernels (Eqs. 21-24) and the Adam step against the oracle.

Bars: loss values within 2e-5 relative (FP32 arithmetic, 64-bit fixed-point sums); gradients
||g - o|| / ||o|| <= 1e-3 per tensor; Adam parameters within 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
from oracle import objective as O
from oracle import shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

LOSS_TOL = 2e-5
GRAD_TOL = 1e-3


def _rel(g, o):
    g = np.asarray(g, np.float64).ravel()
    o = np.asarray(o, np.float64).ravel()
    return np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)


def _ctx():
    from paper_2608_24109_b300 import native as N
    return N, N.exm_create(0)


@pytest.mark.parametrize("shape", [(2, 37, 53), (1, 16, 32), (1, 5, 3), (4, 512, 512)])
def test_image_loss_parity(shape):
    N, ctx = _ctx()
    V, H, W = shape
    rng = np.random.default_rng(sum(shape))
    pred = rng.uniform(0.0, 1.5, size=(V, H, W, 3)).astype(np.float32)
    target = np.clip(pred + rng.normal(0, 0.2, size=pred.shape), 0, None).astype(np.float32)
    pred[0, 0, :2] = 0.001  # the linear branch of the sRGB curve
    p_d, t_d = torch.as_tensor(pred, device="cuda"), torch.as_tensor(target, device="cuda")
    loss = torch.zeros(3, device="cuda")
    grad = torch.empty_like(p_d)
    N.exm_image_loss(ctx, p_d, t_d, 0.2, loss, grad)
    N.exm_sync(ctx)
    po = torch.as_tensor(pred, dtype=torch.float64).requires_grad_(True)
    tot, l1, ds = O.image_loss(po, torch.as_tensor(target, dtype=torch.float64), 0.2)
    (go,) = torch.autograd.grad(tot, po)
    gl = loss.cpu().numpy()
    for k, ref in enumerate((tot.item(), l1.item(), ds.item())):
        assert abs(gl[k] - ref) <= LOSS_TOL * abs(ref) + 1e-7, (k, gl[k], ref)
    assert _rel(grad.cpu().numpy(), go.numpy()) <= GRAD_TOL
    N.exm_destroy(ctx)


def _continuous_metallic(sc, seed=9):
    """The synthetic metallic map is Bernoulli (0 or 1): neighbouring fetches inside a plateau
    are equal up to rounding, where |P(p) - P(q)| has no derivative and FP32 and FP64 rounding
    pick different subgradients.  Parity tests of the TV gradient use a continuous map."""
    sc.maps = sc.maps.copy()
    sc.maps[..., 4] = np.random.default_rng(seed).uniform(0.0, 1.0, size=sc.maps.shape[:2]).astype(np.float32)
    return sc


def _render_tiny(sc, maps=None):
    from paper_2608_24109_b300.render import Renderer
    r = Renderer.from_scene(sc)
    M = torch.as_tensor(sc.maps if maps is None else maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    img = r.forward(M, E)
    r.sync()
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    return r, M, E, img, tab, dec


@pytest.mark.parametrize("metallic,dtype", [(True, torch.float32), (False, torch.float32), (True, torch.bfloat16)])
def test_material_tv_parity(metallic, dtype):
    from paper_2608_24109_b300 import native as N
    sc = _continuous_metallic(scenes.config("tiny", res=96, views=2))
    sc.metallic = metallic
    Mq = torch.as_tensor(sc.maps).to(dtype)
    r, M, E, img, tab, dec = _render_tiny(sc, Mq)
    loss = torch.zeros(1, device="cuda")
    gm = torch.zeros(sc.maps.shape, dtype=torch.float32, device="cuda")
    N.exm_material_tv(r.ctx, M, r.frame, r.params.flags, 0.1, loss, gm)
    r.sync()
    Mo = Mq.to(torch.float64).requires_grad_(True)
    tv = O.material_tv(sc, dec, Mo, metallic)
    (go,) = torch.autograd.grad(0.1 * tv, Mo)
    assert abs(loss.item() - tv.item()) <= LOSS_TOL * tv.item()
    assert _rel(gm.cpu().numpy(), go.numpy()) <= GRAD_TOL


@pytest.mark.parametrize("shape", [(32, 64), (128, 256), (1, 7), (5, 1)])
def test_env_regularizers_parity(shape):
    N, ctx = _ctx()
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    E = np.exp(rng.normal(0, 1, size=(H, W, 3))).astype(np.float32)
    E_d = torch.as_tensor(E, device="cuda")
    loss = torch.zeros(2, device="cuda")
    g = torch.zeros_like(E_d)
    N.exm_env_regularizers(ctx, E_d, 0.1, 0.07, loss, g)
    N.exm_env_regularizers(ctx, E_d, 0.1, 0.07, loss, g)  # accumulates: twice the gradient
    N.exm_sync(ctx)
    Eo = torch.as_tensor(E, dtype=torch.float64).requires_grad_(True)
    tv, ch = O.env_tv(Eo), O.chroma(Eo)
    (go,) = torch.autograd.grad(0.1 * tv + 0.07 * ch, Eo)
    gl = loss.cpu().numpy()
    assert abs(gl[0] - tv.item()) <= LOSS_TOL * tv.item() + 1e-7
    assert abs(gl[1] - ch.item()) <= LOSS_TOL * ch.item() + 1e-7
    assert _rel(g.cpu().numpy() * 0.5, go.numpy()) <= GRAD_TOL
    N.exm_destroy(ctx)


def test_adam_parity_and_clamp():
    N, ctx = _ctx()
    rng = np.random.default_rng(5)
    theta = rng.uniform(0.0, 1.0, size=(1000, 8)).astype(np.float32)
    theta[:10, :5] = 0.9999
    th_d = torch.as_tensor(theta, device="cuda")
    m_d, v_d = torch.zeros_like(th_d), torch.zeros_like(th_d)
    to = torch.as_tensor(theta, dtype=torch.float64)
    mo, vo = torch.zeros_like(to), torch.zeros_like(to)
    for step in range(1, 4):
        g = rng.normal(size=theta.shape).astype(np.float32)
        if step == 1:
            g[:10, :5] = -5.0  # pushes past the upper bound
        N.exm_adam_step(ctx, th_d, torch.as_tensor(g, device="cuda"), m_d, v_d, 0.01, step, O.MAP_LO, O.MAP_HI)
        to, mo, vo = O.adam_step(to, torch.as_tensor(g, dtype=torch.float64), mo, vo, step, 0.01, O.MAP_LO, O.MAP_HI)
    N.exm_sync(ctx)
    got = th_d.cpu().numpy().astype(np.float64)
    assert np.allclose(got, to.numpy(), rtol=1e-6, atol=1e-7)
    assert (got[:10, :5] <= 1.0).all()
    N.exm_destroy(ctx)


def test_stage2_gradients_match_oracle():
    """One full objective evaluation: render, image term, adjoint, material TV, env terms."""
    from paper_2608_24109_b300.objective import Stage2Optimizer
    from paper_2608_24109_b300.render import Renderer
    sc = _continuous_metallic(scenes.config("tiny", res=64, views=2))
    r = Renderer.from_scene(sc)
    M = torch.as_tensor(sc.maps, device="cuda").clone()
    E = torch.as_tensor(sc.env, device="cuda").clone()
    target = r.forward(torch.as_tensor(sc.maps_target, device="cuda"), E).clone()
    opt = Stage2Optimizer(r, M, E, total_steps=100)
    opt.gradients(target)
    r.sync()
    img = opt.image.cpu().numpy().astype(np.float64)
    # oracle: the image term's gradient at the GPU image, pushed through the oracle adjoint
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    pi = torch.as_tensor(img).requires_grad_(True)
    tot, _, _ = O.image_loss(pi, torch.as_tensor(target.cpu().numpy(), dtype=torch.float64), 0.2)
    (grgb,) = torch.autograd.grad(tot, pi)
    Vt, Mt, Et = shade.scene_tensors(sc)
    _, gM, gE = shade.backward(sc, tab, dec, Vt, Mt, Et, grgb.numpy()[pix[:, 0], pix[:, 1], pix[:, 2]])
    Mo = torch.as_tensor(sc.maps, dtype=torch.float64).requires_grad_(True)
    Eo = torch.as_tensor(sc.env, dtype=torch.float64).requires_grad_(True)
    reg = 0.1 * O.material_tv(sc, dec, Mo) + 0.1 * O.env_tv(Eo) + 0.1 * (1 - 0 / 100) * O.chroma(Eo)
    gMr, gEr = torch.autograd.grad(reg, (Mo, Eo))
    assert _rel(opt.grad_maps.cpu().numpy(), (gM + gMr).numpy()) <= GRAD_TOL
    assert _rel(opt.grad_env.cpu().numpy(), (gE + gEr).numpy()) <= GRAD_TOL


def test_stage2_iterations_reduce_the_objective():
    from paper_2608_24109_b300.objective import Stage2Optimizer
    from paper_2608_24109_b300.render import Renderer
    sc = scenes.config("tiny", res=64, views=4)
    r = Renderer.from_scene(sc)
    E = torch.as_tensor(sc.env, device="cuda").clone()
    target = r.forward(torch.as_tensor(sc.maps_target, device="cuda"), E).clone()
    M = torch.as_tensor(sc.maps, device="cuda").clone()
    opt = Stage2Optimizer(r, M, E, lr_maps=1e-2, optimize_env=False, total_steps=30)
    first = None
    for _ in range(30):
        opt.step(target)
        if first is None:
            first = opt.total_loss()
    opt.gradients(target)
    last = opt.total_loss()
    assert np.isfinite(last) and last < 0.9 * first, (first, last)
    mm = M.cpu().numpy()
    assert (mm[..., :5] >= 0).all() and (mm[..., :5] <= 1).all()
