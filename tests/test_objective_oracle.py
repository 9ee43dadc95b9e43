"""Pins of the oracle's Stage-II objective (Eqs. 21-24) and Adam step against values fixed by
their definitions: the sRGB standard, brute-force windowed SSIM, closed forms of TV and
chroma on constructed inputs, Adam's first-step form, and central differences."""
import math

import numpy as np
import torch

from oracle import objective as O

DT = torch.float64


def test_srgb_curve():
    x = torch.tensor([0.0, 1.0, 0.5, 0.0031308, 0.0031308 * (1 + 1e-9)], dtype=DT)
    y = O.srgb(x)
    assert y[0] == 0.0
    assert abs(y[1].item() - 1.0) < 1e-15
    # the two branches meet at the breakpoint (to the rounding of the standard's constants)
    assert abs(y[3].item() - y[4].item()) < 1e-7
    # 50% linear is sRGB 0.7354 (188 / 255 = 0.737 after 8-bit quantisation)
    assert abs(y[2].item() - 0.7353569830524495) < 1e-12
    assert round(y[2].item() * 255) == 188


def _ssim_brute(x, y):
    """Windowed SSIM by explicit loops over pixels and window taps, zero outside the image."""
    g = O.gaussian_window().numpy()
    V, H, W, C = x.shape
    r = O.SSIM_WIN // 2
    tot, n = 0.0, 0
    for v in range(V):
        for c in range(C):
            for i in range(H):
                for j in range(W):
                    mx = my = sxx = syy = sxy = 0.0
                    for a in range(-r, r + 1):
                        for b in range(-r, r + 1):
                            ii, jj = i + a, j + b
                            if 0 <= ii < H and 0 <= jj < W:
                                w = g[a + r] * g[b + r]
                                p, q = x[v, ii, jj, c], y[v, ii, jj, c]
                                mx += w * p
                                my += w * q
                                sxx += w * p * p
                                syy += w * q * q
                                sxy += w * p * q
                    sxx -= mx * mx
                    syy -= my * my
                    sxy -= mx * my
                    c1, c2 = O.SSIM_C1, O.SSIM_C2
                    tot += ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
                    n += 1
    return tot / n


def test_ssim_against_brute_force():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, size=(1, 9, 13, 2))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    s = O.ssim(torch.as_tensor(x), torch.as_tensor(y)).item()
    assert abs(s - _ssim_brute(x, y)) < 1e-12
    assert abs(O.ssim(torch.as_tensor(x), torch.as_tensor(x)).item() - 1.0) < 1e-12
    # the window is a normalised Gaussian with the stated sigma
    g = O.gaussian_window()
    assert abs(g.sum().item() - 1.0) < 1e-15
    assert abs((g[5] / g[6]).item() - math.exp(1.0 / (2 * 1.5 ** 2))) < 1e-12


def test_log_l1_constant_images():
    p = torch.full((2, 5, 7, 3), 0.3, dtype=DT)
    t = torch.full((2, 5, 7, 3), 1.7, dtype=DT)
    total, log_l1, dssim = O.image_loss(p, t, lambda_ssim=0.0)
    assert abs(log_l1.item() - abs(math.log(1.3) - math.log(2.7))) < 1e-15
    assert abs(total.item() - log_l1.item()) < 1e-15


def test_screen_tv_ramp_and_masks():
    V, H, W = 1, 6, 9
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = torch.as_tensor((0.3 * xx - 0.7 * yy)[None, :, :, None])
    full = torch.ones((V, H, W), dtype=torch.bool)
    assert abs(O.screen_tv(img, full).item() - (0.3 + 0.7)) < 1e-14
    # a checkerboard coverage has no pair of covered neighbours
    cb = torch.as_tensor(((xx + yy) % 2 == 0)[None])
    assert O.screen_tv(img, cb).item() == 0.0
    # two covered rows only: the vertical pairs between them, horizontal pairs within them
    two = torch.zeros((V, H, W), dtype=torch.bool)
    two[0, 2:4] = True
    assert abs(O.screen_tv(img, two).item() - 1.0) < 1e-14


def test_env_tv_wraps_in_longitude():
    H, W = 4, 8
    for col in (0, 3, W - 1):
        E = torch.zeros((H, W, 3), dtype=DT)
        E[1, col, 0] = 1.0
        tv = O.env_tv(E).item()
        assert abs(tv - (2.0 / (H * W * 3) + 2.0 / ((H - 1) * W * 3))) < 1e-15, col
    assert O.env_tv(torch.full((H, W, 3), 0.4, dtype=DT)).item() == 0.0


def test_chroma_closed_forms():
    E = torch.zeros((4, 8, 3), dtype=DT)
    E[..., 0] = 1.0
    assert abs(O.chroma(E).item() - 2.0 / 3.0) < 1e-15
    assert O.chroma(torch.full((4, 8, 3), 0.25, dtype=DT)).item() < 1e-32


def test_adam_first_steps_and_clamp():
    rng = np.random.default_rng(1)
    theta = torch.as_tensor(rng.uniform(0.2, 0.8, size=(5, 8)))
    g = torch.as_tensor(rng.normal(size=(5, 8)))
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    lr = 0.01
    t1, m, v = O.adam_step(theta, g, m, v, 1, lr)
    assert torch.allclose(t1, theta - lr * g / (g.abs() + 1e-8), rtol=0, atol=1e-15)
    # a constant gradient keeps the bias-corrected step at lr * g / (|g| + eps)
    t2, m, v = O.adam_step(t1, g, m, v, 2, lr)
    assert torch.allclose(t2, t1 - lr * g / (g.abs() + 1e-8), rtol=0, atol=1e-14)
    # clamping to the material ranges
    big = torch.full((1, 8), 0.999, dtype=DT)
    t3, _, _ = O.adam_step(big, -torch.ones((1, 8), dtype=DT), torch.zeros_like(big), torch.zeros_like(big), 1, 0.5,
                           O.MAP_LO, O.MAP_HI)
    assert torch.all(t3[0, :5] == 1.0) and torch.all(t3[0, 5:] > 1.0)


def test_objective_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    V, H, W = 1, 12, 14
    pred = torch.as_tensor(rng.uniform(0.05, 1.5, size=(V, H, W, 3)), dtype=DT).requires_grad_(True)
    target = torch.as_tensor(rng.uniform(0.05, 1.5, size=(V, H, W, 3)), dtype=DT)
    E = torch.as_tensor(rng.uniform(0.1, 2.0, size=(4, 8, 3)), dtype=DT).requires_grad_(True)

    def f(p, e):
        return O.image_loss(p, target)[0] + 0.1 * O.env_tv(e) + 0.1 * O.chroma(e)

    L = f(pred, E)
    gp, gE = torch.autograd.grad(L, (pred, E))
    h = 1e-6
    for (which, idx) in [("p", (0, 3, 4, 1)), ("p", (0, 0, 0, 2)), ("p", (0, 11, 13, 0)), ("E", (2, 7, 1)),
                         ("E", (0, 0, 0))]:
        def at(delta):
            p2, e2 = pred.detach().clone(), E.detach().clone()
            (p2 if which == "p" else e2)[idx] += delta
            return f(p2, e2).item()
        num = (at(h) - at(-h)) / (2 * h)
        ana = (gp if which == "p" else gE)[idx].item()
        assert abs(num - ana) <= 1e-6 * max(1.0, abs(ana)) + 1e-9, (which, idx, num, ana)


def test_material_tv_on_a_rendered_view():
    import oracle
    from oracle import shade
    from paper_2608_24109_b300 import scenes
    sc = scenes.config("tiny", res=48, views=1)
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    pix = oracle.covered_pixels(keys)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys[pix[:, 0], pix[:, 1], pix[:, 2]])
    # a constant material projects to a constant screen image: zero TV
    flat = torch.full(sc.maps.shape, 0.5, dtype=DT)
    assert O.material_tv(sc, dec, flat).item() < 1e-15  # bilinear weights round to within an ulp
    # the projected image is the bilinear fetch at the primary hits: its gradient reaches the
    # maps only through the primary footprints, i.e. where the direct-only render's does
    maps = torch.as_tensor(sc.maps, dtype=DT).requires_grad_(True)
    tv = O.material_tv(sc, dec, maps)
    assert tv.item() > 0
    (gm,) = torch.autograd.grad(tv, maps)
    Vt, Mt, Et = shade.scene_tensors(sc)
    _, gM_render, _ = shade.backward(sc, tab, dec, Vt, Mt, Et, np.ones((dec.pix.shape[0], 3)))
    support_tv = gm.abs().sum(-1) > 0
    support_render = gM_render.abs().sum(-1) > 0
    assert support_tv.any() and not (support_tv & ~support_render).any()
    # metallic is regularised only with metallic optimisation on
    g_nomet = torch.autograd.grad(O.material_tv(sc, dec, maps, metallic=False), maps)[0]
    assert g_nomet[..., 4].abs().sum() == 0 and gm[..., 4].abs().sum() > 0
