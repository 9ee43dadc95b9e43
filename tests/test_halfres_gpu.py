"""Half-resolution indirect light (EXM_FLAG_HALF_RES_INDIRECT) against the oracle: full-frame
radiance at even and odd image sizes, and the adjoint into maps, environment and vertices."""
import numpy as np
import pytest
import torch

import oracle
from oracle import halfres, shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

RAD_TOL = 1e-4
GRAD_TOL = 1e-3


def _scene(W, H, views=2):
    sc = scenes.config("indirect", n=24, map_res=128, env_w=64, env_h=32, views=views, res=W, n_direct=16,
                       n_bounce=8, n_light=4)
    if H != W:
        sc.cams = np.stack([scenes.look_at_camera(c[0:3], W, H) for c in sc.cams])
        sc.width, sc.height = W, H
    sc.half_res_indirect = True
    return sc


def _gpu(sc):
    from paper_2608_24109_b300.render import Renderer
    r = Renderer.from_scene(sc)
    M = torch.as_tensor(sc.maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    out = r.forward(M, E)
    r.sync()
    return r, M, E, out


def _check_radiance(g, o):
    mean = np.abs(o).mean()
    tol = RAD_TOL * np.maximum(np.abs(o), 1e-3 * mean)
    bad = np.abs(g - o) > tol
    assert not bad.any(), f"{bad.sum()} of {bad.size} values outside tolerance"


@pytest.mark.parametrize("W,H", [(64, 64), (61, 47)])
def test_halfres_forward_parity(W, H):
    sc = _scene(W, H)
    r, M, E, out = _gpu(sc)
    tab = oracle.EnvTable(sc.env)
    V, Mo, Eo = shade.scene_tensors(sc)
    full, hdec = halfres.render_halfres(sc, tab, V, Mo, Eo)
    assert (hdec.stri >= 0).sum() > 50
    _check_radiance(out.cpu().numpy().astype(np.float64), full.detach().numpy())
    # the half-resolution pass changes the image: it is not the full-resolution estimator
    sc.half_res_indirect = False
    r2, _, _, out2 = _gpu(sc)
    assert (out2 - out).abs().max().item() > 1e-4


def test_halfres_backward_parity():
    sc = _scene(56, 56, views=2)
    r, M, E, out = _gpu(sc)
    g = np.random.default_rng(4).normal(size=out.shape).astype(np.float32)
    gm = torch.zeros_like(M)
    gE = torch.zeros_like(E)
    gV = torch.zeros((sc.V.shape[0], 3), device="cuda")
    r.backward(M, torch.as_tensor(g, device="cuda"), gm, gE, gV)
    r.sync()
    tab = oracle.EnvTable(sc.env)
    V, Mo, Eo = (t.requires_grad_(True) for t in shade.scene_tensors(sc))
    full, hdec = halfres.render_halfres(sc, tab, V, Mo, Eo)
    assert (hdec.stri >= 0).sum() > 50
    oV, oM, oE = torch.autograd.grad((full * torch.as_tensor(g, dtype=torch.float64)).sum(), (V, Mo, Eo))
    for got, ref, what in ((gm, oM, "maps"), (gE, oE, "env"), (gV, oV, "V")):
        a = got.cpu().numpy().astype(np.float64).ravel()
        b = ref.numpy().ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        assert rel <= GRAD_TOL, (what, rel)
