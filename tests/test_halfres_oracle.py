"""Pins of the half-resolution indirect oracle: the upsampling against PyTorch's bilinear
interpolation (an independent routine) and partition of unity, the camera halving as a
projective identity, and its reductions (lambda_ind = 0 and a convex mesh give the direct
image)."""
import numpy as np
import torch
import torch.nn.functional as Fn

import oracle
from oracle import halfres, shade
from paper_2608_24109_b300 import scenes

DT = torch.float64


def test_upsample_matches_bilinear_interpolation_for_even_sizes():
    rng = np.random.default_rng(0)
    img = torch.as_tensor(rng.normal(size=(2, 5, 7, 3)))
    up = halfres.upsample(img, 14, 10)
    ref = Fn.interpolate(img.permute(0, 3, 1, 2), scale_factor=2, mode="bilinear", align_corners=False)
    assert torch.allclose(up, ref.permute(0, 2, 3, 1), rtol=0, atol=1e-14)


def test_upsample_partition_of_unity_and_odd_sizes():
    img = torch.full((1, 4, 5, 3), 0.37, dtype=DT)
    for W, H in ((9, 7), (10, 8), (1, 1)):
        up = halfres.upsample(img[:, :(H + 1) // 2, :(W + 1) // 2], W, H)
        assert up.shape == (1, H, W, 3)
        assert torch.allclose(up, torch.full_like(up, 0.37), rtol=0, atol=1e-15)
    # an odd width's last column reads the last half column alone
    ramp = torch.arange(3, dtype=DT)[None, None, :, None].expand(1, 1, 3, 1)
    up = halfres.upsample(ramp, 5, 1)[0, 0, :, 0]
    assert torch.allclose(up, torch.tensor([0.0, 0.25, 0.75, 1.25, 1.75], dtype=DT))


def test_half_cameras_project_to_half_coordinates():
    sc = scenes.config("tiny", res=97, views=2)
    hs = halfres.half_scene(sc)
    assert (hs.width, hs.height) == (49, 49) and hs.n_direct == 0
    rng = np.random.default_rng(1)
    p = rng.normal(size=(20, 3)) * 0.5
    for c, h in zip(sc.cams, hs.cams):
        eye, right, up, fwd = c[0:3], c[3:6], c[6:9], c[9:12]
        q = p - eye
        x, y, w = q @ right, q @ up, q @ fwd
        u, v = c[14] + c[12] * x / w, c[15] - c[13] * y / w
        uh, vh = h[14] + h[12] * x / w, h[15] - h[13] * y / w
        assert np.allclose(uh, u / 2, atol=1e-5) and np.allclose(vh, v / 2, atol=1e-5)


def _direct_image(sc, tab, V, M, E):
    img, mask, dec = halfres._image(halfres.direct_scene(sc), tab, V, M, E)
    return img


def test_lambda_zero_and_convex_mesh_reduce_to_direct():
    sc = scenes.config("indirect", n=24, map_res=64, env_w=32, env_h=16, views=2, res=40, n_direct=16,
                       n_bounce=8, n_light=4)
    tab = oracle.EnvTable(sc.env)
    V, M, E = shade.scene_tensors(sc)
    full, hdec = halfres.render_halfres(sc, tab, V, M, E)
    direct = _direct_image(sc, tab, V, M, E)
    assert (hdec.stri >= 0).sum() > 20
    assert (full - direct).abs().max() > 1e-4   # the cavity scene has indirect light
    assert torch.all(full >= direct - 1e-15)     # and it only adds light
    sc.lambda_ind = 0.0
    full0, _ = halfres.render_halfres(sc, tab, V, M, E)
    assert torch.equal(full0, direct)
    cv = scenes.config("tiny", res=40, views=1, n_bounce=4, n_light=2)
    tcv = oracle.EnvTable(cv.env)
    Vc, Mc, Ec = shade.scene_tensors(cv)
    fc, _ = halfres.render_halfres(cv, tcv, Vc, Mc, Ec)
    assert torch.equal(fc, _direct_image(cv, tcv, Vc, Mc, Ec))
