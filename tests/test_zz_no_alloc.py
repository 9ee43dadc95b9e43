"""The allocation-free backward entry point (exm_render_backward_noalloc).

Some callers cannot call cudaMalloc while they run (their device memory belongs to another
allocator, or they cannot afford the allocator's implicit synchronisation).  For them the
library offers a backward pass whose only scratch is a static device array.  This test
calls it through the C ABI, twice in a row, and checks each result against the regular
exm_render_backward within the gradient tolerance of the parity tests.  It sits in a file
of its own, collected last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_noalloc_backward_matches_regular_backward_twice():
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer

    sc = scenes.config("tiny", res=96, views=2)
    r = Renderer.from_scene(sc)
    M = torch.as_tensor(sc.maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    out = r.forward(M, E)
    g = torch.as_tensor(np.random.default_rng(0).normal(size=out.shape), dtype=torch.float32, device="cuda")
    ref_m, ref_e = torch.zeros_like(M), torch.zeros_like(E)
    N.exm_render_backward(r.ctx, r.mesh, M, r.env, r.cams, r.params, r.frame, g, ref_m, ref_e, None)
    r.sync()
    assert ref_m.abs().sum() > 0 and ref_e.abs().sum() > 0
    for _ in range(2):
        gm, ge = torch.zeros_like(M), torch.zeros_like(E)
        N.exm_render_backward_noalloc(r.ctx, r.mesh, M, r.env, r.cams, r.params, r.frame, g, gm, ge)
        r.sync()
        assert _rel(gm, ref_m) <= GRAD_TOL
        assert _rel(ge, ref_e) <= GRAD_TOL
    r.close()


def test_noalloc_backward_rejects_oversized_environment():
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer

    sc = scenes.config("tiny", res=32, views=1)
    r = Renderer.from_scene(sc)
    big = N.exm_env_create(r.ctx, 1024, 512)  # 524,288 texels > EXM_STATIC_ENV_MAX_TEXELS
    M = torch.as_tensor(sc.maps, device="cuda")
    g = torch.zeros(r.image_shape(), device="cuda")
    with pytest.raises(N.ExmError) as e:
        N.exm_render_backward_noalloc(r.ctx, r.mesh, M, big, r.cams, r.params, r.frame, g, None, None)
    assert e.value.code == N.EXM_ERR_ARG
    N.exm_env_destroy(big)
    r.close()
