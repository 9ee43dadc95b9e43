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


def test_noalloc_backward_allocates_nothing_on_a_fresh_frame():
    """A frame that has only run a forward pass (no regular backward has allocated its own
    environment-gradient buffer): the allocation-free backward still gives the regular
    backward's gradients, and the device's free memory and torch's allocator are the same
    before and after its calls."""
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer

    sc = scenes.config("tiny", res=80, views=2)
    ra = Renderer.from_scene(sc)  # only forward passes and the allocation-free backward
    rb = Renderer.from_scene(sc)  # the regular backward, for reference
    M = torch.as_tensor(sc.maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    out = ra.forward(M, E)
    rb.forward(M, E)
    g = torch.as_tensor(np.random.default_rng(1).normal(size=out.shape), dtype=torch.float32, device="cuda")
    ref_m, ref_e = torch.zeros_like(M), torch.zeros_like(E)
    rb.backward(M, g, ref_m, ref_e)
    gm, ge = torch.zeros_like(M), torch.zeros_like(E)
    # first call: resolves the static array's address (no allocation either)
    N.exm_render_backward_noalloc(ra.ctx, ra.mesh, M, ra.env, ra.cams, ra.params, ra.frame, g, gm, ge)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        gm.zero_()
        ge.zero_()
        N.exm_render_backward_noalloc(ra.ctx, ra.mesh, M, ra.env, ra.cams, ra.params, ra.frame, g, gm, ge)
        torch.cuda.synchronize()
        assert _rel(gm, ref_m) <= GRAD_TOL
        assert _rel(ge, ref_e) <= GRAD_TOL
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    ra.close()
    rb.close()


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
