"""Stage-I topology round on the GPU against the oracle, bit for bit: vertex positions, faces,
UVs and face-corner UV indices, the EMA state and the counts of splits and merges.  Closed
meshes, a UV atlas with seams, an open grid with boundary edges, and a tight face budget; the
per-face render counts against the oracle's raster."""
import numpy as np
import pytest
import torch

import oracle
from oracle import topology as T
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

f32 = np.float32


def _grid(n=12, seed=0):
    rng = np.random.default_rng(seed)
    xs = np.linspace(0, 1, n)
    V = np.array([[x, y, 0.05 * rng.normal()] for y in xs for x in xs], f32)
    F = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            F += [[a, b, c], [a, c, d]] if (i + j) % 2 else [[a, b, d], [b, c, d]]
    return V, np.array(F, np.int32), V[:, :2].copy(), np.array(F, np.int32)


def _meshes():
    tiny = scenes.config("tiny")
    blob = scenes.config("indirect", n=12, map_res=64, env_w=32, env_h=16, views=1, res=32)
    return {"icosphere": (tiny.V, tiny.F, tiny.UV, tiny.Fuv), "atlas_blob": (blob.V, blob.F, blob.UV, blob.Fuv),
            "open_grid": _grid()}


def _run_gpu(ctx, mesh, G, grad, counts, prm):
    from paper_2608_24109_b300.topology import TopologyRound
    V, F, UV, Fuv = mesh
    tr = TopologyRound(ctx, beta_g=prm.beta_g, w_g=prm.w_g, w_k=prm.w_k, tau_degen=prm.tau_degen,
                       tau_uv=prm.tau_uv, split_percent=prm.split_percent, max_faces=prm.max_faces)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)  # noqa: E731
    out, stats = tr(d(V, torch.float32), d(F, torch.int32), d(UV, torch.float32), d(Fuv, torch.int32),
                    d(G, torch.float32), d(grad, torch.float32), d(counts, torch.int32))
    tr.close()
    return [o.cpu().numpy() for o in out], stats


@pytest.mark.parametrize("name", ["icosphere", "atlas_blob", "open_grid"])
@pytest.mark.parametrize("seed", [0, 1])
def test_topology_round_bit_exact(name, seed):
    from paper_2608_24109_b300 import native as N
    mesh = _meshes()[name]
    V, F = mesh[0], mesh[1]
    rng = np.random.default_rng(seed)
    G = rng.uniform(0, 1, V.shape[0]).astype(f32)
    grad = rng.normal(size=V.shape).astype(f32)
    counts = rng.integers(0, 4, F.shape[0]).astype(np.int64)
    prm = T.TopoParams(split_percent=10)
    ctx = N.exm_create(0)
    (Vg, Fg, UVg, Fuvg, Gg), st = _run_gpu(ctx, mesh, G, grad, counts, prm)
    N.exm_destroy(ctx)
    Vo, Fo, UVo, Fuvo, Go, sto = T.topology_round(*mesh, G, grad, counts, prm)
    assert st == sto, (st, sto)
    assert st["splits"] > 0 and st["merges"] > 0
    assert np.array_equal(Fg, Fo) and np.array_equal(Fuvg, Fuvo)
    assert np.array_equal(Vg.view(np.uint32), Vo.view(np.uint32))
    assert np.array_equal(UVg.view(np.uint32), UVo.view(np.uint32))
    assert np.array_equal(Gg.view(np.uint32), Go.view(np.uint32))


def test_topology_face_budget():
    from paper_2608_24109_b300 import native as N
    mesh = _meshes()["atlas_blob"]
    rng = np.random.default_rng(7)
    G = rng.uniform(0, 1, mesh[0].shape[0]).astype(f32)
    grad = rng.normal(size=mesh[0].shape).astype(f32)
    counts = np.ones(mesh[1].shape[0], np.int64)
    prm = T.TopoParams(split_percent=20, max_faces=mesh[1].shape[0] + 21)
    ctx = N.exm_create(0)
    (Vg, Fg, UVg, Fuvg, Gg), st = _run_gpu(ctx, mesh, G, grad, counts, prm)
    N.exm_destroy(ctx)
    Vo, Fo, UVo, Fuvo, Go, sto = T.topology_round(*mesh, G, grad, counts, prm)
    assert st == sto and st["splits"] == 10  # ten two-face splits fit a budget of 21 new faces
    assert np.array_equal(Fg, Fo) and np.array_equal(Vg.view(np.uint32), Vo.view(np.uint32))


def test_face_render_counts_match_the_raster():
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300.render import Renderer
    sc = scenes.config("tiny", res=96, views=3)
    r = Renderer.from_scene(sc)
    r.forward(torch.as_tensor(sc.maps, device="cuda"), torch.as_tensor(sc.env, device="cuda"))
    counts = torch.zeros(sc.F.shape[0], dtype=torch.int32, device="cuda")
    N.exm_face_render_counts(r.frame, sc.F.shape[0], counts)
    r.sync()
    st, keys = oracle.raster_full(sc.V, sc.F, sc.cams, sc.width, sc.height)
    k = keys[(keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)]
    ref = np.bincount((k & np.uint64(0xFFFFFFFF)).astype(np.int64), minlength=sc.F.shape[0])
    assert np.array_equal(counts.cpu().numpy(), ref)
    assert (ref == 0).any() and (ref > 0).any()


@pytest.mark.parametrize("max_faces", [4, 5, 6])
def test_topology_face_budget_hand_worked(max_faces):
    """The hand-worked budget case of the oracle's pins (a +2 split ranked before a +1 split):
    the GPU keeps the same prefix of the accepted splits."""
    from paper_2608_24109_b300 import native as N
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [3, 0, 0], [4, 0, 0], [3, 1, 0]], f32)
    F = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6]], np.int32)
    grad = np.zeros((7, 3), f32)
    grad[0:3] = [1, 0, 0]
    grad[4:7] = [0.5, 0, 0]
    mesh = (V, F, V[:, :2].copy(), F.copy())
    G = np.zeros(7, f32)
    counts = np.ones(3, np.int64)
    prm = T.TopoParams(split_percent=100, max_faces=max_faces)
    ctx = N.exm_create(0)
    (Vg, Fg, UVg, Fuvg, Gg), st = _run_gpu(ctx, mesh, G, grad, counts, prm)
    N.exm_destroy(ctx)
    Vo, Fo, UVo, Fuvo, Go, sto = T.topology_round(*mesh, G, grad, counts, prm)
    assert st == sto and st["splits"] == {4: 0, 5: 1, 6: 2}[max_faces]
    assert np.array_equal(Fg, Fo) and np.array_equal(Vg.view(np.uint32), Vo.view(np.uint32))
