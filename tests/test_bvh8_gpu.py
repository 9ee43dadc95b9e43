"""The 8-wide compressed BVH (child boxes quantised to 8 bits on a per-node grid, rounded
outwards) against the 4-wide one and the oracle.  Its box tests are conservative and its
triangle tests are the same watertight tests, so every decision -- visibility bits, secondary
hit ids -- and hence every radiance value is bit-identical to the 4-wide tree's, and equal to
the brute-force oracle's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _render(sc, width, maps=None, env=None, dtype=torch.float32):
    from paper_2608_24109_b300.render import Renderer
    r = Renderer.from_scene(sc, bvh_width=width)
    M = torch.as_tensor(sc.maps if maps is None else maps).to(dtype).cuda().contiguous()
    E = _dev(sc.env if env is None else env)
    out = r.forward(M, E).clone()
    r.sync()
    return r, out


@pytest.mark.parametrize("name,kw", [("geometry", {}), ("indirect", {"views": 2}), ("precision", {"views": 2}),
                                      ("tiny", {})])
def test_widths_give_bit_identical_images(name, kw):
    """Full-size workloads (fewer views for the larger two): the forward images of the two
    trees are equal bit for bit, and so are the decisions behind them."""
    sc = scenes.config(name, **kw)
    r4, out4 = _render(sc, 4)
    r8, out8 = _render(sc, 8)
    assert torch.equal(out4, out8)
    # the covered-pixel lists hold the same pixels in the order the compaction wrote them
    p4, d4, s4, h4 = r4.saved_state()
    p8, d8, s8, h8 = r8.saved_state()
    o4, o8 = torch.argsort(p4), torch.argsort(p8)
    assert torch.equal(p4[o4], p8[o8])
    assert torch.equal(d4[o4], d8[o8]) and torch.equal(s4[o4], s8[o8])
    assert (h4 is None and h8 is None) or torch.equal(h4[o4], h8[o8])
    r4.close()
    r8.close()


def test_eight_wide_decisions_equal_the_oracles():
    sc = scenes.config("indirect", n=24, map_res=128, env_w=64, env_h=32, views=2, res=56, n_direct=40, n_bounce=6,
                       n_light=3)
    r, out = _render(sc, 8)
    pixels, dbits, sbits, hits = r.saved_state()
    p = pixels.cpu().numpy()
    view, rem = p // (sc.width * sc.height), p % (sc.width * sc.height)
    pix = np.stack([view, rem // sc.width, rem % sc.width], 1).astype(np.int32)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, pix)
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys)
    w = dbits.cpu().numpy().astype(np.uint64)
    k = np.arange(sc.n_direct)
    bits = ((w[:, k // 32] >> (k % 32).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
    assert np.array_equal(bits, dec.dvis)
    gh = hits.cpu().numpy()
    tie = (dec.sgap < 1e-6) & (dec.stri >= 0)
    assert ((gh == dec.stri) | tie).all()
    V, Mo, Eo = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, V, Mo, Eo).numpy()
    g = out.cpu().numpy()[pix[:, 0], pix[:, 1], pix[:, 2]]
    tol = 1e-4 * np.maximum(np.abs(I), 1e-3 * np.abs(I).mean())
    assert (np.abs(g - I) <= tol).all()
    r.close()


def test_eight_wide_single_triangle_and_occluder():
    """A one-triangle mesh (one node, one triangle child) and a floor under an occluding quad
    (the any-hit tracer's hit path): the same images as with the 4-wide tree."""
    V = np.array([[-1.0, -0.8, 0.0], [1.0, -0.8, 0.0], [0.1, 0.9, 0.0]])
    rng = np.random.default_rng(11)
    maps = scenes.material_maps(rng, 32)
    env = scenes.env_map(rng, 32, 16, 1.0)
    cam = scenes.look_at_camera((0.3, 0.2, 2.5), 48, 40)
    one = scenes._finish("one", V, np.array([[0, 1, 2]]), np.array([[0.05, 0.05], [0.95, 0.1], [0.5, 0.95]]),
                         np.array([[0, 1, 2]]), maps, maps, env, cam[None], 48, 40, seed=11, n_direct=32)
    Vf = [[-1, 0, -1], [-1, 0, 1], [1, 0, 1], [1, 0, -1], [-0.5, 0.25, -0.5], [0.5, 0.25, -0.5], [0.5, 0.25, 0.5],
          [-0.5, 0.25, 0.5]]
    Ff = [[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]]
    UVf = [[0.02, 0.02], [0.02, 0.98], [0.98, 0.98], [0.98, 0.02], [0.3, 0.3], [0.7, 0.3], [0.7, 0.7], [0.3, 0.7]]
    cam2 = scenes.look_at_camera((-1.3, 1.6, 0.9), 56, 48)
    floor = scenes._finish("floor", np.array(Vf, float), np.array(Ff), np.array(UVf), np.array(Ff), maps, maps, env,
                           cam2[None], 56, 48, seed=5, n_direct=64, n_bounce=4, n_light=2)
    for sc in (one, floor):
        r4, out4 = _render(sc, 4)
        r8, out8 = _render(sc, 8)
        assert torch.equal(out4, out8) and float(out8.abs().sum()) > 0
        r4.close()
        r8.close()


def test_eight_wide_asset_round_trip_and_cycle():
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc = scenes.config("tiny", res=24, views=1, n_direct=4)
    r, ref = _render(sc, 8)
    info, secs = assets.export_mesh(r.mesh)
    assert info.node_bytes == 80
    M = _dev(sc.maps)
    good = assets.import_mesh(r.ctx, info, secs)
    out = torch.empty_like(ref)
    N.exm_render_forward(r.ctx, good, M, r.env, r.cams, r.params, r.frame, out)
    r.sync()
    assert torch.equal(out, ref)
    # the root made its own only child, whose box is the root's: a cycle with every index in range
    # that every ray entering the root's box follows until the traversal's cap ends it
    nodes = secs[4].view(np.uint32).reshape(info.n_nodes, 20)
    nodes[0, 4] = 0           # child_base
    nodes[0, 6] = 1           # one node child, no triangle children
    lo_words = [8, 9, 10, 11, 12, 13]    # qlo.x, qlo.y, qlo.z (two words each)
    hi_words = [14, 15, 16, 17, 18, 19]  # qhi.x, qhi.y, qhi.z
    nodes[0, lo_words] = 0xFFFFFF00     # slot 0 at plane 0, the empty slots at 255
    nodes[0, [9, 11, 13]] = 0xFFFFFFFF
    nodes[0, hi_words] = 0x000000FF     # slot 0 at plane 255, the empty slots at 0
    nodes[0, [15, 17, 19]] = 0
    bad = assets.import_mesh(r.ctx, info, secs)
    N.exm_render_forward(r.ctx, bad, M, r.env, r.cams, r.params, r.frame, out)
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_TRAVERSAL_LIMIT
    # an out-of-range child base is refused at import
    nodes[0, 4] = info.n_nodes
    with pytest.raises(N.ExmError) as e:
        assets.import_mesh(r.ctx, info, secs)
    assert e.value.code == N.EXM_ERR_ARG
    for m in (good, bad):
        N.exm_mesh_destroy(m)
    r.close()
