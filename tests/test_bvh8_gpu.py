"""The three BVH layouts against each other and the oracle: 4-wide nodes with FP32 boxes, the
same 4-wide tree with child boxes quantised to 8 bits per plane (64-byte nodes), and the 8-wide
compressed tree (child boxes quantised on a per-node grid, rounded outwards).  The box tests of
all three are conservative and their triangle tests are the same watertight tests, so every
decision -- visibility bits, secondary hit ids -- and hence every radiance value is
bit-identical across layouts, and equal to the brute-force oracle's."""
import numpy as np
import pytest
import torch

import oracle
from oracle import shade
from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _render(sc, width, maps=None, env=None, dtype=torch.float32, layout=None, collapse=None):
    from paper_2608_24109_b300.render import Renderer
    r = Renderer.from_scene(sc, bvh_width=width, bvh_layout=layout, bvh_collapse=collapse)
    M = torch.as_tensor(sc.maps if maps is None else maps).to(dtype).cuda().contiguous()
    E = _dev(sc.env if env is None else env)
    out = r.forward(M, E).clone()
    r.sync()
    return r, out


@pytest.mark.parametrize("name,kw", [("geometry", {}), ("indirect", {"views": 2}), ("precision", {"views": 2}),
                                      ("tiny", {})])
def test_layouts_give_bit_identical_images(name, kw):
    """Full-size workloads (fewer views for the larger two): the forward images of the three
    layouts are equal bit for bit, and so are the decisions behind them."""
    from paper_2608_24109_b300 import native as N
    sc = scenes.config(name, **kw)
    r4, out4 = _render(sc, None, layout=N.BVH_4)
    p4, d4, s4, h4 = r4.saved_state()
    o4 = torch.argsort(p4)
    for layout in (N.BVH_4Q, N.BVH_8Q):
        rq, outq = _render(sc, None, layout=layout)
        assert torch.equal(out4, outq)
        # the covered-pixel lists hold the same pixels in the order the compaction wrote them
        pq, dq, sq, hq = rq.saved_state()
        oq = torch.argsort(pq)
        assert torch.equal(p4[o4], pq[oq])
        assert torch.equal(d4[o4], dq[oq]) and torch.equal(s4[o4], sq[oq])
        assert (h4 is None and hq is None) or torch.equal(h4[o4], hq[oq])
        rq.close()
    r4.close()


@pytest.mark.parametrize("layout", [2, 3])  # BVH_4Q, BVH_8Q
def test_quantised_layout_decisions_equal_the_oracles(layout):
    sc = scenes.config("indirect", n=24, map_res=128, env_w=64, env_h=32, views=2, res=56, n_direct=40, n_bounce=6,
                       n_light=3)
    r, out = _render(sc, None, layout=layout)
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
        r4, out4 = _render(sc, None, layout=1)
        for layout in (2, 3):
            rq, outq = _render(sc, None, layout=layout)
            assert torch.equal(out4, outq) and float(outq.abs().sum()) > 0
            rq.close()
        r4.close()


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


def _unskew(a, n_nodes, per_node):
    """Records of `per_node` float4 (4 or 8) in their logical order: chunk j (two float4) of node
    q is stored at j xor (q mod 4) (128-byte nodes) or j xor (q/2 mod 2) (64-byte nodes)."""
    a = a.reshape(n_nodes, per_node // 2, 8)
    q = np.arange(n_nodes)
    out = np.empty_like(a)
    for j in range(per_node // 2):
        pos = j ^ (q & 3) if per_node == 8 else j ^ ((q >> 1) & 1)
        out[:, j] = a[q, pos]
    return out.reshape(n_nodes, per_node * 4)


def test_quantised_boxes_contain_the_fp32_boxes_with_a_step_of_margin():
    """The same tree in both 4-wide layouts (the builds number the nodes in a different order, so
    the nodes are paired by walking both trees from the root): each pair has the same leaf
    references, and every decoded 8-bit child box of the quantised node contains the FP32 child
    box with at least one grid step on every side (the margin that covers the traversal's folded
    plane evaluation)."""
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc = scenes.config("geometry", views=1, res=64)
    r4, _ = _render(sc, None, layout=N.BVH_4)
    rq, _ = _render(sc, None, layout=N.BVH_4Q)
    i4, s4 = assets.export_mesh(r4.mesh)
    iq, sq = assets.export_mesh(rq.mesh)
    assert i4.node_bytes == 128 and iq.node_bytes == 64 and i4.n_nodes == iq.n_nodes
    n = i4.n_nodes
    f4 = _unskew(s4[4].view(np.float32), n, 8)       # lo.x[4] lo.y[4] lo.z[4] hi.x[4] hi.y[4] hi.z[4] ref[4] pad
    fq = _unskew(sq[4].view(np.float32), n, 4)       # p.xyz step.x ref[4] qlo.xyz qhi.x qhi.y qhi.z step.y step.z
    ref4 = f4[:, 24:28].view(np.int32)
    refq = fq[:, 4:8].view(np.int32)
    # pair the nodes: root with root, then child slot by child slot
    pair = np.full(n, -1, np.int64)
    pair[0] = 0
    todo = [0]
    while todo:
        a = todo.pop()
        b = pair[a]
        ra, rb = ref4[a], refq[b]
        assert np.array_equal(ra < 0, rb < 0) and np.array_equal(ra[ra < 0], rb[rb < 0])
        assert np.array_equal(ra == 0x7FFFFFFF, rb == 0x7FFFFFFF)
        for c in range(4):
            if 0 <= ra[c] < 0x7FFFFFFF:
                assert pair[ra[c]] == -1
                pair[ra[c]] = rb[c]
                todo.append(int(ra[c]))
    assert (pair >= 0).all() and len(set(pair.tolist())) == n
    fq = fq[pair]
    p = fq[:, 0:3].astype(np.float64)
    step = np.stack([fq[:, 3], fq[:, 14], fq[:, 15]], 1).astype(np.float64)
    assert (np.log2(step) == np.round(np.log2(step))).all()   # powers of two
    qw = fq[:, 8:14].view(np.uint32)                           # qlo.x qlo.y qlo.z qhi.x qhi.y qhi.z
    qb = ((qw[:, :, None] >> (8 * np.arange(4))) & 0xFF).astype(np.float64)   # [node, word, child]
    live = ref4 != 0x7FFFFFFF
    assert np.array_equal(live, fq[:, 4:8].view(np.int32) != 0x7FFFFFFF)
    for a in range(3):
        lo4 = f4[:, 4 * a:4 * a + 4].astype(np.float64)
        hi4 = f4[:, 12 + 4 * a:16 + 4 * a].astype(np.float64)
        dlo = p[:, a:a + 1] + qb[:, a] * step[:, a:a + 1]
        dhi = p[:, a:a + 1] + qb[:, 3 + a] * step[:, a:a + 1]
        assert (dlo[live] <= lo4[live] - step[:, a:a + 1].repeat(4, 1)[live]).all()
        assert (dhi[live] >= hi4[live] + step[:, a:a + 1].repeat(4, 1)[live]).all()
        # empty slots decode to inverted boxes
        assert (qb[:, a][~live] == 255).all() and (qb[:, 3 + a][~live] == 0).all()
    r4.close()
    rq.close()


def test_quantised_four_wide_asset_round_trip_and_cycle():
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc = scenes.config("tiny", res=24, views=1, n_direct=4)
    r, ref = _render(sc, None, layout=N.BVH_4Q)
    info, secs = assets.export_mesh(r.mesh)
    assert info.node_bytes == 64
    M = _dev(sc.maps)
    good = assets.import_mesh(r.ctx, info, secs)
    out = torch.empty_like(ref)
    N.exm_render_forward(r.ctx, good, M, r.env, r.cams, r.params, r.frame, out)
    r.sync()
    assert torch.equal(out, ref)
    # node 0 (unskewed: chunk 0 first): the root's node children made the root
    refs = secs[4].view(np.int32).reshape(info.n_nodes, 16)[0, 4:8]
    refs[(refs >= 0) & (refs != 0x7FFFFFFF)] = 0
    bad = assets.import_mesh(r.ctx, info, secs)
    N.exm_render_forward(r.ctx, bad, M, r.env, r.cams, r.params, r.frame, out)
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_TRAVERSAL_LIMIT
    # an out-of-range node reference, and more nodes than a tree over nf leaves has, are refused
    refs[0] = info.n_nodes
    with pytest.raises(N.ExmError) as e:
        assets.import_mesh(r.ctx, info, secs)
    assert e.value.code == N.EXM_ERR_ARG
    for m in (good, bad):
        N.exm_mesh_destroy(m)
    r.close()


@pytest.mark.parametrize("name,kw", [("geometry", {"views": 2}), ("indirect", {"views": 1}), ("tiny", {})])
def test_sah_and_greedy_collapses_render_the_same_images(name, kw):
    """The SAH and the greedy 4-wide collapse of the same binary tree (the SAH one with leaves of
    up to four consecutive triangle records): the same decisions and images bit for bit; both
    trees pass the import checks (every reference in range) and reference every node and
    triangle record exactly once, and the SAH one is not worse by its own cost measure (node
    visits plus 0.6 triangle tests, counted over the frame's rays), up to 2%."""
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc = scenes.config(name, **kw)
    outs, work = [], []
    for mode in (N.BVH_COLLAPSE_GREEDY, N.BVH_COLLAPSE_SAH):
        r, out = _render(sc, None, layout=N.BVH_4, collapse=mode)
        info, secs = assets.export_mesh(r.mesh)
        m2 = assets.import_mesh(r.ctx, info, secs)
        N.exm_mesh_destroy(m2)
        # a tree: every node but the root referenced once, every triangle record once (a leaf
        # ~(k | (c - 1) << 28) names the c records from k)
        refs = _unskew(secs[4].view(np.float32), info.n_nodes, 8)[:, 24:28].view(np.int32).ravel()
        refs = refs[refs != 0x7FFFFFFF]
        inner, lt = refs[refs >= 0], (~refs[refs < 0]).astype(np.int64)
        first, count = lt & ((1 << 28) - 1), (lt >> 28) + 1
        assert count.max() <= 4 and (mode == N.BVH_COLLAPSE_SAH or count.max() == 1)
        records = np.concatenate([np.arange(f, f + c) for f, c in zip(first, count)])
        assert np.array_equal(np.sort(inner), np.arange(1, info.n_nodes))
        assert np.array_equal(np.sort(records), np.arange(info.nf))
        if mode == N.BVH_COLLAPSE_SAH:
            assert (count > 1).any()  # some leaves hold several triangles
        r.params.flags |= N.FLAG_COUNT_WORK
        M = torch.as_tensor(sc.maps).cuda().contiguous()
        r.forward(M, _dev(sc.env))
        r.sync()
        work.append(N.exm_frame_work(r.frame))
        outs.append(out)
        r.close()
    assert torch.equal(outs[0], outs[1])
    cost_g, cost_s = (w[0] + 0.6 * w[1] for w in work)  # node visits + c_tri / c_node x triangle tests
    assert cost_s <= cost_g * 1.02


@pytest.mark.parametrize("nf", [2, 3, 4, 5, 7, 9, 17])
def test_small_meshes_all_trees_agree(nf):
    """Meshes of a few triangles (a binary tree of one or two levels, where the SAH collapse may
    cut leaves of several triangles below the root): the greedy and SAH 4-wide trees and the
    8-wide tree render the same image, and it is not empty."""
    from paper_2608_24109_b300 import native as N
    rng = np.random.default_rng(nf)
    c = rng.uniform(-0.6, 0.6, (nf, 1, 3))
    V = (c + rng.uniform(-0.5, 0.5, (nf, 3, 3))).reshape(-1, 3)
    F = np.arange(3 * nf).reshape(nf, 3)
    maps = scenes.material_maps(rng, 32)
    env = scenes.env_map(rng, 32, 16, 1.0)
    cams = np.stack([scenes.look_at_camera((0.3, 0.4, 2.5), 40, 40), scenes.look_at_camera((-0.4, 0.2, -2.5), 40, 40)])
    sc = scenes._finish("few", V, F, rng.uniform(0.0, 1.0, (3 * nf, 2)), F, maps, maps, env, cams, 40, 40, seed=nf,
                        n_direct=32, n_bounce=2, n_light=2)
    outs = []
    for layout, collapse in ((N.BVH_4, N.BVH_COLLAPSE_GREEDY), (N.BVH_4, N.BVH_COLLAPSE_SAH),
                             (N.BVH_4Q, N.BVH_COLLAPSE_SAH), (N.BVH_8Q, None)):
        r, out = _render(sc, None, layout=layout, collapse=collapse)
        outs.append(out)
        r.close()
    assert float(outs[0].abs().sum()) > 0
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
