"""Pins of the Stage-I topology oracle (Sec. 4.1-4.3): the arccos formula against the true
function, Eq. 1-4 closed forms (EMA, octahedron curvature, equilateral degeneracy), hand-
derived results of one split and one collapse, the seam rule of Eqs. 5-6, the mu constraint,
and the invariants of a round on a closed mesh."""
import math

import numpy as np

from oracle import topology as T

f32 = np.float32


def test_acos_formula():
    x = np.linspace(-1, 1, 20001).astype(f32)
    got = np.array([T.acos_f32(v) for v in x], np.float64)
    assert np.abs(got - np.arccos(x.astype(np.float64))).max() < 5e-7
    assert T.acos_f32(1.0) == 0.0 and abs(float(T.acos_f32(-1.0)) - math.pi) < 3e-7


def test_ema_and_face_measures():
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]], f32)
    F = np.array([[0, 1, 2]])
    nrm, area, elen, degen = T.face_geometry(V, F)
    assert abs(degen[0] - math.sqrt(3) / 4) < 1e-6 and abs(area[0] - math.sqrt(3) / 4) < 1e-6
    assert np.allclose(nrm[0], [0, 0, 1])
    # Eq. 1 with |grad| = 5 from G = 1
    out = T.topology_round(V, F, np.zeros((3, 2), f32), F, np.ones(3, f32),
                           np.array([[3, 4, 0]] * 3, f32), np.ones(1), T.TopoParams(split_percent=0))
    assert np.allclose(out[4], 0.95 + 0.05 * 5, atol=1e-6)


def test_octahedron_curvature_and_flat_grid():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], f32)
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    nrm, area, elen, degen = T.face_geometry(V, F)
    faces_of, deg = T.edge_table(F, 6)
    K = T.curvature(F, nrm, faces_of)
    assert np.allclose(K, math.acos(1.0 / 3.0), atol=1e-6)
    assert (deg == 4).all()
    Vg = np.array([[x, y, 0] for y in range(3) for x in range(3)], f32)
    Fg = np.array([[0, 1, 4], [0, 4, 3], [1, 2, 5], [1, 5, 4], [3, 4, 7], [3, 7, 6], [4, 5, 8], [4, 8, 7]])
    n2, *_ = T.face_geometry(Vg, Fg)
    fo2, _ = T.edge_table(Fg, 9)
    assert (T.curvature(Fg, n2, fo2) == 0).all()


def _quad(uv_seam=False):
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], f32)
    F = np.array([[0, 1, 2], [0, 2, 3]])
    if not uv_seam:
        UV = V[:, :2].copy()
        Fuv = F.copy()
    else:  # the second face lives on another UV island
        UV = np.concatenate([V[:, :2], V[:, :2] * 0.5 + 0.5]).astype(f32)
        Fuv = np.array([[0, 1, 2], [4, 6, 7]])
    return V, F, UV, Fuv


def test_split_of_a_quad_diagonal():
    V, F, UV, Fuv = _quad()
    grad = np.array([[1, 0, 0], [1, 0, 0], [1, 0, 0], [0, 0, 0]], f32)  # face 0 scores higher
    V2, F2, UV2, Fuv2, G2, st = T.topology_round(V, F, UV, Fuv, np.zeros(4, f32), grad, np.ones(2))
    assert st == {"splits": 1, "merges": 0, "faces_deleted": 0}
    # face 0 = (0,1,2) splits its edge (2,0) (l/mean degree: 1/2.5, 1/2.5, sqrt(2)/3) at the
    # common projection (0.5, 0.5) of vertices 1 and 3
    assert np.array_equal(V2[4], f32([0.5, 0.5, 0]))
    assert F2.tolist() == [[2, 4, 1], [0, 4, 3], [4, 0, 1], [4, 2, 3]]
    assert UV2.shape == (5, 2) and np.array_equal(UV2[4], f32([0.5, 0.5]))  # not a seam: one shared UV
    assert Fuv2.tolist() == F2.tolist()
    assert abs(G2[4] - 0.05) < 1e-7  # mean of the endpoints' EMA (0.05 and 0.05)


def test_split_across_a_uv_seam_keeps_two_uvs():
    V, F, UV, Fuv = _quad(uv_seam=True)
    grad = np.array([[1, 0, 0], [1, 0, 0], [1, 0, 0], [0, 0, 0]], f32)
    V2, F2, UV2, Fuv2, G2, st = T.topology_round(V, F, UV, Fuv, np.zeros(4, f32), grad, np.ones(2))
    assert st["splits"] == 1
    # u at mu = 1/2 between the corners of vertices 2 and 0, in each face's own island
    assert np.array_equal(UV2[-2], f32([0.5, 0.5])) and np.array_equal(UV2[-1], f32([0.75, 0.75]))
    assert Fuv2[0].tolist()[1] == Fuv2[2].tolist()[0] == UV2.shape[0] - 2
    assert Fuv2[1].tolist()[1] == Fuv2[3].tolist()[0] == UV2.shape[0] - 1


def test_split_outside_the_mu_range_is_discarded():
    # face 0 = (a, b, c) on a long edge (a, b); a fan around c raises deg(c) to 5 so that (a, b)
    # has the best l_e / mean degree (4/4 against 3.74/4.5 and 1.08/4.5).  Both opposite vertices
    # c and d project to (0.4, 0): mu = 0.1 < 0.25, so the split is discarded
    V = np.array([[0, 0, 0], [4, 0, 0], [0.4, 1, 0], [0.4, -1, 0], [-0.6, 1.5, 0], [0.4, 2.2, 0], [1.4, 1.5, 0]], f32)
    F = np.array([[0, 1, 2], [1, 0, 3], [2, 1, 6], [2, 6, 5], [2, 5, 4], [2, 4, 0]])
    grad = np.zeros((7, 3), f32)
    grad[2] = [1, 0, 0]  # faces around c score highest; face 0 first by index
    faces_of, deg = T.edge_table(F, 7)
    assert deg[:3].tolist() == [4, 4, 5]
    vs, mu = T.split_vertex(V, F, 0, 0, 1, 0)
    assert abs(mu - 0.1) < 1e-6
    V2, F2, UV2, Fuv2, G2, st = T.topology_round(V, F, V[:, :2], F, np.zeros(7, f32), grad, np.ones(6))
    assert st["splits"] == 0 and np.array_equal(F2, F)


def test_collapse_of_a_sliver_on_the_boundary():
    # a square fanned around a centre vertex 4 pushed against the bottom edge: face (0,1,4) is a
    # sliver (D_f = 0.005) with the boundary edge (0,1); vertices 0 and 1 both have degree 3,
    # so the higher index, 1, merges into 0
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0.5, 0.01, 0]], f32)
    F = np.array([[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]])
    prm = T.TopoParams(split_percent=0)
    V2, F2, UV2, Fuv2, G2, st = T.topology_round(V, F, V[:, :2], F, np.zeros(5, f32), np.zeros((5, 3), f32),
                                                 np.ones(4), prm)
    assert st == {"splits": 0, "merges": 1, "faces_deleted": 1}
    assert np.array_equal(V2, V[[0, 2, 3, 4]])
    # (1,2,4) -> (0,1,3) after the merge and the compaction; (2,3,4) -> (1,2,3); (3,0,4) -> (2,0,3)
    assert F2.tolist() == [[0, 1, 3], [1, 2, 3], [2, 0, 3]]
    # reconnected corners keep their UV index (the corner of vertex 1 keeps UV 1); all five UVs
    # stay referenced, so none is dropped
    assert Fuv2.tolist() == [[1, 2, 4], [2, 3, 4], [3, 0, 4]]
    assert np.array_equal(UV2, V[:, :2])


def _euler(F, nv):
    E = {(min(a, b), max(a, b)) for f in F for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))}
    return nv - len(E) + len(F)


def test_round_invariants_on_a_closed_mesh():
    from paper_2608_24109_b300 import scenes
    sc = scenes.config("indirect", n=10, map_res=64, env_w=32, env_h=16, views=1, res=32)
    rng = np.random.default_rng(3)
    G = rng.uniform(0, 1, sc.V.shape[0]).astype(f32)
    grad = rng.normal(size=sc.V.shape).astype(f32)
    counts = rng.integers(0, 4, sc.F.shape[0])
    V2, F2, UV2, Fuv2, G2, st = T.topology_round(sc.V, sc.F, sc.UV, sc.Fuv, G, grad, counts)
    assert st["splits"] > 0 and st["merges"] > 0
    assert _euler(F2, V2.shape[0]) == _euler(sc.F, sc.V.shape[0])
    assert F2.min() >= 0 and F2.max() < V2.shape[0] and Fuv2.min() >= 0 and Fuv2.max() < UV2.shape[0]
    assert len(np.unique(Fuv2)) == UV2.shape[0]  # every UV referenced
    assert (F2[:, 0] != F2[:, 1]).all() and (F2[:, 1] != F2[:, 2]).all() and (F2[:, 0] != F2[:, 2]).all()
    nf2 = sc.F.shape[0] + 2 * st["splits"] - st["faces_deleted"]
    assert F2.shape[0] == nf2
    assert V2.shape[0] == sc.V.shape[0] + st["splits"] - st["merges"]


def _budget_case():
    # a quad (faces 0, 1) and a lone triangle (face 2).  Rank order: face 0 (its diagonal, shared
    # with face 1: +2 faces), face 1 (claimed by face 0's split), face 2 (its hypotenuse, a
    # boundary edge: +1 face).  So the accepted splits are [face 0 (+2), face 2 (+1)]
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [3, 0, 0], [4, 0, 0], [3, 1, 0]], f32)
    F = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6]])
    grad = np.zeros((7, 3), f32)
    grad[0:3] = [1, 0, 0]
    grad[4:7] = [0.5, 0, 0]
    return V, F, V[:, :2].copy(), F.copy(), grad


def test_face_budget_keeps_the_prefix_of_the_accepted_splits():
    """R40's budget rule, hand-worked where the two readings of "max 200K faces" differ: with
    room for one more face, skipping the +2 split and taking the later +1 split would give one
    split; keeping the prefix of the accepted splits that fits gives none.  With room for two
    faces the first split fits and the second does not; with room for three both fit."""
    V, F, UV, Fuv, grad = _budget_case()
    expect = {4: (0, 3), 5: (1, 5), 6: (2, 6)}
    for max_faces, (splits, faces) in expect.items():
        prm = T.TopoParams(split_percent=100, max_faces=max_faces)
        V2, F2, UV2, Fuv2, G2, st = T.topology_round(V, F, UV, Fuv, np.zeros(7, f32), grad, np.ones(3), prm)
        assert (st["splits"], F2.shape[0]) == (splits, faces), max_faces
    # with room for two faces the applied split is face 0's diagonal (new vertex at the centre)
    prm = T.TopoParams(split_percent=100, max_faces=5)
    V2, F2, *_ = T.topology_round(V, F, UV, Fuv, np.zeros(7, f32), grad, np.ones(3), prm)
    assert np.array_equal(V2[7], f32([0.5, 0.5, 0]))
