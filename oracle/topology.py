"""Oracle, part 5: one Stage-I topology round (Sec. 4.1-4.3: Eqs. 1-6), sequential and in FP32
with every operation in a fixed order, so that the GPU round can be compared bit for bit.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The round, as read from the paper (each choice the paper leaves open is a reading listed
with the design):

1. Eq. 1: G_v <- beta_g G_v + (1 - beta_g) |grad_v L|.
2. Per face: unit normal, area, edge lengths; D_f = Area / l_max^2 (Eq. 4).  Two faces are
   adjacent when they share an edge used by exactly two faces; any other edge is a boundary
   edge.  deg(v) is the number of distinct neighbours of v.
3. Eq. 2: K_f = mean over adjacent faces of arccos(n_f . n_f'), arccos by the published
   8-term formula of Abramowitz and Stegun (4.4.46, absolute error <= 2e-8).
4. Eq. 3: S_f = w_g G_f + w_k K_f with G_f the mean of the corners' G_v.
5. Splitting: faces with area >= the lower median area are candidates, ranked by S_f
   (descending, ties by index); the first ceil(5% of the faces) are tried in rank order.  The
   split edge maximises l_e / mean degree (ties: edge order (0,1), (1,2), (2,0)); the new
   vertex is the mean of the projections of the two opposite vertices onto the edge line
   (the midpoint on a boundary edge); mu = |v_s - v_a| / |v_b - v_a| outside [0.25, 0.75]
   discards the split.  A split is skipped when one of its faces was already claimed by an
   accepted split (greedy in rank order).  The accepted splits are then applied in rank order
   while the face count stays within the face budget; the rest are dropped.  Edge choice, v_s
   and mu use the mesh at the start of the round.
6. UV maintenance (Eqs. 5-6): u_s interpolated at mu in the UV space of each old face; two
   candidates closer than tau_uv share one averaged UV, else each side keeps its own.
7. Merging, on the mesh after the splits: unmodified faces with C_rend = 0 or D_f < tau_degen
   and area <= the lower median area, ranked by D_f (ascending, ties by index).  The collapse
   edge is the shortest boundary edge if the face has one, else its shortest edge; the
   lower-degree endpoint v_r (ties: the higher index) merges into v_s, which keeps its
   position.  A merge is skipped when a face around v_r was already modified in the round.
8. Faces left with a repeated vertex are deleted; faces, vertices and UVs are compacted in
   order (unreferenced UVs dropped); reconnected corners keep their UV indices.

Split children: a face (x0, x1, x2) split on its edge (x_k, x_k+1) keeps its slot for
(x_k, v_s, x_k+2) and appends (v_s, x_k+1, x_k+2), which preserves the orientation.  New
vertices, faces and UVs are appended in the order of the accepted splits.  A new vertex's
G_v is the mean of the edge endpoints'.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

f32 = np.float32

# Abramowitz and Stegun 4.4.46: arccos x = sqrt(1 - x) (a0 + a1 x + ... + a7 x^7), 0 <= x <= 1
ACOS_A = [f32(1.5707963050), f32(-0.2145988016), f32(0.0889789874), f32(-0.0501743046),
          f32(0.0308918810), f32(-0.0170881256), f32(0.0066700901), f32(-0.0012624911)]
PI_F = f32(3.14159265358979)


@dataclass
class TopoParams:
    beta_g: float = 0.95
    w_g: float = 0.6
    w_k: float = 0.4
    tau_degen: float = 0.05
    tau_uv: float = 1e-4
    split_percent: int = 5
    max_faces: int = 200000


def acos_f32(x):
    """arccos of an FP32 value in [-1, 1] (Horner in FP32, no fused operations)."""
    x = f32(x)
    ax = f32(abs(x))
    p = ACOS_A[7]
    for a in ACOS_A[6::-1]:
        p = f32(f32(p * ax) + a)
    r = f32(np.sqrt(f32(f32(1.0) - ax)) * p)
    return f32(PI_F - r) if x < 0 else r


def _sub(a, b):
    return [f32(a[0] - b[0]), f32(a[1] - b[1]), f32(a[2] - b[2])]


def _dot(a, b):
    return f32(f32(f32(a[0] * b[0]) + f32(a[1] * b[1])) + f32(a[2] * b[2]))


def _cross(a, b):
    return [f32(f32(a[1] * b[2]) - f32(a[2] * b[1])), f32(f32(a[2] * b[0]) - f32(a[0] * b[2])),
            f32(f32(a[0] * b[1]) - f32(a[1] * b[0]))]


def _len(a):
    return f32(np.sqrt(_dot(a, a)))


def face_geometry(V, F):
    """Unit normals, areas, edge lengths [nf, 3] (edges (0,1), (1,2), (2,0)) and D_f."""
    nf = F.shape[0]
    nrm = np.zeros((nf, 3), f32)
    area = np.zeros(nf, f32)
    elen = np.zeros((nf, 3), f32)
    degen = np.zeros(nf, f32)
    for f in range(nf):
        p = [V[F[f, k]] for k in range(3)]
        c = _cross(_sub(p[1], p[0]), _sub(p[2], p[0]))
        ln = _len(c)
        if ln > 0:
            nrm[f] = [f32(c[0] / ln), f32(c[1] / ln), f32(c[2] / ln)]
        area[f] = f32(f32(0.5) * ln)
        for k in range(3):
            elen[f, k] = _len(_sub(p[(k + 1) % 3], p[k]))
        lm = max(elen[f, 0], elen[f, 1], elen[f, 2])
        degen[f] = f32(area[f] / f32(lm * lm)) if lm > 0 else f32(0.0)
    return nrm, area, elen, degen


def edge_table(F, nv):
    """Undirected edge -> list of (face, local edge); vertex valence."""
    faces_of = {}
    for f in range(F.shape[0]):
        for k in range(3):
            a, b = int(F[f, k]), int(F[f, (k + 1) % 3])
            faces_of.setdefault((min(a, b), max(a, b)), []).append((f, k))
    deg = np.zeros(nv, np.int64)
    for (a, b) in faces_of:
        deg[a] += 1
        deg[b] += 1
    return faces_of, deg


def _neighbour(faces_of, F, f, k):
    """The face across local edge k of f (-1 on a boundary edge) and its local edge."""
    a, b = int(F[f, k]), int(F[f, (k + 1) % 3])
    lst = faces_of[(min(a, b), max(a, b))]
    if len(lst) != 2:
        return -1, -1
    g, kg = lst[0] if lst[0][0] != f else lst[1]
    return g, kg


def curvature(F, nrm, faces_of):
    nf = F.shape[0]
    K = np.zeros(nf, f32)
    for f in range(nf):
        s, cnt = f32(0.0), 0
        for k in range(3):
            g, _ = _neighbour(faces_of, F, f, k)
            if g < 0:
                continue
            d = _dot(nrm[f], nrm[g])
            d = f32(min(max(d, f32(-1.0)), f32(1.0)))
            s = f32(s + acos_f32(d))
            cnt += 1
        K[f] = f32(s / f32(cnt)) if cnt else f32(0.0)
    return K


def lower_median(x):
    s = np.sort(np.asarray(x, f32))
    return s[(len(s) - 1) // 2]


def split_vertex(V, F, f, k, g, kg):
    """v_s and mu for splitting face f on its local edge k (g: face across, -1 on a boundary)."""
    va, vb = V[F[f, k]], V[F[f, (k + 1) % 3]]
    e = _sub(vb, va)
    ee = _dot(e, e)

    def proj(p):
        t = f32(_dot(_sub(p, va), e) / ee)
        return [f32(va[i] + f32(t * e[i])) for i in range(3)]

    if g < 0:
        vs = [f32(f32(va[i] + vb[i]) * f32(0.5)) for i in range(3)]
    else:
        tc = proj(V[F[f, (k + 2) % 3]])
        td = proj(V[F[g, (kg + 2) % 3]])
        vs = [f32(f32(tc[i] + td[i]) * f32(0.5)) for i in range(3)]
    mu = f32(_len(_sub(vs, va)) / f32(np.sqrt(ee)))
    return vs, mu


def topology_round(V, F, UV, Fuv, G, grad_V, render_counts, prm: TopoParams = TopoParams()):
    """One round; returns (V, F, UV, Fuv, G, stats) as new arrays."""
    V = np.asarray(V, f32).copy()
    F = np.asarray(F, np.int64).copy()
    UV = np.asarray(UV, f32).copy()
    Fuv = np.asarray(Fuv, np.int64).copy()
    nv, nf = V.shape[0], F.shape[0]
    # 1. Eq. 1
    b = f32(prm.beta_g)
    gn = np.array([_len(grad_V[v].astype(f32)) for v in range(nv)], f32)
    G = np.array([f32(f32(b * f32(G[v])) + f32(f32(f32(1.0) - b) * gn[v])) for v in range(nv)], f32)
    # 2.-4.
    nrm, area, elen, degen = face_geometry(V, F)
    faces_of, deg = edge_table(F, nv)
    K = curvature(F, nrm, faces_of)
    wg, wk = f32(prm.w_g), f32(prm.w_k)
    S = np.zeros(nf, f32)
    for f in range(nf):
        Gf = f32(f32(f32(G[F[f, 0]] + G[F[f, 1]]) + G[F[f, 2]]) / f32(3.0))
        S[f] = f32(f32(wg * Gf) + f32(wk * K[f]))
    # 5.-6. splits
    amed = lower_median(area)
    cand = [f for f in range(nf) if area[f] >= amed]
    cand.sort(key=lambda f: (-float(S[f]), f))
    cand = cand[:(nf * prm.split_percent + 99) // 100]
    # greedy selection in rank order on the mesh at the start of the round
    claimed = np.zeros(nf, bool)
    accepted = []
    for f in cand:
        score = [f32(elen[f, k] / f32(f32(deg[F[f, k]] + deg[F[f, (k + 1) % 3]]) * f32(0.5))) for k in range(3)]
        k = 0
        for c in (1, 2):
            if score[c] > score[k]:
                k = c
        g, kg = _neighbour(faces_of, F, f, k)
        vs, mu = split_vertex(V, F, f, k, g, kg)
        if not (f32(0.25) <= mu <= f32(0.75)):
            continue
        if claimed[f] or (g >= 0 and claimed[g]):
            continue
        claimed[f] = True
        if g >= 0:
            claimed[g] = True
        accepted.append((f, k, g, kg, vs, mu))
    # the face budget keeps a prefix of the accepted splits
    applied, faces_now = [], nf
    for sp in accepted:
        add = 2 if sp[2] >= 0 else 1
        if faces_now + add > prm.max_faces:
            break
        faces_now += add
        applied.append(sp)
    touched = np.zeros(nf, bool)
    F0, Fuv0 = F.copy(), Fuv.copy()  # the mesh at the start of the round (F is rewritten below)
    new_V, new_G, new_F, new_Fuv, new_UV = [], [], [], [], []
    n_split = 0
    for (f, k, g, kg, vs, mu) in applied:
        touched[f] = True
        if g >= 0:
            touched[g] = True
        s_idx = nv + len(new_V)
        new_V.append(vs)
        va_i, vb_i = int(F0[f, k]), int(F0[f, (k + 1) % 3])
        new_G.append(f32(f32(G[va_i] + G[vb_i]) * f32(0.5)))
        # UVs at mu in each old face's UV space (Eqs. 5-6)
        one_m = f32(f32(1.0) - mu)

        def interp(face):
            ca = [c for c in range(3) if F0[face, c] == va_i][0]
            cb = [c for c in range(3) if F0[face, c] == vb_i][0]
            ua, ub = UV[Fuv0[face, ca]], UV[Fuv0[face, cb]]
            return [f32(f32(one_m * ua[i]) + f32(mu * ub[i])) for i in range(2)]

        u1 = interp(f)
        uv_base = UV.shape[0] + len(new_UV)
        if g >= 0:
            u2 = interp(g)
            d = [f32(u1[0] - u2[0]), f32(u1[1] - u2[1])]
            if f32(np.sqrt(f32(f32(d[0] * d[0]) + f32(d[1] * d[1])))) < f32(prm.tau_uv):
                new_UV.append([f32(f32(u1[i] + u2[i]) * f32(0.5)) for i in range(2)])
                uf, ug = uv_base, uv_base
            else:
                new_UV.append(u1)
                new_UV.append(u2)
                uf, ug = uv_base, uv_base + 1
        else:
            new_UV.append(u1)
            uf = uv_base
        for face, kk, us in ((f, k, uf),) + (((g, kg, ug),) if g >= 0 else ()):
            x = [int(F0[face, (kk + j) % 3]) for j in range(3)]
            t = [int(Fuv0[face, (kk + j) % 3]) for j in range(3)]
            F[face] = [x[0], s_idx, x[2]]
            Fuv[face] = [t[0], us, t[2]]
            new_F.append([s_idx, x[1], x[2]])
            new_Fuv.append([us, t[1], t[2]])
        n_split += 1
    if new_V:
        V = np.concatenate([V, np.asarray(new_V, f32)])
        G = np.concatenate([G, np.asarray(new_G, f32)])
        F = np.concatenate([F, np.asarray(new_F, np.int64)])
        Fuv = np.concatenate([Fuv, np.asarray(new_Fuv, np.int64)])
        UV = np.concatenate([UV, np.asarray(new_UV, f32).reshape(-1, 2)])
        touched = np.concatenate([touched, np.ones(len(new_F), bool)])
    # 7. merges on the post-split mesh
    nv2, nf2 = V.shape[0], F.shape[0]
    nrm, area, elen, degen = face_geometry(V, F)
    faces_of, deg = edge_table(F, nv2)
    counts = np.concatenate([np.asarray(render_counts, np.int64), np.zeros(nf2 - nf, np.int64)])
    amed = lower_median(area)
    tau = f32(prm.tau_degen)
    mcand = [f for f in range(nf2) if not touched[f] and area[f] <= amed and (counts[f] == 0 or degen[f] < tau)]
    mcand.sort(key=lambda f: (float(degen[f]), f))
    star = {}
    for f in range(nf2):
        for k in range(3):
            star.setdefault(int(F[f, k]), []).append(f)
    target = {}
    n_merge = 0
    for f in mcand:
        bnd = [k for k in range(3) if _neighbour(faces_of, F, f, k)[0] < 0]
        ks = bnd if bnd else [0, 1, 2]
        k = ks[0]
        for c in ks[1:]:
            if elen[f, c] < elen[f, k]:
                k = c
        a, bb = int(F[f, k]), int(F[f, (k + 1) % 3])
        if deg[a] < deg[bb] or (deg[a] == deg[bb] and a > bb):
            vr, vs_ = a, bb
        else:
            vr, vs_ = bb, a
        if any(touched[g] for g in star[vr]):
            continue
        for g in star[vr]:
            touched[g] = True
        target[vr] = vs_
        n_merge += 1
    # 8. apply, delete, compact
    vmap = np.arange(nv2)
    for vr, vs_ in target.items():
        vmap[vr] = vs_
    F = vmap[F]
    keep = (F[:, 0] != F[:, 1]) & (F[:, 1] != F[:, 2]) & (F[:, 2] != F[:, 0])
    F, Fuv = F[keep], Fuv[keep]
    alive = np.ones(nv2, bool)
    alive[list(target.keys())] = False
    newidx = np.cumsum(alive) - 1
    V, G = V[alive], G[alive]
    F = newidx[F]
    used = np.zeros(UV.shape[0], bool)
    used[Fuv.ravel()] = True
    uvidx = np.cumsum(used) - 1
    UV = UV[used]
    Fuv = uvidx[Fuv]
    return V, F.astype(np.int32), UV, Fuv.astype(np.int32), G, dict(splits=n_split, merges=n_merge,
                                                                    faces_deleted=int((~keep).sum()))
