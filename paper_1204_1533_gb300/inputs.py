"""Seeded synthetic inputs: node sets, meshes and initial states.

This module produces the *data* that both the CUDA library and its CPU test
oracle consume: the 1-D solution-node set {s_i}, isoparametric node
coordinates of structured quad/hex meshes (optionally perturbed, curved,
periodic, or with per-element re-oriented local coordinates), boundary tags,
and nodal initial / manufactured states. It evaluates nothing of the Line-DG
scheme itself (no quadrature, no basis, no metric, no flux, no residual).

Mesh dictionaries have the keys
  D         : int, 2 or 3
  p         : int, polynomial degree
  s         : float64[p+1], increasing node set on [0,1], s[0]=0, s[p]=1,
              symmetric (s[p-i] == 1 - s[i] exactly)
  nodes     : float64[E, (p+1)^D, D], node coordinates x_ijk, local node index
              i + (p+1) j + (p+1)^2 k (i runs along reference direction 1)
  vertices  : int64[E, 2^D] global vertex ids; local corner c sits at the
              reference corner (c & 1, (c >> 1) & 1, (c >> 2) & 1); periodic
              images share ids
  btag      : int32[E, 2D]; face f = 2 d + end (end 0 at X_d = 0, end 1 at
              X_d = 1); -1 = interior (matched through vertex ids), >= 0 =
              boundary tag
Elements of the structured generators are numbered e = ex + nx (ey + ny ez).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

MESH_SEED = 1204
STATE_SEED = 1533


# ---------------------------------------------------------------------------
# node sets
# ---------------------------------------------------------------------------
def gll_nodes(p: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre points mapped to [0,1] (the node set chosen for
    s_i; the paper only requires an increasing set with s_0=0, s_p=1).
    Made exactly symmetric so that reversed face orientations map node i to
    node p-i."""
    if p < 1:
        raise ValueError("p >= 1 required")
    from numpy.polynomial import legendre as leg
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.sort(np.real(leg.legroots(leg.legder(c)))) if p >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    s = 0.5 * (x + 1.0)
    s[0], s[p] = 0.0, 1.0
    for i in range(1, (p + 1) // 2):
        s[p - i] = 1.0 - s[i]
    if p % 2 == 0:
        s[p // 2] = 0.5
    return s


def equispaced_nodes(p: int) -> np.ndarray:
    s = np.linspace(0.0, 1.0, p + 1)
    for i in range(1, (p + 1) // 2):
        s[p - i] = 1.0 - s[i]
    if p % 2 == 0:
        s[p // 2] = 0.5
    return s


# ---------------------------------------------------------------------------
# structured meshes
# ---------------------------------------------------------------------------
def _corner_bits(D):
    return [tuple((c >> b) & 1 for b in range(D)) for c in range(1 << D)]


def structured_mesh(n, p, lo, hi, periodic, perturb=0.0, seed=MESH_SEED,
                    node_map=None, s=None, btag_of_face=None, ycoords=None):
    """Tensor-product mesh of len(n) dimensions.

    n        : elements per dimension
    lo, hi   : domain box
    periodic : per-dimension periodicity flags (periodic images share ids)
    perturb  : vertex perturbation, a fraction of the local spacing h; every
               coordinate of every perturbable vertex moves by U(-perturb h,
               +perturb h). A vertex is perturbable when it is interior in
               every non-periodic dimension; periodic perturbations repeat.
    node_map : optional callable (xyz[..., D]) -> xyz applied to the node
               coordinates after multilinear placement (curved elements)
    btag_of_face(d, end) -> tag for faces on non-periodic domain sides
    ycoords  : optional explicit vertex coordinates along dimension 1
    """
    D = len(n)
    n = tuple(int(v) for v in n)
    s = gll_nodes(p) if s is None else np.asarray(s, dtype=np.float64)
    rng = np.random.default_rng(seed)
    nv = [n[d] if periodic[d] else n[d] + 1 for d in range(D)]
    h = [(hi[d] - lo[d]) / n[d] for d in range(D)]
    # vertex perturbations on the id grid (periodic images identical)
    shape_ids = tuple(nv[::-1])  # [z][y][x]
    delta = rng.uniform(-1.0, 1.0, size=shape_ids + (D,))
    movable = np.ones(shape_ids, dtype=bool)
    for d in range(D):
        if not periodic[d]:
            ax = D - 1 - d
            sl = [slice(None)] * D
            sl[ax] = 0
            movable[tuple(sl)] = False
            sl[ax] = nv[d] - 1
            movable[tuple(sl)] = False
    for d in range(D):
        delta[..., d] *= perturb * h[d]
    delta[~movable] = 0.0

    def coord_axis(d, idx):
        if d == 1 and ycoords is not None:
            return ycoords[idx]
        return lo[d] + idx * h[d]

    E = int(np.prod(n))
    npe = (p + 1) ** D
    nodes = np.zeros((E, npe, D))
    verts = np.zeros((E, 1 << D), dtype=np.int64)
    btag = -np.ones((E, 2 * D), dtype=np.int32)
    corners = _corner_bits(D)
    # reference node coordinates, local index i + (p+1) j + (p+1)^2 k
    ref = np.array([[s[(a // (p + 1) ** b) % (p + 1)] for b in range(D)]
                    for a in range(npe)])
    for e, eidx in enumerate(itertools.product(*[range(n[d]) for d in reversed(range(D))])):
        eidx = eidx[::-1]  # (ex, ey, ez)
        cpos = np.zeros((1 << D, D))
        for c, bits in enumerate(corners):
            g = [eidx[d] + bits[d] for d in range(D)]
            gid = [g[d] % nv[d] if periodic[d] else g[d] for d in range(D)]
            vid = 0
            for d in reversed(range(D)):
                vid = vid * nv[d] + gid[d]
            verts[e, c] = vid
            dl = delta[tuple(gid[::-1])]
            for d in range(D):
                cpos[c, d] = coord_axis(d, g[d]) + dl[d]
        # multilinear placement of the nodes between the corners
        w = np.ones((npe, 1 << D))
        for c, bits in enumerate(corners):
            for d in range(D):
                w[:, c] *= ref[:, d] if bits[d] else (1.0 - ref[:, d])
        nodes[e] = w @ cpos
        for d in range(D):
            if periodic[d]:
                continue
            if eidx[d] == 0:
                btag[e, 2 * d] = 0 if btag_of_face is None else btag_of_face(d, 0)
            if eidx[d] == n[d] - 1:
                btag[e, 2 * d + 1] = 0 if btag_of_face is None else btag_of_face(d, 1)
    if node_map is not None:
        nodes = node_map(nodes)
    return {"D": D, "p": int(p), "s": s, "nodes": np.ascontiguousarray(nodes),
            "vertices": verts, "btag": btag,
            "shape": n, "periodic": tuple(bool(x) for x in periodic),
            "lo": tuple(lo), "hi": tuple(hi)}


# ---------------------------------------------------------------------------
# per-element re-orientation (exercises general face orientations)
# ---------------------------------------------------------------------------
def _rotations(D):
    """Orientation-preserving symmetries of the reference square / cube as
    (perm, flip): new axis a takes old axis perm[a], reversed if flip[a]."""
    out = []
    for perm in itertools.permutations(range(D)):
        inv = sum(1 for i in range(D) for j in range(i + 1, D) if perm[i] > perm[j])
        for flip in itertools.product([0, 1], repeat=D):
            if (inv + sum(flip)) % 2 == 0:
                out.append((perm, flip))
    return out


def reorient(mesh, seed=MESH_SEED + 7):
    """Give each element a random orientation-preserving local coordinate
    system. Returns (new_mesh, maps) where maps[e] is the node permutation
    new_local -> old_local, usable with permute_nodal()."""
    D, p = mesh["D"], mesh["p"]
    rng = np.random.default_rng(seed)
    rots = _rotations(D)
    E = mesh["nodes"].shape[0]
    npe = (p + 1) ** D
    nodes = np.empty_like(mesh["nodes"])
    verts = np.empty_like(mesh["vertices"])
    btag = np.empty_like(mesh["btag"])
    maps = np.empty((E, npe), dtype=np.int64)
    for e in range(E):
        perm, flip = rots[rng.integers(len(rots))]
        for a in range(npe):
            newidx = [(a // (p + 1) ** b) % (p + 1) for b in range(D)]
            old = [0] * D
            for ax in range(D):
                v = newidx[ax]
                old[perm[ax]] = (p - v) if flip[ax] else v
            maps[e, a] = sum(old[b] * (p + 1) ** b for b in range(D))
        nodes[e] = mesh["nodes"][e][maps[e]]
        for c in range(1 << D):
            newb = [(c >> b) & 1 for b in range(D)]
            old = [0] * D
            for ax in range(D):
                old[perm[ax]] = (1 - newb[ax]) if flip[ax] else newb[ax]
            verts[e, c] = mesh["vertices"][e, sum(old[b] << b for b in range(D))]
        for ax in range(D):
            for end in range(2):
                oend = (1 - end) if flip[ax] else end
                btag[e, 2 * ax + end] = mesh["btag"][e, 2 * perm[ax] + oend]
    out = dict(mesh)
    out.update(nodes=nodes, vertices=verts, btag=btag)
    out.pop("shape", None)
    return out, maps


def permute_nodal(field, maps):
    """Apply reorient() node maps to a nodal field [E, ..., (p+1)^D]."""
    out = np.empty_like(field)
    for e in range(field.shape[0]):
        out[e] = field[e][..., maps[e]]
    return out


# ---------------------------------------------------------------------------
# unstructured meshes (non-grid topology: vertices of valence 3, 5, 6, ...)
# ---------------------------------------------------------------------------
def _multilinear(cpos, s, D):
    """Node coordinates [(p+1)^D, D] of the multilinear element with corner
    positions cpos [2^D, D] (local corner c at reference corner bits of c)."""
    p = len(s) - 1
    npe = (p + 1) ** D
    ref = np.array([[s[(a // (p + 1) ** b) % (p + 1)] for b in range(D)] for a in range(npe)])
    w = np.ones((npe, 1 << D))
    for c, bits in enumerate(_corner_bits(D)):
        for d in range(D):
            w[:, c] *= ref[:, d] if bits[d] else (1.0 - ref[:, d])
    return w @ cpos


def _grid_vertices(n, D, L, periodic, perturb, rng):
    """Perturbed vertex grid: (ids [...], positions [..., D]) indexed by the
    unwrapped integer grid point; periodic images share ids and offsets."""
    nv = n if periodic else n + 1
    h = L / n
    delta = rng.uniform(-1.0, 1.0, size=(nv,) * D + (D,)) * perturb * h
    if not periodic:
        inner = np.zeros((nv,) * D, dtype=bool)
        inner[(slice(1, nv - 1),) * D] = True
        delta[~inner] = 0.0

    def vid(g):
        w = [int(v) % nv if periodic else int(v) for v in g]
        out = 0
        for d in reversed(range(D)):
            out = out * nv + w[d]
        return out

    def pos(g):
        w = tuple(int(v) % nv if periodic else int(v) for v in g)
        return np.array([g[d] * h for d in range(D)], dtype=np.float64) + delta[w[::-1]]
    return vid, pos, nv ** D


def _finish_mesh(D, p, s, corners_list, lo, hi, periodic):
    """Mesh dictionary from elements given as (vertex ids [2^D], corner
    positions [2^D, D]); faces seen once get boundary tag 0."""
    E = len(corners_list)
    npe = (p + 1) ** D
    nodes = np.zeros((E, npe, D))
    verts = np.zeros((E, 1 << D), dtype=np.int64)
    for e, (ids, cpos) in enumerate(corners_list):
        verts[e] = ids
        nodes[e] = _multilinear(np.asarray(cpos), s, D)
    count = {}
    for e in range(E):
        for f in range(2 * D):
            d, end = divmod(f, 2)
            key = tuple(sorted(int(verts[e, c]) for c in range(1 << D) if ((c >> d) & 1) == end))
            count[key] = count.get(key, 0) + 1
    btag = -np.ones((E, 2 * D), dtype=np.int32)
    for e in range(E):
        for f in range(2 * D):
            d, end = divmod(f, 2)
            key = tuple(sorted(int(verts[e, c]) for c in range(1 << D) if ((c >> d) & 1) == end))
            if count[key] == 1:
                btag[e, f] = 0
    return {"D": D, "p": int(p), "s": s, "nodes": np.ascontiguousarray(nodes), "vertices": verts,
            "btag": btag, "periodic": (bool(periodic),) * D, "lo": tuple(lo), "hi": tuple(hi)}


def unstructured_quad_mesh(n=2, p=3, L=1.0, periodic=False, perturb=0.1, refine=0, seed=MESH_SEED):
    """Unstructured straight-sided quadrilaterals on [0,L]^2.

    An n x n vertex grid (interior vertices, or all vertices when periodic,
    perturbed by U(-perturb h, perturb h) per coordinate) is split into
    triangles along a seeded random diagonal per cell; every triangle is
    split into three quadrilaterals through its edge midpoints and centroid
    (vertices of valence 3 at the centroids, 4-8 elsewhere). `refine`
    uniform refinements then split every quadrilateral into four through
    its edge midpoints and centre, so a refined mesh tiles the same
    bilinear elements (the nested sequence of a convergence study).
    6 n^2 4^refine elements. Periodic meshes need n >= 3."""
    rng = np.random.default_rng(seed)
    s = gll_nodes(p)
    vid, pos, nid = _grid_vertices(n, 2, L, periodic, perturb, rng)
    next_id = [nid]
    mids = {}

    def mid_id(a, b):
        key = (min(a, b), max(a, b))
        if key not in mids:
            mids[key] = next_id[0]
            next_id[0] += 1
        return mids[key]

    def fresh():
        next_id[0] += 1
        return next_id[0] - 1

    quads = []  # (ids [4] in local corner order, positions [4, 2])
    for j in range(n):
        for i in range(n):
            g = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            if rng.integers(2):
                tris = [(g[0], g[1], g[2]), (g[0], g[2], g[3])]
            else:
                tris = [(g[0], g[1], g[3]), (g[1], g[2], g[3])]
            for tri in tris:  # counter-clockwise
                ids = [vid(v) for v in tri]
                P = [pos(v) for v in tri]
                cid = fresh()
                cen = (P[0] + P[1] + P[2]) / 3.0
                for k in range(3):
                    a, b, c = k, (k + 1) % 3, (k + 2) % 3
                    mab, mca = mid_id(ids[a], ids[b]), mid_id(ids[c], ids[a])
                    # local corners (0,0) (1,0) (0,1) (1,1): A, m_AB, m_CA, centroid
                    quads.append(([ids[a], mab, mca, cid],
                                  np.array([P[a], 0.5 * (P[a] + P[b]), 0.5 * (P[c] + P[a]), cen])))
    for _ in range(refine):
        mids = {}
        finer = []
        for ids, P in quads:
            c0, c1, c2, c3 = ids
            m01, m02, m13, m23 = mid_id(c0, c1), mid_id(c0, c2), mid_id(c1, c3), mid_id(c2, c3)
            cc = fresh()
            Q = {"c0": P[0], "c1": P[1], "c2": P[2], "c3": P[3],
                 "m01": 0.5 * (P[0] + P[1]), "m02": 0.5 * (P[0] + P[2]),
                 "m13": 0.5 * (P[1] + P[3]), "m23": 0.5 * (P[2] + P[3]), "cc": 0.25 * P.sum(axis=0)}
            I = {"c0": c0, "c1": c1, "c2": c2, "c3": c3, "m01": m01, "m02": m02, "m13": m13, "m23": m23,
                 "cc": cc}
            for kids in (("c0", "m01", "m02", "cc"), ("m01", "c1", "cc", "m13"),
                         ("m02", "cc", "c2", "m23"), ("cc", "m13", "m23", "c3")):
                finer.append(([I[k] for k in kids], np.array([Q[k] for k in kids])))
        quads = finer
    return _finish_mesh(2, p, s, quads, (0.0, 0.0), (L, L), periodic)


def unstructured_hex_mesh(n=3, p=2, L=1.0, periodic=False, perturb=0.0, seed=MESH_SEED):
    """Unstructured trilinear hexahedra on [0,L]^3: every cell of an n^3
    vertex grid is split into the six tetrahedra of the Kuhn (Freudenthal)
    triangulation, which is conforming across cells, and every tetrahedron
    into four hexahedra, one per tetrahedron vertex, with corners at the
    vertex, its three edge midpoints, its three face centroids and the
    tetrahedron's centroid (non-grid topology: edges shared by 3-8
    hexahedra). 24 n^3 elements. Periodic meshes need n >= 3."""
    rng = np.random.default_rng(seed)
    s = gll_nodes(p)
    vid, pos, nid = _grid_vertices(n, 3, L, periodic, perturb, rng)
    next_id = [nid]
    keyed = {}

    def kid(key):
        if key not in keyed:
            keyed[key] = next_id[0]
            next_id[0] += 1
        return keyed[key]

    hexes = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for perm in itertools.permutations(range(3)):
                    g = [np.array([i, j, k])]
                    for ax in perm:
                        step = np.zeros(3, dtype=int)
                        step[ax] = 1
                        g.append(g[-1] + step)
                    ids = [vid(v) for v in g]
                    P = [pos(v) for v in g]
                    tid = kid(("tet", i, j, k, perm))
                    cen = sum(P) / 4.0
                    for a in range(4):
                        o = [b for b in range(4) if b != a]
                        b1, b2, b3 = o
                        if np.linalg.det(np.array([P[b1] - P[a], P[b2] - P[a], P[b3] - P[a]])) < 0:
                            b2, b3 = b3, b2

                        def em(b):
                            return kid(("e",) + tuple(sorted((ids[a], ids[b]))))

                        def fm(b, c):
                            return kid(("f",) + tuple(sorted((ids[a], ids[b], ids[c]))))
                        # local corners by bits (x, y, z): x -> b1, y -> b2, z -> b3
                        cid = [ids[a], em(b1), em(b2), fm(b1, b2), em(b3), fm(b1, b3), fm(b2, b3), tid]
                        cp = [P[a], 0.5 * (P[a] + P[b1]), 0.5 * (P[a] + P[b2]), (P[a] + P[b1] + P[b2]) / 3.0,
                              0.5 * (P[a] + P[b3]), (P[a] + P[b1] + P[b3]) / 3.0, (P[a] + P[b2] + P[b3]) / 3.0, cen]
                        hexes.append((cid, np.array(cp)))
    return _finish_mesh(3, p, s, hexes, (0.0, 0.0, 0.0), (L, L, L), periodic)


# ---------------------------------------------------------------------------
# workload meshes (sizes and perturbations of the benchmark workloads)
# ---------------------------------------------------------------------------
def poisson_square_mesh(n=8, p=3, perturb=0.15, seed=MESH_SEED):
    """Unit square, n x n straight-sided quads, interior vertices perturbed by
    U(-perturb h, +perturb h); all sides Dirichlet (tag 0)."""
    return structured_mesh((n, n), p, (0.0, 0.0), (1.0, 1.0), (False, False),
                           perturb=perturb, seed=seed)


def vortex_mesh(n=64, p=4, L=10.0, perturb=0.1, seed=MESH_SEED):
    """Periodic [0,L]^2, n x n quads, all vertices perturbed by U(-0.1h,0.1h)."""
    return structured_mesh((n, n), p, (0.0, 0.0), (L, L), (True, True),
                           perturb=perturb, seed=seed)


def tgv_node_map(amp=0.05):
    def f(x):
        y = np.empty_like(x)
        y[..., 0] = x[..., 0] + amp * np.sin(x[..., 1]) * np.sin(x[..., 2])
        y[..., 1] = x[..., 1] + amp * np.sin(x[..., 2]) * np.sin(x[..., 0])
        y[..., 2] = x[..., 2] + amp * np.sin(x[..., 0]) * np.sin(x[..., 1])
        return y
    return f


def tgv_mesh(n=32, p=3, amp=0.05):
    """Periodic [0,2pi]^3, n^3 hexes, nodes curved by the cyclic map
    x + amp sin(y) sin(z)."""
    L = 2.0 * math.pi
    return structured_mesh((n, n, n), p, (0.0, 0.0, 0.0), (L, L, L), (True, True, True),
                           node_map=tgv_node_map(amp))


def channel_wall_coords(ny=32, ratio=1.1):
    """Vertex y-coordinates on [-1,1], geometric growth `ratio` from each wall."""
    half = ny // 2
    dy = np.array([ratio ** k for k in range(half)])
    dy /= dy.sum()
    y = np.concatenate([[-1.0], -1.0 + np.cumsum(dy)])
    y[-1] = 0.0
    return np.concatenate([y, -y[-2::-1]])


def channel_mesh(nx=64, ny=32, nz=32, p=4, amp=0.1, wavelength=1.0, ratio=1.1):
    """[0,4] x [-1,1] x [0,2] channel, periodic in x and z, walls (tag 1) at
    y = +-1 + amp sin(2 pi x / wavelength) blended linearly to the centre line,
    wall-normal geometric stretching `ratio` from each wall."""
    yc = channel_wall_coords(ny, ratio)

    def bump(x):
        y = x.copy()
        y[..., 1] = x[..., 1] + amp * np.sin(2 * math.pi * x[..., 0] / wavelength) * np.abs(x[..., 1])
        return y
    return structured_mesh((nx, ny, nz), p, (0.0, -1.0, 0.0), (4.0, 1.0, 2.0), (True, False, True),
                           node_map=bump, ycoords=yc, btag_of_face=lambda d, end: 1)


# ---------------------------------------------------------------------------
# states (conserved variables, layout [E, n_c, (p+1)^D])
# ---------------------------------------------------------------------------
def _to_conserved(rho, vel, p, gamma):
    E_ = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [E_], axis=1)


def vortex_state(mesh, gamma=1.4, mach=0.5, eps=5.0, rc=1.0, x0=5.0, y0=5.0,
                 theta=math.atan(0.5), t=0.0):
    """Isentropic vortex of the Euler test (vortex strength eps, size rc),
    free stream rho=1, |u|=1, p = 1/(gamma M^2)."""
    x = mesh["nodes"][..., 0]
    y = mesh["nodes"][..., 1]
    uinf = 1.0
    ub, vb = uinf * math.cos(theta), uinf * math.sin(theta)
    pinf = 1.0 / (gamma * mach ** 2)
    dx, dy = (x - x0) - ub * t, (y - y0) - vb * t
    f = (1.0 - dx ** 2 - dy ** 2) / rc ** 2
    u = uinf * (math.cos(theta) - eps * dy / (2 * math.pi * rc) * np.exp(f / 2))
    v = uinf * (math.sin(theta) + eps * dx / (2 * math.pi * rc) * np.exp(f / 2))
    base = 1.0 - eps ** 2 * (gamma - 1.0) * mach ** 2 / (8 * math.pi ** 2) * np.exp(f)
    rho = base ** (1.0 / (gamma - 1.0))
    p = pinf * base ** (gamma / (gamma - 1.0))
    return _to_conserved(rho, [u, v], p, gamma)


def tgv_state(mesh, gamma=1.4, mach=0.1, V0=1.0, rho0=1.0):
    """Single-mode Taylor-Green vortex (L=1), isothermal density."""
    x, y, z = (mesh["nodes"][..., d] for d in range(3))
    p0 = rho0 * V0 ** 2 / (gamma * mach ** 2)
    u = V0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -V0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = p0 + rho0 * V0 ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = rho0 * p / p0
    return _to_conserved(rho, [u, v, w], p, gamma)


def channel_state(mesh, gamma=1.4, mach=0.3, amp=0.01, seed=STATE_SEED):
    """Laminar parabolic profile (centre-line speed 1) plus a seeded 1%
    smooth perturbation; rho = 1, p = 1/(gamma M^2)."""
    x, y, z = (mesh["nodes"][..., d] for d in range(3))
    rng = np.random.default_rng(seed)
    u = np.clip(1.0 - y ** 2, 0.0, None)
    pert = np.zeros_like(u)
    for _ in range(4):
        kx, kz = rng.integers(1, 3, size=2)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        pert += np.sin(2 * math.pi * kx * x / 4.0 + ph[0]) * np.sin(math.pi * kz * z + ph[1])
    u = u * (1.0 + amp * pert)
    v = amp * pert * np.clip(1.0 - y ** 2, 0.0, None)
    w = np.zeros_like(u)
    rho = np.ones_like(u)
    p = np.full_like(u, 1.0 / (gamma * mach ** 2))
    return _to_conserved(rho, [u, v, w], p, gamma)


def poisson_mapped_square_mesh(n=8, p=3, amp=0.08):
    """Unit square, n x n quads whose nodes are moved by the smooth map
    (x + amp sin(pi x) sin(2 pi y), y + amp sin(2 pi x) sin(pi y)): curved
    isoparametric elements that stay nested under refinement (every n
    samples the same map, unlike a per-level random perturbation); the map
    keeps each side of the square on itself. All sides Dirichlet (tag 0)."""
    m = structured_mesh((n, n), p, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=0.0)
    X, Y = m["nodes"][..., 0].copy(), m["nodes"][..., 1].copy()
    m["nodes"][..., 0] = X + amp * np.sin(math.pi * X) * np.sin(2.0 * math.pi * Y)
    m["nodes"][..., 1] = Y + amp * np.sin(2.0 * math.pi * X) * np.sin(math.pi * Y)
    return m


def poisson_paper_solution(mesh, alpha=0.1, beta=0.3, a=5.1, b=-6.2, c=4.3, d=3.4):
    """The manufactured solution of the paper's Poisson study (Sec. 5.1, its
    printed constants): u = exp(alpha sin(a x + b y) + beta cos(c x + d y)),
    with its gradient and f = -lap u at the nodes. Returns (u [E, 1, npe],
    grad u [E, 1, 2, npe], f [E, 1, npe]); u is also the Dirichlet data."""
    x, y = mesh["nodes"][..., 0], mesh["nodes"][..., 1]
    s1, c1 = np.sin(a * x + b * y), np.cos(a * x + b * y)
    s2, c2 = np.sin(c * x + d * y), np.cos(c * x + d * y)
    u = np.exp(alpha * s1 + beta * c2)
    px = alpha * a * c1 - beta * c * s2
    py = alpha * b * c1 - beta * d * s2
    lap_phi = -alpha * (a * a + b * b) * s1 - beta * (c * c + d * d) * c2
    f = -u * (px * px + py * py + lap_phi)
    return u[:, None], np.stack([u * px, u * py], axis=1)[:, None], f[:, None]


def poisson_exact(mesh):
    """Manufactured u = sin(pi x) sin(pi y), [E, 1, (p+1)^2]."""
    x, y = mesh["nodes"][..., 0], mesh["nodes"][..., 1]
    return (np.sin(math.pi * x) * np.sin(math.pi * y))[:, None, :]


def poisson_source(mesh):
    """f = -lap u = 2 pi^2 sin(pi x) sin(pi y)."""
    return 2.0 * math.pi ** 2 * poisson_exact(mesh)


def poisson_exact_grad(mesh):
    x, y = mesh["nodes"][..., 0], mesh["nodes"][..., 1]
    gx = math.pi * np.cos(math.pi * x) * np.sin(math.pi * y)
    gy = math.pi * np.sin(math.pi * x) * np.cos(math.pi * y)
    return np.stack([gx, gy], axis=1)[:, None, :, :]  # [E, 1, D, nodes]


def smooth_perturbation(mesh, state, amp=0.05, seed=STATE_SEED, nmodes=3, periods=None):
    """state + amp * max|state_c| * (mean of seeded smooth modes), one mode set
    per component c. periods: per-dimension domain lengths for
    periodic-compatible wavenumbers (default: the mesh box)."""
    rng = np.random.default_rng(seed)
    D = mesh["D"]
    X = mesh["nodes"]
    if periods is None:
        periods = [mesh["hi"][d] - mesh["lo"][d] for d in range(D)]
    out = state.copy()
    for c in range(state.shape[1]):
        m = np.zeros(X.shape[:2])
        for _ in range(nmodes):
            k = rng.integers(1, 3, size=D)
            ph = rng.uniform(0, 2 * math.pi, size=D)
            term = np.ones(X.shape[:2])
            for d in range(D):
                term = term * np.sin(2 * math.pi * k[d] * X[..., d] / periods[d] + ph[d])
            m += term
        scale = max(float(np.abs(state[:, c]).max()), 1e-3)
        out[:, c] = state[:, c] + amp * scale * m / nmodes
    return out


def random_state(shape, seed=STATE_SEED, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)
