"""Mesh topology, switch function and metric terms (oracle; test infrastructure).

Follows:
  * Sec. 2.1: the (p+1)^D node grid x_ijk per element, the coordinate lines
    through it, and the outside traces u^+(1), u^-(0) "given by nodes in the
    neighbouring elements"; Eq. 2 (J = det G, G = grad_X x) and Eqs. 4-6
    (contravariant normals n_d^+ = J G^{-T} N_d^+, n_d^- = J G^{-T} N_d^-).
  * Sec. 2.2: isoparametric map (Eq. 11), metric at the Gauss points of each
    line, n^+- precomputed at the line ends, J at the nodes.
  * Sec. 3: switch function S^+-_d per element, direction and end, with
    S^+ = -S^-, opposite signs on the two sides of a shared face, propagated
    along globally connected lines from an arbitrary start (here: the
    lowest unassigned element and direction, S^+ = +1).

Conventions (shared with the library's documented layout, not its code):
  local node a = i + (p+1) j + (p+1)^2 k; face f = 2 d + end; line l of
  direction d enumerates the other indices, lowest dimension fastest; global
  node id = e (p+1)^D + a; a boundary line end carries -1 - tag.
"""
from __future__ import annotations

import itertools

import numpy as np


class MeshError(ValueError):
    pass


def multi_index(a, D, p):
    return [(a // (p + 1) ** b) % (p + 1) for b in range(D)]


def flat_index(idx, p):
    return sum(int(v) * (p + 1) ** b for b, v in enumerate(idx))


def line_nodes(D, p, d, l):
    """Local node indices of line l in direction d, ordered along xi."""
    others = [b for b in range(D) if b != d]
    rest = [(l // (p + 1) ** r) % (p + 1) for r in range(len(others))]
    out = []
    for t in range(p + 1):
        idx = [0] * D
        idx[d] = t
        for b, v in zip(others, rest):
            idx[b] = v
        out.append(flat_index(idx, p))
    return out


def to_lines(A, D, p, d):
    """[..., (p+1)^D] nodal array -> [..., nl, p+1] lines of direction d."""
    lead = A.shape[:-1]
    Ar = A.reshape(lead + (p + 1,) * D)          # axes [..., dim D-1, ..., dim 0]
    Ar = np.moveaxis(Ar, len(lead) + (D - 1 - d), -1)
    return Ar.reshape(lead + ((p + 1) ** (D - 1), p + 1))


def from_lines(L, D, p, d):
    """Inverse of to_lines."""
    lead = L.shape[:-2]
    shp = lead + (p + 1,) * (D - 1) + (p + 1,)
    Ar = L.reshape(shp)
    Ar = np.moveaxis(Ar, -1, len(lead) + (D - 1 - d))
    return Ar.reshape(lead + ((p + 1) ** D,))


# ---------------------------------------------------------------------------
# connectivity
# ---------------------------------------------------------------------------
def face_corners(D, f):
    d, end = divmod(f, 2)
    return [c for c in range(1 << D) if ((c >> d) & 1) == end]


def face_local_nodes(D, p, f):
    d, end = divmod(f, 2)
    return [a for a in range((p + 1) ** D) if multi_index(a, D, p)[d] == end * p]


def _node_signature(mesh, e, f, a):
    """Multilinear weights of face node a on the face's corner vertices,
    keyed by global vertex id: identifies the physical point independently
    of each element's local orientation."""
    D, p, s = mesh["D"], mesh["p"], mesh["s"]
    d, end = divmod(f, 2)
    idx = multi_index(a, D, p)
    sig = {}
    for c in face_corners(D, f):
        w = 1.0
        for b in range(D):
            if b == d:
                continue
            w *= s[idx[b]] if (c >> b) & 1 else (1.0 - s[idx[b]])
        sig[int(mesh["vertices"][e, c])] = w
    return sig


class Connectivity:
    """nbr_elem[e, f], nbr_face[e, f] (-1 on boundaries) and
    nbr[e, d, l, end] = global id of the outside node of each line end or
    -1 - tag on boundary faces."""

    def __init__(self, mesh):
        D, p = mesh["D"], mesh["p"]
        E = mesh["nodes"].shape[0]
        npe = (p + 1) ** D
        nl = (p + 1) ** (D - 1)
        verts = mesh["vertices"]
        btag = mesh["btag"]
        faces = {}
        for e in range(E):
            for f in range(2 * D):
                key = tuple(sorted(int(verts[e, c]) for c in face_corners(D, f)))
                if len(set(key)) != len(key):
                    raise MeshError("degenerate face")
                faces.setdefault(key, []).append((e, f))
        self.nbr_elem = -np.ones((E, 2 * D), dtype=np.int64)
        self.nbr_face = -np.ones((E, 2 * D), dtype=np.int64)
        for key, lst in faces.items():
            if len(lst) > 2:
                raise MeshError("face shared by more than two elements")
            if len(lst) == 2:
                (e0, f0), (e1, f1) = lst
                self.nbr_elem[e0, f0], self.nbr_face[e0, f0] = e1, f1
                self.nbr_elem[e1, f1], self.nbr_face[e1, f1] = e0, f0
        for e in range(E):
            for f in range(2 * D):
                matched = self.nbr_elem[e, f] >= 0
                if matched and btag[e, f] >= 0:
                    raise MeshError("boundary-tagged face has a neighbour")
                if not matched and btag[e, f] < 0:
                    raise MeshError("unmatched interior face")
        # outside node of each face node, by matching vertex-weight signatures
        self.face_map = {}
        for e in range(E):
            for f in range(2 * D):
                en, fn = self.nbr_elem[e, f], self.nbr_face[e, f]
                if en < 0:
                    continue
                mine = face_local_nodes(D, p, f)
                theirs = face_local_nodes(D, p, fn)
                sig_t = [_node_signature(mesh, en, fn, b) for b in theirs]
                m = {}
                for a in mine:
                    sa = _node_signature(mesh, e, f, a)
                    best, bestd = None, np.inf
                    for b, sb in zip(theirs, sig_t):
                        if set(sb) != set(sa):
                            raise MeshError("face vertex sets differ")
                        dist = max(abs(sa[v] - sb[v]) for v in sa)
                        if dist < bestd:
                            best, bestd = b, dist
                    if bestd > 1e-12:
                        raise MeshError("face nodes do not coincide (node set not symmetric?)")
                    m[a] = best
                self.face_map[(e, f)] = m
        self.nbr = np.zeros((E, D, nl, 2), dtype=np.int64)
        for e in range(E):
            for d in range(D):
                for l in range(nl):
                    ln = line_nodes(D, p, d, l)
                    for end in range(2):
                        f = 2 * d + end
                        a = ln[end * p]
                        if self.nbr_elem[e, f] < 0:
                            self.nbr[e, d, l, end] = -1 - int(btag[e, f])
                        else:
                            self.nbr[e, d, l, end] = self.nbr_elem[e, f] * npe + self.face_map[(e, f)][a]


def switches(mesh, conn):
    """S[e, d, end] in {-1, +1}: scan elements in id order and directions in
    order; the first unassigned (e, d) gets S^+ = +1 at its xi=1 end; the
    sign pattern is then carried along the global line of elements in both
    directions with S^- = -S^+ inside an element and opposite signs on the
    two sides of every shared face."""
    D = mesh["D"]
    E = mesh["nodes"].shape[0]
    S = np.zeros((E, D, 2), dtype=np.int8)
    done = np.zeros((E, D), dtype=bool)
    for e in range(E):
        for d in range(D):
            if done[e, d]:
                continue
            S[e, d, 1], S[e, d, 0] = 1, -1
            done[e, d] = True
            for start_end in (1, 0):
                ce, cd, cend = e, d, start_end
                while True:
                    f = 2 * cd + cend
                    ne = conn.nbr_elem[ce, f]
                    if ne < 0:
                        break
                    nd, nend = divmod(int(conn.nbr_face[ce, f]), 2)
                    want = -S[ce, cd, cend]
                    if done[ne, nd]:
                        if S[ne, nd, nend] != want:
                            raise MeshError("inconsistent switch along a closed line")
                        break
                    S[ne, nd, nend] = want
                    S[ne, nd, 1 - nend] = -want
                    done[ne, nd] = True
                    ce, cd, cend = ne, nd, 1 - nend
    return S


# ---------------------------------------------------------------------------
# metric terms
# ---------------------------------------------------------------------------
def _cofactor(G):
    """det G and J G^{-T} (the cofactor matrix) for G[..., a, b] = dx_a/dX_b,
    written out for 2x2 and 3x3 (works in any float precision)."""
    D = G.shape[-1]
    C = np.zeros_like(G)
    if D == 2:
        C[..., 0, 0] = G[..., 1, 1]
        C[..., 0, 1] = -G[..., 1, 0]
        C[..., 1, 0] = -G[..., 0, 1]
        C[..., 1, 1] = G[..., 0, 0]
        J = G[..., 0, 0] * G[..., 1, 1] - G[..., 0, 1] * G[..., 1, 0]
    else:
        for a in range(3):
            for b in range(3):
                a1, a2 = [r for r in range(3) if r != a]
                b1, b2 = [c for c in range(3) if c != b]
                minor = G[..., a1, b1] * G[..., a2, b2] - G[..., a1, b2] * G[..., a2, b1]
                C[..., a, b] = minor if (a + b) % 2 == 0 else -minor
        J = sum(G[..., 0, b] * C[..., 0, b] for b in range(3))
    return J, C


class Metrics:
    """J at nodes [E, npe]; contravariant normals at the Gauss points of each
    line ng[d] : [E, nl, nq, D]; n^+ at xi=1 and n^- at xi=0 of each line
    nplus[d], nminus[d] : [E, nl, D]."""

    def __init__(self, mesh, rules):
        # The metric terms are formed in extended precision and rounded to
        # float64 once: the residual subtracts flux values of size |F| |n|
        # from each other, so independent float64 roundings of n (node
        # coordinates of size L, spacings h) would show up in R amplified by
        # about (L / h) |F| / |R|.
        D, p = mesh["D"], mesh["p"]
        X = mesh["nodes"].astype(np.longdouble)    # [E, npe, D]
        E = X.shape[0]
        # G at the nodes: dx_a/dX_b by the nodal derivative matrix along b
        Gn = np.zeros((E, (p + 1) ** D, D, D), dtype=np.longdouble)
        for b in range(D):
            for a in range(D):
                xl = to_lines(X[..., a], D, p, b)    # [E, nl, p+1]
                dl = np.einsum("ij,elj->eli", rules.Dn_x, xl)
                Gn[:, :, a, b] = from_lines(dl, D, p, b)
        J, cof_n = _cofactor(Gn)
        if np.any(J <= 0):
            raise MeshError("non-positive mapping Jacobian at a node")
        self.J = J.astype(np.float64)
        self.ng, self.nplus, self.nminus = [], [], []
        for d in range(D):
            # G at (xi_q along d, nodes in the other directions)
            Gq = np.zeros((E, (p + 1) ** (D - 1), rules.nq, D, D), dtype=np.longdouble)
            for a in range(D):
                xl = to_lines(X[..., a], D, p, d)
                Gq[..., a, d] = np.einsum("qj,elj->elq", rules.dPhi_x, xl)
                for b in range(D):
                    if b == d:
                        continue
                    gl = to_lines(Gn[:, :, a, b], D, p, d)
                    Gq[..., a, b] = np.einsum("qj,elj->elq", rules.Phi_x, gl)
            _, cof_q = _cofactor(Gq)
            self.ng.append(cof_q[..., :, d].astype(np.float64))     # [E, nl, nq, D]
            cl = np.stack([to_lines(cof_n[:, :, a, d], D, p, d) for a in range(D)], axis=-1)
            self.nplus.append(cl[:, :, p, :].astype(np.float64))     # N_d^+ at xi = 1
            self.nminus.append((-cl[:, :, 0, :]).astype(np.float64))  # N_d^- at xi = 0


def pattern_counts(mesh, conn):
    """Distinct scalar-node columns coupled to each node by a first-order
    Line-DG operator: the nodes of its D lines plus the outside node at each
    line end it lies on (Sec. 2.3). Returns [E, npe] counts."""
    D, p = mesh["D"], mesh["p"]
    E = mesh["nodes"].shape[0]
    npe = (p + 1) ** D
    nl = (p + 1) ** (D - 1)
    cols = [[set() for _ in range(npe)] for _ in range(E)]
    for e in range(E):
        for d in range(D):
            for l in range(nl):
                ln = line_nodes(D, p, d, l)
                ext = [e * npe + a for a in ln]
                for end in range(2):
                    g = conn.nbr[e, d, l, end]
                    if g >= 0:
                        ext.append(int(g))
                for a in ln:
                    cols[e][a].update(ext)
    return np.array([[len(c) for c in row] for row in cols])
