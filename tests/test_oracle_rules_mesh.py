"""Pins for the oracle's 1-D rules, connectivity, switches and metrics
(CPU only)."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle.mesh import Connectivity, Metrics, line_nodes, pattern_counts, switches
from oracle.rules import Rules, gauss_legendre_01, lagrange, n_gauss

GOLD = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


@pytest.mark.parametrize("nq", range(2, 15))
def test_gauss_matches_numpy(nq):
    x, w = gauss_legendre_01(nq)
    xr, wr = np.polynomial.legendre.leggauss(nq)
    assert np.allclose(x, (xr + 1) / 2, atol=2e-16, rtol=0)
    assert np.allclose(w, wr / 2, atol=5e-16, rtol=0)


def test_gauss_point_count():
    # Sec. 2.2: precision 3p -> ceil((3p+1)/2) points
    assert [n_gauss(p) for p in range(1, 9)] == [math.ceil((3 * p + 1) / 2) for p in range(1, 9)]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_lagrange_and_mass(p):
    s = I.gll_nodes(p)
    phi, dphi = lagrange(s, s)
    assert np.allclose(phi, np.eye(p + 1), atol=1e-14)
    xs = np.linspace(0, 1, 17)
    phi, dphi = lagrange(s, xs)
    assert np.allclose(phi.sum(1), 1.0, atol=1e-13)
    assert np.allclose(dphi.sum(1), 0.0, atol=1e-11)
    assert np.allclose(dphi @ s, 1.0, atol=1e-11)
    r = Rules(p, s)
    # mass matrix against an independent higher-order rule
    xr, wr = np.polynomial.legendre.leggauss(3 * p + 3)
    ph, _ = lagrange(s, (xr + 1) / 2)
    Mref = ph.T @ (wr[:, None] / 2 * ph)
    assert np.allclose(r.M, Mref, atol=1e-15)
    assert abs(r.M.sum() - 1.0) < 1e-14
    assert np.allclose(r.M @ np.ones(p + 1), r.wnod, atol=1e-15)
    b = np.random.default_rng(p).standard_normal((3, p + 1))
    assert np.allclose(r.mass_solve(b) @ r.M.T, b, atol=1e-12)
    # int r = F+ + F- for the v = 1 test function: 1^T M M^-1 e = 1
    L1 = r.mass_solve(np.eye(p + 1)[p])
    L0 = r.mass_solve(np.eye(p + 1)[0])
    assert abs(r.wnod @ L1 - 1) < 1e-12 and abs(r.wnod @ L0 - 1) < 1e-12
    # 1-D free-stream identity: M^-1 dPhi^T W 1 = L1 - L0
    Kd1 = r.mass_solve((r.dPhi * r.wq[:, None]).T @ np.ones(r.nq))
    assert np.allclose(Kd1, L1 - L0, atol=1e-10)


def _costtab():
    rows = np.loadtxt(f"{GOLD}/costtab.txt", comments="#")
    return {int(r[0]): (int(r[1]), int(r[4])) for r in rows}


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_costtab_2d(p):
    # Table 1: every node of a first-order Line-DG operator couples to 2p+5 nodes
    m = I.vortex_mesh(3, p, perturb=0.1)
    cnt = pattern_counts(m, Connectivity(m))
    assert np.all(cnt == _costtab()[p][0])
    m2, _ = I.reorient(m)
    assert np.all(pattern_counts(m2, Connectivity(m2)) == _costtab()[p][0])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_costtab_3d(p):
    m = I.structured_mesh((3, 3, 3), p, (0, 0, 0), (1, 1, 1), (True,) * 3, perturb=0.1)
    m2, _ = I.reorient(m)
    assert np.all(pattern_counts(m2, Connectivity(m2)) == _costtab()[p][1])


def test_costtab_closed_forms():
    # the printed table follows (Dp+1)+2D, (Dp+1)+2D(p+1), (p+1)^D+2D(p+1)^(D-1)
    rows = np.loadtxt(f"{GOLD}/costtab.txt", comments="#").astype(int)
    for p, l2, s2, n2, l3, s3, n3 in rows:
        assert l2 == 2 * p + 1 + 4 and l3 == 3 * p + 1 + 6
        assert s2 == 2 * p + 1 + 4 * (p + 1) and s3 == 3 * p + 1 + 6 * (p + 1)
        # nodal DG: (p+1)^D + 2D (p+1)^(2(D-1)) / (p+1)^D face couplings per node
        assert n2 == (p + 1) ** 2 + 4 and n3 == (p + 1) ** 3 + 6 * (p + 1)


@pytest.mark.parametrize("D,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_neighbour_nodes_coincide(D, periodic):
    p = 2
    n = (3,) * D
    m = I.structured_mesh(n, p, (0,) * D, (1,) * D, (periodic,) * D, perturb=0.1)
    m, _ = I.reorient(m)
    c = Connectivity(m)
    X = m["nodes"]
    npe = (p + 1) ** D
    for e in range(X.shape[0]):
        for d in range(D):
            for l in range((p + 1) ** (D - 1)):
                ln = line_nodes(D, p, d, l)
                for end in range(2):
                    g = c.nbr[e, d, l, end]
                    if g < 0:
                        continue
                    eo, ao = divmod(int(g), npe)
                    diff = X[eo, ao] - X[e, ln[end * p]]
                    if periodic:
                        diff = diff - np.round(diff)   # unit box periods
                    assert np.abs(diff).max() < 1e-13
                    # the outside node's own line through this face points back
                    fo = c.nbr_face[e, 2 * d + end]
                    back = c.face_map[(eo, fo)][ao]
                    assert back == ln[end * p]


@pytest.mark.parametrize("D", [2, 3])
def test_switch_function(D):
    m = I.structured_mesh((3,) * D, 2, (0,) * D, (1,) * D, (True,) * D, perturb=0.1)
    c = Connectivity(m)
    S = switches(m, c)
    assert np.all(S[:, :, 1] == 1) and np.all(S[:, :, 0] == -1)   # aligned mesh
    m2, _ = I.reorient(m)
    c2 = Connectivity(m2)
    S2 = switches(m2, c2)
    assert np.all(S2[:, :, 0] == -S2[:, :, 1])
    for e in range(S2.shape[0]):
        for f in range(2 * D):
            eo, fo = c2.nbr_elem[e, f], c2.nbr_face[e, f]
            if eo >= 0:
                assert S2[e, f // 2, f % 2] == -S2[eo, fo // 2, fo % 2]
    assert np.any(S2[:, :, 1] == -1)   # re-orientation does flip some


@pytest.mark.parametrize("D", [2, 3])
def test_metrics_affine(D):
    rng = np.random.default_rng(3)
    A = np.eye(D) + 0.2 * rng.standard_normal((D, D))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    p = 3
    m = I.structured_mesh((2,) * D, p, (0,) * D, (1,) * D, (False,) * D,
                          node_map=lambda x: x @ A.T)
    r = Rules(p, m["s"])
    met = Metrics(m, r)
    h = 0.5
    G = A * h                                     # dx/dX for a reference cell of size h
    J = np.linalg.det(G)
    cof = J * np.linalg.inv(G).T
    assert np.allclose(met.J, J, rtol=1e-13)
    for d in range(D):
        assert np.allclose(met.ng[d], cof[:, d], rtol=1e-12, atol=1e-14)
        assert np.allclose(met.nplus[d], cof[:, d], rtol=1e-12, atol=1e-14)
        assert np.allclose(met.nminus[d], -cof[:, d], rtol=1e-12, atol=1e-14)
    if D == 3:
        # n_1 = dx/dX2 x dx/dX3 (Sec. 2.1)
        assert np.allclose(cof[:, 0], np.cross(G[:, 1], G[:, 2]))
