"""Pins for the oracle on unstructured meshes (CPU only).

The paper's Poisson study (Sec. 5.1) runs on an unstructured quadrilateral
mesh refined uniformly, and the method is stated for unstructured hexahedral
meshes (Sec. 2.1, the switch construction of Sec. 3). The synthetic
unstructured meshes here have non-grid topology: quadrilaterals from split
triangles (vertices of valence 3 to 8) and hexahedra from split Kuhn
tetrahedra (edges shared by 3 to 8 elements). Each pin rests on a closed
form, an invariant of the scheme or a printed table, never on the oracle's
own output."""
import math
import os

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle.mesh import Connectivity, line_nodes, pattern_counts, switches
from oracle.residual import (Discretization, conservation_weights, full_residual, gradient,
                             residual)

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}
POISSON = {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}}


def _free_stream(E, npe, D):
    rho, v, p = 1.1, [0.8, -0.3, 0.25][:D], 2.5
    U = np.zeros((E, D + 2, npe))
    U[:, 0] = rho
    for a in range(D):
        U[:, 1 + a] = rho * v[a]
    U[:, D + 1] = p / 0.4 + 0.5 * rho * sum(x * x for x in v)
    return U


def test_meshes_are_unstructured_and_conforming():
    # 2-D: some vertex of valence 3 (triangle centroids) and some of valence
    # other than 4; every interior face matched exactly once
    m = I.unstructured_quad_mesh(3, 2, L=1.0, periodic=True)
    val = np.bincount(m["vertices"].ravel())
    assert 3 in set(val) and max(val) > 4
    c = Connectivity(m)
    assert np.all(c.nbr_elem >= 0)
    m3 = I.unstructured_hex_mesh(3, 1, periodic=True)
    # hexahedra sharing each edge: a structured mesh has 4 everywhere
    cnt = {}
    for e in range(m3["vertices"].shape[0]):
        v = m3["vertices"][e]
        for a, b in ((0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7),
                     (0, 4), (1, 5), (2, 6), (3, 7)):
            k = (min(v[a], v[b]), max(v[a], v[b]))
            cnt[k] = cnt.get(k, 0) + 1
    assert {3, 4}.issubset(set(cnt.values())) and max(cnt.values()) > 4
    assert np.all(Connectivity(m3).nbr_elem >= 0)


@pytest.mark.parametrize("D,p", [(2, 1), (2, 3), (2, 5), (3, 1), (3, 2)])
def test_costtab_on_unstructured_meshes(D, p):
    # Table 1: 2p+5 (2-D) and 3p+7 (3-D) couplings per node on any conforming mesh
    rows = np.loadtxt(f"{GOLD}/costtab.txt", comments="#").astype(int)
    gold = {int(r[0]): (int(r[1]), int(r[4])) for r in rows}
    m = (I.unstructured_quad_mesh(3, p, periodic=True, perturb=0.1) if D == 2
         else I.unstructured_hex_mesh(3, p, periodic=True, perturb=0.05))
    assert np.all(pattern_counts(m, Connectivity(m)) == gold[p][D - 2])


@pytest.mark.parametrize("D", [2, 3])
def test_neighbour_nodes_coincide_on_unstructured(D):
    m = (I.unstructured_quad_mesh(2, 3, perturb=0.15) if D == 2
         else I.unstructured_hex_mesh(1, 2))
    p = m["p"]
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
                        assert m["btag"][e, 2 * d + end] == 0
                        continue
                    eo, ao = divmod(int(g), npe)
                    assert np.abs(X[eo, ao] - X[e, ln[end * p]]).max() < 1e-13


@pytest.mark.parametrize("D", [2, 3])
def test_switch_function_on_unstructured(D):
    # Sec. 3: S+ = -S- per element and direction, opposite signs on the two
    # sides of every shared face; the lines of elements close on themselves
    m = (I.unstructured_quad_mesh(3, 2, periodic=True) if D == 2
         else I.unstructured_hex_mesh(3, 1, periodic=True))
    c = Connectivity(m)
    S = switches(m, c)
    assert np.all(S[:, :, 0] == -S[:, :, 1])
    for e in range(S.shape[0]):
        for f in range(2 * D):
            eo, fo = c.nbr_elem[e, f], c.nbr_face[e, f]
            assert S[e, f // 2, f % 2] == -S[eo, fo // 2, fo % 2]


@pytest.mark.parametrize("D,p", [(2, 2), (2, 4), (3, 2)])
def test_free_stream_on_unstructured(D, p):
    m = (I.unstructured_quad_mesh(3, p, L=10.0, periodic=True, perturb=0.15) if D == 2
         else I.unstructured_hex_mesh(3, p, periodic=True, perturb=0.1))
    disc = Discretization(m, EULER)
    R = residual(disc, _free_stream(disc.E, disc.npe, D))
    assert np.abs(R).max() < 1e-11 * (p + 1) ** 2


def test_weighted_conservation_on_unstructured():
    m = I.unstructured_quad_mesh(3, 3, L=10.0, periodic=True, perturb=0.15)
    eq = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.05, "Pr": 0.72}
    U = I.smooth_perturbation(m, I.vortex_state(m), 0.05, periods=[10, 10])
    disc = Discretization(m, eq)
    R = full_residual(disc, U)
    W = conservation_weights(disc)[:, None, :]
    assert np.abs((W * R).sum(axis=(0, 2))).max() < 1e-13 * (W * np.abs(R)).sum()


@pytest.mark.parametrize("p", [2, 3])
def test_poisson_polynomial_reproduction_on_unstructured(p):
    # u in P_p on bilinear quads: the LDG gradient is grad u and R = 0 exactly
    m = I.unstructured_quad_mesh(2, p, perturb=0.15)
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    c3 = 1.0 if p >= 3 else 0.0
    u = (c3 * x ** 2 * y - 0.5 * y ** p + 0.3 * x * y + x ** p)[:, None]
    f = -(c3 * 2 * y - 0.5 * p * (p - 1) * y ** (p - 2) + p * (p - 1) * x ** (p - 2))[:, None]
    disc = Discretization(m, POISSON)
    Q = gradient(disc, u, u)
    assert np.allclose(Q[:, 0, 0], c3 * 2 * x * y + 0.3 * y + p * x ** (p - 1), atol=1e-11)
    assert np.allclose(Q[:, 0, 1], c3 * x ** 2 - 0.5 * p * y ** (p - 1) + 0.3 * x, atol=1e-11)
    assert np.abs(residual(disc, u, Q, u, f)).max() < 1e-10


def _poisson_unstructured(refine, p):
    import scipy.sparse.linalg as spla
    m = I.unstructured_quad_mesh(2, p, perturb=0.15, refine=refine)
    disc = Discretization(m, POISSON)
    gD = np.zeros((disc.E, 1, disc.npe))
    f = I.poisson_source(m)
    U0 = np.zeros_like(gD)
    A = JAC.A_full(disc, U0, gD, f)
    U = spla.spsolve(A.tocsc(), -full_residual(disc, U0, gD, f).ravel()).reshape(U0.shape)
    eu = np.abs(U - I.poisson_exact(m)).max()
    eq_ = np.abs(gradient(disc, U, gD) - I.poisson_exact_grad(m)).max()
    return eu, eq_


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2, 3])
def test_poisson_rates_on_refined_unstructured_mesh(p):
    # Table 2's setting: an unstructured quadrilateral mesh refined
    # uniformly; rates of the minimal-dissipation scheme p+1 (u) and p (q)
    gold = {int(r[0]): r[1:] for r in np.loadtxt(f"{GOLD}/poisson_rates.txt", comments="#")}
    levels = (1, 2, 3) if p == 1 else (0, 1, 2)
    res = [_poisson_unstructured(r, p) for r in levels]
    ru = math.log2(res[1][0] / res[2][0])
    rq = math.log2(res[1][1] / res[2][1])
    assert abs(ru - gold[p][2]) < 0.6, (res, ru)
    assert abs(rq - gold[p][5]) < 0.6, (res, rq)
