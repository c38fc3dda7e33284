"""Pins for the oracle's Neumann boundary (Eqs. 29-30, C22 = 0), CPU only.

The Neumann data is the prescribed flux G at the boundary nodes (for
Poisson F = -q, so G = -grad u of a manufactured u). Pins: polynomial
reproduction (u in P_p on bilinear quads with exact Dirichlet and Neumann
data gives q = grad u and R = 0 exactly, on sides of both kinds and at the
corner where two Neumann sides meet), the convergence rate p + 1 of the
mixed Dirichlet/Neumann problem, and the Jacobian against central
differences."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle.residual import Discretization, full_residual, gradient, residual


def neumann_square(n, p, perturb=0.15, seed=1204):
    """Unit square; the sides x = 1 and y = 1 carry tag 1 (Neumann), the
    others tag 0 (Dirichlet)."""
    return I.structured_mesh((n, n), p, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=perturb, seed=seed,
                             btag_of_face=lambda d, end: 1 if end == 1 else 0)


def poisson_eq(gN):
    return {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet", 1: "neumann"}, "gN": gN}


@pytest.mark.parametrize("p", [2, 3])
def test_neumann_polynomial_reproduction(p):
    m, _ = I.reorient(neumann_square(3, p, perturb=0.2))
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    c3 = 1.0 if p >= 3 else 0.0
    u = (c3 * x ** 2 * y - 0.5 * y ** p + 0.3 * x * y + x ** p)[:, None]
    ux = c3 * 2 * x * y + 0.3 * y + p * x ** (p - 1)
    uy = c3 * x ** 2 - 0.5 * p * y ** (p - 1) + 0.3 * x
    f = -(c3 * 2 * y - 0.5 * p * (p - 1) * y ** (p - 2) + p * (p - 1) * x ** (p - 2))[:, None]
    gN = -np.stack([ux, uy], axis=1)[:, None]            # F = -grad u
    disc = Discretization(m, poisson_eq(gN))
    assert (m["btag"] == 1).any() and (m["btag"] == 0).any()
    Q = gradient(disc, u, u)
    assert np.allclose(Q[:, 0, 0], ux, atol=1e-11)
    assert np.allclose(Q[:, 0, 1], uy, atol=1e-11)
    assert np.abs(residual(disc, u, Q, u, f)).max() < 1e-10
    # a wrong sign of the data breaks it
    bad = Discretization(m, poisson_eq(-gN))
    assert np.abs(residual(bad, u, gradient(bad, u, u), u, f)).max() > 1e-3


def _solve(n, p):
    import scipy.sparse.linalg as spla
    m = neumann_square(n, p)
    gq = I.poisson_exact_grad(m)                       # [E, 1, D, npe]
    disc = Discretization(m, poisson_eq(-gq))
    gD = np.zeros((disc.E, 1, disc.npe))
    f = I.poisson_source(m)
    U0 = np.zeros_like(gD)
    A = JAC.A_full(disc, U0, gD, f)
    U = spla.spsolve(A.tocsc(), -full_residual(disc, U0, gD, f).ravel()).reshape(U0.shape)
    return np.abs(U - I.poisson_exact(m)).max()


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3])
def test_mixed_dirichlet_neumann_converges_at_p_plus_1(p):
    e = [_solve(n, p) for n in (4, 8, 16)]
    rate = math.log2(e[1] / e[2])
    assert abs(rate - (p + 1)) < 0.6, (e, rate)


def test_neumann_jacobian_matches_central_differences():
    m, _ = I.reorient(neumann_square(3, 2))
    gN = np.random.default_rng(5).standard_normal((m["nodes"].shape[0], 1, 2, 9))
    disc = Discretization(m, poisson_eq(gN))
    gD = np.zeros((disc.E, 1, disc.npe))
    U = np.random.default_rng(6).standard_normal(gD.shape)
    A = JAC.A_full(disc, U, gD)
    v = np.random.default_rng(7).standard_normal(U.size)
    h = 1e-6
    fd = (full_residual(disc, U + h * v.reshape(U.shape), gD) -
          full_residual(disc, U - h * v.reshape(U.shape), gD)).ravel() / (2 * h)
    assert np.abs(A @ v - fd).max() < 1e-7 * np.abs(fd).max()
