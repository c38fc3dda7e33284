"""Pins for the oracle's stabilised LDG scheme, C11 = C22 = 1/20 (Sec. 3
Eqs. 25-26 and 30, Sec. 4.1 Eq. 36, Table 2's lower half), CPU only.

With C22 != 0 the trace u^ depends on the normal viscous flux on both sides
of a face, so Q = D(U, Q) is coupled and the steady problem is the split
system (R(U, Q), Q - D(U, Q)) = 0, solved here by a sparse direct solve of
its Jacobian [[K11, K12], [-K21, I - K22]] as in the paper. Pins: exact
polynomial solutions, the reduction to the minimal-dissipation scheme, the
sign of the C22 term (the stabilising sign keeps every eigenvalue of the
steady operator in the left half-plane, the printed one does not), and the
rates of Table 2's lower half with the higher q-rate it reports."""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle.residual import Discretization, coupled_residual, full_residual, gradient

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def stab_eq(C=1.0 / 20.0, **kw):
    eq = {"kind": "poisson", "C11": C, "C22": C, "C11b": 1.0, "bc": {0: "dirichlet"}}
    eq.update(kw)
    return eq


def coupled_solve(disc, gD, f):
    U0 = np.zeros((disc.E, 1, disc.npe))
    Q0 = np.zeros((disc.E, 1, disc.D, disc.npe))
    J = JAC.coupled(disc, U0, Q0, gD, f)
    R0, G0 = coupled_residual(disc, U0, Q0, gD, f)
    X = spla.spsolve(J.tocsc(), -np.concatenate([R0.ravel(), G0.ravel()]))
    return X[:U0.size].reshape(U0.shape), X[U0.size:].reshape(Q0.shape)


@pytest.mark.parametrize("mesh", ["reoriented", "unstructured", "neumann"])
def test_polynomial_solutions_are_exact(mesh):
    # u in P_p on bilinear quads: (u, grad u) makes both parts of the split
    # residual vanish (every jump is zero), Dirichlet and Neumann sides alike
    p = 3
    if mesh == "reoriented":
        m = I.reorient(I.poisson_square_mesh(3, p, perturb=0.2))[0]
    elif mesh == "unstructured":
        m = I.unstructured_quad_mesh(2, p, perturb=0.15)
    else:
        m = I.reorient(I.structured_mesh((3, 3), p, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=0.2,
                                         btag_of_face=lambda d, end: 1 if end == 1 else 0))[0]
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    u = (x ** 2 * y - 0.5 * y ** 3 + 0.3 * x * y + x ** 3)[:, None]
    ux, uy = 2 * x * y + 0.3 * y + 3 * x ** 2, x ** 2 - 1.5 * y ** 2 + 0.3 * x
    f = -(2 * y - 3 * y + 6 * x)[:, None]
    Q = np.stack([ux, uy], axis=1)[:, None]
    disc = Discretization(m, stab_eq(bc={0: "dirichlet", 1: "neumann"}, gN=-Q))
    R, G = coupled_residual(disc, u, Q, u, f)
    assert np.abs(R).max() < 1e-9 and np.abs(G).max() < 1e-10


def test_zero_c22_is_the_minimal_dissipation_scheme():
    m = I.unstructured_quad_mesh(2, 2, perturb=0.15)
    f = I.poisson_source(m)
    gD = np.zeros_like(f)
    U, Q = coupled_solve(Discretization(m, stab_eq(C=1e-300)), gD, f)
    disc0 = Discretization(m, stab_eq(C=0.0))
    A = JAC.A_full(disc0, gD, gD, f)
    U0 = spla.spsolve(A.tocsc(), -full_residual(disc0, gD, gD, f).ravel()).reshape(gD.shape)
    assert np.abs(U - U0).max() < 1e-11 * np.abs(U0).max()
    assert np.abs(Q - gradient(disc0, U0, gD)).max() < 1e-9 * np.abs(Q).max()


@pytest.mark.parametrize("C22", [0.05, 1.0])
def test_c22_sign_keeps_the_steady_operator_dissipative(C22):
    # the steady operator after eliminating Q, A = K11 + K12 (I - K22)^-1 K21:
    # every eigenvalue in the left half-plane with the stabilising sign; the
    # printed sign (the same term with -C22) puts eigenvalues on the right
    m = I.reorient(I.poisson_square_mesh(3, 2, perturb=0.15))[0]
    out = []
    for c in (C22, -C22):
        disc = Discretization(m, stab_eq(C=0.05, C22=c))
        gD = np.zeros((disc.E, 1, disc.npe))
        J = JAC.coupled(disc, gD, np.zeros((disc.E, 1, 2, disc.npe)), gD).toarray()
        n = gD.size
        A = J[:n, :n] - J[:n, n:] @ np.linalg.solve(J[n:, n:], J[n:, :n])
        out.append(np.linalg.eigvals(A).real.max())
    assert out[0] < 0.0 < out[1], out


def _rates(p, levels, C):
    res = []
    for r in levels:
        m = I.unstructured_quad_mesh(2, p, perturb=0.15, refine=r)
        f = I.poisson_source(m)
        U, Q = coupled_solve(Discretization(m, stab_eq(C=C)), np.zeros_like(f), f)
        res.append((np.abs(U - I.poisson_exact(m)).max(), np.abs(Q - I.poisson_exact_grad(m)).max()))
    return (math.log2(res[-2][0] / res[-1][0]), math.log2(res[-2][1] / res[-1][1]))


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2, 3])
def test_table2_stabilised_rates_on_refined_unstructured_mesh(p):
    # Table 2, lower half: u keeps ~p+1, q gains over the minimal-dissipation
    # scheme (p), on an unstructured mesh refined uniformly
    gold = {int(r[0]): r[1:] for r in np.loadtxt(f"{GOLD}/poisson_rates_stabilized.txt", comments="#")}
    levels = (1, 2, 3) if p < 3 else (0, 1, 2)
    ru, rq = _rates(p, levels, 1.0 / 20.0)
    _, rq0 = _rates(p, levels, 1e-300)
    assert abs(ru - gold[p][2]) < 0.6, (ru, gold[p])
    assert abs(rq - gold[p][5]) < 0.6, (rq, gold[p])
    assert rq > rq0 + 0.25, (rq, rq0)
