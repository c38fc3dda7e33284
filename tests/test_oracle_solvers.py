"""Pins for the oracle's split matvec, masked preconditioner, ILU(0), GMRES
and Newton-BDF2 (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle import solvers as S
from oracle.residual import Discretization, full_residual, gradient

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}


def test_line_pattern_counts():
    # an element's Line-DG block: every node couples to the Dp+1 nodes of its lines
    for D in (2, 3):
        for p in (1, 2, 3, 4):
            pat = S.line_pattern(D, p)
            assert all(len(r) == D * p + 1 for r in pat)
            assert all(i in r for i, r in enumerate(pat))


def _ns_small():
    m = I.structured_mesh((3, 3), 2, (0, 0), (1, 1), (True, True), perturb=0.1)
    m, _ = I.reorient(m)
    eq = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.02, "Pr": 0.72}
    disc = Discretization(m, eq)
    npe = disc.npe
    base = np.zeros((disc.E, 4, npe))
    base[:, 0], base[:, 1], base[:, 2], base[:, 3] = 1.0, 0.5, -0.2, 1.0 / (1.4 * 0.3 ** 2) / 0.4 + 0.145
    U = I.smooth_perturbation(m, base, 0.1, periods=[1, 1])
    return disc, U


def test_split_matvec_equals_dense_newton_matrix():
    disc, U = _ns_small()
    Q = gradient(disc, U)
    K11, K12, K21 = JAC.K11(disc, U, Q), JAC.K12(disc, U, Q), JAC.K21(disc)
    A = JAC.dense_brute_force(lambda X: full_residual(disc, X), U)
    x = np.random.default_rng(0).standard_normal(U.size)
    a_dt = 0.7
    y = S.split_matvec(K11, K12, K21, x, 1.0, -a_dt)
    assert np.allclose(y, x - a_dt * (A @ x), atol=1e-10 * np.abs(y).max())


def test_masked_blocks_keep_in_pattern_product_entries():
    disc, U = _ns_small()
    Q = gradient(disc, U)
    A = (JAC.K11(disc, U, Q) + JAC.K12(disc, U, Q) @ JAC.K21(disc)).toarray()
    Ab = S.masked_blocks(disc, A, 1.0, -0.3)
    pat = S.line_pattern(disc.D, disc.p)
    nc, npe = disc.nc, disc.npe
    e = 4
    blk = A.reshape(disc.E, nc, npe, disc.E, nc, npe)[e, :, :, e]
    for i in range(npe):
        for j in range(npe):
            ref = -0.3 * blk[:, i, :, j] + (np.eye(nc) if i == j else 0)
            if j in pat[i]:
                assert np.allclose(Ab[e, i, j], ref, atol=1e-14)
            else:
                assert not np.any(Ab[e, i, j])


def test_ilu0_reproduces_matrix_on_pattern():
    # ILU(0) is characterised by (L U)_ij = A_ij for every (i, j) in the pattern
    rng = np.random.default_rng(1)
    D, p, nc = 2, 3, 3
    pat = S.line_pattern(D, p)
    npe = (p + 1) ** D
    Ab = np.zeros((1, npe, npe, nc, nc))
    for i in range(npe):
        for j in pat[i]:
            Ab[0, i, j] = 0.1 * rng.standard_normal((nc, nc))
        Ab[0, i, i] += 3 * np.eye(nc)
    F = S.ilu0(Ab, pat)[0]
    L = np.zeros((npe * nc, npe * nc))
    Uu = np.zeros_like(L)
    for i in range(npe):
        for j in pat[i]:
            blk = F[i, j]
            if j < i:
                L[i * nc:(i + 1) * nc, j * nc:(j + 1) * nc] = blk
            else:
                Uu[i * nc:(i + 1) * nc, j * nc:(j + 1) * nc] = blk
        L[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc] = np.eye(nc)
    LU = (L @ Uu).reshape(npe, nc, npe, nc)
    for i in range(npe):
        for j in pat[i]:
            assert np.allclose(LU[i, :, j, :], Ab[0, i, j], atol=1e-13)
    # and the apply is the exact (LU)^-1
    r = rng.standard_normal((1, nc, npe))
    z = S.ilu_apply(S.ilu0(Ab, pat), pat, r)
    zz = np.linalg.solve(L @ Uu, r[0].T.ravel()).reshape(npe, nc).T
    assert np.allclose(z[0], zz, atol=1e-12)


@pytest.mark.parametrize("D,p", [(2, 4), (3, 2), (3, 3), (3, 4)])
def test_ilu_apply_by_wavefront_levels_equals_row_order(D, p):
    # the property a wavefront apply rests on: with level(i) = ix + iy + iz,
    # every lower neighbour of row i in the line pattern lies on a lower
    # level and every upper one on a higher level, so the rows of one level
    # are independent in both triangular solves; solving level by level
    # (every row of a level from the values of the earlier levels) gives the
    # row-ordered solve of ilu_apply
    rng = np.random.default_rng(7)
    N, nc = p + 1, 3
    pat = S.line_pattern(D, p)
    npe = N ** D
    lev = [i % N + (i // N) % N + (i // (N * N) if D == 3 else 0) for i in range(npe)]
    for i in range(npe):
        assert sum(k < i for k in pat[i]) == lev[i]   # the diagonal's slot is the level
        for k in pat[i]:
            if k < i:
                assert lev[k] < lev[i]
            elif k > i:
                assert lev[k] > lev[i]
    Ab = np.zeros((2, npe, npe, nc, nc))
    for e in range(2):
        for i in range(npe):
            for j in pat[i]:
                Ab[e, i, j] = 0.1 * rng.standard_normal((nc, nc))
            Ab[e, i, i] += 3 * np.eye(nc)
    F = S.ilu0(Ab, pat)
    r = rng.standard_normal((2, nc, npe))
    z_ref = S.ilu_apply(F, pat, r)
    for e in range(2):
        y = r[e].T.copy()
        for l in range(1, max(lev) + 1):
            rows = [i for i in range(npe) if lev[i] == l]
            upd = {i: sum(F[e, i, k] @ y[k] for k in pat[i] if k < i) for i in rows}
            for i in rows:
                y[i] = y[i] - upd[i]
        x = y.copy()
        for l in range(max(lev), -1, -1):
            rows = [i for i in range(npe) if lev[i] == l]
            new = {i: np.linalg.solve(F[e, i, i], x[i] - sum((F[e, i, j] @ x[j] for j in pat[i] if j > i),
                                                              np.zeros(nc))) for i in rows}
            for i in rows:
                x[i] = new[i]
        assert np.allclose(x.T, z_ref[e], rtol=0, atol=1e-12 * np.abs(z_ref[e]).max())


def test_ilu0_is_exact_lu_when_pattern_is_full():
    # with p = 1 in 1-D-like blocks (D=2, p=1 gives 3 of 4 couplings; use a
    # dense random block instead): ILU(0) on a full pattern equals LU
    rng = np.random.default_rng(2)
    n, nc = 5, 2
    pat = [list(range(n)) for _ in range(n)]
    Ab = 0.2 * rng.standard_normal((1, n, n, nc, nc))
    for i in range(n):
        Ab[0, i, i] += 2 * np.eye(nc)
    F = S.ilu0(Ab, pat)
    r = rng.standard_normal((1, nc, n))
    z = S.ilu_apply(F, pat, r)
    dense = Ab[0].transpose(0, 2, 1, 3).reshape(n * nc, n * nc)
    assert np.allclose(z[0].T.ravel(), np.linalg.solve(dense, r[0].T.ravel()), atol=1e-12)


def test_gmres_full_space_equals_direct_solve():
    rng = np.random.default_rng(3)
    n = 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    x, its, rel = S.gmres(lambda v: A @ v, b, tol=1e-14, restart=n)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-11)
    P = np.linalg.inv(A + 0.05 * rng.standard_normal((n, n)))
    x2, its2, _ = S.gmres(lambda v: A @ v, b, precond=lambda v: P @ v, tol=1e-12, restart=n)
    assert np.allclose(x2, np.linalg.solve(A, b), atol=1e-10)
    assert its2 < its


def _vortex_small():
    m = I.vortex_mesh(4, 2, perturb=0.1)
    disc = Discretization(m, EULER)
    return disc, I.vortex_state(m)


def test_newton_bdf2_converges_quadratically_with_fresh_jacobian():
    disc, U0 = _vortex_small()
    F = lambda X: full_residual(disc, X)
    jac = lambda X: (JAC.K11(disc, X), None, None)
    pat = S.line_pattern(disc.D, disc.p)

    def pc(K, shift, scale):
        Fct = S.ilu0(S.masked_blocks(disc, K[0], shift, scale), pat)
        return lambda v: S.ilu_apply(Fct, pat, v.reshape(U0.shape)).ravel()
    U1, st = S.newton_bdf2(F, jac, U0, None, 0.2, first=True, rtol=1e-12, gmres_tol=1e-12,
                           restart=200, reuse=1, precond_builder=pc)
    h = np.array(st["hist"])
    assert st["newton"] <= 5
    # quadratic: each error roughly the square of the previous (relative)
    rel = h / h[0]
    assert rel[2] < 10 * rel[1] ** 2 + 1e-13
    # the update solves the BDF1 stage equation
    G = U1 - U0 - 0.2 * F(U1)
    assert np.linalg.norm(G) <= 1e-12 * np.linalg.norm(0.2 * F(U0)) * 1.01


def test_preconditioner_reduces_gmres_iterations():
    # qualitative statement of Sec. 5.5: without the preconditioner many more
    # GMRES iterations are needed for the same tolerance
    disc, U0 = _vortex_small()
    K = JAC.K11(disc, U0)
    pat = S.line_pattern(disc.D, disc.p)
    dt = 0.5
    Fct = S.ilu0(S.masked_blocks(disc, K, 1.0, -dt), pat)
    mv = lambda v: S.split_matvec(K, None, None, v, 1.0, -dt)
    b = np.random.default_rng(4).standard_normal(U0.size)
    _, it_p, _ = S.gmres(mv, b, lambda v: S.ilu_apply(Fct, pat, v.reshape(U0.shape)).ravel(),
                         tol=1e-8, restart=300)
    _, it_n, _ = S.gmres(mv, b, None, tol=1e-8, restart=300)
    assert it_n > 2 * it_p


def test_dirk3_tableau_order_conditions_and_stability():
    """Alexander's three-stage DIRK (Sec. 4.1): the order-3 conditions, the
    defining cubic of its diagonal, stiff accuracy and L-stability."""
    A, b, c = S.dirk3_tableau()
    a = S.DIRK3_ALPHA
    assert abs(a ** 3 - 3 * a ** 2 + 1.5 * a - 1.0 / 6.0) < 1e-14
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert abs(b.sum() - 1.0) < 1e-15
    assert abs(b @ c - 0.5) < 1e-14
    assert abs(b @ c ** 2 - 1.0 / 3.0) < 1e-14
    assert abs(b @ A @ c - 1.0 / 6.0) < 1e-14
    assert np.array_equal(A[2], b)                     # stiffly accurate

    def R(z):                                          # stability function
        return 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    assert abs(R(-1e8)) < 1e-7                         # L-stable
    for y in np.linspace(0.0, 50.0, 101):
        assert abs(R(1j * y)) <= 1.0 + 1e-12           # A-stable on the imaginary axis
    # R(z) = e^z + O(z^4)
    for z in (1e-2, -1e-2):
        assert abs(R(z) - math.exp(z)) < 2 * abs(z) ** 4


def test_dirk3_third_order_on_dg_advection():
    """The DIRK3 driver on the DG advection semi-discretisation (a linear
    ODE system): halving dt divides the error by about 8."""
    m = I.structured_mesh((3, 3), 3, (0, 0), (1, 1), (True, True), perturb=0.1)
    disc = Discretization(m, {"kind": "advection", "adv": [1.0, 0.6]})
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    U0 = np.sin(2 * math.pi * x + 0.3)[:, None] * np.cos(2 * math.pi * y)[:, None]
    F = lambda X: full_residual(disc, X)
    K = JAC.K11(disc, U0)
    jac = lambda X: (K, None, None)

    def run(nsteps, T=0.2):
        U = U0.copy()
        for _ in range(nsteps):
            U, st = S.dirk3_step(F, jac, U, T / nsteps, rtol=1e-13, gmres_tol=1e-14, restart=200, reuse=100)
            assert all(s["newton"] <= 2 for s in st)
        return U
    ref = run(64)
    e1 = np.abs(run(4) - ref).max()
    e2 = np.abs(run(8) - ref).max()
    assert 2.7 < math.log2(e1 / e2) < 3.5, (e1, e2)


def test_rk4_amplification_is_the_quartic_taylor_polynomial():
    """On y' = M y one step multiplies by 1 + hM + (hM)^2/2 + (hM)^3/6 + (hM)^4/24."""
    rng = np.random.default_rng(4)
    M = rng.standard_normal((6, 6))
    y = rng.standard_normal(6)
    h = 0.1
    hm = h * M
    P = np.eye(6) + hm + hm @ hm / 2 + hm @ hm @ hm / 6 + hm @ hm @ hm @ hm / 24
    assert np.allclose(S.rk4_step(lambda v: M @ v, y, h), P @ y, rtol=1e-14, atol=1e-14)


def test_rk4_fourth_order_on_dg_advection():
    m = I.structured_mesh((3, 3), 3, (0, 0), (1, 1), (True, True), perturb=0.1)
    disc = Discretization(m, {"kind": "advection", "adv": [1.0, 0.6]})
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    U0 = np.sin(2 * math.pi * x + 0.3)[:, None] * np.cos(2 * math.pi * y)[:, None]
    F = lambda X: full_residual(disc, X)

    def run(nsteps, T=0.1):
        U = U0.copy()
        for _ in range(nsteps):
            U = S.rk4_step(F, U, T / nsteps)
        return U
    ref = run(256)
    e1 = np.abs(run(32) - ref).max()
    e2 = np.abs(run(64) - ref).max()
    assert 3.7 < math.log2(e1 / e2) < 4.4, (e1, e2)


def test_bdf2_second_order_on_dg_advection():
    """The BDF2 Newton driver (a BDF1 first level, then BDF2) on the DG
    advection semi-discretisation, against the exact flow of that linear ODE
    system (matrix exponential of its dense Jacobian): halving dt divides
    the error by about 4 (the BDF1 start contributes O(dt^2) once)."""
    import scipy.linalg as sla
    m = I.structured_mesh((3, 3), 2, (0, 0), (1, 1), (True, True), perturb=0.1)
    disc = Discretization(m, {"kind": "advection", "adv": [1.0, 0.6]})
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    U0 = np.sin(2 * math.pi * x + 0.3)[:, None] * np.cos(2 * math.pi * y)[:, None]
    F = lambda X: full_residual(disc, X)
    K = JAC.K11(disc, U0)
    jac = lambda X: (K, None, None)
    T = 0.2
    exact = (sla.expm(T * K.toarray()) @ U0.ravel()).reshape(U0.shape)

    def run(nsteps):
        dt = T / nsteps
        Unm1, Un = None, U0.copy()
        for k in range(nsteps):
            U1, st = S.newton_bdf2(F, jac, Un, Unm1, dt, first=(k == 0), rtol=1e-13, gmres_tol=1e-14,
                                   restart=200, reuse=100)
            assert st["newton"] <= 2
            Unm1, Un = Un, U1
        return Un
    e1 = np.abs(run(20) - exact).max()
    e2 = np.abs(run(40) - exact).max()
    assert 1.8 < math.log2(e1 / e2) < 2.3, (e1, e2)
