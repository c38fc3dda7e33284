"""Pins for the oracle's fluxes, residual, gradient and Jacobians (CPU only).

Each pin rests on something other than the oracle itself: a closed form,
an invariant of the scheme, a textbook 1-D DG computed here from scratch,
polynomial exactness, finite differences, or brute force.
"""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle import physics as ph
from oracle.residual import (Discretization, conservation_weights, full_residual, gradient,
                             residual)

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}
EULER_LF = {"kind": "euler", "gamma": 1.4, "flux": "lf"}


def ns_eq(mu=0.05):
    return {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": mu, "Pr": 0.72}


def _free_stream(E, npe, D, gamma=1.4):
    rho, v, p = 1.1, [0.8, -0.3, 0.25][:D], 2.5
    U = np.zeros((E, D + 2, npe))
    U[:, 0] = rho
    for a in range(D):
        U[:, 1 + a] = rho * v[a]
    U[:, D + 1] = p / (gamma - 1) + 0.5 * rho * sum(x * x for x in v)
    return U


# ---------------------------------------------------------------------------
# pointwise fluxes
# ---------------------------------------------------------------------------
def _rand_states(D, k, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, k)
    v = rng.uniform(-1, 1, (D, k))
    p = rng.uniform(0.5, 3.0, k)
    u = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * (v * v).sum(0)]])
    return u


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("flux", ["roe", "lf"])
def test_numflux_consistency_and_antisymmetry(D, flux):
    eq = {"kind": "euler", "gamma": 1.4, "flux": flux}
    ua, ub = _rand_states(D, 50, 1), _rand_states(D, 50, 2)
    n = np.random.default_rng(3).standard_normal((D, 50))
    f = ph.inviscid_numflux(eq, ua, ua, n)
    assert np.allclose(f, ph.euler_flux_n(ua, n, 1.4), rtol=1e-13, atol=1e-13)
    f1 = ph.inviscid_numflux(eq, ua, ub, n)
    f2 = ph.inviscid_numflux(eq, ub, ua, -n)
    assert np.allclose(f1, -f2, rtol=1e-12, atol=1e-12)


def test_roe_supersonic_upwinding():
    # all characteristic speeds positive along n: the flux is F(u_in).n
    D = 2
    rho, p = np.array([1.0, 1.3]), np.array([1.0, 0.8])
    vx = np.array([3.0, 3.2])
    u_in = np.stack([rho[:1], rho[:1] * vx[:1], [0.0], p[:1] / 0.4 + 0.5 * rho[:1] * vx[:1] ** 2])
    u_out = np.stack([rho[1:], rho[1:] * vx[1:], [0.0], p[1:] / 0.4 + 0.5 * rho[1:] * vx[1:] ** 2])
    n = np.array([[2.0], [0.0]])
    f = ph.roe_flux(u_out, u_in, n, 1.4)
    assert np.allclose(f, ph.euler_flux_n(u_in, n, 1.4), rtol=1e-13)
    f = ph.roe_flux(u_in, u_out, -n, 1.4)   # flow towards this side: upwind = outside
    assert np.allclose(f, ph.euler_flux_n(u_in, -n, 1.4), rtol=1e-13)


def test_ns_viscous_flux_from_primitive_gradients():
    # build q = grad(conserved) from chosen primitive gradients by the chain
    # rule and compare with tau / heat flux written from the definitions
    rng = np.random.default_rng(5)
    D, g, mu, Pr = 3, 1.4, 0.3, 0.72
    rho, v, p = 1.2, rng.standard_normal(D), 2.0
    grho, gv, gp = rng.standard_normal(D), rng.standard_normal((D, D)), rng.standard_normal(D)
    E = p / (g - 1) + 0.5 * rho * v @ v
    u = np.concatenate([[rho], rho * v, [E]])[:, None]
    q = np.zeros((D + 2, D))
    q[0] = grho
    for a in range(D):
        q[1 + a] = v[a] * grho + rho * gv[a]
    q[D + 1] = gp / (g - 1) + 0.5 * grho * (v @ v) + rho * (gv.T @ v)
    n = rng.standard_normal((D, 1))
    F = ph.ns_viscous_flux_n(u, q[:, :, None], n, g, mu, Pr)[:, 0]
    div = np.trace(gv)
    tau = mu * (gv + gv.T - 2 / 3 * div * np.eye(D))
    e = p / ((g - 1) * rho)
    ge = gp / ((g - 1) * rho) - p * grho / ((g - 1) * rho ** 2)
    heat = -(mu / Pr) * g * ge
    ref = np.concatenate([[0.0], -tau @ n[:, 0], [(heat - tau.T @ v) @ n[:, 0]]])
    assert np.allclose(F, ref, rtol=1e-12, atol=1e-12)
    assert e > 0


# ---------------------------------------------------------------------------
# residual invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("eq", [EULER, EULER_LF])
def test_free_stream_2d_perturbed(p, eq):
    m, _ = I.reorient(I.vortex_mesh(4, p, perturb=0.15))
    disc = Discretization(m, eq)
    R = residual(disc, _free_stream(disc.E, disc.npe, 2))
    assert np.abs(R).max() < 2e-12 * (p + 1) ** 2


@pytest.mark.parametrize("p", [2, 3])
def test_free_stream_3d_trilinear(p):
    m = I.structured_mesh((3, 3, 3), p, (0,) * 3, (1,) * 3, (True,) * 3, perturb=0.15)
    m, _ = I.reorient(m)
    disc = Discretization(m, EULER)
    R = residual(disc, _free_stream(disc.E, disc.npe, 3))
    assert np.abs(R).max() < 1e-11 * (p + 1) ** 2


def test_free_stream_3d_curved_converges():
    # 3-D curved maps do not preserve free stream exactly; the defect must
    # vanish under refinement at (at least) order p
    p, errs = 2, []
    for n in (4, 8):
        m = I.tgv_mesh(n, p, amp=0.1)
        disc = Discretization(m, EULER)
        errs.append(np.abs(residual(disc, _free_stream(disc.E, disc.npe, 3))).max())
    assert errs[1] < errs[0] * 2.0 ** -(p - 0.3)


@pytest.mark.parametrize("case", ["euler2d", "lf2d", "ns3d", "reoriented_ns2d"])
def test_weighted_conservation(case):
    if case in ("euler2d", "lf2d"):
        m = I.vortex_mesh(4, 3, perturb=0.15)
        eq = EULER if case == "euler2d" else EULER_LF
        U = I.smooth_perturbation(m, I.vortex_state(m, x0=5, y0=5), 0.05)
    elif case == "ns3d":
        m = I.tgv_mesh(3, 2)
        eq = ns_eq()
        U = I.smooth_perturbation(m, I.tgv_state(m), 0.05)
    else:
        m0 = I.vortex_mesh(4, 2, perturb=0.15)
        U0 = I.smooth_perturbation(m0, I.vortex_state(m0), 0.05)
        m, maps = I.reorient(m0)
        U = I.permute_nodal(U0, maps)
        eq = ns_eq()
    disc = Discretization(m, eq)
    R = full_residual(disc, U)
    W = conservation_weights(disc)[:, None, :]
    tot = np.abs((W * R).sum(axis=(0, 2)))
    assert tot.max() < 1e-13 * (W * np.abs(R)).sum()


def test_advection_polynomial_exactness():
    # u in P_p on a bilinear mesh with exact inflow data: R = -a.grad u at the nodes
    p = 3
    a = np.array([0.7, -0.4])
    m, maps = I.reorient(I.poisson_square_mesh(4, p, perturb=0.2))
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    u = (1 + x + 2 * y - x * y + x ** 3 - 0.5 * y ** 2 * x)[:, None]
    ux = 1 - y + 3 * x ** 2 - 0.5 * y ** 2
    uy = 2 - x - y * x
    eq = {"kind": "advection", "adv": a, "bc": {0: "dirichlet"}}
    disc = Discretization(m, eq)
    R = residual(disc, u, None, u)
    assert np.allclose(R[:, 0], -(a[0] * ux + a[1] * uy), atol=1e-11)


def _textbook_dg_1d(x_edges, s, uvals, flux, numflux):
    """Standard nodal DG on a periodic 1-D grid, written in physical
    coordinates with its own quadrature: returns du/dt at the nodes."""
    K, p = len(x_edges) - 1, len(s) - 1
    xg, wg = np.polynomial.legendre.leggauss(math.ceil((3 * p + 1) / 2))   # precision 3p
    from oracle.rules import lagrange   # basis values only
    out = np.zeros_like(uvals)
    for k in range(K):
        xl, xr = x_edges[k], x_edges[k + 1]
        h = xr - xl
        xi = (xg + 1) / 2
        phi, dphi = lagrange(s, xi)
        M = h * phi.T @ (wg[:, None] / 2 * phi)
        uq = np.einsum("qi,ci->cq", phi, uvals[k])
        Fq = flux(uq)
        vol = np.einsum("qi,q,cq->ci", dphi / h, wg / 2 * h, Fq)
        fr = numflux(uvals[(k + 1) % K][:, 0], uvals[k][:, p])
        fl = numflux(uvals[k][:, 0], uvals[k - 1][:, p])
        b = vol.copy()
        b[:, p] -= fr
        b[:, 0] += fl
        out[k] = np.linalg.solve(M, b.T).T
    return out


def test_reduces_to_textbook_1d_dg():
    # a state that depends on x only, on an affine mesh: Line-DG equals
    # standard 1-D DG along the x lines (the scheme's defining property).
    # This pins the line operator; the numerical flux is the oracle's own
    # Roe flux here, which tests/test_oracle_fluxes.py pins on its own
    p, nx, ny, L = 3, 5, 3, 10.0
    m = I.structured_mesh((nx, ny), p, (0, 0), (L, 6.0), (True, True))
    x = m["nodes"][..., 0]
    rho = 1 + 0.2 * np.sin(2 * math.pi * x / L)
    vx = 0.5 + 0.1 * np.cos(2 * math.pi * x / L)
    pr = 1 + 0.1 * np.sin(4 * math.pi * x / L)
    U = np.stack([rho, rho * vx, 0 * rho, pr / 0.4 + 0.5 * rho * vx ** 2], axis=1)
    disc = Discretization(m, EULER)
    R = residual(disc, U)
    # 1-D textbook on the x grid (row of elements ey = 0, line j = 0)
    s = m["s"]
    edges = np.linspace(0, L, nx + 1)
    u1 = np.stack([U[k][[0, 1, 3]][:, :p + 1] for k in range(nx)])
    f1 = lambda u: np.stack([u[1], u[1] ** 2 / u[0] + 0.4 * (u[2] - 0.5 * u[1] ** 2 / u[0]),
                             (u[2] + 0.4 * (u[2] - 0.5 * u[1] ** 2 / u[0])) * u[1] / u[0]])

    def nf(uo, ui):
        full = lambda w: np.array([w[0], w[1], 0.0, w[2]])[:, None]
        return ph.roe_flux(full(uo), full(ui), np.array([[1.0], [0.0]]), 1.4)[[0, 1, 3], 0]
    ref = _textbook_dg_1d(edges, s, u1, f1, nf)
    got = np.stack([R[k][[0, 1, 3]][:, :p + 1] for k in range(nx)])
    assert np.allclose(got, ref, atol=1e-12)


def test_euler_vortex_truncation_converges():
    # R(u_exact) vs the exact du/dt of the translating vortex: O(h^p) or better
    p, errs = 2, []
    for n in (8, 16, 32):
        m = I.vortex_mesh(n, p, perturb=0.1)
        disc = Discretization(m, EULER)
        eps = 1e-4
        dudt = (I.vortex_state(m, t=eps) - I.vortex_state(m, t=-eps)) / (2 * eps)
        errs.append(np.abs(residual(disc, I.vortex_state(m)) - dudt).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p - 0.3, rates


# ---------------------------------------------------------------------------
# Poisson (LDG, the perturbed unit square)
# ---------------------------------------------------------------------------
POISSON = {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}}


@pytest.mark.parametrize("p", [2, 3])
def test_poisson_polynomial_reproduction(p):
    m, _ = I.reorient(I.poisson_square_mesh(3, p, perturb=0.2))
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    c3 = 1.0 if p >= 3 else 0.0          # keep the total degree <= p
    u = (c3 * x ** 2 * y - 0.5 * y ** p + 0.3 * x * y + x ** p)[:, None]
    f = -(c3 * 2 * y - 0.5 * p * (p - 1) * y ** (p - 2) + p * (p - 1) * x ** (p - 2))[:, None]
    disc = Discretization(m, POISSON)
    Q = gradient(disc, u, u)
    assert np.allclose(Q[:, 0, 0], c3 * 2 * x * y + 0.3 * y + p * x ** (p - 1), atol=1e-11)
    assert np.allclose(Q[:, 0, 1], c3 * x ** 2 - 0.5 * p * y ** (p - 1) + 0.3 * x, atol=1e-11)
    assert np.abs(residual(disc, u, Q, u, f)).max() < 1e-10


def _poisson_solve(n, p):
    import scipy.sparse.linalg as spla
    m = I.poisson_square_mesh(n, p)
    disc = Discretization(m, POISSON)
    gD = np.zeros((disc.E, 1, disc.npe))
    f = I.poisson_source(m)
    U0 = np.zeros_like(gD)
    A = JAC.A_full(disc, U0, gD, f)
    R0 = full_residual(disc, U0, gD, f)
    U = spla.spsolve(A.tocsc(), -R0.ravel()).reshape(U0.shape)
    eu = np.abs(U - I.poisson_exact(m)).max()
    eq_ = np.abs(gradient(disc, U, gD) - I.poisson_exact_grad(m)).max()
    return eu, eq_, np.abs(full_residual(disc, U, gD, f)).max()


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2, 3])
def test_poisson_convergence_rates(p):
    # Table 2 (C11 = C22 = 0): rates ~ p+1 for u and ~ p for q
    gold = {int(r[0]): r[1:] for r in np.loadtxt(
        __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                   "poisson_rates.txt"), comments="#")}
    res = [_poisson_solve(n, p) for n in (4, 8, 16)]
    assert max(r[2] for r in res) < 1e-9
    ru = np.log2(res[0][0] / res[1][0]), np.log2(res[1][0] / res[2][0])
    rq = np.log2(res[0][1] / res[1][1]), np.log2(res[1][1] / res[2][1])
    assert abs(ru[1] - gold[p][2]) < 0.6, (ru, gold[p])
    assert abs(rq[1] - gold[p][5]) < 0.6, (rq, gold[p])


# ---------------------------------------------------------------------------
# Jacobians
# ---------------------------------------------------------------------------
def _small_case(kind):
    if kind == "euler":
        m, _ = I.reorient(I.vortex_mesh(3, 2, perturb=0.15))
        U = I.smooth_perturbation(m, I.vortex_state(m, x0=5, y0=5), 0.05)
        return Discretization(m, EULER), U, None
    if kind == "ns":
        m = I.structured_mesh((3, 3, 3), 1, (0,) * 3, (2 * math.pi,) * 3, (True,) * 3, perturb=0.1)
        U = I.smooth_perturbation(m, I.tgv_state(m, mach=0.3), 0.05)
        return Discretization(m, ns_eq(0.1)), U, None
    m, _ = I.reorient(I.poisson_square_mesh(3, 2))
    U = I.poisson_exact(m) + 0.1
    return Discretization(m, POISSON), U, np.zeros_like(U)


@pytest.mark.parametrize("kind", ["euler", "ns", "poisson"])
def test_jacobian_vs_central_differences(kind):
    disc, U, gD = _small_case(kind)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(U.shape)
    h = 1e-6 * np.abs(U).max()
    F = lambda X: full_residual(disc, X, gD)
    fd = (F(U + h * v) - F(U - h * v)).ravel() / (2 * h)
    if disc.nc > 1 and kind == "ns" or kind == "poisson":
        Q = gradient(disc, U, gD)
        Kv = JAC.K11(disc, U, Q, gD) @ v.ravel() + JAC.K12(disc, U, Q, gD) @ (JAC.K21(disc, gD) @ v.ravel())
    else:
        Kv = JAC.K11(disc, U) @ v.ravel()
    assert np.abs(Kv - fd).max() < 1e-6 * np.abs(fd).max()


def test_jacobian_colouring_equals_dense():
    disc, U, _ = _small_case("euler")
    K = JAC.K11(disc, U).toarray()
    Kd = JAC.dense_brute_force(lambda X: residual(disc, X), U)
    assert np.array_equal(K, Kd)


def test_k21_state_and_component_independent():
    disc, U, _ = _small_case("ns")
    K21 = JAC.K21(disc).tocsr()
    # D is affine with zero boundary data: D(U) = K21 U exactly
    assert np.allclose(K21 @ U.ravel(), gradient(disc, U).ravel(), atol=1e-12)
    # same scalar operator for every component
    E, nc, D, npe = disc.E, disc.nc, disc.D, disc.npe
    blk = K21.toarray().reshape(E, nc, D, npe, E, nc, npe)
    for c in range(1, nc):
        assert np.array_equal(blk[:, c, :, :, :, c], blk[:, 0, :, :, :, 0])
        assert not np.any(blk[:, c, :, :, :, 0])


@pytest.mark.parametrize("kind", ["ns", "poisson"])
def test_reduced_jacobian_is_split_product(kind):
    # Eq. 40: A = K11 + K12 K21
    disc, U, gD = _small_case(kind)
    Q = gradient(disc, U, gD)
    A = JAC.A_full(disc, U, gD)
    S = JAC.K11(disc, U, Q, gD) + JAC.K12(disc, U, Q, gD) @ JAC.K21(disc, gD)
    assert np.abs((A - S).toarray()).max() < 1e-12 * np.abs(A.toarray()).max()


@pytest.mark.slow
@pytest.mark.parametrize("C11b", [0.1, 10.0])
def test_poisson_rates_insensitive_to_boundary_penalty(C11b):
    # the Dirichlet penalty only needs to be positive (Sec. 3): the u-rate
    # p + 1 of Table 2 holds for penalties two decades apart
    import scipy.sparse.linalg as spla
    p, errs = 2, []
    for n in (4, 8, 16):
        m = I.poisson_square_mesh(n, p)
        disc = Discretization(m, dict(POISSON, C11b=C11b))
        gD = np.zeros((disc.E, 1, disc.npe))
        f = I.poisson_source(m)
        A = JAC.A_full(disc, gD, gD, f)
        U = spla.spsolve(A.tocsc(), -full_residual(disc, gD, gD, f).ravel()).reshape(gD.shape)
        errs.append(np.abs(U - I.poisson_exact(m)).max())
    assert abs(math.log2(errs[1] / errs[2]) - (p + 1)) < 0.6, errs


@pytest.mark.parametrize("bc", ["dirichlet", "mixed"])
def test_poisson_operator_is_dissipative(bc):
    # dU/dt = R(U) with R the LDG form of lap u: the dense Jacobian on a tiny
    # mesh is nonsingular and every eigenvalue has a negative real part (the
    # semi-discrete heat equation decays), with Dirichlet or mixed sides
    m = I.reorient(I.structured_mesh((2, 2), 2, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=0.15,
                                     btag_of_face=(lambda d, end: 1 if end == 1 else 0) if bc == "mixed" else None))[0]
    eq = dict(POISSON, bc={0: "dirichlet", 1: "neumann"})
    disc = Discretization(m, eq)
    gD = np.zeros((disc.E, 1, disc.npe))
    A = JAC.dense_brute_force(lambda X: full_residual(disc, X.reshape(gD.shape), gD).ravel(), gD.ravel())
    lam = np.linalg.eigvals(A)
    assert lam.real.max() < 0.0, lam.real.max()
    assert np.linalg.cond(A) < 1e8
