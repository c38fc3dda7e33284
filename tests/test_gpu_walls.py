"""GPU parity of the Jacobian path on meshes with no-slip walls.

At a wall the gradient's trace is the wall state of the inside trace, a
nonlinear function of it, so the oracle's references come from complex
steps of its full residual (which contains the wall fluxes and traces
exactly): the Newton matrix times a vector by one complex step, each
element's diagonal block by a complex step per column, then the oracle's
masking, ILU(0) and solve, and a Newton-BDF2 solution with that Jacobian.
Tolerances as for periodic meshes: matvec 1e-5 (FP32) / 1e-11 (FP64),
factors 1e-5 / 1e-10 per block row, apply 1e-4 / 1e-10, Newton 1e-7."""
import math
import types

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle import solvers as S
from oracle.residual import Discretization, full_residual
from submesh import H_CS, diag_block

pytestmark = pytest.mark.gpu

SHIFT, SCALE = 1.0, -0.02


@pytest.fixture(scope="module")
def L():
    from paper_1204_1533_gb300 import build, ldg
    build.build()
    return ldg


def _ns(mu=0.02):
    return {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": mu, "Pr": 0.72, "bc": {1: "wall"}}


def _case(name):
    if name == "channel3d_p2":
        m = I.channel_mesh(3, 4, 3, 2)
        return m, _ns(), I.smooth_perturbation(m, I.channel_state(m), 0.02)
    if name == "ns2d_walls_p3":
        m = I.structured_mesh((3, 4), 3, (0.0, -1.0), (3.0, 1.0), (True, False), perturb=0.1,
                              btag_of_face=lambda d, end: 1)
        x, y = m["nodes"][..., 0], m["nodes"][..., 1]
        rho = 1.0 + 0.05 * np.sin(2 * math.pi * x / 3.0)
        u = (1.0 - y ** 2) * (1.0 + 0.1 * np.cos(2 * math.pi * x / 3.0))
        v = 0.05 * (1.0 - y ** 2) * np.sin(2 * math.pi * x / 3.0)
        p = np.full_like(u, 1.0 / (1.4 * 0.3 ** 2))
        U = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], axis=1)
        return m, _ns(0.05), U
    # Euler with walls: the inviscid wall (pressure flux only)
    m = I.structured_mesh((3, 3), 2, (0.0, -1.0), (3.0, 1.0), (True, False), perturb=0.1,
                          btag_of_face=lambda d, end: 1)
    U = I.smooth_perturbation(m, _euler_state(m), 0.02)
    return m, {"kind": "euler", "gamma": 1.4, "flux": "roe", "bc": {1: "wall"}}, U


def _euler_state(m):
    x, y = m["nodes"][..., 0], m["nodes"][..., 1]
    rho = 1.0 + 0.05 * np.cos(2 * math.pi * x / 3.0)
    u = 1.0 - 0.3 * y ** 2
    v = 0.02 * np.sin(math.pi * y) * np.sin(2 * math.pi * x / 3.0)
    p = 1.0 / (1.4 * 0.4 ** 2) * np.ones_like(u)
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], axis=1)


CASES = ["channel3d_p2", "ns2d_walls_p3", "euler2d_walls_p2"]


@pytest.mark.parametrize("name", CASES)
def test_walls_matvec_and_preconditioner(L, name):
    import torch
    m, eq, U = _case(name)
    disc = Discretization(m, eq)
    h = L.ldg_setup(m, eq)
    Ut = torch.from_numpy(U).cuda()
    # the residual with walls first (the oracle is its reference here too)
    R = torch.empty_like(Ut)
    L.ldg_residual(h, Ut, R)
    Ro = full_residual(disc, np.asarray(U, np.longdouble)).astype(np.float64)
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * np.abs(Ro).max()
    x = np.random.default_rng(7).standard_normal(U.shape)
    Ax = np.imag(full_residual(disc, U + 1j * H_CS * x)) / H_CS
    y_ref = SHIFT * x + SCALE * Ax
    pat = S.line_pattern(m["D"], m["p"])
    one = types.SimpleNamespace(E=1, nc=U.shape[1], npe=U.shape[2], D=m["D"], p=m["p"])
    # every element of the small cases; on the channel six elements with a wall face
    walled = np.nonzero((m["btag"] == 1).any(axis=1))[0]
    els = np.arange(disc.E) if disc.E <= 12 else np.random.default_rng(3).choice(walled, 6, replace=False)
    Fo = np.concatenate([S.ilu0(S.masked_blocks(one, diag_block(disc, U, e), SHIFT, SCALE), pat) for e in els])
    zo = S.ilu_apply(Fo, pat, x[els])
    Fo_p = np.stack([Fo[:, i, pat[i]] for i in range(disc.npe)], axis=1)
    for prec, tv, tf, ta in ((L.PREC_FP32, 1e-5, 1e-5, 1e-4), (L.PREC_FP64, 1e-11, 1e-10, 1e-10)):
        dt = torch.float32 if prec == L.PREC_FP32 else torch.float64
        xt = torch.from_numpy(x).to(dt).cuda()
        J = L.ldg_jacobian(h, Ut, prec)
        y = torch.empty_like(xt)
        L.ldg_jacvec(h, J, SHIFT, SCALE, xt, y, prec)
        P = L.ldg_precond(h, J, SHIFT, SCALE)
        z = torch.empty_like(xt)
        L.ldg_precond_apply(h, P, xt, z, prec)
        torch.cuda.synchronize()
        err_y = np.abs(y.double().cpu().numpy() - y_ref).max() / np.abs(y_ref).max()
        assert err_y <= tv, (name, prec, err_y)
        Fg = L.ldg_pc_export(P, prec).astype(np.float64)[els]
        scale_r = np.abs(Fo_p).max(axis=(2, 3, 4), keepdims=True)
        err_f = (np.abs(Fg - Fo_p) / scale_r).max()
        assert err_f <= tf, (name, prec, err_f)
        err_z = np.abs(z.double().cpu().numpy()[els] - zo).max() / np.abs(zo).max()
        assert err_z <= ta, (name, prec, err_z)


@pytest.mark.parametrize("mode", [0, 1])
def test_walls_newton_step(L, mode):
    """One BDF1 and one BDF2 level of the walled 2-D Navier-Stokes case
    against the oracle's Newton solution with its complex-step Jacobian."""
    import torch
    m, eq, U0 = _case("ns2d_walls_p3")
    disc = Discretization(m, eq)
    dt = 0.01
    F = lambda X: full_residual(disc, X)
    A = JAC.A_full(disc, U0)
    jac = lambda X: (A, None, None)         # frozen Jacobian: converges, more iterations
    U1o, _ = S.newton_bdf2(F, jac, U0, None, dt, first=True, rtol=1e-12, gmres_tol=1e-12, restart=600,
                           reuse=1000, maxit=60)
    U2o, _ = S.newton_bdf2(F, jac, U1o, U0, dt, first=False, rtol=1e-12, gmres_tol=1e-12, restart=600,
                           reuse=1000, maxit=60)
    h = L.ldg_setup(m, eq)
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    st1 = L.ldg_newton_step(h, U1, Un, None, None, dt, L.solver_opts(mode=mode, first_step=True))
    U2 = torch.empty_like(Un)
    st2 = L.ldg_newton_step(h, U2, U1, Un, None, dt, L.solver_opts(mode=mode, force_rebuild=False))
    for st in (st1, st2):
        assert st["res_final"] <= 1e-8 * st["res0"]
        assert st["newton_its"] <= 10
    d1 = np.abs(U1.cpu().numpy() - U1o).max() / np.abs(U1o).max()
    d2 = np.abs(U2.cpu().numpy() - U2o).max() / np.abs(U2o).max()
    assert d1 < 1e-7 and d2 < 1e-7, (d1, d2)
