"""GPU parity of the line-sparse Jacobian (K11, K12, K21), the split
Jacobian-vector product, the element-block ILU(0) preconditioner and the
Newton-BDF2 step against the oracle (complex-step Jacobians, textbook
ILU(0) and GMRES). Tolerances: 1e-5 relative per block row for FP32 values
(the stated FP32 Jacobian/preconditioner bound), 1e-11 for the FP64 build;
integer structure bit-exact."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1204_1533_gb300 import inputs as I
from oracle import jacobian as JAC
from oracle import solvers as S
from oracle.mesh import line_nodes
from oracle.residual import Discretization, full_residual, gradient

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1204_1533_gb300 import build, ldg
    build.build()
    return ldg


def ns(mu=0.05):
    return {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": mu, "Pr": 0.72}


EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}


def _fs(m, nc, v=(0.5, -0.2, 0.3), p=2.0):
    D = m["D"]
    E, npe = m["nodes"].shape[:2]
    U = np.zeros((E, nc, npe))
    U[:, 0] = 1.0
    for a in range(D):
        U[:, 1 + a] = v[a]
    U[:, D + 1] = p / 0.4 + 0.5 * sum(x * x for x in v[:D])
    return U


def _case(name):
    if name == "euler2d_p3":
        m = I.reorient(I.vortex_mesh(4, 3, perturb=0.15))[0]
        return m, EULER, I.smooth_perturbation(m, I.vortex_state(m), 0.05, periods=[10, 10]), None
    if name == "lf2d_p2":
        m = I.vortex_mesh(3, 2, perturb=0.15)
        return m, dict(EULER, flux="lf"), I.smooth_perturbation(m, I.vortex_state(m), 0.05), None
    if name == "ns2d_p2":
        m = I.reorient(I.structured_mesh((3, 3), 2, (0, 0), (1, 1), (True, True), perturb=0.1))[0]
        return m, ns(), I.smooth_perturbation(m, _fs(m, 4), 0.1, periods=[1, 1]), None
    if name == "ns3d_p2":
        m = I.structured_mesh((3, 3, 3), 2, (0,) * 3, (2 * math.pi,) * 3, (True,) * 3, perturb=0.1)
        return m, ns(0.02), I.smooth_perturbation(m, I.tgv_state(m, mach=0.3), 0.05), None
    if name == "poisson_p3":
        m = I.poisson_square_mesh(4, 3)
        gD = np.zeros((16, 1, 16))
        eq = {"kind": "poisson", "bc": {0: "dirichlet"}, "gD": gD, "source": I.poisson_source(m)}
        return m, eq, I.poisson_exact(m) + 0.1, gD
    if name == "unstructured_ns2d_p2":
        m = I.unstructured_quad_mesh(3, 2, periodic=True, perturb=0.1)
        return m, ns(), I.smooth_perturbation(m, _fs(m, 4), 0.1, periods=[1, 1]), None
    if name == "unstructured_euler3d_p2_farfield":
        m = I.unstructured_hex_mesh(1, 2)
        g = _fs(m, 5)
        return m, dict(EULER, bc={0: "dirichlet"}, gD=g), I.smooth_perturbation(m, g, 0.05, periods=[1, 1, 1]), g
    if name == "poisson_neumann_p3":
        m = I.reorient(I.structured_mesh((4, 4), 3, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=0.15,
                                         btag_of_face=lambda d, end: 1 if end == 1 else 0))[0]
        gD = np.zeros((16, 1, 16))
        eq = {"kind": "poisson", "bc": {0: "dirichlet", 1: "neumann"}, "gD": gD, "source": I.poisson_source(m),
              "gN": -I.poisson_exact_grad(m)}
        return m, eq, I.poisson_exact(m) + 0.1, gD
    if name == "ns2d_neumann_p2":
        m = I.reorient(I.structured_mesh((3, 3), 2, (0.0, 0.0), (1.0, 1.0), (True, False), perturb=0.1,
                                         btag_of_face=lambda d, end: 1 if end == 1 else 0))[0]
        g = _fs(m, 4)
        eq = dict(ns(), bc={0: "dirichlet", 1: "neumann"}, gD=g, gN=I.random_state((9, 4, 2, 9), seed=8))
        return m, eq, I.smooth_perturbation(m, g, 0.1, periods=[1, 1]), g
    raise KeyError(name)


def _oeq(eq):
    o = {k: v for k, v in eq.items() if k not in ("gD", "source")}
    o.setdefault("bc", {0: "dirichlet"})
    return o


def _sparse_from_export(disc, K11, K12, K21):
    """Scatter the library's line-block arrays into sparse matrices with the
    oracle's flat index conventions (layout documented in include/ldg.h)."""
    D, p, nc, npe, nl, E = disc.D, disc.p, disc.nc, disc.npe, disc.nl, disc.E
    n = p + 1
    nbr, sw = disc.conn.nbr, disc.S
    r11, c11, v11, r12, c12, v12, r21, c21, v21 = ([] for _ in range(9))
    for e in range(E):
        for d in range(D):
            for l in range(nl):
                Lx = (e * D + d) * nl + l
                ln = line_nodes(D, p, d, l)
                for i in range(n):
                    for c in range(nc):
                        row = (e * nc + c) * npe + ln[i]
                        for j in range(n):
                            for cp in range(nc):
                                r11.append(row)
                                c11.append((e * nc + cp) * npe + ln[j])
                                v11.append(K11[((i * n + j) * nc + c) * nc + cp, Lx])
                        for end in range(2):
                            g = nbr[e, d, l, end]
                            if g < 0:
                                continue
                            eo, ao = divmod(int(g), npe)
                            for cp in range(nc):
                                r11.append(row)
                                c11.append((eo * nc + cp) * npe + ao)
                                v11.append(K11[n * n * nc * nc + ((end * n + i) * nc + c) * nc + cp, Lx])
                        if K12 is None:
                            continue
                        ncd = nc * D
                        for j in range(n):
                            for cp in range(nc):
                                for b in range(D):
                                    r12.append(row)
                                    c12.append(((e * nc + cp) * D + b) * npe + ln[j])
                                    v12.append(K12[((i * n + j) * nc + c) * ncd + cp * D + b, Lx])
                        for end in range(2):
                            g = nbr[e, d, l, end]
                            if g < 0 or sw[e, d, end] != 1:
                                continue
                            eo, ao = divmod(int(g), npe)
                            for cp in range(nc):
                                for b in range(D):
                                    r12.append(row)
                                    c12.append(((eo * nc + cp) * D + b) * npe + ao)
                                    v12.append(K12[n * n * nc * ncd + (i * nc + c) * ncd + cp * D + b, Lx])
                    if K21 is None:
                        continue
                    for c in range(nc):
                        for b in range(D):
                            row = ((e * nc + c) * D + b) * npe + ln[i]
                            for j in range(n):
                                r21.append(row)
                                c21.append((e * nc + c) * npe + ln[j])
                                v21.append(K21[(i * n + j) * D + b, Lx])
                            for end in range(2):
                                g = nbr[e, d, l, end]
                                if g < 0 or sw[e, d, end] != -1:
                                    continue
                                eo, ao = divmod(int(g), npe)
                                r21.append(row)
                                c21.append((eo * nc + c) * npe + ao)
                                v21.append(K21[n * n * D + i * D + b, Lx])
    N, NQ = E * nc * npe, E * nc * D * npe
    out = [sp.csr_matrix((np.array(v11, np.float64), (r11, c11)), shape=(N, N))]
    if K12 is not None:
        out.append(sp.csr_matrix((np.array(v12, np.float64), (r12, c12)), shape=(N, NQ)))
        out.append(sp.csr_matrix((np.array(v21, np.float64), (r21, c21)), shape=(NQ, N)))
    else:
        out += [None, None]
    return out


def _row_rel(A, B):
    """max over rows of max|A_r - B_r| / max|B_r| (rows with B_r = 0 use 1)."""
    A, B = sp.csr_matrix(A), sp.csr_matrix(B)
    Dm = abs(A - B).max(axis=1).toarray().ravel()
    Bm = abs(B).max(axis=1).toarray().ravel()
    Bm[Bm == 0] = 1.0
    return float((Dm / Bm).max())


def _gpu_jac(L, h, U, prec):
    import torch
    Ut = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    J = L.ldg_jacobian(h, Ut, prec)
    torch.cuda.synchronize()
    return J


@pytest.mark.parametrize("name", ["euler2d_p3", "lf2d_p2", "ns2d_p2", "ns3d_p2", "poisson_p3",
                                  "unstructured_ns2d_p2", "unstructured_euler3d_p2_farfield",
                                  "poisson_neumann_p3", "ns2d_neumann_p2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_jacobian_matches_complex_step(L, name, prec):
    m, eq, U, gD = _case(name)
    disc = Discretization(m, _oeq(eq))
    Q = gradient(disc, U, gD) if disc.eq["kind"] in ("ns", "poisson") else None
    src = eq.get("source")
    h = L.ldg_setup(m, eq)
    J = _gpu_jac(L, h, U, prec)
    K11, K12, K21 = _sparse_from_export(disc, *L.ldg_jac_export(J))
    tol = 1e-5 if prec == 0 else 1e-11
    assert _row_rel(K11, JAC.K11(disc, U, Q, gD, src)) < tol
    if K12 is not None:
        assert _row_rel(K12, JAC.K12(disc, U, Q, gD, src)) < tol
        assert _row_rel(K21, JAC.K21(disc, gD)) < tol


def test_line_block_row_counts(L):
    # structural: every K11 row of the line-block format stores D(p+1) n_c
    # in-line entries (diagonal once per direction) plus 2 D n_c face entries
    m, eq, U, _ = _case("ns3d_p2")
    h = L.ldg_setup(m, eq)
    J = _gpu_jac(L, h, U, 0)
    K11, K12, K21 = L.ldg_jac_export(J)
    n, nc, D = 3, 5, 3
    assert K11.shape[0] == (n * n + 2 * n) * nc * nc
    per_row = (D * n * nc + 2 * D * nc)
    assert K11.shape[0] * K11.shape[1] == h.ndof * per_row


@pytest.mark.parametrize("name", ["euler2d_p3", "ns2d_p2", "ns3d_p2", "poisson_p3", "unstructured_ns2d_p2",
                                  "unstructured_euler3d_p2_farfield", "poisson_neumann_p3", "ns2d_neumann_p2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_split_jacvec(L, name, prec):
    import torch
    m, eq, U, gD = _case(name)
    disc = Discretization(m, _oeq(eq))
    Q = gradient(disc, U, gD) if disc.eq["kind"] in ("ns", "poisson") else None
    K11o = JAC.K11(disc, U, Q, gD)
    K12o = JAC.K12(disc, U, Q, gD) if Q is not None else None
    K21o = JAC.K21(disc, gD) if Q is not None else None
    x = np.random.default_rng(7).standard_normal(U.size)
    shift, scale = 1.0, -0.37
    yo = S.split_matvec(K11o, K12o, K21o, x, shift, scale)
    h = L.ldg_setup(m, eq)
    J = _gpu_jac(L, h, U, prec)
    dt = torch.float32 if prec == 0 else torch.float64
    xt = torch.from_numpy(x).to(dt).cuda()
    y = torch.empty_like(xt)
    L.ldg_jacvec(h, J, shift, scale, xt, y, prec)
    torch.cuda.synchronize()
    err = np.abs(y.double().cpu().numpy() - yo).max() / np.abs(yo).max()
    assert err < (2e-5 if prec == 0 else 1e-11), err
    if prec == 0:
        # FP64 vectors against the FP32 matrix (the refinement residual)
        y64 = torch.empty(x.size, dtype=torch.float64, device="cuda")
        L.ldg_jacvec(h, J, shift, scale, torch.from_numpy(x).cuda(), y64, 1)
        assert np.abs(y64.cpu().numpy() - yo).max() / np.abs(yo).max() < 2e-5


@pytest.mark.parametrize("name", ["euler2d_p3", "ns2d_p2", "ns3d_p2", "poisson_p3", "unstructured_ns2d_p2",
                                  "unstructured_euler3d_p2_farfield", "poisson_neumann_p3", "ns2d_neumann_p2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_preconditioner_factors_and_apply(L, name, prec):
    import torch
    m, eq, U, gD = _case(name)
    disc = Discretization(m, _oeq(eq))
    Q = gradient(disc, U, gD) if disc.eq["kind"] in ("ns", "poisson") else None
    A = JAC.K11(disc, U, Q, gD)
    if Q is not None:
        A = A + JAC.K12(disc, U, Q, gD) @ JAC.K21(disc, gD)
    shift, scale = 1.0, -0.3
    pat = S.line_pattern(disc.D, disc.p)
    Fo = S.ilu0(S.masked_blocks(disc, A, shift, scale), pat)
    h = L.ldg_setup(m, eq)
    J = _gpu_jac(L, h, U, prec)
    P = L.ldg_precond(h, J, shift, scale)
    Fg = L.ldg_pc_export(P, prec).astype(np.float64)
    # scatter the oracle's dense element blocks into the pattern layout
    Fo_p = np.stack([Fo[:, i, pat[i]] for i in range(disc.npe)], axis=1)
    tol = 1e-5 if prec == 0 else 1e-10
    scale_r = np.abs(Fo_p).max(axis=(2, 3, 4), keepdims=True)
    assert (np.abs(Fg - Fo_p) / scale_r).max() < tol
    r = np.random.default_rng(3).standard_normal(U.shape)
    zo = S.ilu_apply(Fo, pat, r)
    dt = torch.float32 if prec == 0 else torch.float64
    rt = torch.from_numpy(r).to(dt).cuda()
    z = torch.empty_like(rt)
    L.ldg_precond_apply(h, P, rt, z, prec)
    torch.cuda.synchronize()
    zg = z.double().cpu().numpy()
    # end to end against the FP64 factors: the triangular solves amplify the
    # factors' FP32 rounding (1e-5 above), hence 1e-4 here
    assert np.abs(zg - zo).max() / np.abs(zo).max() < (1e-4 if prec == 0 else 1e-10)
    # the apply alone: the oracle's triangular solves in FP64 on the GPU's own
    # factors and the rounded input, so only the apply's own arithmetic differs
    Fd = np.zeros_like(Fo)
    for i in range(disc.npe):
        Fd[:, i, pat[i]] = Fg[:, i]
    zr = S.ilu_apply(Fd, pat, rt.double().cpu().numpy())
    assert np.abs(zg - zr).max() / np.abs(zr).max() < (1e-5 if prec == 0 else 1e-12)


@pytest.mark.parametrize("ortho", ["cgs2", "selective", "selective_always"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", ["euler2d_p3", "ns2d_p2", "unstructured_ns2d_p2"])
def test_newton_bdf2_step(L, mode, name, ortho):
    """One BDF1 then one BDF2 level to ||G|| <= 1e-8 ||G(U^n)||, compared with
    the oracle's Newton solution of the same stage equation solved to 1e-12,
    with CGS2 (every Arnoldi column orthogonalised twice), with the selective
    second pass (at most as many second passes as columns), and with the
    selective scheme's criterion factor 1, which sends every column through
    the not-accepted branch (a skipped update sweep, then the second pass)."""
    import torch
    m, eq, U0, _ = _case(name)
    disc = Discretization(m, _oeq(eq))
    dt = 0.05 if name.startswith("euler") else 0.01
    F = lambda X: full_residual(disc, X)

    def jac(X):
        if disc.eq["kind"] == "ns":
            Qx = gradient(disc, X)
            return JAC.K11(disc, X, Qx), JAC.K12(disc, X, Qx), JAC.K21(disc)
        return JAC.K11(disc, X), None, None
    U1o, _ = S.newton_bdf2(F, jac, U0, None, dt, first=True, rtol=1e-12, gmres_tol=1e-10, restart=400, reuse=1)
    U2o, _ = S.newton_bdf2(F, jac, U1o, U0, dt, first=False, rtol=1e-12, gmres_tol=1e-10, restart=400, reuse=1)
    h = L.ldg_setup(m, eq)
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    oo = {"ortho": L.ORTHO_CGS2 if ortho == "cgs2" else L.ORTHO_SELECTIVE,
          "reorth_factor": 1.0 if ortho == "selective_always" else 0.0}
    st1 = L.ldg_newton_step(h, U1, Un, None, None, dt, L.solver_opts(mode=mode, first_step=True, **oo))
    U2 = torch.empty_like(Un)
    st2 = L.ldg_newton_step(h, U2, U1, Un, None, dt, L.solver_opts(mode=mode, force_rebuild=False, **oo))
    for st in (st1, st2):
        assert st["res_final"] <= 1e-8 * st["res0"]
        assert st["newton_its"] <= 10
        if ortho == "selective":
            assert 0 <= st["reorth_its"] <= st["gmres_its"]
        else:
            assert st["reorth_its"] == st["gmres_its"]
    d1 = np.abs(U1.cpu().numpy() - U1o).max() / np.abs(U1o).max()
    d2 = np.abs(U2.cpu().numpy() - U2o).max() / np.abs(U2o).max()
    assert d1 < 1e-7 and d2 < 1e-7, (d1, d2)


def _oracle_newton_parts(disc):
    F = lambda X: full_residual(disc, X)

    def jac(X):
        if disc.eq["kind"] == "ns":
            Qx = gradient(disc, X)
            return JAC.K11(disc, X, Qx), JAC.K12(disc, X, Qx), JAC.K21(disc)
        return JAC.K11(disc, X), None, None
    return F, jac


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", ["euler2d_p3", "ns2d_p2"])
def test_dirk3_step(L, mode, name):
    """One step of the paper's three-stage DIRK (Sec. 4.1) against the
    oracle's DIRK3 with every stage solved to 1e-12."""
    import torch
    m, eq, U0, _ = _case(name)
    disc = Discretization(m, _oeq(eq))
    dt = 0.05 if name.startswith("euler") else 0.01
    F, jac = _oracle_newton_parts(disc)
    Uo, _ = S.dirk3_step(F, jac, U0, dt, rtol=1e-12, gmres_tol=1e-10, restart=400, reuse=1)
    h = L.ldg_setup(m, eq)
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    st = L.ldg_dirk3_step(h, U1, Un, dt, L.solver_opts(mode=mode))
    assert st["res_final"] <= 1e-8 * st["res0"]
    assert st["newton_its"] <= 30
    d = np.abs(U1.cpu().numpy() - Uo).max() / np.abs(Uo).max()
    assert d < 1e-7, d


def test_dirk3_paper_policy(L):
    """The paper's Newton policy (five GMRES iterations per Newton step,
    Jacobian re-use until more than 15 Newton iterations) reaches the same
    levels as the default solver over two DIRK3 steps."""
    import torch
    m, eq, U0, _ = _case("euler2d_p3")
    h = L.ldg_setup(m, eq)
    out = {}
    for name, opts in (("default", L.solver_opts(mode=0)), ("paper", L.paper_policy_opts(mode=0))):
        U = torch.from_numpy(U0).cuda()
        for _ in range(2):
            Un, U = U, torch.empty_like(U)
            st = L.ldg_dirk3_step(h, U, Un, 0.05, opts)
            assert st["res_final"] <= 1e-8 * st["res0"], (name, st)
            if name == "paper":
                assert st["gmres_its"] == 5 * st["newton_its"]
        out[name] = U.cpu().numpy()
    assert np.abs(out["paper"] - out["default"]).max() <= 1e-7 * np.abs(out["default"]).max()


@pytest.mark.parametrize("name", ["euler2d_p3", "ns2d_p2"])
def test_rk4_step(L, name):
    """The explicit RK4 step against the oracle's (FP64 residuals only)."""
    import torch
    m, eq, U0, _ = _case(name)
    disc = Discretization(m, _oeq(eq))
    dt = 1e-3
    Uo = S.rk4_step(lambda X: full_residual(disc, X), U0, dt)
    h = L.ldg_setup(m, eq)
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    L.ldg_rk4_step(h, U1, Un, dt)
    L.ldg_rk4_step(h, Un, Un, dt)            # in place gives the same level
    torch.cuda.synchronize()
    assert np.array_equal(U1.cpu().numpy(), Un.cpu().numpy())
    # each stage adds dt times a residual that matches the oracle to 1e-12
    # of its scale
    Rmax = np.abs(full_residual(disc, U0)).max()
    assert np.abs(U1.cpu().numpy() - Uo).max() <= 1e-12 * dt * Rmax * 4 + 1e-15 * np.abs(Uo).max()


def test_rk4_vortex_convergence_on_gpu(L):
    """The paper's explicit vortex study on the GPU residual: RK4 to t = 0.5
    against the exact translated vortex on 16^2 and 32^2 elements, p = 3;
    halving h divides the error by close to 2^(p+1)."""
    import torch
    errs = []
    for n in (16, 32):
        m = I.vortex_mesh(n, 3, perturb=0.0)
        h = L.ldg_setup(m, EULER)
        U = torch.from_numpy(I.vortex_state(m)).cuda()
        T, steps = 0.5, 25 * n
        for _ in range(steps):
            L.ldg_rk4_step(h, U, U, T / steps)
        exact = I.vortex_state(m, t=T)
        errs.append(np.abs(U.cpu().numpy() - exact).max())
    rate = math.log2(errs[0] / errs[1])
    assert rate > 3.7, (errs, rate)      # the oracle's run of this study gives 4.1


@pytest.mark.parametrize("mode", [0, 1])
def test_poisson_steady_solve_and_rates(L, mode):
    """The Poisson workload on the GPU: -lap u = f on the perturbed unit square,
    p = 3, solved by the steady driver (one step without the time
    derivative); the solution matches the oracle's direct solve, and the
    error falls at the rate of the paper's Table 2 (p + 1)."""
    import scipy.sparse.linalg as spla
    import torch
    errs = []
    for n in (4, 8, 16):
        m = I.poisson_square_mesh(n, 3)
        f = I.poisson_source(m)
        gD = np.zeros_like(f)
        eq = {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}, "gD": gD, "source": f}
        h = L.ldg_setup(m, eq)
        U = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        st = L.ldg_steady_solve(h, U, 1.0, 1.0, 0, L.solver_opts(mode=mode, rtol=1e-12, max_newton=20))
        assert st["res_final"] <= 1e-12 * st["res0"]
        Ug = U.cpu().numpy()
        errs.append(np.abs(Ug - I.poisson_exact(m)).max())
        if n == 4:
            disc = Discretization(m, {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}})
            A = JAC.A_full(disc, np.zeros_like(f), gD, f)
            Uo = spla.spsolve(A.tocsc(), -full_residual(disc, np.zeros_like(f), gD, f).ravel()).reshape(f.shape)
            assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    gold = np.loadtxt(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                                 "poisson_rates.txt"), comments="#")
    rate = math.log2(errs[1] / errs[2])
    assert abs(rate - gold[2][3]) < 0.6, (errs, rate)       # p = 3, last refinement: 4.0


@pytest.mark.parametrize("mode", [0, 1])
def test_poisson_solve_on_refined_unstructured_mesh(L, mode):
    """The paper's Poisson setting (Sec. 5.1): an unstructured quadrilateral
    mesh refined uniformly, p = 3, solved on the GPU; the solution matches
    the oracle's direct solve on the once-refined mesh, and the error falls at
    the u-rate of Table 2 (p + 1). On the twice-refined mesh restarted
    GMRES(30) with the element-block ILU(0) stagnates (the oracle's GMRES as
    well: the relative residual stays at 0.79), so the solve uses GMRES(64),
    and its target there is 1e-10: rounding keeps the oracle's own Krylov
    solve near 2e-12."""
    import scipy.sparse.linalg as spla
    import torch
    errs = []
    for refine in (0, 1, 2):
        m = I.unstructured_quad_mesh(2, 3, perturb=0.15, refine=refine)
        f = I.poisson_source(m)
        gD = np.zeros_like(f)
        eq = {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}, "gD": gD, "source": f}
        h = L.ldg_setup(m, eq)
        U = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        rtol = 1e-12 if refine < 2 else 1e-10
        st = L.ldg_steady_solve(h, U, 1.0, 1.0, 0, L.solver_opts(mode=mode, rtol=rtol, max_newton=30, restart=64))
        assert st["res_final"] <= rtol * st["res0"]
        Ug = U.cpu().numpy()
        errs.append(np.abs(Ug - I.poisson_exact(m)).max())
        if refine == 1:
            disc = Discretization(m, {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet"}})
            A = JAC.A_full(disc, np.zeros_like(f), gD, f)
            Uo = spla.spsolve(A.tocsc(), -full_residual(disc, np.zeros_like(f), gD, f).ravel()).reshape(f.shape)
            assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    rate = math.log2(errs[1] / errs[2])
    assert abs(rate - 4.0) < 0.6, (errs, rate)


@pytest.mark.parametrize("mode", [0, 1])
def test_poisson_solve_mixed_dirichlet_neumann(L, mode):
    """Neumann sides (Eqs. 29-30) on the GPU: -lap u = f on the perturbed
    unit square, p = 3, Dirichlet on x = 0 and y = 0, the flux of the
    manufactured solution prescribed on x = 1 and y = 1; the solution matches
    the oracle's direct solve and converges at about p + 1."""
    import scipy.sparse.linalg as spla
    import torch
    errs = []
    for n in (4, 8, 16):
        m = I.structured_mesh((n, n), 3, (0.0, 0.0), (1.0, 1.0), (False, False), perturb=0.15,
                              btag_of_face=lambda d, end: 1 if end == 1 else 0)
        f = I.poisson_source(m)
        gD = np.zeros_like(f)
        gN = -I.poisson_exact_grad(m)
        eq = {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet", 1: "neumann"}, "gD": gD, "source": f,
              "gN": gN}
        h = L.ldg_setup(m, eq)
        U = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
        st = L.ldg_steady_solve(h, U, 1.0, 1.0, 0, L.solver_opts(mode=mode, rtol=1e-12, max_newton=30, restart=64))
        assert st["res_final"] <= 1e-12 * st["res0"]
        Ug = U.cpu().numpy()
        errs.append(np.abs(Ug - I.poisson_exact(m)).max())
        if n == 4:
            disc = Discretization(m, {"kind": "poisson", "C11b": 1.0, "bc": {0: "dirichlet", 1: "neumann"},
                                      "gN": gN})
            A = JAC.A_full(disc, np.zeros_like(f), gD, f)
            Uo = spla.spsolve(A.tocsc(), -full_residual(disc, np.zeros_like(f), gD, f).ravel()).reshape(f.shape)
            assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    rate = math.log2(errs[1] / errs[2])
    assert abs(rate - 4.0) < 0.6, (errs, rate)


def test_steady_continuation_euler(L):
    """Pseudo-time continuation on a compressible case: a perturbed uniform
    flow in a box whose boundary data is that uniform flow; backward Euler
    with growing steps, then the step without the time derivative, drive the
    residual to the target and the state to the uniform flow."""
    import torch
    m = I.structured_mesh((4, 4), 2, (0.0, 0.0), (4.0, 4.0), (False, False), perturb=0.1)
    g = I.vortex_state(m, eps=0.0)
    eq = dict(EULER, bc={0: "dirichlet"}, gD=g)
    h = L.ldg_setup(m, eq)
    U = torch.from_numpy(I.smooth_perturbation(m, g, 0.02, periods=[4, 4])).cuda()
    R = torch.empty_like(U)
    L.ldg_residual(h, U, R)
    r0 = float(R.abs().max())
    # dt 0.1 .. 25.6 then the step without the time derivative (beyond
    # dt ~ 50 the backward Euler Newton stalls here, in the oracle too)
    st = L.ldg_steady_solve(h, U, 0.1, 2.0, 9, L.solver_opts(mode=0, max_newton=50))
    assert st["res_final"] <= 1e-8 * st["res0"], st
    L.ldg_residual(h, U, R)
    assert float(R.abs().max()) <= 1e-6 * r0, (r0, float(R.abs().max()), st)
    assert float((U - torch.from_numpy(g).cuda()).abs().max()) <= 1e-6 * float(np.abs(g).max())
