"""The library side of a partitioned run, on one GPU: every part of a
3-way element partition, set up as its own sub-mesh (owned elements plus
two rings of ghosts, cut faces as a Dirichlet tag of their own, the global
switch function passed in), gives through ldg_residual the rows of its owned
elements of the global residual (the oracle's, in extended precision, within
the residual tolerance 1e-12; and the library's own global rows to 1e-13),
given the ghost states a halo exchange delivers (copied here from the global
state; the exchange itself is tested on CPU ranks in test_partition.py)."""
import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from paper_1204_1533_gb300 import partition as PT

pytestmark = pytest.mark.gpu

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}
NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.05, "Pr": 0.72}


@pytest.fixture(scope="module")
def L():
    from paper_1204_1533_gb300 import build, ldg
    build.build()
    return ldg


def _case(name):
    if name == "euler2d":
        m = I.vortex_mesh(6, 3)
        return m, EULER, I.smooth_perturbation(m, I.vortex_state(m, x0=5.0, y0=5.0), 0.05), 1
    if name == "ns2d_unstructured":
        m = I.unstructured_quad_mesh(3, 3, L=10.0, periodic=True, perturb=0.1)
        return m, NS, I.smooth_perturbation(m, I.vortex_state(m), 0.05, periods=[10, 10]), 2
    m = I.unstructured_hex_mesh(3, 2, L=6.283185307179586, periodic=True, perturb=0.1)
    return m, NS, I.smooth_perturbation(m, I.tgv_state(m, mach=0.3), 0.05), 2


@pytest.mark.parametrize("name", ["euler2d", "ns2d_unstructured", "ns3d_unstructured"])
def test_part_residuals_equal_global_rows(L, name):
    import torch

    from oracle.residual import Discretization, full_residual
    m, eq, U, layers = _case(name)
    E = m["nodes"].shape[0]
    Ro = full_residual(Discretization(m, eq), np.asarray(U, dtype=np.longdouble)).astype(np.float64)
    sw = L.ldg_setup_host(m, eq)["sw"]
    h = L.ldg_setup(m, eq)
    Ug = torch.from_numpy(U).cuda()
    Rg = torch.empty_like(Ug)
    L.ldg_residual(h, Ug, Rg)
    Rg = Rg.cpu().numpy()
    owner = PT.block_partition(E, 3)
    adj = PT.face_neighbours(m)
    seen = np.zeros(E, dtype=bool)
    for r in range(3):
        plan = PT.halo_plan(m, owner, r, layers, adj, switches=sw)
        hl = L.ldg_setup(plan.submesh, dict(eq, bc={**eq.get("bc", {}), plan.cut_tag: "dirichlet"}))
        Ul = torch.from_numpy(np.ascontiguousarray(U[plan.local])).cuda()
        Rl = torch.full_like(Ul, float("nan"))
        L.ldg_residual(hl, Ul, Rl)
        own = plan.local[:plan.n_owned]
        got = Rl.cpu().numpy()[:plan.n_owned]
        assert np.abs(got - Ro[own]).max() <= 1e-12 * np.abs(Ro).max()
        assert np.abs(got - Rg[own]).max() <= 1e-13 * np.abs(Rg).max()
        seen[own] = True
    assert seen.all()


@pytest.mark.parametrize("name", ["ns2d_unstructured", "ns3d_unstructured"])
@pytest.mark.parametrize("prec", [0, 1])
def test_split_product_and_jacobian_at_given_gradient(L, name, prec):
    # ldg_k21_apply then ldg_jacvec_g equals ldg_jacvec; ldg_jacobian_uq at
    # Q = D(U) is ldg_jacobian bit for bit
    import torch
    m, eq, U, _ = _case(name)
    h = L.ldg_setup(m, eq)
    Ut = torch.from_numpy(U).cuda()
    J = L.ldg_jacobian(h, Ut, prec)
    Q = torch.empty((h.E, h.nc, h.D, h.npe), dtype=torch.float64, device="cuda")
    L.ldg_gradient(h, Ut, Q)
    J2 = L.ldg_jacobian_uq(h, Ut, Q, prec)
    for a, b in zip(L.ldg_jac_export(J), L.ldg_jac_export(J2)):
        if a is not None:
            assert np.array_equal(a, b)
    dt = torch.float32 if prec == 0 else torch.float64
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(U.shape)).to(dt).cuda()
    y = torch.empty_like(x)
    L.ldg_jacvec(h, J, 1.0, -0.02, x, y, prec)
    g = torch.empty((h.E, h.nc, h.D, h.npe), dtype=dt, device="cuda")
    L.ldg_k21_apply(h, J, x, g, prec)
    y2 = torch.empty_like(x)
    L.ldg_jacvec_g(h, J, 1.0, -0.02, x, g, y2, prec)
    torch.cuda.synchronize()
    assert torch.equal(y, y2)


@pytest.mark.parametrize("name", ["euler2d", "ns2d_unstructured"])
def test_partitioned_driver_on_library_operators(L, name):
    # the partitioned BDF2 level (paper_1204_1533_gb300/partitioned_solver.py)
    # on the library's operators as one part, against ldg_newton_step in FP64
    # with the same stopping rule (the multi-part exchanges are tested on CPU
    # ranks in test_partition_krylov.py)
    import torch

    from paper_1204_1533_gb300 import partitioned_solver as PS
    m, eq, U, _ = _case(name)
    sw = L.ldg_setup_host(m, eq)["sw"]
    plan = PS.trace_plan(m, np.zeros(m["nodes"].shape[0], np.int64), 0, switches=sw)
    part = PS.Partitioned(plan, PS.LdgPartOps(plan, eq), single=True)
    dt = 0.1
    Un = torch.from_numpy(U).cuda()
    U1, st = PS.newton_bdf2(part, Un, None, dt, first=True, rtol=1e-12, gmres_tol=1e-6)
    h = L.ldg_setup(m, eq)
    Ur = torch.empty_like(Un)
    sr = L.ldg_newton_step(h, Ur, Un, None, None, dt, L.solver_opts(mode=L.MODE_FP64, first_step=True, rtol=1e-12,
                                                                    gmres_tol=1e-6))
    assert st["res_final"] <= 1e-12 * st["res0"] and sr["res_final"] <= 1e-12 * sr["res0"]
    assert float((U1 - Ur).abs().max()) <= 1e-10 * float(Ur.abs().max())
