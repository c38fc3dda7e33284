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
