"""The partitioned residual on CPU ranks (gloo): element partition, ghost
rings, halo exchange, and the global norm by one all-reduce
(paper_1204_1533_gb300/partition.py). The local residual of each rank's
sub-mesh is the oracle's here (on a GPU it is the library's); the owned rows
must equal the global residual, and an explicit RK4 step (Sec. 4.1) taken
rank by rank must equal the global one."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from paper_1204_1533_gb300 import partition as PT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}
NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.05, "Pr": 0.72}


def _case(name):
    if name == "euler2d":
        m = I.vortex_mesh(6, 2)
        return m, EULER, I.smooth_perturbation(m, I.vortex_state(m, x0=5.0, y0=5.0), 0.05), 1
    if name == "ns2d_unstructured":
        m = I.unstructured_quad_mesh(3, 2, L=10.0, periodic=True, perturb=0.1)
        return m, NS, I.smooth_perturbation(m, I.vortex_state(m), 0.05, periods=[10, 10]), 2
    m = I.tgv_mesh(4, 2)
    return m, NS, I.smooth_perturbation(m, I.tgv_state(m, mach=0.3), 0.05), 2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1204_1533_gb300 import build
    build.build()


def test_given_switches_are_used_and_checked():
    # a part of an unstructured mesh derives switches that differ from the
    # global ones; given the global ones, the set-up takes them
    from paper_1204_1533_gb300 import ldg
    m, eq, _, _ = _case("ns2d_unstructured")
    sw = ldg.ldg_setup_host(m, eq)["sw"]
    owner = PT.block_partition(m["nodes"].shape[0], 2)
    differs = False
    for r in range(2):
        plan = PT.halo_plan(m, owner, r, 2, switches=sw)
        eqs = dict(eq, bc={plan.cut_tag: "dirichlet"})
        assert np.array_equal(ldg.ldg_setup_host(plan.submesh, eqs)["sw"], sw[plan.local])
        derived = ldg.ldg_setup_host(dict(plan.submesh, switches=None), eqs)["sw"]
        differs |= not np.array_equal(derived, sw[plan.local])
    assert differs
    bad = plan.submesh["switches"].copy()
    bad[0, 0, :] *= -1
    with pytest.raises(ldg.LdgError) as e:
        ldg.ldg_setup_host(dict(plan.submesh, switches=bad), eqs)
    assert e.value.code == -3


def test_plans_are_consistent():
    m, _, _, _ = _case("ns2d_unstructured")
    E = m["nodes"].shape[0]
    owner = PT.block_partition(E, 3)
    adj = PT.face_neighbours(m)
    plans = [PT.halo_plan(m, owner, r, 2, adj) for r in range(3)]
    owned = np.concatenate([p.local[:p.n_owned] for p in plans])
    assert sorted(owned.tolist()) == list(range(E))
    for a in plans:
        for b in plans:
            if a.rank == b.rank:
                continue
            sent = a.local[a.send.get(b.rank, [])].tolist()
            got = b.local[b.recv.get(a.rank, [])].tolist()
            assert sent == got
        # ghosts within two face steps of the owned set, cut faces tagged
        assert (a.submesh["btag"] == a.cut_tag).any()


def _local_residual(plan, eq):
    from oracle.residual import Discretization, full_residual
    disc = Discretization(plan.submesh, dict(eq, bc={plan.cut_tag: "dirichlet"}))
    disc.S = plan.submesh["switches"]      # the global switch function (Sec. 3)
    gD = np.zeros((len(plan.local), disc.nc, disc.npe))

    def f(U_local):
        import torch
        return torch.from_numpy(full_residual(disc, U_local.numpy(), gD))
    return f


def _worker(rank, ws, port, name, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    from oracle.residual import Discretization
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        m, eq, U, layers = _case(name)
        sw = Discretization(m, eq).S               # the oracle's global switch function
        owner = PT.block_partition(m["nodes"].shape[0], ws)
        plan = PT.halo_plan(m, owner, rank, layers, switches=sw)
        res = _local_residual(plan, eq)
        Uo = torch.from_numpy(U[plan.local[:plan.n_owned]].copy())
        R = PT.partitioned_residual(Uo, plan, res)
        nrm = PT.global_norm(R)
        # explicit RK4 step, every stage a partitioned residual
        dt = 1e-3
        K1 = R
        K2 = PT.partitioned_residual(Uo + 0.5 * dt * K1, plan, res)
        K3 = PT.partitioned_residual(Uo + 0.5 * dt * K2, plan, res)
        K4 = PT.partitioned_residual(Uo + dt * K3, plan, res)
        U1 = Uo + dt / 6.0 * (K1 + 2.0 * K2 + 2.0 * K3 + K4)
        q.put((rank, plan.local[:plan.n_owned], R.numpy(), nrm, U1.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name,ws", [("euler2d", 2), ("ns2d_unstructured", 2), ("ns3d", 2),
                                     ("ns2d_unstructured", 3)])
def test_partitioned_residual_and_rk4_step_equal_global(name, ws):
    import torch.multiprocessing as mp

    from oracle.residual import Discretization, full_residual
    from oracle.solvers import rk4_step
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, name, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, eq, U, _ = _case(name)
    disc = Discretization(m, eq)
    Rg = full_residual(disc, U)
    U1g = rk4_step(lambda X: full_residual(disc, X), U, 1e-3)
    R = np.zeros_like(Rg)
    U1 = np.zeros_like(U)
    for rank, ids, Rr, nrm, U1r in out:
        R[ids] = Rr
        U1[ids] = U1r
        assert nrm == pytest.approx(np.linalg.norm(Rg), rel=1e-12)
    assert np.abs(R - Rg).max() <= 1e-13 * np.abs(Rg).max()
    assert np.abs(U1 - U1g).max() <= 1e-13 * np.abs(U1g).max()
