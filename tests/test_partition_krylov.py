"""The partitioned BDF2 Newton-GMRES level on CPU ranks (gloo):
face-node trace exchanges of U and Q for the residual, of x and K21 x for
the split matvec (Eq. 41), element-local block ILU(0) (Sec. 4.2), and
all-reduced Gram-Schmidt dots and Newton norms
(paper_1204_1533_gb300/partitioned_solver.py). Each part's local operators
are the oracle's here (on a GPU they are the library's); the partitioned
level must equal the single-part one."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from paper_1204_1533_gb300 import partition as PT
from paper_1204_1533_gb300 import partitioned_solver as PS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}
NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.05, "Pr": 0.72}


def _case(name):
    if name == "euler2d":
        m = I.vortex_mesh(6, 2)
        return m, EULER, I.smooth_perturbation(m, I.vortex_state(m, x0=5.0, y0=5.0), 0.05), 0.2
    m = I.unstructured_quad_mesh(3, 2, L=10.0, periodic=True, perturb=0.1)
    return m, NS, I.smooth_perturbation(m, I.vortex_state(m), 0.05, periods=[10, 10]), 0.1


class OracleOps:
    """A part's local operators from the oracle (CPU tensors, FP64)."""

    def __init__(self, plan, eq):
        from oracle import solvers as S
        from oracle.residual import Discretization
        self.disc = Discretization(plan.submesh, dict(eq, bc={plan.cut_tag: "dirichlet"}))
        self.disc.S = plan.submesh["switches"]          # the global switch function
        self.viscous = eq["kind"] in ("ns", "poisson")
        self.gD = np.zeros((len(plan.local), self.disc.nc, self.disc.npe))
        self.pat = S.line_pattern(self.disc.D, self.disc.p)

    def gradient(self, U):
        import torch

        from oracle.residual import gradient
        return torch.from_numpy(gradient(self.disc, U.numpy(), self.gD))

    def residual(self, U, Q):
        import torch

        from oracle.residual import full_residual, residual
        if self.viscous:
            return torch.from_numpy(residual(self.disc, U.numpy(), Q.numpy(), self.gD))
        return torch.from_numpy(full_residual(self.disc, U.numpy(), self.gD))

    def jacobian(self, U, Q):
        from oracle import jacobian as JAC
        with np.errstate(all="ignore"):
            self.K11 = JAC.K11(self.disc, U.numpy(), None if Q is None else Q.numpy(), self.gD)
            if self.viscous:
                self.K12 = JAC.K12(self.disc, U.numpy(), Q.numpy(), self.gD)
                self.K21 = JAC.K21(self.disc, self.gD)

    def precond(self, shift, scale):
        from oracle import solvers as S
        A = self.K11 + self.K12 @ self.K21 if self.viscous else self.K11
        with np.errstate(all="ignore"):
            self.F = S.ilu0(S.masked_blocks(self.disc, A, shift, scale), self.pat)

    def k21(self, x):
        import torch
        d = self.disc
        return torch.from_numpy((self.K21 @ x.numpy().ravel()).reshape(x.shape[0], d.nc, d.D, d.npe))

    def jacvec_g(self, shift, scale, x, g):
        import torch
        Ax = self.K11 @ x.numpy().ravel()
        if self.viscous:
            Ax = Ax + self.K12 @ g.numpy().ravel()
        return torch.from_numpy(shift * x.numpy() + scale * Ax.reshape(x.shape))

    def apply(self, r):
        import torch

        from oracle import solvers as S
        with np.errstate(all="ignore"):
            return torch.from_numpy(S.ilu_apply(self.F, self.pat, r.numpy()))


def _level(part, U, dt):
    """Two levels: BDF1 from U, then BDF2."""
    import torch
    Un = torch.from_numpy(U.copy())
    U1, s1 = PS.newton_bdf2(part, Un, None, dt, first=True, rtol=1e-12, gmres_tol=1e-6)
    U2, s2 = PS.newton_bdf2(part, U1, Un, dt, first=False, rtol=1e-12, gmres_tol=1e-6)
    return U2.numpy(), (s1, s2)


def _worker(rank, ws, port, name, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle.residual import Discretization
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        m, eq, U, dt = _case(name)
        sw = Discretization(m, eq).S
        owner = PT.block_partition(m["nodes"].shape[0], ws)
        plan = PS.trace_plan(m, owner, rank, switches=sw)
        part = PS.Partitioned(plan, OracleOps(plan, eq))
        U2, st = _level(part, U[plan.local[:plan.n_owned]], dt)
        q.put((rank, plan.local[:plan.n_owned], U2, st))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_trace_plans_are_consistent():
    m, _, _, _ = _case("ns2d")
    E = m["nodes"].shape[0]
    owner = PT.block_partition(E, 3)
    adj = PT.face_neighbours(m)
    plans = [PS.trace_plan(m, owner, r, adj) for r in range(3)]
    for a in plans:
        for b in plans:
            if a.rank != b.rank and b.rank in a.send:
                sent = [(int(a.local[k]), f) for k, f in a.send[b.rank]]
                got = [(int(b.local[k]), f) for k, f in b.recv[a.rank]]
                assert sent == got
                assert all(k < a.n_owned for k, _ in a.send[b.rank])
                assert all(k >= b.n_owned for k, _ in b.recv[a.rank])
        # one ring of ghosts: every ghost is a face neighbour of an owned element
        owned = set(int(e) for e in a.local[:a.n_owned])
        for g in a.local[a.n_owned:]:
            assert owned & set(adj[0][int(g)])


@pytest.mark.parametrize("name,ws", [("euler2d", 2), ("ns2d", 2), ("ns2d", 3)])
def test_partitioned_bdf2_level_equals_single_part(name, ws):
    import torch.multiprocessing as mp

    from oracle.residual import Discretization
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, name, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=900) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, eq, U, dt = _case(name)
    sw = Discretization(m, eq).S
    plan = PS.trace_plan(m, np.zeros(m["nodes"].shape[0], np.int64), 0, switches=sw)
    ref, st_ref = _level(PS.Partitioned(plan, OracleOps(plan, eq), single=True), U, dt)
    got = np.zeros_like(ref)
    for rank, ids, U2, st in out:
        got[ids] = U2
        assert st[1]["newton_its"] == st_ref[1]["newton_its"]
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
