"""A BDF2 Newton-GMRES level on a partitioned mesh (one part per rank).

The Line-DG operator couples an element to a face neighbour only through
the node at each line end (Sec. 2.3), so the data a part needs from the
other parts are the face-node traces of its cut faces, (p+1)^(D-1) nodes
per face:
  * residual (Eq. 36 split form): the traces of U, then, after each part has
    formed its gradient Q = D(U) (Eq. 32), the traces of Q;
  * split Jacobian-vector product (Eq. 41): the traces of x, then, after
    g = K21 x, the traces of g; y = x - alpha dt (K11 x + K12 g);
  * Jacobian: the traces of U and Q before the assembly;
  * the element-block preconditioner (Sec. 4.2) is element-local: no
    exchange;
  * GMRES: one all-reduce of the batched dot products per Gram-Schmidt
    sweep; Newton: one all-reduce per norm.
A part holds its owned elements and one ring of ghost elements (the face
neighbours of its owned ones), of which only the face nodes on the cut
faces carry data; the owned rows of every local operator read no other
ghost value. Faces of ghosts that leave the part get a Dirichlet tag of
their own, as in partition.halo_plan.

The local operators are given as an object (duck-typed, see PartOps): on a
GPU the single-GPU library on the part's sub-mesh (LdgPartOps below), in
the CPU tests any implementation of the same operators. The exchanges use
torch.distributed point-to-point calls posted as one group and all-reduces
(gloo on CPU tensors, NCCL on device tensors); every part runs the same
sequence of collectives.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import partition as PT


def face_nodes(D, p, f):
    """Local node ids (ascending) on face f = 2 d + end of an element."""
    d, end = divmod(f, 2)
    N = p + 1
    idx = np.arange(N ** D)
    return idx[(idx // N ** d) % N == end * p]


@dataclass
class TracePlan:
    rank: int
    local: np.ndarray          # global ids of the local elements: owned, then ghosts
    n_owned: int
    submesh: dict
    cut_tag: int
    D: int
    p: int
    send: dict = field(default_factory=dict)   # dst -> [(local position of an owned element, face)]
    recv: dict = field(default_factory=dict)   # src -> [(local position of a ghost, face)]


def trace_plan(mesh, owner, rank, adjacency=None, switches=None):
    """The part of `rank`: its owned elements, one ring of ghosts and the
    face-trace lists. For every face between an element e owned here and an
    element a owned by rank s, s sends the nodes of a on that face and this
    rank sends those of e; both sides list the pairs (element, face) in
    increasing (global element id, face), so every send list matches the
    receiver's list element for element."""
    adj = PT.face_neighbours(mesh) if adjacency is None else adjacency
    _, partner = adj
    hp = PT.halo_plan(mesh, owner, rank, 1, adj, switches)
    pos = {int(e): k for k, e in enumerate(hp.local)}
    D, p = int(mesh["D"]), int(mesh["p"])
    tp = TracePlan(rank=rank, local=hp.local, n_owned=hp.n_owned, submesh=hp.submesh, cut_tag=hp.cut_tag, D=D, p=p)
    send, recv = {}, {}
    for e in hp.local[:hp.n_owned]:
        e = int(e)
        for f in range(2 * D):
            if (e, f) not in partner:
                continue
            a, fa = partner[(e, f)]
            s = int(owner[a])
            if s == rank:
                continue
            recv.setdefault(s, []).append((int(a), int(fa)))
            send.setdefault(s, []).append((e, f))
    for s in recv:
        tp.recv[s] = [(pos[a], fa) for a, fa in sorted(recv[s])]
        tp.send[s] = [(pos[e], f) for e, f in sorted(send[s])]
    return tp


def _index(plan, lst, device):
    import torch
    fn = [face_nodes(plan.D, plan.p, f) for f in range(2 * plan.D)]
    rows = torch.tensor([[pos] for pos, _ in lst], dtype=torch.long, device=device)
    nodes = torch.tensor(np.stack([fn[f] for _, f in lst]), dtype=torch.long, device=device)
    return rows, nodes


def trace_exchange(X, plan, group=None):
    """Fill the face-node traces of the ghosts of X [n_local, C, npe] (a torch
    tensor whose owned blocks are current) from the parts that own them:
    all sends and receives of the exchange are posted as one group."""
    import torch.distributed as dist
    ops, recvd = [], []
    for dst, lst in sorted(plan.send.items()):
        rows, nodes = _index(plan, lst, X.device)
        ops.append(dist.P2POp(dist.isend, X[rows, :, nodes].contiguous(), dst, group=group))
    for src, lst in sorted(plan.recv.items()):
        rows, nodes = _index(plan, lst, X.device)
        buf = X.new_empty((len(lst), nodes.shape[1], X.shape[1]))
        recvd.append((rows, nodes, buf))
        ops.append(dist.P2POp(dist.irecv, buf, src, group=group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for rows, nodes, buf in recvd:
        X[rows, :, nodes] = buf
    return X


class Partitioned:
    """The global operators restricted to one part's owned rows.

    ops (PartOps): viscous (bool) and, on the part's local arrays
    [n_local, ...]: gradient(U) -> Q, residual(U, Q) -> R, jacobian(U, Q),
    precond(shift, scale), k21(x) -> g, jacvec_g(shift, scale, x, g) -> y,
    apply(r) -> z (the element-block preconditioner), all with the owned
    rows exact when the ghosts' face traces are current. group: the
    torch.distributed group, or None for a single part (no communication)."""

    def __init__(self, plan, ops, group=None, single=False):
        self.plan, self.ops, self.group, self.single = plan, ops, group, single
        self.n = plan.n_owned

    def _local(self, X_owned):
        X = X_owned.new_zeros((len(self.plan.local),) + tuple(X_owned.shape[1:]))
        X[:self.n] = X_owned
        return X

    def _exchange(self, X):
        if not self.single:
            trace_exchange(X.reshape(X.shape[0], -1, X.shape[-1]), self.plan, self.group)
        return X

    def allreduce(self, t):
        if not self.single:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def dots(self, V, w):
        """[V_j . w]_j over all parts: one all-reduce of the batched dots."""
        return self.allreduce((V.reshape(V.shape[0], -1) * w.reshape(1, -1)).sum(1))

    def norm(self, x):
        return math.sqrt(float(self.allreduce((x * x).sum().reshape(1))[0]))

    def _state(self, U_owned):
        U = self._local(U_owned)
        # ghost nodes other than the exchanged traces are never read by an
        # owned row; the part's mean state keeps their (discarded) rows finite
        U[self.n:] = U_owned.mean(dim=(0, 2), keepdim=True)
        U = self._exchange(U)
        Q = None
        if self.ops.viscous:
            Q = self._exchange(self.ops.gradient(U))
        return U, Q

    def residual(self, U_owned):
        U, Q = self._state(U_owned)
        return self.ops.residual(U, Q)[:self.n]

    def jacobian(self, U_owned):
        U, Q = self._state(U_owned)
        self.ops.jacobian(U, Q)

    def matvec(self, x_owned, shift, scale):
        x = self._exchange(self._local(x_owned))
        g = self._exchange(self.ops.k21(x)) if self.ops.viscous else None
        return self.ops.jacvec_g(shift, scale, x, g)[:self.n]

    def apply(self, r_owned):
        return self.ops.apply(self._local(r_owned))[:self.n]


def gmres(part, b, shift, scale, tol, m):
    """Right-preconditioned GMRES(m) on (shift I + scale A) x = b with one
    restart cycle from x = 0: classical Gram-Schmidt twice, every sweep's dot
    products reduced together; the Hessenberg least-squares problem is
    replicated on every part. Returns (x, iterations, relative residual)."""
    import torch
    beta = part.norm(b)
    if beta == 0.0:
        return torch.zeros_like(b), 0, 0.0
    V = b.new_zeros((m + 1,) + tuple(b.shape))
    Z = b.new_zeros((m,) + tuple(b.shape))
    V[0] = b / beta
    H = np.zeros((m + 1, m))
    cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
    g[0] = beta
    k_used, rel = 0, 1.0
    for k in range(m):
        Z[k] = part.apply(V[k])
        w = part.matvec(Z[k], shift, scale)
        h = np.zeros(k + 1)
        for _ in range(2):
            hk = part.dots(V[:k + 1], w)
            w = w - (V[:k + 1].reshape(k + 1, -1) * hk.reshape(-1, 1)).sum(0).reshape(w.shape)
            h += hk.double().cpu().numpy()
        hn = part.norm(w)
        H[:k + 1, k] = h
        H[k + 1, k] = hn
        if hn > 0:
            V[k + 1] = w / hn
        for j in range(k):
            a, c = H[j, k], H[j + 1, k]
            H[j, k], H[j + 1, k] = cs[j] * a + sn[j] * c, -sn[j] * a + cs[j] * c
        den = math.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
        H[k, k], H[k + 1, k] = den, 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        k_used = k + 1
        rel = abs(g[k + 1]) / beta
        if rel <= tol or hn == 0.0:
            break
    y = np.zeros(k_used)
    for i in range(k_used - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:]) / H[i, i]
    yt = torch.from_numpy(y).to(device=b.device, dtype=b.dtype)
    x = (Z[:k_used].reshape(k_used, -1) * yt.reshape(-1, 1)).sum(0).reshape(b.shape)
    return x, k_used, rel


def newton_bdf2(part, U_n, U_nm1, dt, first=False, rtol=1e-8, gmres_tol=1e-3, restart=30, max_cycles=10,
                max_newton=30):
    """One BDF2 level (BDF1 when `first`) of the owned rows, as
    ldg_newton_step in FP64: G(U) = U - c1 U^n - c2 U^{n-1} - alpha dt R(U),
    the stopping rule ||G|| <= rtol ||G(U^n)||, the Jacobian and
    preconditioner built once at the extrapolated start, each linear solve
    restarted GMRES cycles from the true residual to gmres_tol ||G||.
    Returns (U, stats)."""
    alpha = 1.0 if first else 2.0 / 3.0
    c1, c2 = (1.0, 0.0) if first else (4.0 / 3.0, -1.0 / 3.0)
    adt = alpha * dt

    def G(U):
        out = U - c1 * U_n - adt * part.residual(U)
        if not first:
            out = out - c2 * U_nm1
        return out
    res0 = part.norm(G(U_n))
    target = rtol * res0
    U = U_n.clone() if first else 2.0 * U_n - U_nm1
    stats = {"res0": res0, "newton_its": 0, "gmres_its": 0}
    built = False
    for it in range(max_newton + 1):
        Gu = G(U)
        gn = part.norm(Gu)
        stats["res_final"] = gn
        if gn <= target:
            return U, stats
        if it == max_newton:
            break
        if not built:
            part.jacobian(U)
            part.ops.precond(1.0, -adt)
            built = True
        delta = U.new_zeros(U.shape)
        for _ in range(max_cycles):
            r = -Gu - part.matvec(delta, 1.0, -adt)
            rn = part.norm(r)
            if rn <= gmres_tol * gn or rn == 0.0:
                break
            x, its, _ = gmres(part, r, 1.0, -adt, gmres_tol * gn / rn, restart)
            delta = delta + x
            stats["gmres_its"] += its
        U = U + delta
        stats["newton_its"] += 1
    raise RuntimeError(f"partitioned Newton did not reach {target:.3e} in {max_newton} iterations")


class LdgPartOps:
    """The local operators of a part by the single-GPU library on the part's
    sub-mesh, FP64 (device tensors): ldg_gradient, ldg_residual(_uq),
    ldg_jacobian_uq, ldg_precond, ldg_k21_apply, ldg_jacvec_g and
    ldg_precond_apply. Per-element data of the equations (g_D, source, g_N)
    are restricted to the part's elements; the cut faces are Dirichlet faces
    with zero data (they touch only ghost rows)."""

    def __init__(self, plan, eq):
        from . import ldg
        self.L = ldg
        eqs = dict(eq)
        for k in ("gD", "source", "gN"):
            if eqs.get(k) is not None:
                eqs[k] = np.ascontiguousarray(np.asarray(eqs[k])[plan.local])
        bc = dict(eqs.get("bc", {}))
        bc[plan.cut_tag] = "dirichlet"
        eqs["bc"] = bc
        self.h = ldg.ldg_setup(plan.submesh, eqs)
        self.viscous = eq["kind"] in ("ns", "poisson")
        self.J = self.P = None

    def gradient(self, U):
        h = self.h
        Q = U.new_empty((U.shape[0], h.nc, h.D, h.npe))
        return self.L.ldg_gradient(h, U, Q)

    def residual(self, U, Q):
        R = U.new_empty(U.shape)
        if self.viscous:
            return self.L.ldg_residual_uq(self.h, U, Q, R)
        return self.L.ldg_residual(self.h, U, R)

    def jacobian(self, U, Q):
        self.J = self.L.ldg_jacobian_uq(self.h, U, Q, self.L.PREC_FP64, self.J)

    def precond(self, shift, scale):
        self.P = self.L.ldg_precond(self.h, self.J, shift, scale, self.P)

    def k21(self, x):
        h = self.h
        g = x.new_empty((x.shape[0], h.nc, h.D, h.npe))
        return self.L.ldg_k21_apply(h, self.J, x, g, self.L.PREC_FP64)

    def jacvec_g(self, shift, scale, x, g):
        y = x.new_empty(x.shape)
        return self.L.ldg_jacvec_g(self.h, self.J, shift, scale, x, g, y, self.L.PREC_FP64)

    def apply(self, r):
        z = r.new_empty(r.shape)
        return self.L.ldg_precond_apply(self.h, self.P, r, z, self.L.PREC_FP64)
