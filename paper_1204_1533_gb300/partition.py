"""Element partitioning and halo exchange for running the Line-DG residual
on several ranks (one GPU per rank).

The scheme couples an element to its face neighbours only through the node
at each line end (Sec. 2.3), and the viscous residual reaches one step
further through the neighbours' LDG gradients. A rank therefore owns a set
of elements and keeps ghost copies of the elements within `layers` face
steps of them (1 for first-order equations, 2 for second-order ones): after
a halo exchange of the ghosts' states the rank evaluates the residual of its
local sub-mesh with the single-GPU library, and the rows of its owned
elements are exactly those of the global residual. Faces cut by the
sub-mesh become Dirichlet faces of a tag of their own; they touch only the
outermost ghosts, whose residual rows are discarded.

The switch function (Sec. 3) is a global property of the mesh: a sub-mesh
must use the global switches restricted to its elements, which halo_plan
stores in the sub-mesh (`switches`, passed to ldg_setup) when it is given
the global function (ldg_setup_host exports it without a GPU).

Host logic only: the plan is integer work on the host, the exchange moves
whole element blocks [n_c, (p+1)^D] with torch.distributed point-to-point
calls (gloo on CPU tensors, NCCL on device tensors), and the norm is one
all-reduce.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _face_key(verts, e, f, D):
    d, end = divmod(f, 2)
    return tuple(sorted(int(verts[e, c]) for c in range(1 << D) if ((c >> d) & 1) == end))


def face_neighbours(mesh):
    """Face-adjacent elements from the vertex ids of the faces: nbrs[e] is
    the sorted list of the elements sharing a face with e, partner[(e, f)]
    the (element, face) on the other side of face f of e (absent on the
    boundary)."""
    D = int(mesh["D"])
    verts = mesh["vertices"]
    E = verts.shape[0]
    faces = {}
    for e in range(E):
        for f in range(2 * D):
            faces.setdefault(_face_key(verts, e, f, D), []).append((e, f))
    nbrs = [set() for _ in range(E)]
    partner = {}
    for ef in faces.values():
        for a in ef:
            for b in ef:
                if a != b:
                    partner[a] = b
                    if a[0] != b[0]:
                        nbrs[a[0]].add(b[0])
    return [sorted(s) for s in nbrs], partner


def block_partition(n_elem, nparts):
    """owner[e]: contiguous blocks of element ids (slabs of the structured
    generators, whose elements are numbered lexicographically)."""
    return (np.arange(n_elem, dtype=np.int64) * nparts) // n_elem


@dataclass
class HaloPlan:
    rank: int
    local: np.ndarray                 # global ids of the local elements: owned, then ghosts
    n_owned: int
    submesh: dict                     # the local mesh (cut faces tagged `cut_tag`)
    cut_tag: int
    recv: dict = field(default_factory=dict)   # src rank -> local positions of its elements
    send: dict = field(default_factory=dict)   # dst rank -> local positions of my owned elements


def _rings(nbrs, owned, layers):
    """Elements within `layers` face steps of the set `owned`, outside it."""
    have = set(int(e) for e in owned)
    front = list(have)
    out = []
    for _ in range(layers):
        nxt = []
        for e in front:
            for o in nbrs[e]:
                if o not in have:
                    have.add(o)
                    nxt.append(o)
        out += nxt
        front = nxt
    return sorted(out)


def halo_plan(mesh, owner, rank, layers, adjacency=None, switches=None):
    """The local sub-mesh of `rank` (owned elements, then `layers` rings of
    ghosts, each group in increasing global id) and the exchange lists.
    Every rank builds every plan from the same global mesh, so the send list
    of one rank towards another is, element for element, that rank's receive
    list from it. switches: the global switch function [E, D, 2] (int8)."""
    nbrs, partner = face_neighbours(mesh) if adjacency is None else adjacency
    D = int(mesh["D"])
    owned = np.nonzero(owner == rank)[0]
    local = np.concatenate([owned, np.array(_rings(nbrs, owned, layers), dtype=np.int64)]).astype(np.int64)
    pos = {int(e): k for k, e in enumerate(local)}
    btag = mesh["btag"][local].copy()
    cut_tag = int(max(int(mesh["btag"].max()), -1) + 1)
    for k, e in enumerate(local):
        for f in range(2 * D):
            if btag[k, f] < 0 and int(partner[(int(e), f)][0]) not in pos:
                btag[k, f] = cut_tag
    sub = {key: mesh[key] for key in ("D", "p", "s")}
    sub.update(nodes=mesh["nodes"][local], vertices=mesh["vertices"][local], btag=btag)
    if switches is not None:
        sub["switches"] = np.ascontiguousarray(np.asarray(switches, dtype=np.int8)[local])
    plan = HaloPlan(rank=rank, local=local, n_owned=len(owned), submesh=sub, cut_tag=cut_tag)
    for k in range(len(owned), len(local)):   # ghosts: increasing global id within each ring
        plan.recv.setdefault(int(owner[local[k]]), []).append(k)
    for src in plan.recv:
        plan.recv[src] = sorted(plan.recv[src], key=lambda k: int(local[k]))
    for dst in range(int(owner.max()) + 1):
        if dst == rank:
            continue
        need = [e for e in _rings(nbrs, np.nonzero(owner == dst)[0], layers) if owner[e] == rank]
        if need:
            plan.send[dst] = [pos[e] for e in sorted(need)]
    return plan


def halo_exchange(U_local, plan, group=None):
    """Fill the ghost blocks of U_local [n_local, ...] (a torch tensor; the
    owned blocks must be current) from their owners. Messages are whole
    element blocks in increasing global element id. All sends and receives
    of the exchange are posted as one group (batch_isend_irecv): under NCCL
    point-to-point calls issued one by one queue on each pair's stream, and
    two ranks that both send first could wait on each other; a group lets the
    backend match them."""
    import torch.distributed as dist
    ops, recvd = [], []
    for dst, rows in sorted(plan.send.items()):
        ops.append(dist.P2POp(dist.isend, U_local[rows].contiguous(), dst, group=group))
    for src, rows in sorted(plan.recv.items()):
        buf = U_local.new_empty((len(rows),) + tuple(U_local.shape[1:]))
        recvd.append((rows, buf))
        ops.append(dist.P2POp(dist.irecv, buf, src, group=group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    for rows, buf in recvd:
        U_local[rows] = buf
    return U_local


def partitioned_residual(U_owned, plan, local_residual, U_local=None, group=None):
    """R of the owned elements: halo exchange into the local state, the
    residual of the local sub-mesh by `local_residual(U_local) -> R_local`
    (on a GPU: ldg_residual of a handle set up on plan.submesh), and its
    owned rows."""
    if U_local is None:
        U_local = U_owned.new_empty((len(plan.local),) + tuple(U_owned.shape[1:]))
    U_local[:plan.n_owned] = U_owned
    halo_exchange(U_local, plan, group)
    return local_residual(U_local)[:plan.n_owned]


def global_norm(x_owned, group=None, local_sq=None):
    """||x||_2 over all ranks: each rank's sum of squares of its owned
    entries, then one all-reduce. local_sq(x) -> float gives that sum on the
    rank (on a GPU: ldg_norm2 of the owned slice, squared); by default it is
    taken on the tensor's own device."""
    import math

    import torch
    import torch.distributed as dist
    if local_sq is None:
        sq = float((x_owned.double() ** 2).sum())
    else:
        sq = float(local_sq(x_owned))
    s = torch.tensor([sq], dtype=torch.float64, device=x_owned.device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return math.sqrt(float(s))
