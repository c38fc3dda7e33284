"""LDG gradient D(U) and residual R(U, Q) of the Line-DG scheme (oracle;
test infrastructure).

Per direction d and per line of nodes the oracle
  1. interpolates the nodal values to the Gauss points (Eq. 8),
  2. evaluates the contravariant flux F . n_d at each Gauss point (Eq. 4),
  3. forms the right-hand side of the 1-D Galerkin problem, Eq. 7 with
     v = phi_i: F^.n^+(u^+(1), u(1)) phi_i(1) + F^.n^-(u^-(0), u(0)) phi_i(0)
     - sum_q w_q f~(xi_q) phi_i'(xi_q), and solves M r = b (Cholesky),
  4. accumulates R = -(1/J) sum_d r^(d) + S (Eqs. 10 and 31).
The gradient pass applies the same Galerkin procedure to u (x) n_d (Eq. 19)
with the trace u^ of Eq. 20, and q = (1/J) sum_d d^(d) (Eq. 32).

Numerical fluxes (Sec. 3, Eqs. 25-28, C12 = n S/2, C22 = 0):
  interior, switch S = S^+-_d of this element and end:
      F^vis . n = F^vis(outside) . n  if S = +1, F^vis(inside) . n if S = -1,
                  plus C11 (u_in - u_out)            (dissipative sign; with the
                  non-unit normal n of Eq. 7 this is a penalty per unit
                  reference length, C11 / h in physical units)
      u^        = inside if S = +1, outside if S = -1
  Dirichlet boundary (Eqs. 27-28):
      F^vis . n = F^vis(u_in, q_in) . n + C11_b |n| (u_in - g_D),  u^ = g_D,
      inviscid part: the Riemann flux with outside trace g_D.
  Stabilised scheme (C11, C22 != 0, Sec. 3 and Table 2's lower half): at
  interior ends
      u^ = (switch value) + C22 (F^vis(inside) - F^vis(outside)) . n/|n|,
  the sign that makes C22 a penalty on the jump of the normal flux (the
  printed sign, with the outside as the positive side as the switch form
  implies, gives an unstable operator); at Neumann ends
      u^ = u_in + C22 (F^vis(inside) . n/|n| - g_N).
  D then depends on Q, and a solve couples U and Q (Eq. 36).
  Neumann boundary (Eqs. 29-30 with C22 = 0): the prescribed flux enters as
  a flux vector G at the boundary nodes (data gN[E, nc, D, npe]; a scalar
  normal flux g_N is G = g_N n/|n|), so that a node where two Neumann faces
  meet carries one datum for both:
      F^ . n = G . n (n the non-unit normal of the line end),  u^ = u_in.
  No-slip adiabatic wall (Navier-Stokes; not in the paper):
      inviscid part: pressure-only flux (0, p_in n, 0),
      u^ = (rho_in, 0, 0, 0, rho E_in - |rho v_in|^2 / (2 rho_in)),
      F^vis . n = F^vis(u^, q_in) . n with the energy (heat) component
                  replaced by the work term only (adiabatic), plus the
                  C11_b |n| (u_in - u^) penalty on the momentum components.

All arrays may carry extra leading batch axes (complex-step columns):
U[..., E, nc, npe], Q[..., E, nc, D, npe].
"""
from __future__ import annotations

import numpy as np

from . import physics as ph
from .mesh import Connectivity, Metrics, from_lines, switches, to_lines
from .rules import Rules


class Discretization:
    """Everything the residual needs that does not depend on the state."""

    def __init__(self, mesh, eq):
        self.mesh = mesh
        self.eq = dict(eq)
        self.D, self.p = mesh["D"], mesh["p"]
        self.E = mesh["nodes"].shape[0]
        self.npe = (self.p + 1) ** self.D
        self.nl = (self.p + 1) ** (self.D - 1)
        self.nc = ph.n_components(eq, self.D)
        self.rules = Rules(self.p, mesh["s"])
        self.conn = Connectivity(mesh)
        self.S = switches(mesh, self.conn)
        self.met = Metrics(mesh, self.rules)
        self.C11 = float(eq.get("C11", 0.0))
        self.C11b = float(eq.get("C11b", 1.0))
        self.C22 = float(eq.get("C22", 0.0))
        self.bc = dict(eq.get("bc", {0: "dirichlet"}))
        self.gN = None if eq.get("gN") is None else np.asarray(eq["gN"], dtype=np.float64)

    @property
    def ndof(self):
        return self.E * self.nc * self.npe


# ---------------------------------------------------------------------------
def _gather(A, g):
    """A[..., E, C, npe] at global node ids g (any shape) -> [C, ..., *g.shape]."""
    lead = A.shape[:-3]
    E, C, npe = A.shape[-3:]
    flat = np.moveaxis(A, -2, -3).reshape(lead + (C, E * npe))
    gg = np.where(g >= 0, g, 0)
    return np.moveaxis(flat[..., gg], len(lead), 0)


def _lead(x, nlead):
    """Insert nlead singleton batch axes after the component axis."""
    return x.reshape(x.shape[:1] + (1,) * nlead + x.shape[1:])


def _bc_kind(disc, codes):
    tags = -1 - codes
    kinds = np.full(codes.shape, "", dtype=object)
    for t, k in disc.bc.items():
        kinds[tags == t] = k
    return kinds


def _wall_state(u_in, D):
    rho = u_in[0]
    ke = 0.5 * sum(u_in[1 + a] * u_in[1 + a] for a in range(D)) / rho
    out = [rho] + [np.zeros_like(rho) for _ in range(D)] + [u_in[D + 1] - ke]
    return np.stack(out)


def _end_traces(disc, U, d, end, uL):
    """(u_in, u_out, codes) at the given end of every line of direction d;
    component axis first: [C, ..., E, nl]."""
    p = disc.p
    g = disc.conn.nbr[:, d, :, end]                      # [E, nl]
    u_in = np.moveaxis(uL[..., end * p], -2, 0)            # [C, ..., E, nl]
    u_out = _gather(U, g)                                  # [C, ..., E, nl]
    return u_in, u_out, g


def gradient(disc, U, gD=None, Q=None):
    """Q = D(U) (Eqs. 19, 20, 26, 28, 32), shape [..., E, nc, D, npe]; with
    C22 != 0 the trace depends on the given Q as well: D(U, Q) of Eq. 36."""
    D, p, r = disc.D, disc.p, disc.rules
    stab = disc.C22 != 0.0
    if stab and Q is None:
        raise ValueError("C22 != 0: the gradient depends on Q")
    if stab:
        lead = np.broadcast_shapes(U.shape[:-3], Q.shape[:-4])
        U = np.broadcast_to(U, lead + U.shape[-3:])
        Qin = np.broadcast_to(Q, lead + Q.shape[-4:])
        dtype = np.result_type(U, Qin)
    else:
        lead = U.shape[:-3]
        dtype = U.dtype
    Q = np.zeros(lead + (disc.E, disc.nc, D, disc.npe), dtype=dtype)
    for d in range(D):
        uL = to_lines(U, D, p, d)                          # [..., E, nc, nl, p+1]
        uq = np.einsum("qi,...i->...q", r.Phi, uL)          # [..., E, nc, nl, nq]
        ng = np.moveaxis(disc.met.ng[d], -1, 0)             # [D, E, nl, nq]
        # b_i = uhat^+ n^+ phi_i(1) + uhat^- n^- phi_i(0) - sum_q w_q u_q n_q phi_i'(xi_q)
        b = np.zeros(lead + (disc.E, disc.nc, D, disc.nl, p + 1), dtype=dtype)
        for a in range(D):
            w = uq * ng[a][:, None]                          # [..., E, nc, nl, nq]
            b[..., a, :, :] -= np.einsum("qi,q,...q->...i", r.dPhi, r.wq, w)
        for end in (0, 1):
            u_in, u_out, g = _end_traces(disc, U, d, end, uL)
            Sw = disc.S[:, d, end][:, None]                  # [E, 1]
            uhat = np.where(Sw == 1, u_in, u_out)
            bnd = g < 0
            nend = disc.met.nplus[d] if end == 1 else disc.met.nminus[d]   # [E, nl, D]
            if stab:
                # C22 times the jump of the normal viscous flux (Eq. 26)
                n = np.moveaxis(nend, -1, 0)                                 # [D, E, nl]
                q_in = np.moveaxis(np.moveaxis(to_lines(Qin, D, p, d)[..., end * p], -3, 0), -2, 1)
                sc = ph.norm(n)
                f_in = ph.viscous_flux_n(disc.eq, u_in, q_in, n) / sc
                f_out = ph.viscous_flux_n(disc.eq, u_out, _gather_q(Qin, g), n) / sc
                uhat = uhat + disc.C22 * (f_in - f_out)
            if np.any(bnd):
                kinds = _bc_kind(disc, g)
                if gD is not None:
                    gd = _lead(_gather(gD, _self_ids(disc, d, end)), len(lead))
                for kind in set(kinds[bnd]):
                    m = bnd & (kinds == kind)
                    if kind == "dirichlet":
                        uhat = np.where(m, gd, uhat)
                    elif kind == "wall":
                        uhat = np.where(m, _wall_state(u_in, D), uhat)
                    elif kind == "neumann":
                        un = u_in
                        if stab:   # Eq. 30
                            sid = _self_ids(disc, d, end)
                            gn = _lead(_neumann_flux(disc, sid, n), len(lead)) / sc
                            un = u_in + disc.C22 * (f_in - gn)
                        uhat = np.where(m, un, uhat)
                    else:
                        raise ValueError(f"unknown boundary kind {kind!r}")
            for a in range(D):
                contrib = np.moveaxis(uhat * nend[..., a], 0, -2)          # [..., E, nc, nl]
                b[..., a, :, end * p] += contrib
        dd = r.mass_solve(b)                                               # [..., E, nc, D, nl, p+1]
        Q += from_lines(dd, D, p, d)
    return Q / disc.met.J[:, None, None, :]


def _self_ids(disc, d, end):
    """Global ids of the line-end nodes themselves [E, nl]."""
    from .mesh import line_nodes
    ids = np.zeros((disc.E, disc.nl), dtype=np.int64)
    for l in range(disc.nl):
        a = line_nodes(disc.D, disc.p, d, l)[end * disc.p]
        ids[:, l] = np.arange(disc.E) * disc.npe + a
    return ids


def residual(disc, U, Q=None, gD=None, source=None):
    """R(U, Q) = -(1/J) sum_d r^(d) + S (Eqs. 7, 10, 31), [..., E, nc, npe]."""
    D, p, r, eq = disc.D, disc.p, disc.rules, disc.eq
    visc = ph.has_viscous(eq)
    lead = np.broadcast_shapes(U.shape[:-3], Q.shape[:-4] if Q is not None else ())
    U = np.broadcast_to(U, lead + U.shape[-3:])
    if Q is not None:
        Q = np.broadcast_to(Q, lead + Q.shape[-4:])
    dtype = np.result_type(U, Q if Q is not None else U)
    acc = np.zeros(lead + (disc.E, disc.nc, disc.npe), dtype=dtype)
    for d in range(D):
        uL = to_lines(U, D, p, d)                                   # [..., E, nc, nl, p+1]
        uq = np.moveaxis(np.einsum("qi,...i->...q", r.Phi, uL), -3, 0)   # [nc, ..., E, nl, nq]
        ng = np.moveaxis(disc.met.ng[d], -1, 0)                      # [D, E, nl, nq]
        fq = ph.inviscid_flux_n(eq, uq, ng)
        if visc:
            QL = to_lines(Q, D, p, d)                               # [..., E, nc, D, nl, p+1]
            qq = np.einsum("qi,...i->...q", r.Phi, QL)
            qq = np.moveaxis(np.moveaxis(qq, -4, 0), -3, 1)          # [nc, D, ..., E, nl, nq]
            fq = fq + ph.viscous_flux_n(eq, uq, qq, ng)
        b = -np.einsum("qi,q,...q->...i", r.dPhi, r.wq, np.moveaxis(fq, 0, -3))   # [..., E, nc, nl, p+1]
        for end in (0, 1):
            u_in, u_out, g = _end_traces(disc, U, d, end, uL)
            n = np.moveaxis(disc.met.nplus[d] if end == 1 else disc.met.nminus[d], -1, 0)  # [D, E, nl]
            bnd = g < 0
            Fh = ph.inviscid_numflux(eq, u_out, u_in, n)
            if visc:
                q_in = np.moveaxis(np.moveaxis(to_lines(Q, D, p, d)[..., end * p], -3, 0), -2, 1)
                q_out = _gather_q(Q, g)
                Sw = disc.S[:, d, end][:, None]
                fv_out = ph.viscous_flux_n(eq, u_out, q_out, n)
                fv_in = ph.viscous_flux_n(eq, u_in, q_in, n)
                # interior penalty per unit reference length (C11 / h physically)
                Fv = np.where(Sw == 1, fv_out, fv_in) + disc.C11 * (u_in - u_out)
                Fh = Fh + Fv
            if np.any(bnd):
                kinds = _bc_kind(disc, g)
                sid = _self_ids(disc, d, end)
                for kind in set(kinds[bnd]):
                    m = bnd & (kinds == kind)
                    if kind == "dirichlet":
                        gd = _lead(_gather(gD, sid), len(lead))
                        Fb = ph.inviscid_numflux(eq, gd, u_in, n)
                        if visc:
                            Fb = Fb + ph.viscous_flux_n(eq, u_in, q_in, n) \
                                + disc.C11b * ph.norm(n) * (u_in - gd)
                    elif kind == "wall":
                        Fb = _wall_flux(disc, u_in, q_in if visc else None, n)
                    elif kind == "neumann":
                        Fb = _lead(_neumann_flux(disc, sid, n), len(lead))
                    else:
                        raise ValueError(f"unknown boundary kind {kind!r}")
                    Fh = np.where(m, Fb, Fh)
            b[..., end * p] += np.moveaxis(Fh, 0, -2)
        rr = r.mass_solve(b)
        acc = acc + from_lines(rr, D, p, d)
    R = -acc / disc.met.J[:, None, :]
    if source is not None:
        R = R + source
    return R


def _gather_q(Q, g):
    """Q[..., E, nc, D, npe] at global node ids g -> [nc, D, ..., *g.shape]."""
    lead = Q.shape[:-4]
    E, C, D, npe = Q.shape[-4:]
    flat = np.moveaxis(Q, -1, -3)                     # [..., E, npe, nc, D]
    flat = flat.reshape(lead + (E * npe, C, D))
    gg = np.where(g >= 0, g, 0)
    out = flat[..., gg, :, :]                        # [..., *g.shape, nc, D]
    return np.moveaxis(np.moveaxis(out, -2, 0), -1, 1)


def _neumann_flux(disc, sid, n):
    """G . n at the line-end nodes sid [E, nl] (zero without data): [nc, E, nl]."""
    if disc.gN is None:
        return np.zeros((disc.nc,) + sid.shape)
    G = _gather_q(disc.gN, sid)                       # [nc, D, E, nl]
    return sum(G[:, a] * n[a] for a in range(disc.D))


def _wall_flux(disc, u_in, q_in, n):
    """No-slip adiabatic wall flux (see module docstring)."""
    eq, D = disc.eq, disc.D
    rho, v, p = ph.primitive(u_in, eq["gamma"])
    F = [np.zeros_like(rho * n[0])] + [p * n[a] for a in range(D)] + [np.zeros_like(rho * n[0])]
    F = np.stack(F)
    if q_in is not None:
        ub = _wall_state(u_in, D)
        Fv = ph.viscous_flux_n(eq, ub, q_in, n)
        # adiabatic: drop the heat-flux part; with zero wall velocity the
        # work term vanishes as well
        Fv[D + 1] = 0.0 * Fv[D + 1]
        pen = disc.C11b * ph.norm(n) * (u_in - ub)
        pen[0] = 0.0 * pen[0]
        pen[D + 1] = 0.0 * pen[D + 1]
        F = F + Fv + pen
    return F


def coupled_residual(disc, U, Q, gD=None, source=None):
    """The split system of Eq. 36 as one residual: (R(U, Q), Q - D(U, Q)),
    zero at a steady solution; with C22 != 0 the two parts are coupled."""
    return residual(disc, U, Q, gD, source), Q - gradient(disc, U, gD, Q)


def full_residual(disc, U, gD=None, source=None):
    """F(U) = R(U, D(U)) (Eq. 36); first-order systems skip D."""
    if ph.has_viscous(disc.eq):
        return residual(disc, U, gradient(disc, U, gD), gD, source)
    return residual(disc, U, None, gD, source)


def conservation_weights(disc):
    """(prod_d w_{i_d}) J at every node, w_i = int phi_i: the weights under
    which the Line-DG residual telescopes (sum_i w_i r_i^(d) = F^+ + F^-)."""
    D, p = disc.D, disc.p
    w = disc.rules.wnod
    W = np.ones(disc.npe)
    for a in range(disc.npe):
        for b in range(D):
            W[a] *= w[(a // (p + 1) ** b) % (p + 1)]
    return W[None, :] * disc.met.J
