"""Jacobian matrices of the Line-DG discretisation by complex step (oracle;
test infrastructure).

Sec. 4.1 (Eq. 35) defines K11 = dR/dU, K12 = dR/dQ, K21 = dD/dU
(K22 = 0 when C22 = 0) and Eq. 40 the reduced Jacobian
A = dR(U, D(U))/dU = K11 + K12 K21. The oracle obtains every column as
Im f(x + i h e_k) / h with h = 1e-30 (exact to rounding; no subtraction),
perturbing many columns at once when their elements are far enough apart
that their rows cannot overlap (greedy colouring of the face graph).

Flat index conventions: U[E, nc, npe] -> (e nc + c) npe + a;
Q[E, nc, D, npe] -> ((e nc + c) D + b) npe + a.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .residual import gradient, residual

H_CS = 1e-30


def _element_balls(disc, radius):
    """Elements within face-graph distance `radius` of each element."""
    nb = disc.conn.nbr_elem
    balls = []
    for e in range(disc.E):
        seen = {e}
        front = [e]
        for _ in range(radius):
            nxt = []
            for x in front:
                for y in nb[x]:
                    if y >= 0 and y not in seen:
                        seen.add(int(y))
                        nxt.append(int(y))
            front = nxt
        balls.append(sorted(seen))
    return balls


def _coloring(disc, radius):
    balls = _element_balls(disc, radius)
    color = -np.ones(disc.E, dtype=np.int64)
    for e in range(disc.E):
        used = {color[x] for x in balls[e] if color[x] >= 0}
        c = 0
        while c in used:
            c += 1
        color[e] = c
    return color


def colored_jacobian(disc, fun, x0, reach, batch=48):
    """Sparse d fun / d x at x0. x0: [E, *local_in] real; fun maps
    [B, E, *local_in] complex -> [B, E, *local_out] complex. `reach` bounds
    how many face-neighbour steps an input's influence can travel."""
    E = disc.E
    loc_in = x0.shape[1:]
    nin = int(np.prod(loc_in))
    color = _coloring(disc, 2 * reach)
    balls = _element_balls(disc, reach)
    ncol = int(color.max()) + 1
    tasks = [(c, k) for c in range(ncol) for k in range(nin)]
    rows, cols, vals = [], [], []
    out_local = None
    for t0 in range(0, len(tasks), batch):
        tb = tasks[t0:t0 + batch]
        X = np.repeat(x0[None].astype(np.complex128), len(tb), axis=0)
        Xf = X.reshape(len(tb), E, nin)
        for j, (c, k) in enumerate(tb):
            Xf[j, color == c, k] += 1j * H_CS
        Y = np.imag(fun(Xf.reshape(X.shape))) / H_CS
        if out_local is None:
            out_local = int(np.prod(Y.shape[2:]))
        Yf = Y.reshape(len(tb), E, out_local)
        for j, (c, k) in enumerate(tb):
            for e in np.nonzero(color == c)[0]:
                for r_e in balls[e]:
                    v = Yf[j, r_e]
                    nz = np.nonzero(v)[0]
                    rows.append(r_e * out_local + nz)
                    cols.append(np.full(len(nz), e * nin + k))
                    vals.append(v[nz])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(E * out_local, E * nin))


def K11(disc, U, Q=None, gD=None, source=None):
    """dR/dU at fixed Q."""
    return colored_jacobian(disc, lambda X: residual(disc, X, Q, gD, source), U, 1)


def K12(disc, U, Q, gD=None, source=None):
    """dR/dQ at fixed U."""
    return colored_jacobian(disc, lambda X: residual(disc, U, X, gD, source), Q, 1)


def K21(disc, gD=None):
    """dD/dU: the discrete gradient is affine in U, so its Jacobian is
    state-independent (Sec. 4.2); evaluated at U = 0."""
    U0 = np.zeros((disc.E, disc.nc, disc.npe))
    f = lambda X: gradient(disc, X, gD).reshape(X.shape[0], disc.E, -1)
    return colored_jacobian(disc, f, U0, 1)


def coupled(disc, U, Q, gD=None, source=None):
    """Jacobian of the split system (R(U, Q), Q - D(U, Q)) of Eq. 36 with
    respect to (U, Q): [[K11, K12], [-K21, I - K22]] (Sec. 4.1; K22 != 0
    when C22 != 0)."""
    k11 = colored_jacobian(disc, lambda X: residual(disc, X, Q, gD, source), U, 1)
    k12 = colored_jacobian(disc, lambda X: residual(disc, U, X, gD, source), Q, 1)
    k21 = colored_jacobian(disc, lambda X: gradient(disc, X, gD, Q), U, 1)
    k22 = colored_jacobian(disc, lambda X: gradient(disc, U, gD, X), Q, 1)
    return sp.bmat([[k11, k12], [-k21, sp.eye(Q.size) - k22]]).tocsr()


def A_full(disc, U, gD=None, source=None):
    """dR(U, D(U))/dU directly (the reduced Jacobian of Eq. 40)."""
    def f(X):
        Qx = gradient(disc, X, gD)
        return residual(disc, X, Qx, gD, source)
    return colored_jacobian(disc, f, U, 2)


def dense_brute_force(fun, x0):
    """Dense Jacobian column by column (tiny problems)."""
    n = x0.size
    cols = []
    for k in range(n):
        X = x0.astype(np.complex128).ravel().copy()
        X[k] += 1j * H_CS
        cols.append(np.imag(fun(X.reshape(x0.shape))).ravel() / H_CS)
    return np.stack(cols, axis=1)
