"""Implicit solver pieces (oracle; test infrastructure).

  * split matrix-vector product (I - alpha dt A) p = p - alpha dt (K11 p +
    K12 (K21 p)) without forming A (Sec. 4.2, Eq. 41);
  * the block-Jacobi preconditioning matrix: A restricted to the element
    diagonal blocks and, inside each block, to the Line-DG pattern (node i
    couples to the nodes of its D lines); entries of K12 K21 that fall inside
    that pattern are kept, fill outside it and every inter-element coupling
    is dropped (Sec. 4.2);
  * ILU(0) of each element block in that pattern (textbook IKJ form with
    n_c x n_c blocks, node order i + (p+1) j + (p+1)^2 k), forward/backward
    substitution;
  * restarted right-preconditioned GMRES with modified Gram-Schmidt and
    Givens rotations (Saad and Schultz);
  * Newton's method on the BDF2 stage equation
    G(U) = U - 4/3 U^n + 1/3 U^{n-1} - 2/3 dt F(U) (BDF1 on the first step),
    solving (I - 2/3 dt A) delta = -G(U) (the form of Eq. 39 with the stage
    residual on the right-hand side), stopping at ||G|| <= rtol ||G(U^n)||;
  * the paper's own integrator, Alexander's three-stage L-stable DIRK (Sec.
    4.1, Eqs. dirk1-dirk2 and their tableau): every stage equation
    U_i - alpha dt F(U_i) = U^n + dt sum_{j<i} a_ij K_j is the BDF1 form
    above with U^n replaced by its right-hand side and dt by alpha dt;
  * the classical explicit fourth-order Runge-Kutta step the paper uses for
    explicit time-stepping (Sec. 4.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import line_nodes


def split_matvec(K11, K12, K21, x, shift, scale):
    """shift x + scale (K11 x + K12 (K21 x)); K12/K21 may be None."""
    y = K11 @ x
    if K12 is not None:
        y = y + K12 @ (K21 @ x)
    return shift * x + scale * y


def line_pattern(D, p):
    """pat[i] = sorted local nodes sharing a coordinate line with node i."""
    npe = (p + 1) ** D
    pat = [set() for _ in range(npe)]
    for d in range(D):
        for l in range((p + 1) ** (D - 1)):
            ln = line_nodes(D, p, d, l)
            for a in ln:
                pat[a].update(ln)
    return [sorted(s) for s in pat]


def masked_blocks(disc, A, shift, scale):
    """Element blocks Ab[e, i, j, c, c'] = shift delta_ij delta_cc' +
    scale A[(e,c,i), (e,c',j)] for j in pattern(i), zero elsewhere."""
    E, nc, npe = disc.E, disc.nc, disc.npe
    pat = line_pattern(disc.D, disc.p)
    A = sp.csr_matrix(A)
    Ab = np.zeros((E, npe, npe, nc, nc))
    for e in range(E):
        rows = [(e * nc + c) * npe + i for c in range(nc) for i in range(npe)]
        blk = A[rows][:, rows].toarray().reshape(nc, npe, nc, npe)
        for i in range(npe):
            for j in pat[i]:
                Ab[e, i, j] = scale * blk[:, i, :, j]
            Ab[e, i, i] += shift * np.eye(nc)
    return Ab


def ilu0(Ab, pat):
    """Block ILU(0) of every element block, in place on a copy. Returns the
    combined factors: strictly lower part = L (unit diagonal implied),
    upper part including the diagonal = U."""
    F = Ab.copy()
    npe = F.shape[1]
    for e in range(F.shape[0]):
        a = F[e]
        for i in range(1, npe):
            pi = set(pat[i])
            for k in pat[i]:
                if k >= i:
                    break
                a[i, k] = a[i, k] @ np.linalg.inv(a[k, k])
                for j in pat[i]:
                    if j > k:
                        a[i, j] = a[i, j] - a[i, k] @ a[k, j]
    return F


def ilu_apply(F, pat, r):
    """z = (LU)^{-1} r per element; r, z: [E, nc, npe]."""
    E, npe = F.shape[0], F.shape[1]
    z = np.zeros_like(r)
    for e in range(E):
        y = np.zeros((npe, r.shape[1]))
        for i in range(npe):
            acc = r[e, :, i].copy()
            for k in pat[i]:
                if k < i:
                    acc -= F[e, i, k] @ y[k]
            y[i] = acc
        x = np.zeros_like(y)
        for i in reversed(range(npe)):
            acc = y[i].copy()
            for j in pat[i]:
                if j > i:
                    acc -= F[e, i, j] @ x[j]
            x[i] = np.linalg.solve(F[e, i, i], acc)
        z[e] = x.T
    return z


def gmres(matvec, b, precond=None, tol=1e-3, restart=30, maxiter=1, x0=None):
    """Right-preconditioned restarted GMRES; returns (x, iterations, relres)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    M = (lambda v: v) if precond is None else precond
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, 0.0
    its = 0
    rel = 1.0
    for _ in range(maxiter):
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= tol:
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            Z[k] = M(V[k])
            w = matvec(Z[k])
            for j in range(k + 1):
                Hm[j, k] = w @ V[j]
                w = w - Hm[j, k] * V[j]
            Hm[k + 1, k] = np.linalg.norm(w)
            if Hm[k + 1, k] > 0:
                V[k + 1] = w / Hm[k + 1, k]
            for j in range(k):
                t = cs[j] * Hm[j, k] + sn[j] * Hm[j + 1, k]
                Hm[j + 1, k] = -sn[j] * Hm[j, k] + cs[j] * Hm[j + 1, k]
                Hm[j, k] = t
            den = np.hypot(Hm[k, k], Hm[k + 1, k])
            cs[k], sn[k] = Hm[k, k] / den, Hm[k + 1, k] / den
            Hm[k, k] = den
            Hm[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_used = k + 1
            rel = abs(g[k + 1]) / bnorm
            if rel <= tol:
                break
        y = np.zeros(k_used)
        for i in reversed(range(k_used)):
            y[i] = (g[i] - Hm[i, i + 1:k_used] @ y[i + 1:]) / Hm[i, i]
        x = x + Z[:k_used].T @ y
        if rel <= tol:
            break
    return x, its, rel


def bdf2_residual(F_U, U, Un, Unm1, dt, first):
    """G(U) for BDF2 (BDF1 when first)."""
    if first:
        return U - Un - dt * F_U
    return U - (4.0 / 3.0) * Un + (1.0 / 3.0) * Unm1 - (2.0 / 3.0) * dt * F_U


def newton_bdf2(F, jac, Un, Unm1, dt, first=False, rtol=1e-8, gmres_tol=1e-3,
                restart=30, reuse=15, maxit=50, precond_builder=None, U0=None):
    """One implicit BDF2 level by Newton-GMRES (FP64). F(U) -> F(U) array,
    jac(U) -> (K11, K12, K21) sparse, precond_builder(K, shift, scale) ->
    callable or None. Returns (U, stats)."""
    alpha = 1.0 if first else 2.0 / 3.0
    target = rtol * np.linalg.norm(bdf2_residual(F(Un), Un, Un, Unm1, dt, first))
    U = (Un.copy() if first or Unm1 is None else 2.0 * Un - Unm1) if U0 is None else U0.copy()
    stats = {"newton": 0, "gmres": 0, "jac": 0, "hist": []}
    K = None
    P = None
    age = 0
    for _ in range(maxit):
        G = bdf2_residual(F(U), U, Un, Unm1, dt, first)
        gn = np.linalg.norm(G)
        stats["hist"].append(gn)
        if gn <= target:
            return U, stats
        if K is None or age >= reuse:
            K = jac(U)
            P = precond_builder(K, 1.0, -alpha * dt) if precond_builder else None
            stats["jac"] += 1
            age = 0
        mv = lambda v: split_matvec(K[0], K[1], K[2], v, 1.0, -alpha * dt)
        dx, its, _ = gmres(mv, -G.ravel(), P, tol=gmres_tol, restart=restart)
        stats["gmres"] += its
        stats["newton"] += 1
        age += 1
        U = U + dx.reshape(U.shape)
    raise RuntimeError("Newton did not converge")


# ---------------------------------------------------------------------------
# DIRK3 (Sec. 4.1)
# ---------------------------------------------------------------------------
DIRK3_ALPHA = 0.435866521508459


def dirk3_tableau():
    """(A, b, c) of the three-stage method: diagonal alpha; tau2 = (1 +
    alpha) / 2; b1 = -(6 alpha^2 - 16 alpha + 1) / 4; b2 = (6 alpha^2 - 20
    alpha + 5) / 4; last row of A equal to b (stiffly accurate)."""
    a = DIRK3_ALPHA
    tau2 = (1.0 + a) / 2.0
    b1 = -(6.0 * a * a - 16.0 * a + 1.0) / 4.0
    b2 = (6.0 * a * a - 20.0 * a + 5.0) / 4.0
    A = np.array([[a, 0.0, 0.0], [tau2 - a, a, 0.0], [b1, b2, a]])
    b = np.array([b1, b2, a])
    c = np.array([a, tau2, 1.0])
    return A, b, c


def dirk3_step(F, jac, Un, dt, rtol=1e-8, gmres_tol=1e-3, restart=30, reuse=15, maxit=50,
               precond_builder=None):
    """One DIRK3 step: stages K_i = F(U_i) with U_i = U^n + dt sum_{j<=i}
    a_ij K_j, each solved by Newton on G_i(U) = U - B_i - a_ii dt F(U),
    B_i = U^n + dt sum_{j<i} a_ij K_j, from the start U = B_i; then
    U^{n+1} = U^n + dt sum_j b_j K_j. Returns (U^{n+1}, per-stage stats)."""
    A, b, _ = dirk3_tableau()
    K, stats = [], []
    for i in range(3):
        B = Un + dt * sum(A[i, j] * K[j] for j in range(i)) if i else Un.copy()
        Ui, st = newton_bdf2(F, jac, B, None, A[i, i] * dt, first=True, rtol=rtol, gmres_tol=gmres_tol,
                             restart=restart, reuse=reuse, maxit=maxit, precond_builder=precond_builder)
        K.append(F(Ui))
        stats.append(st)
    return Un + dt * sum(b[j] * K[j] for j in range(3)), stats


def rk4_step(F, U, dt):
    """Classical RK4: k1 = F(U), k2 = F(U + dt/2 k1), k3 = F(U + dt/2 k2),
    k4 = F(U + dt k3); U + dt/6 (k1 + 2 k2 + 2 k3 + k4)."""
    k1 = F(U)
    k2 = F(U + 0.5 * dt * k1)
    k3 = F(U + 0.5 * dt * k2)
    k4 = F(U + dt * k3)
    return U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

