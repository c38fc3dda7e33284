"""1-D reference element of the Line-DG scheme (oracle; test infrastructure).

Follows Sec. 2.1 (Eqs. 8-9: nodal Lagrange expansion on [0,1]) and Sec. 2.2
(Gauss-Legendre integration of precision 3p with ceil((3p+1)/2) points; the
mass matrix is the same for every line, component and element and is
Cholesky-factorised once).
"""
from __future__ import annotations

import math

import numpy as np


def n_gauss(p: int) -> int:
    """Number of Gauss points: ceil((3p+1)/2) (Sec. 2.2)."""
    return (3 * p + 2) // 2


def gauss_legendre_01(nq: int, dtype=np.float64):
    """Gauss-Legendre points/weights on [0,1], by Newton's method on P_nq
    evaluated with the three-term Legendre recurrence (in `dtype`)."""
    k = np.arange(1, nq + 1, dtype=dtype)
    x = np.cos(dtype(np.pi) * (k - dtype(0.25)) / (nq + dtype(0.5)))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for m in range(2, nq + 1):
            p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
        dp = nq * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 16 * np.finfo(dtype).eps:
            break
    for _ in range(3):   # polish at the working precision
        p0 = np.ones_like(x)
        p1 = x.copy()
        for m in range(2, nq + 1):
            p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
        dp = nq * (x * p1 - p0) / (x * x - 1.0)
        x = x - p1 / dp
    p0 = np.ones_like(x)
    p1 = x.copy()
    for m in range(2, nq + 1):
        p0, p1 = p1, ((2 * m - 1) * x * p1 - (m - 1) * p0) / m
    dp = nq * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return 0.5 * (x[order] + 1.0), 0.5 * w[order]


def lagrange(s, x, dtype=np.float64):
    """phi_i(x_q) and phi_i'(x_q) for the nodal basis phi_i(s_j) = delta_ij,
    written out as products (returns arrays [len(x), len(s)])."""
    s = np.asarray(s, dtype=dtype)
    x = np.atleast_1d(np.asarray(x, dtype=dtype))
    n = len(s)
    phi = np.ones((len(x), n), dtype=dtype)
    dphi = np.zeros((len(x), n), dtype=dtype)
    for i in range(n):
        for j in range(n):
            if j != i:
                phi[:, i] *= (x - s[j]) / (s[i] - s[j])
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(x), 1 / (s[i] - s[k]), dtype=dtype)
            for j in range(n):
                if j != i and j != k:
                    term *= (x - s[j]) / (s[i] - s[j])
            dphi[:, i] += term
    return phi, dphi


class Rules:
    """All 1-D quantities for degree p and node set s.

    s, xq, wq  : nodes, Gauss points, Gauss weights on [0,1]
    Phi, dPhi  : phi_i(xq), phi_i'(xq), shape [nq, p+1]
    M          : mass matrix M_ij = int phi_i phi_j (exact with nq points)
    chol       : lower Cholesky factor of M
    Dn         : nodal derivative matrix Dn[i, j] = phi_j'(s_i)
    wnod       : int_0^1 phi_i (interpolatory weights of the node set)
    """

    def __init__(self, p: int, s):
        self.p = int(p)
        self.s = np.asarray(s, dtype=np.float64)
        assert len(self.s) == p + 1
        self.nq = n_gauss(p)
        self.xq, self.wq = gauss_legendre_01(self.nq)
        self.Phi, self.dPhi = lagrange(self.s, self.xq)
        self.M = self.Phi.T @ (self.wq[:, None] * self.Phi)
        self.chol = np.linalg.cholesky(self.M)
        _, self.Dn = lagrange(self.s, self.s)
        self.wnod = self.Phi.T @ self.wq
        # extended-precision copies for the metric terms (rounded once)
        X = np.longdouble
        xq_x, _ = gauss_legendre_01(self.nq, X)
        self.Phi_x, self.dPhi_x = lagrange(self.s, xq_x, X)
        _, self.Dn_x = lagrange(self.s, self.s, X)

    def mass_solve(self, b):
        """Solve M r = b along the last axis of b with the Cholesky factor
        (forward then backward substitution), real or complex b."""
        L = self.chol
        n = self.p + 1
        y = np.zeros(b.shape, dtype=np.result_type(b, np.float64))
        for i in range(n):
            acc = b[..., i].copy()
            for j in range(i):
                acc = acc - L[i, j] * y[..., j]
            y[..., i] = acc / L[i, i]
        r = np.zeros_like(y)
        for i in reversed(range(n)):
            acc = y[..., i].copy()
            for j in range(i + 1, n):
                acc = acc - L[j, i] * r[..., j]
            r[..., i] = acc / L[i, i]
        return r
