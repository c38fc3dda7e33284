"""Pointwise fluxes (oracle; test infrastructure).

Arrays carry the component index on the first axis: u[c, ...], q[c, b, ...]
(q = grad of the conserved variables, b = Cartesian direction), n[a, ...]
(a non-normalised normal). Everything is written so that a complex-step
perturbation passes through analytically: absolute values and maxima are
taken on the real part's sign.

  * Euler / Navier-Stokes: Eqs. 44-48 (Sec. 5.2) with the readings
    d(rho u_i u_j + p delta_ij)/dx_j for the momentum flux, the standard
    symmetric stress tau_ij = mu (du_i/dx_j + du_j/dx_i - 2/3 delta_ij
    du_k/dx_k), heat flux -(mu/Pr) grad(E + p/rho - |u|^2/2) = -(mu gamma /
    Pr) grad e, constant mu; F = F^inv + F^vis written as one flux in
    du/dt + div F = 0, so the viscous part carries its own sign.
  * Roe's approximate Riemann solver (named in Sec. 5.2) with Roe averages
    and Harten's entropy fix |lambda| -> (lambda^2 + delta^2) / (2 delta)
    for |lambda| < delta = 0.1 c~; a unit-normal flux is scaled by |n|
    (Eq. 13).
  * Local Lax-Friedrichs (Rusanov) with lambda = max(|v.n|+c) of the two
    traces (an alternative flux the paper does not use).
  * Poisson: F = -q, source f (Eq. 42). Scalar advection F = a u with the
    upwind flux (used by exactness pins).
Argument order of every numerical flux is F^.n(u_out, u_in; n) with n the
outward normal: the first trace sits on the side n points to (Eqs. 5-7).
"""
from __future__ import annotations

import numpy as np


def cabs(x):
    """|x| that keeps the imaginary (derivative) part analytic."""
    return np.where(np.real(x) >= 0, x, -x)


def cmax(a, b):
    return np.where(np.real(a) >= np.real(b), a, b)


def norm(n):
    return np.sqrt(sum(n[a] * n[a] for a in range(n.shape[0])))


# ---------------------------------------------------------------------------
# Euler
# ---------------------------------------------------------------------------
def primitive(u, gamma):
    D = u.shape[0] - 2
    rho = u[0]
    v = [u[1 + a] / rho for a in range(D)]
    p = (gamma - 1.0) * (u[D + 1] - 0.5 * sum(u[1 + a] * v[a] for a in range(D)))
    return rho, v, p


def euler_flux_n(u, n, gamma):
    """F^inv(u) . n."""
    D = n.shape[0]
    rho, v, p = primitive(u, gamma)
    vn = sum(v[a] * n[a] for a in range(D))
    out = [rho * vn]
    for a in range(D):
        out.append(u[1 + a] * vn + p * n[a])
    out.append((u[D + 1] + p) * vn)
    return np.stack(out)


def roe_flux(u_out, u_in, n, gamma, entropy_fix=0.1):
    """Roe flux F^.n(u_out, u_in; n) = |n| * [ (F(u_in)+F(u_out)).nbar / 2
    - |A_roe(nbar)| (u_out - u_in) / 2 ]."""
    D = n.shape[0]
    nn = norm(n)
    nb = n / nn
    rl, vl, pl = primitive(u_in, gamma)
    rr, vr, pr = primitive(u_out, gamma)
    Hl = (u_in[D + 1] + pl) / rl
    Hr = (u_out[D + 1] + pr) / rr
    sl, sr = np.sqrt(rl), np.sqrt(rr)
    rt = sl * sr
    vt = [(sl * vl[a] + sr * vr[a]) / (sl + sr) for a in range(D)]
    Ht = (sl * Hl + sr * Hr) / (sl + sr)
    q2 = sum(vt[a] * vt[a] for a in range(D))
    ct = np.sqrt((gamma - 1.0) * (Ht - 0.5 * q2))
    vnt = sum(vt[a] * nb[a] for a in range(D))
    drho = rr - rl
    dp = pr - pl
    dv = [vr[a] - vl[a] for a in range(D)]
    dvn = sum(dv[a] * nb[a] for a in range(D))
    delta = entropy_fix * ct

    def fix(lam):
        al = cabs(lam)
        return np.where(np.real(al) < np.real(delta), (lam * lam + delta * delta) / (2.0 * delta), al)

    l1 = fix(vnt - ct)
    l2 = fix(vnt)
    l5 = fix(vnt + ct)
    a1 = (dp - rt * ct * dvn) / (2.0 * ct * ct)
    a2 = drho - dp / (ct * ct)
    a5 = (dp + rt * ct * dvn) / (2.0 * ct * ct)
    diss = []
    diss.append(l1 * a1 + l2 * a2 + l5 * a5)
    for a in range(D):
        diss.append(l1 * a1 * (vt[a] - ct * nb[a]) + l2 * a2 * vt[a]
                    + l2 * rt * (dv[a] - dvn * nb[a]) + l5 * a5 * (vt[a] + ct * nb[a]))
    vdv = sum(vt[a] * dv[a] for a in range(D))
    diss.append(l1 * a1 * (Ht - ct * vnt) + l2 * a2 * 0.5 * q2
                + l2 * rt * (vdv - vnt * dvn) + l5 * a5 * (Ht + ct * vnt))
    diss = np.stack(diss)
    fl = euler_flux_n(u_in, nb, gamma)
    fr = euler_flux_n(u_out, nb, gamma)
    return nn * (0.5 * (fl + fr) - 0.5 * diss)


def lf_flux(u_out, u_in, n, gamma):
    """Local Lax-Friedrichs: (F(u_in)+F(u_out)).n/2 - lambda |n| (u_out-u_in)/2."""
    D = n.shape[0]
    nn = norm(n)
    rl, vl, pl = primitive(u_in, gamma)
    rr, vr, pr = primitive(u_out, gamma)
    cl = np.sqrt(gamma * pl / rl)
    cr = np.sqrt(gamma * pr / rr)
    vnl = sum(vl[a] * n[a] for a in range(D)) / nn
    vnr = sum(vr[a] * n[a] for a in range(D)) / nn
    lam = cmax(cabs(vnl) + cl, cabs(vnr) + cr)
    return 0.5 * (euler_flux_n(u_in, n, gamma) + euler_flux_n(u_out, n, gamma)) \
        - 0.5 * lam * nn * (u_out - u_in)


# ---------------------------------------------------------------------------
# Navier-Stokes viscous flux
# ---------------------------------------------------------------------------
def ns_viscous_flux_n(u, q, n, gamma, mu, Pr):
    """F^vis(u, q) . n with q = grad of the conserved variables."""
    D = n.shape[0]
    rho = u[0]
    v = [u[1 + a] / rho for a in range(D)]
    Et = u[D + 1] / rho
    gv = [[(q[1 + a, b] - v[a] * q[0, b]) / rho for b in range(D)] for a in range(D)]
    ge = [(q[D + 1, b] - Et * q[0, b]) / rho - sum(v[a] * gv[a][b] for a in range(D))
          for b in range(D)]
    div = sum(gv[a][a] for a in range(D))
    tau = [[mu * (gv[a][b] + gv[b][a] - (2.0 / 3.0) * div * (1.0 if a == b else 0.0))
            for b in range(D)] for a in range(D)]
    heat = [-(mu * gamma / Pr) * ge[b] for b in range(D)]
    mom = [-sum(tau[a][b] * n[b] for b in range(D)) for a in range(D)]
    ener = sum((heat[b] - sum(v[a] * tau[a][b] for a in range(D))) * n[b] for b in range(D))
    mom = [np.broadcast_to(x, ener.shape) for x in mom]
    return np.stack([np.zeros_like(ener)] + mom + [ener])


# ---------------------------------------------------------------------------
# equation-level dispatch
# ---------------------------------------------------------------------------
def inviscid_flux_n(eq, u, n):
    k = eq["kind"]
    if k in ("euler", "ns"):
        return euler_flux_n(u, n, eq["gamma"])
    if k == "advection":
        a = eq["adv"]
        return sum(a[b] * n[b] for b in range(n.shape[0])) * u
    return np.zeros_like(u * n[0])


def inviscid_numflux(eq, u_out, u_in, n):
    k = eq["kind"]
    if k in ("euler", "ns"):
        if eq.get("flux", "roe") == "roe":
            return roe_flux(u_out, u_in, n, eq["gamma"])
        return lf_flux(u_out, u_in, n, eq["gamma"])
    if k == "advection":
        a = eq["adv"]
        an = sum(a[b] * n[b] for b in range(n.shape[0]))
        return np.where(np.real(an) >= 0, an * u_in, an * u_out)
    return np.zeros_like(u_in * n[0])


def viscous_flux_n(eq, u, q, n):
    k = eq["kind"]
    if k == "ns":
        return ns_viscous_flux_n(u, q, n, eq["gamma"], eq["mu"], eq["Pr"])
    if k == "poisson":
        return -sum(q[:, b] * n[b] for b in range(n.shape[0]))
    return np.zeros_like(u * n[0])


def has_viscous(eq):
    return eq["kind"] in ("ns", "poisson")


def n_components(eq, D):
    return {"euler": D + 2, "ns": D + 2, "poisson": 1, "advection": 1}[eq["kind"]]
