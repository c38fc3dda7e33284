"""Pins for the oracle's Riemann fluxes that reach every term of Roe's
dissipation, the shear-wave part included (CPU only).

Roe's solver (Sec. 5.2 names it; the scheme follows Roe's construction):
the dissipation is |A(u~)| (u_out - u_in) with A(u~) the Jacobian of the
normal Euler flux at the Roe-averaged state u~, the state for which
A(u~) (u_R - u_L) = F(u_R) - F(u_L) holds exactly ("property U"). The
reference here is built without the oracle's arithmetic: the flux from its
definition in primitive variables, the Jacobian by complex step of that
flux, |A| from numpy's eigendecomposition, and the Roe state from the
textbook averages, itself checked by property U. Random state pairs carry
velocity jumps in every direction, so the shear waves (the eigenvalue v.n
repeated D - 1 times) carry a jump of their own.
"""
import numpy as np
import pytest

from oracle import physics as ph

GAMMA = 1.4


def _states(D, k, seed, vscale=1.0, vshift=None):
    """Conserved states from primitive draws; returns (u, rho, v, p)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, k)
    v = vscale * rng.uniform(-1, 1, (D, k))
    if vshift is not None:
        v = v + np.asarray(vshift, dtype=float)[:, None]
    p = rng.uniform(0.5, 3.0, k)
    E = p / (GAMMA - 1) + 0.5 * rho * (v * v).sum(0)
    return np.concatenate([[rho], rho * v, [E]]), rho, v, p


def _flux_primitive(rho, v, p, nb):
    """Normal Euler flux from its definition: (rho v.n, rho v v.n + p n,
    (E + p) v.n), E = p/(gamma-1) + rho |v|^2 / 2."""
    vn = (v * nb).sum(0)
    E = p / (GAMMA - 1) + 0.5 * rho * (v * v).sum(0)
    return np.concatenate([[rho * vn], rho * v * vn + p * nb, [(E + p) * vn]])


def _flux_conserved(u, nb):
    D = u.shape[0] - 2
    rho = u[0]
    v = u[1:1 + D] / rho
    p = (GAMMA - 1) * (u[D + 1] - 0.5 * rho * (v * v).sum(0))
    return _flux_primitive(rho, v, p, nb)


def _jacobian(u, nb):
    """dF.n/du at one state by complex step (exact to rounding)."""
    m = u.shape[0]
    A = np.zeros((m, m))
    for k in range(m):
        du = np.zeros(m, dtype=complex)
        du[k] = 1e-30j
        A[:, k] = np.imag(_flux_conserved((u + du)[:, None], nb[:, None])[:, 0]) / 1e-30
    return A


def _roe_state(rho_l, v_l, p_l, rho_r, v_r, p_r):
    """Textbook Roe averages (sqrt(rho) weights of v and H), as a conserved
    state, and its sound speed."""
    sl, sr = np.sqrt(rho_l), np.sqrt(rho_r)
    H_l = (p_l / (GAMMA - 1) + 0.5 * rho_l * v_l @ v_l + p_l) / rho_l
    H_r = (p_r / (GAMMA - 1) + 0.5 * rho_r * v_r @ v_r + p_r) / rho_r
    rho = sl * sr
    v = (sl * v_l + sr * v_r) / (sl + sr)
    H = (sl * H_l + sr * H_r) / (sl + sr)
    c2 = (GAMMA - 1) * (H - 0.5 * v @ v)
    p = rho * c2 / GAMMA
    E = rho * H - p
    return np.concatenate([[rho], rho * v, [E]]), np.sqrt(c2)


def _abs_matrix(A, fn):
    """R fn(Lambda) R^-1 from numpy's eigendecomposition (real spectrum)."""
    lam, R = np.linalg.eig(A)
    assert np.abs(lam.imag).max() < 1e-10 * np.abs(lam).max()
    return np.real(R @ np.diag(fn(lam.real)) @ np.linalg.inv(R)), lam.real


def _oracle_dissipation(u_out, u_in, n, fix):
    """|A| (u_out - u_in) as the oracle's Roe flux applies it:
    F^ = |n| [ (F(u_in) + F(u_out)).nb / 2 - diss / 2 ]."""
    nb = n / np.sqrt((n * n).sum(0))
    nn = np.sqrt((n * n).sum(0))
    with np.errstate(divide="ignore", invalid="ignore"):
        F = ph.roe_flux(u_out, u_in, n, GAMMA, entropy_fix=fix)
    return ph.euler_flux_n(u_in, nb, GAMMA) + ph.euler_flux_n(u_out, nb, GAMMA) - 2.0 * F / nn


@pytest.mark.parametrize("D", [2, 3])
def test_physical_flux_from_primitive_definition(D):
    u, rho, v, p = _states(D, 40, 11)
    n = np.random.default_rng(12).standard_normal((D, 40))
    assert np.allclose(ph.euler_flux_n(u, n, GAMMA), _flux_primitive(rho, v, p, n), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("D", [2, 3])
def test_roe_average_has_property_u(D):
    # the reference Roe state below is the one of Roe's construction:
    # A(u~) (u_R - u_L) = F(u_R) - F(u_L) for any pair, any direction
    ul, rl, vl, pl = _states(D, 12, 21)
    ur, rr, vr, pr = _states(D, 12, 22)
    nrm = np.random.default_rng(23).standard_normal((D, 12))
    for k in range(12):
        nb = nrm[:, k] / np.linalg.norm(nrm[:, k])
        ut, _ = _roe_state(rl[k], vl[:, k], pl[k], rr[k], vr[:, k], pr[k])
        A = _jacobian(ut, nb)
        dF = _flux_conserved(ur[:, k:k + 1], nb[:, None])[:, 0] - _flux_conserved(ul[:, k:k + 1], nb[:, None])[:, 0]
        assert np.allclose(A @ (ur[:, k] - ul[:, k]), dF, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3])
def test_roe_dissipation_is_abs_jacobian_at_roe_state(D):
    # entropy fix off: the oracle's wave-by-wave dissipation must equal
    # |A(u~)| du with |A| from the eigendecomposition; every term of it,
    # the shear waves' included, moves the result
    k = 30
    u_in, rl, vl, pl = _states(D, k, 31)
    u_out, rr, vr, pr = _states(D, k, 32)
    n = 0.5 + np.random.default_rng(33).standard_normal((D, k))
    diss = _oracle_dissipation(u_out, u_in, n, 0.0)
    for j in range(k):
        nb = n[:, j] / np.linalg.norm(n[:, j])
        ut, _ = _roe_state(rl[j], vl[:, j], pl[j], rr[j], vr[:, j], pr[j])
        absA, _ = _abs_matrix(_jacobian(ut, nb), np.abs)
        ref = absA @ (u_out[:, j] - u_in[:, j])
        assert np.allclose(diss[:, j], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("D", [2, 3])
def test_roe_shear_wave_alone(D):
    # a pure shear jump (same rho, p and normal velocity; tangential
    # velocity differs) is carried by the repeated eigenvalue v.n alone:
    # the dissipation is |v~.n| rho~ (0, dv_t, v~.dv_t) with nothing from
    # the acoustic waves
    rng = np.random.default_rng(41)
    for _ in range(10):
        nb = rng.standard_normal(D)
        nb /= np.linalg.norm(nb)
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 3.0)
        v_l = rng.uniform(-1, 1, D)
        dvt = rng.uniform(-1, 1, D)
        dvt -= (dvt @ nb) * nb
        v_r = v_l + dvt
        cons = lambda v: np.concatenate([[rho], rho * v, [p / (GAMMA - 1) + 0.5 * rho * v @ v]])
        u_l, u_r = cons(v_l), cons(v_r)
        diss = _oracle_dissipation(u_r[:, None], u_l[:, None], nb[:, None], 0.0)[:, 0]
        vt = 0.5 * (v_l + v_r)           # equal densities: the Roe velocity is the mean
        ref = abs(vt @ nb) * rho * np.concatenate([[0.0], dvt, [vt @ dvt]])
        assert np.allclose(diss, ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3])
def test_roe_entropy_fix_is_harten(D):
    # near-stagnation normal velocity puts the shear/entropy eigenvalue
    # v.n below delta = 0.1 c~: the dissipation is R f(Lambda) R^-1 du
    # with Harten's f(l) = (l^2 + delta^2) / (2 delta) for |l| < delta
    k = 20
    u_in, rl, vl, pl = _states(D, k, 51, vscale=0.03)
    u_out, rr, vr, pr = _states(D, k, 52, vscale=0.03)
    n = np.random.default_rng(53).standard_normal((D, k))
    diss = _oracle_dissipation(u_out, u_in, n, 0.1)
    hit = 0
    for j in range(k):
        nb = n[:, j] / np.linalg.norm(n[:, j])
        ut, ct = _roe_state(rl[j], vl[:, j], pl[j], rr[j], vr[:, j], pr[j])
        delta = 0.1 * ct
        f = lambda l: np.where(np.abs(l) < delta, (l * l + delta * delta) / (2 * delta), np.abs(l))
        absA, lam = _abs_matrix(_jacobian(ut, nb), f)
        hit += int((np.abs(lam) < delta).any())
        ref = absA @ (u_out[:, j] - u_in[:, j])
        assert np.allclose(diss[:, j], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    assert hit == k


@pytest.mark.parametrize("D", [2, 3])
def test_roe_supersonic_upwinding_with_tangential_jumps(D):
    # every eigenvalue of A(u~) positive along n (normal Mach number ~3 on
    # both sides, tangential velocities differing at random): |A| = A, so
    # by property U the flux is the inside state's physical flux
    rng = np.random.default_rng(61)
    k = 16
    nrm = rng.standard_normal((D, k))
    nb = nrm / np.sqrt((nrm * nrm).sum(0))
    u_in, rl, vl, pl = _states(D, k, 62)
    u_out, rr, vr, pr = _states(D, k, 63)

    def push(rho, v, p):
        c = np.sqrt(GAMMA * p / rho)
        v = v + (3.0 * c - (v * nb).sum(0)) * nb   # normal velocity 3c, tangential kept
        return v, np.concatenate([[rho], rho * v, [p / (GAMMA - 1) + 0.5 * rho * (v * v).sum(0)]])

    vl, u_in = push(rl, vl, pl)
    vr, u_out = push(rr, vr, pr)
    assert (np.abs((vl - vr) - ((vl - vr) * nb).sum(0) * nb).max(0) > 1e-3).all()   # real shear jumps
    scale = 2.5
    f = ph.roe_flux(u_out, u_in, scale * nb, GAMMA)
    assert np.allclose(f, scale * _flux_primitive(rl, vl, pl, nb), rtol=1e-12, atol=1e-12)
    # the same pair seen from the other side: flow leaves through -n,
    # so the upwind state is the outside one
    f = ph.roe_flux(u_in, u_out, -scale * nb, GAMMA)
    assert np.allclose(f, -scale * _flux_primitive(rl, vl, pl, nb), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3])
def test_lax_friedrichs_wave_speed(D):
    # local Lax-Friedrichs: (F(u_in) + F(u_out)).n / 2 - lam |n| (u_out - u_in) / 2
    # with lam = max over the two traces of |v.n^| + c, c = sqrt(gamma p / rho)
    k = 40
    u_in, rl, vl, pl = _states(D, k, 71)
    u_out, rr, vr, pr = _states(D, k, 72)
    n = 1.7 * np.random.default_rng(73).standard_normal((D, k))
    nn = np.sqrt((n * n).sum(0))
    nb = n / nn
    lam = np.maximum(np.abs((vl * nb).sum(0)) + np.sqrt(GAMMA * pl / rl),
                     np.abs((vr * nb).sum(0)) + np.sqrt(GAMMA * pr / rr))
    ref = 0.5 * nn * (_flux_primitive(rl, vl, pl, nb) + _flux_primitive(rr, vr, pr, nb)) \
        - 0.5 * lam * nn * (u_out - u_in)
    assert np.allclose(ph.lf_flux(u_out, u_in, n, GAMMA), ref, rtol=1e-12, atol=1e-12)
