"""Pins for the oracle's no-slip adiabatic wall (and the pressure-only wall
of the Euler equations), CPU only. The paper gives no wall condition; the
builder's wall flux carries no mass and, at the wall's zero velocity, no
energy (no work, no heat flux), so two invariants follow from the scheme's
telescoping: a fluid at rest with uniform pressure stays at rest (R = 0 on a
2-D isoparametric mesh, where free stream is preserved exactly), and on a
mesh periodic in the other directions the weighted sums of the mass and
energy rows of R vanish for any state while momentum is not conserved (the
walls push)."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle.residual import Discretization, conservation_weights, full_residual

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe", "bc": {1: "wall"}}
NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.02, "Pr": 0.72, "bc": {1: "wall"}}


def _bump_channel_2d(p):
    def bump(x):
        y = x.copy()
        y[..., 1] = x[..., 1] + 0.1 * np.sin(2 * math.pi * x[..., 0] / 3.0) * np.abs(x[..., 1])
        return y
    return I.structured_mesh((4, 4), p, (0.0, -1.0), (3.0, 1.0), (True, False), perturb=0.1,
                             node_map=bump, btag_of_face=lambda d, end: 1)


def _at_rest(m, nc, rho=1.2, p=2.0):
    E, npe = m["nodes"].shape[:2]
    U = np.zeros((E, nc, npe))
    U[:, 0] = rho
    U[:, nc - 1] = p / 0.4
    return U


@pytest.mark.parametrize("eq", [EULER, NS], ids=["euler", "ns"])
@pytest.mark.parametrize("p", [2, 3])
def test_fluid_at_rest_stays_at_rest(eq, p):
    m = _bump_channel_2d(p)
    disc = Discretization(m, eq)
    R = full_residual(disc, _at_rest(m, 4))
    assert np.abs(R).max() < 1e-11


@pytest.mark.parametrize("case", ["euler2d", "ns2d", "ns3d_channel"])
def test_walls_conserve_mass_and_energy_not_momentum(case):
    if case == "ns3d_channel":
        m = I.channel_mesh(3, 4, 3, 2)
        eq = NS
        U = I.smooth_perturbation(m, I.channel_state(m), 0.05, periods=[4, 2, 2])
    else:
        m = _bump_channel_2d(3)
        eq = EULER if case == "euler2d" else NS
        U0 = I.vortex_state(m, x0=1.5, y0=0.0, mach=0.3, eps=1.0)
        U = I.smooth_perturbation(m, U0, 0.05, periods=[3, 2])
    disc = Discretization(m, eq)
    R = full_residual(disc, U)
    W = conservation_weights(disc)[:, None, :]
    tot = (W * R).sum(axis=(0, 2))
    scale = (W * np.abs(R)).sum(axis=(0, 2))
    nc = R.shape[1]
    assert abs(tot[0]) < 1e-12 * scale[0]
    assert abs(tot[nc - 1]) < 1e-12 * scale[nc - 1]
    assert max(abs(tot[1:nc - 1])) > 1e-6 * scale[1:nc - 1].max()
