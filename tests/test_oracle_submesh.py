"""The sampling behind the full-size GPU parity tests, checked on the oracle
alone: an element's residual, its row of the Newton matvec A x and its
diagonal block of A, evaluated on a sub-mesh cut around it (5^D elements,
3^D for the block), equal the values on the whole periodic mesh."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle.residual import Discretization, full_residual
from submesh import H_CS, diag_block, oracle_eq, submesh


def _cases():
    m2 = I.vortex_mesh(8, 2)
    yield ("euler2d", m2, {"kind": "euler", "gamma": 1.4, "flux": "roe"},
           I.smooth_perturbation(m2, I.vortex_state(m2, x0=4.0, y0=4.0), 0.05), (3, 4))
    m3 = I.structured_mesh((6, 6, 6), 2, (0.0,) * 3, (2 * math.pi,) * 3, (True,) * 3, perturb=0.1)
    yield ("ns3d", m3, {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.05, "Pr": 0.72},
           I.smooth_perturbation(m3, I.tgv_state(m3, mach=0.3), 0.05), (2, 3, 3))


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_submesh_reproduces_element_quantities(case):
    name, m, eq, U, center = case
    disc = Discretization(m, eq)
    sub5, ids5, k5 = submesh(m, center, 2)
    e = ids5[k5]
    disc5 = Discretization(sub5, oracle_eq(eq))
    U5 = U[ids5]
    R_full = full_residual(disc, U)[e]
    R_sub = full_residual(disc5, U5, U5)[k5]
    assert np.abs(R_full - R_sub).max() <= 1e-12 * np.abs(R_full).max()
    x = np.random.default_rng(2).standard_normal(U.shape)
    Ax_full = np.imag(full_residual(disc, U + 1j * H_CS * x))[e] / H_CS
    Ax_sub = np.imag(full_residual(disc5, U5 + 1j * H_CS * x[ids5], U5))[k5] / H_CS
    assert np.abs(Ax_full - Ax_sub).max() <= 1e-12 * np.abs(Ax_full).max()
    sub3, ids3, k3 = submesh(m, center, 1)
    disc3 = Discretization(sub3, oracle_eq(eq))
    B_sub = diag_block(disc3, U[ids3], k3)
    B_full = diag_block(disc, U, e)
    assert np.abs(B_full - B_sub).max() <= 1e-12 * np.abs(B_full).max()
    # and the block is what a directional derivative sees on the element
    xe = np.zeros_like(U)
    xe[e] = x[e]
    Axe = np.imag(full_residual(disc, U + 1j * H_CS * xe))[e] / H_CS
    assert np.allclose(B_full @ x[e].reshape(-1), Axe.reshape(-1), rtol=1e-12, atol=1e-12 * np.abs(Axe).max())
