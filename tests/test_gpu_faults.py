"""Failure detection without a GPU fault: bad states and exhausted
iteration caps come back as status codes from the host-side checks (every
cap is a host counter; no kernel waits on anything), and the handle stays
usable afterwards."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}


@pytest.fixture(scope="module")
def L():
    from paper_1204_1533_gb300 import build, ldg
    build.build()
    return ldg


def test_nonfinite_state_and_newton_cap(L):
    import torch
    m = I.vortex_mesh(4, 2, L=5.0)
    U0 = I.vortex_state(m, x0=2.5, y0=2.5)
    h = L.ldg_setup(m, EULER)
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    bad = Un.clone()
    bad[1, 0, 3] = float("nan")
    with pytest.raises(L.LdgError) as e:
        L.ldg_newton_step(h, U1, bad, None, None, 0.05, L.solver_opts(mode=L.MODE_FP64, first_step=True))
    assert e.value.code == -4                                  # LDG_ERR_NONFINITE
    # one Newton iteration cannot reach a 1e-14 reduction
    with pytest.raises(L.LdgError) as e:
        L.ldg_newton_step(h, U1, Un, None, None, 0.05,
                          L.solver_opts(mode=L.MODE_FP64, first_step=True, rtol=1e-14, max_newton=1))
    assert e.value.code == -6                                  # LDG_ERR_NEWTON_MAXIT
    # the handle still works
    st = L.ldg_newton_step(h, U1, Un, None, None, 0.05, L.solver_opts(mode=L.MODE_MIXED, first_step=True))
    assert st["res_final"] <= 1e-8 * st["res0"]
    assert bool(torch.isfinite(U1).all())


def test_coupled_solve_cycle_cap(L):
    import torch
    m = I.poisson_square_mesh(4, 2)
    f = I.poisson_source(m)
    eq = {"kind": "poisson", "C11": 0.05, "C22": 0.05, "C11b": 1.0, "bc": {0: "dirichlet"}, "source": f,
          "gD": np.zeros_like(f)}
    h = L.ldg_setup(m, eq)
    U = torch.zeros(f.shape, dtype=torch.float64, device="cuda")
    Q = torch.zeros((16, 1, 2, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LdgError) as e:
        L.ldg_coupled_solve(h, U, Q, rtol=1e-14, restart=2, max_cycles=1)
    assert e.value.code == -6
    st = L.ldg_coupled_solve(h, U, Q, rtol=1e-10, restart=64, max_cycles=50)
    assert st["res_final"] <= 1e-10 * st["res0"] and math.isfinite(st["res_final"])
