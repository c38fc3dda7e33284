"""ldg_residual_noalloc: the residual without any device allocation.

Some callers may not call cudaMalloc once they are running (another
allocator owns the device memory, or the loop must not allocate); this entry
point gives them the residual with its gradient scratch in a fixed device
array. Its output must equal ldg_residual's within the residual tolerance,
on two consecutive calls (the second call finds the first call's data in
the shared array), and it must refuse problems larger than the array."""
import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 0.02, "Pr": 0.72}


def test_noalloc_residual_matches_residual_on_two_calls():
    import torch

    from paper_1204_1533_gb300 import build, ldg
    build.build()
    m = I.reorient(I.vortex_mesh(4, 3, perturb=0.15))[0]
    h = ldg.ldg_setup(m, NS)
    for seed in (11, 12):
        U = torch.from_numpy(I.smooth_perturbation(m, I.vortex_state(m), 0.05, seed=seed,
                                                   periods=[10, 10])).cuda()
        R_ref = torch.empty_like(U)
        ldg.ldg_residual(h, U, R_ref)
        R = torch.full_like(U, float("nan"))
        ldg.ldg_residual_noalloc(h, U, R)
        torch.cuda.synchronize()
        ref = R_ref.cpu().numpy()
        got = R.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_residual_refuses_oversized_problems():
    import torch

    from paper_1204_1533_gb300 import build, ldg
    build.build()
    m = I.tgv_mesh(11, 3)      # 1331 elements x 5 x 3 x 64 > 2^20 gradient values
    h = ldg.ldg_setup(m, dict(NS, mu=1 / 1600))
    U = torch.from_numpy(I.tgv_state(m)).cuda()
    R = torch.empty_like(U)
    with pytest.raises(ldg.LdgError) as err:
        ldg.ldg_residual_noalloc(h, U, R)
    assert err.value.code == -9


def _compare(ldg, h, U):
    import torch
    R_ref = torch.empty_like(U)
    ldg.ldg_residual(h, U, R_ref)
    R = torch.full_like(U, float("nan"))
    ldg.ldg_residual_noalloc(h, U, R)
    torch.cuda.synchronize()
    ref, got = R_ref.cpu().numpy(), R.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_euler_3d_and_reuse_after_a_larger_call():
    # Euler (first order: no scratch used), 3-D Navier-Stokes (the 3-D
    # gradient layout in the shared array), then a smaller 2-D problem after
    # the larger one left its gradient in the array
    import torch

    from paper_1204_1533_gb300 import build, ldg
    build.build()
    m2 = I.reorient(I.vortex_mesh(4, 3, perturb=0.15))[0]
    U2 = torch.from_numpy(I.smooth_perturbation(m2, I.vortex_state(m2), 0.05, seed=21, periods=[10, 10])).cuda()
    _compare(ldg, ldg.ldg_setup(m2, {"kind": "euler", "gamma": 1.4, "flux": "roe"}), U2)
    m3 = I.tgv_mesh(6, 3)      # 216 elements x 5 x 3 x 64 = 207,360 gradient values
    U3 = torch.from_numpy(I.smooth_perturbation(m3, I.tgv_state(m3), 0.05, seed=22,
                                                periods=[2 * np.pi] * 3)).cuda()
    _compare(ldg, ldg.ldg_setup(m3, dict(NS, mu=1 / 1600)), U3)
    _compare(ldg, ldg.ldg_setup(m2, NS), U2)


def test_noalloc_allocates_no_device_memory():
    import torch

    from paper_1204_1533_gb300 import build, ldg
    build.build()
    m = I.tgv_mesh(4, 3)
    h = ldg.ldg_setup(m, dict(NS, mu=1 / 1600))
    U = torch.from_numpy(I.tgv_state(m)).cuda()
    R = torch.empty_like(U)
    ldg.ldg_residual_noalloc(h, U, R)       # first call on the device: address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ldg.ldg_residual_noalloc(h, U, R)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
