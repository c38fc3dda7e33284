"""The element shape of the channel workload: 3-D Navier-Stokes at p = 4
with no-slip walls, through the C ABI in FP32 and FP64. The FP64 element
block of the preconditioner (325 KB) does not fit in shared memory and is
assembled and factored in place in global memory. References as in the
wall tests: the oracle's complex steps of its full residual for A x and for
the diagonal blocks of sampled wall elements, then its masking, ILU(0) and
solve. Mesh: a 3 x 2 x 3 channel (every element has a wall face), one
sampled element for the factors and the solve, the whole mesh for A x."""
import types

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import solvers as S
from oracle.residual import Discretization, full_residual
from submesh import H_CS, diag_block

pytestmark = pytest.mark.gpu

SHIFT, SCALE = 1.0, -0.02


@pytest.fixture(scope="module")
def L():
    from paper_1204_1533_gb300 import build, ldg
    build.build()
    return ldg


def test_channel_p4_matvec_and_preconditioner(L):
    import torch
    m = I.channel_mesh(3, 2, 3, 4)
    eq = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 1.0 / 5000.0, "Pr": 0.72, "bc": {1: "wall"}}
    U = I.smooth_perturbation(m, I.channel_state(m), 0.02)
    disc = Discretization(m, eq)
    h = L.ldg_setup(m, eq)
    Ut = torch.from_numpy(U).cuda()
    x = np.random.default_rng(11).standard_normal(U.shape)
    Ax = np.imag(full_residual(disc, U + 1j * H_CS * x)) / H_CS
    y_ref = SHIFT * x + SCALE * Ax
    pat = S.line_pattern(3, 4)
    one = types.SimpleNamespace(E=1, nc=5, npe=125, D=3, p=4)
    walled = np.nonzero((m["btag"] == 1).any(axis=1))[0]
    els = np.random.default_rng(1).choice(walled, 1, replace=False)
    Fo = np.concatenate([S.ilu0(S.masked_blocks(one, diag_block(disc, U, e), SHIFT, SCALE), pat) for e in els])
    zo = S.ilu_apply(Fo, pat, x[els])
    Fo_p = np.stack([Fo[:, i, pat[i]] for i in range(125)], axis=1)
    for prec, tv, tf, ta in ((L.PREC_FP32, 1e-5, 1e-5, 1e-4), (L.PREC_FP64, 1e-11, 1e-10, 1e-10)):
        dt = torch.float32 if prec == L.PREC_FP32 else torch.float64
        xt = torch.from_numpy(x).to(dt).cuda()
        J = L.ldg_jacobian(h, Ut, prec)
        y = torch.empty_like(xt)
        L.ldg_jacvec(h, J, SHIFT, SCALE, xt, y, prec)
        P = L.ldg_precond(h, J, SHIFT, SCALE)
        z = torch.empty_like(xt)
        L.ldg_precond_apply(h, P, xt, z, prec)
        torch.cuda.synchronize()
        err_y = np.abs(y.double().cpu().numpy() - y_ref).max() / np.abs(y_ref).max()
        assert err_y <= tv, (prec, err_y)
        Fg = L.ldg_pc_export(P, prec).astype(np.float64)[els]
        scale_r = np.abs(Fo_p).max(axis=(2, 3, 4), keepdims=True)
        err_f = (np.abs(Fg - Fo_p) / scale_r).max()
        assert err_f <= tf, (prec, err_f)
        err_z = np.abs(z.double().cpu().numpy()[els] - zo).max() / np.abs(zo).max()
        assert err_z <= ta, (prec, err_z)
