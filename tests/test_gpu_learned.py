"""What the trained line MLP gains over plain BDF2 extrapolation.

A small version of the learned-predictor experiment (an 8^3 Taylor-Green
mesh, 24 solver-generated trajectories at Re ~ U[400, 1600], dt = 0.03, a
4000-step Adam run) evaluated on the held-out Re = 1200: the network's
initial guesses must have a clearly smaller nodal error and BDF2 residual
than the extrapolation on average, the residual check must keep a large
weight on the network's guess, and the converged solutions must agree to
the Newton tolerance. The size of the gain is an empirical claim (no closed
form pins it). With the target-aware forcing (each linear solve asked only
for the reduction the stopping rule still needs) the smaller start residual
turns into fewer GMRES iterations: the network's starts must not need more
iterations in total than extrapolation's."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_guess_beats_extrapolation():
    from paper_1204_1533_gb300 import build, learned
    build.build()
    out, _, _ = learned.experiment(n=8, n_traj=24, steps=10, dt=0.03, train_steps=4000, lines=4096,
                                   eval_steps=10, verbose=True)
    assert out["loss_last"] < 0.1 * out["loss_first"]
    assert out["mean_err_ratio_mlp_over_extrap"] < 0.5, out
    assert out["mean_res_ratio_mlp_over_extrap"] < 0.8, out
    assert out["mean_mlp_weight"] > 0.3
    for r in out["levels"]:
        assert r["diff"] < 1e-6
    tf = out["forcing_target"]
    assert sum(r["gmres_mlp"] for r in tf["levels"]) <= sum(r["gmres_extrap"] for r in tf["levels"]), tf
    assert tf["gmres_extrap"] <= out["gmres_extrap"], (tf["gmres_extrap"], out["gmres_extrap"])
