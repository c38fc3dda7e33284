"""Learned Newton initial guess for the BDF2 Newton-GMRES step.

Orchestration only; every step runs in libldg.so:
  1. trajectories: the implicit solver itself (ldg_newton_step, converged to
     the 1e-8 target) integrates the Taylor-Green vortex for Reynolds numbers
     drawn from U[400, 1600]; for every level n >= 2 the line features of
     (U^n, U^{n-1}, U^{n-2}) and the scaled correction targets of U^{n+1}
     are taken on a random subset of lines (ldg_line_features / _targets);
  2. standardisation from the first trajectory (feature mean / std, output
     scale per component);
  3. training: Adam on the GPU (ldg_mlp_train_step) over random batches;
  4. evaluation on a held-out Reynolds number: each level is solved once with
     the extrapolation predictor and once with the network's guess behind
     the residual check of LDG_PRED_CHECKED (fallback to extrapolation),
     comparing ||G|| of the initial guesses, Newton iterations and time.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import ldg

NS = {"kind": "ns", "gamma": 1.4, "flux": "roe", "Pr": 0.72}


def tgv_problem(n, p=3, re=1600.0):
    m = I.tgv_mesh(n, p)
    return m, dict(NS, mu=1.0 / re), I.tgv_state(m)


def _step(h, Un, Unm1, dt, first, mode, predictor=ldg.PRED_EXTRAP, guess=None, force=False,
          forcing=ldg.FORCING_FIXED):
    import torch
    Unext = torch.empty_like(Un) if guess is None else guess
    st = ldg.ldg_newton_step(h, Unext, Un, Unm1, None, dt,
                             ldg.solver_opts(mode=mode, predictor=predictor, first_step=first,
                                             force_rebuild=force, forcing=forcing))
    return Unext, st


def trajectory(h, U0, re, steps, dt, mode=ldg.MODE_MIXED):
    """Levels U^0 .. U^steps of one Reynolds number (device tensors)."""
    import torch
    ldg.ldg_set_viscosity(h, 1.0 / re)
    Us = [torch.from_numpy(U0).cuda()]
    for k in range(steps):
        nxt, _ = _step(h, Us[-1], Us[-2] if k else None, dt, first=(k == 0), mode=mode, force=(k == 0))
        Us.append(nxt)
    return Us


def fit_scaling(h, mlp, Us):
    """Feature mean / std and per-component output scale from one trajectory."""
    import torch
    n_in, n_out = mlp.n_in, mlp.n_out
    ldg.ldg_mlp_set_scaling(mlp, np.zeros(n_in), np.ones(n_in), np.ones(n_out))
    nl1 = h.E * h.nl
    X = torch.empty((nl1, ldg.MLP_INP), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((nl1, n_out), dtype=torch.float32, device="cuda")
    feats, targs = [], []
    for n in range(2, len(Us) - 1):
        ldg.ldg_line_features(h, mlp, Us[n], Us[n - 1], Us[n - 2], X)
        ldg.ldg_line_targets(h, mlp, Us[n + 1], Us[n], Us[n - 1], T)
        feats.append(X[:, :n_in].float())
        targs.append(T.clone())
    F = torch.cat(feats)
    Tt = torch.cat(targs)
    mean = F.mean(0).double().cpu().numpy()
    std = F.std(0).double().cpu().numpy()
    std = np.where(std > 1e-6 * np.abs(mean).max(), std, 1.0)
    nc = h.nc
    comp = Tt.reshape(Tt.shape[0], -1, nc).permute(2, 0, 1).reshape(nc, -1)
    cs = comp.std(1).double().cpu().numpy()
    cs = np.where(cs > 0, cs, 1.0)
    oscale = np.tile(cs, h.p + 1)
    ldg.ldg_mlp_set_scaling(mlp, mean, std, oscale)
    return mean, std, oscale


def collect(h, mlp, Us, lines_per_level, rng):
    """Features / targets of random lines of every level n >= 2."""
    import torch
    nl1 = h.E * h.nl
    X = torch.empty((nl1, ldg.MLP_INP), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((nl1, mlp.n_out), dtype=torch.float32, device="cuda")
    xs, ts = [], []
    for n in range(2, len(Us) - 1):
        ldg.ldg_line_features(h, mlp, Us[n], Us[n - 1], Us[n - 2], X)
        ldg.ldg_line_targets(h, mlp, Us[n + 1], Us[n], Us[n - 1], T)
        idx = torch.from_numpy(rng.choice(nl1, size=min(lines_per_level, nl1), replace=False)).cuda()
        xs.append(X[idx].clone())
        ts.append(T[idx].clone())
    return xs, ts


def train(mlp, X, T, steps, batch=4096, lr=1e-3, seed=0, log_every=1000):
    """Adam with cosine learning-rate decay on random batches; returns the
    loss history (every log_every steps)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    hist = []
    S = X.shape[0]
    for k in range(steps):
        idx = torch.randint(0, S, (min(batch, S),), generator=g, device="cuda")
        lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / steps))
        ldg.ldg_mlp_train_step(mlp, X[idx].contiguous(), T[idx].contiguous(), lr_k, loss)
        if k % log_every == 0 or k == steps - 1:
            hist.append((k, float(loss.item())))
    return hist


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3


def evaluate(h, mlp, U0, re, steps, dt, mode=ldg.MODE_MIXED, with_fp64=True, forcing=ldg.FORCING_FIXED):
    """Solve the held-out trajectory several times per level: extrapolation
    vs the network's checked guess (both in `mode`) and, with with_fp64, the
    plain FP64 solver with extrapolation, all with the same forcing of the
    linear solves; returns per-level statistics with the wall time of each
    step (the network's prediction included)."""
    import torch
    ldg.ldg_set_viscosity(h, 1.0 / re)
    Us = [torch.from_numpy(U0).cuda()]
    # first use of the predictor kernels and of the torch ops used below
    # (module loading) outside the timing
    warm = torch.empty_like(Us[0])
    ldg.ldg_mlp_predict(h, mlp, Us[0], Us[0], Us[0], warm)
    float((warm - Us[0]).norm())
    torch.cuda.synchronize()
    del warm
    rows = []
    for k in range(steps):
        first = k == 0
        Um1 = Us[-2] if k else None
        (ext, s_ext), ms_ext = _timed(lambda: _step(h, Us[-1], Um1, dt, first, mode, force=True, forcing=forcing))
        if k >= 2:
            pred = torch.empty_like(Us[-1])

            def learned_step():
                guess = torch.empty_like(Us[-1])
                ldg.ldg_mlp_predict(h, mlp, Us[-1], Us[-2], Us[-3], guess)
                pred.copy_(guess)  # the guess before the solver overwrites it
                return _step(h, Us[-1], Um1, dt, first, mode, predictor=ldg.PRED_CHECKED, guess=guess, force=True,
                             forcing=forcing)
            (nn_, s_nn), ms_nn = _timed(learned_step)
            e_mlp = float((pred - ext).norm())
            e_ext = float((2.0 * Us[-1] - Us[-2] - ext).norm())
            row = {"level": k, "res0": s_ext["res0"], "res_extrap": s_ext["res_pred"],
                   "res_mlp": s_nn["res_pred"], "mlp_weight": s_nn["pred_weight"],
                   "err_extrap": e_ext, "err_mlp": e_mlp,
                   "newton_extrap": s_ext["newton_its"], "newton_mlp": s_nn["newton_its"],
                   "gmres_extrap": s_ext["gmres_its"], "gmres_mlp": s_nn["gmres_its"],
                   "ms_extrap": ms_ext, "ms_mlp": ms_nn,
                   "diff": float((nn_ - ext).abs().max() / ext.abs().max())}
            if with_fp64:
                (u64, s64), ms64 = _timed(lambda: _step(h, Us[-1], Um1, dt, first, ldg.MODE_FP64, force=True,
                                                        forcing=forcing))
                row.update({"ms_fp64": ms64, "newton_fp64": s64["newton_its"], "gmres_fp64": s64["gmres_its"],
                            "diff_fp64": float((ext - u64).norm() / u64.norm())})
            rows.append(row)
        Us.append(ext)
    return rows


def init_params(n_in, n_out, seed):
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases, last layer x0.1."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = [(n_in, 128), (128, 128), (128, 128), (128, n_out)]
    for li, (a, b) in enumerate(shapes):
        lim = 1.0 / math.sqrt(a)
        W = rng.uniform(-lim, lim, size=(a, b)) * (0.1 if li == 3 else 1.0)
        parts += [W.ravel(), np.zeros(b)]
    return np.concatenate(parts)


def summarize(rows):
    """Means over the evaluated levels of one held-out trajectory."""
    out = {"mean_res_ratio_mlp_over_extrap": float(np.mean([r["res_mlp"] / r["res_extrap"] for r in rows])),
           "newton_extrap": float(np.mean([r["newton_extrap"] for r in rows])),
           "newton_mlp": float(np.mean([r["newton_mlp"] for r in rows])),
           "gmres_extrap": float(np.mean([r["gmres_extrap"] for r in rows])),
           "gmres_mlp": float(np.mean([r["gmres_mlp"] for r in rows])),
           "mean_err_ratio_mlp_over_extrap": float(np.mean([r["err_mlp"] / r["err_extrap"] for r in rows])),
           "mean_mlp_weight": float(np.mean([r["mlp_weight"] for r in rows])),
           "ms_mixed_extrap": float(np.mean([r["ms_extrap"] for r in rows])),
           "ms_mixed_mlp": float(np.mean([r["ms_mlp"] for r in rows]))}
    if rows and "ms_fp64" in rows[0]:
        out.update({"ms_fp64_extrap": float(np.mean([r["ms_fp64"] for r in rows])),
                    "newton_fp64": float(np.mean([r["newton_fp64"] for r in rows])),
                    "gmres_fp64": float(np.mean([r["gmres_fp64"] for r in rows])),
                    "max_rel_diff_mixed_vs_fp64": float(np.max([r["diff_fp64"] for r in rows]))})
    return out


def experiment(n=16, p=3, n_traj=200, steps=10, dt=0.03, train_steps=20000, lines=4096, seed=2024,
               held_out=1200.0, eval_steps=12, lr=1e-3, verbose=True,
               forcings=(ldg.FORCING_FIXED, ldg.FORCING_TARGET)):
    """Trajectories, training and the held-out evaluation; the summary of the
    first forcing policy is at the top level, the others under
    "forcing_<policy>"."""
    import torch
    m, eq, U0 = tgv_problem(n, p)
    h = ldg.ldg_setup(m, eq)
    n_in, n_out = 3 * (p + 1) * h.nc + h.D * h.D, (p + 1) * h.nc
    mlp = ldg.ldg_mlp_create(n_in, n_out)
    ldg.ldg_mlp_params(mlp, init_params(n_in, n_out, 7))
    rng = np.random.default_rng(seed)
    res = rng.uniform(400.0, 1600.0, size=n_traj)
    t0 = time.perf_counter()
    xs, ts = [], []
    for i, re in enumerate(res):
        Us = trajectory(h, U0, re, steps, dt)
        if i == 0:
            fit_scaling(h, mlp, Us)
        x, t = collect(h, mlp, Us, lines, rng)
        xs += x
        ts += t
        del Us
    X = torch.cat(xs)
    T = torch.cat(ts)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = train(mlp, X, T, train_steps, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"mesh": f"{n}^3", "p": p, "trajectories": n_traj, "levels_per_trajectory": steps, "dt": dt,
           "samples": int(X.shape[0]), "train_steps": train_steps, "t_generate_s": t_gen,
           "t_train_s": t_train, "loss_first": hist[0][1], "loss_last": hist[-1][1],
           "held_out_re": held_out}
    names = {ldg.FORCING_FIXED: "fixed", ldg.FORCING_TARGET: "target"}
    for k, f in enumerate(forcings):
        rows = evaluate(h, mlp, U0, held_out, eval_steps, dt, forcing=f)
        summ = dict(summarize(rows), levels=rows)
        if k == 0:
            out.update(summ)
            out["forcing"] = names[f]
        else:
            out["forcing_" + names[f]] = summ
    if verbose:
        print(json.dumps({k: v for k, v in out.items() if k != "levels" and not k.startswith("forcing_")}),
              flush=True)
        for k, v in out.items():
            if k.startswith("forcing_"):
                print(k, json.dumps({a: b for a, b in v.items() if a != "levels"}), flush=True)
    return out, mlp, h


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--traj", type=int, default=200)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--dt", type=float, default=0.03)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--lines", type=int, default=4096)
    ap.add_argument("--eval-steps", type=int, default=12)
    ap.add_argument("--out", default=None, help="write the result JSON here")
    a = ap.parse_args()
    from . import build
    build.build()
    out, _, _ = experiment(a.n, 3, a.traj, a.steps, a.dt, a.train_steps, a.lines, eval_steps=a.eval_steps)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
