"""Learned per-element sub-grid closure for coarse Taylor-Green runs: data generation from
filtered fine SD runs, training of the 64-128-128-15 network, and evaluation of the coarse
run with and without it against the filtered fine run.

This module only orchestrates calls into the CUDA library (fine and coarse SSPRK(5,4)
time stepping, the box filter, flux means, features, targets, standardisation, the BF16
MLP forward/backward and Adam kernels); no step of the computation runs in Python.

    python -m paper_2608_09615_b300.closure --fine 64 --coarse 16 --re 1600 3000 5000

The paper has no learned component; the definitions (filter, targets, features, injection)
are those of include/sd.h's closure section.
"""
import argparse
import json
import math
import time

import numpy as np

from . import MLP, SD, Physics, closure_targets, colstats, filter_project, filter_matrix, standardise
from . import inputs, tgv


def init_params(seed, widths=(64, 128, 128, 15)):
    """He-uniform initial weights (W of shape (out, in)), zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = math.sqrt(6.0 / a)
        out.append((rng.uniform(-lim, lim, (b, a)).astype(np.float32), np.zeros(b, dtype=np.float32)))
    return out


def stable_dt(ne, p, Ma=0.1, cfl=0.2):
    """Acoustic time step of the periodic [0, 2 pi]^3 grid with u0 = 1 (tgv.time_step)."""
    return tgv.time_step(ne, p, Ma, cfl=cfl)


def run_tgv(ne, p, Re, t_end, every, precision="f32", scheme="compact", closure=None, on_sample=None):
    """SSPRK(5,4) Taylor-Green run on the GPU (tgv.run); returns the diagnostics every
    `every` time units (and calls on_sample(t, U) there)."""
    return tgv.run(ne, p, Re, scheme, t_end, every, precision, closure=closure, on_sample=on_sample)["diag"]


def training_data(fine_ne, coarse_ne, Re_list, t_end, every, pf=4, pc=3):
    """Features X (FP32, (samples, 64)), targets T ((samples, 15)) and the filtered kinetic
    energy curves of fine runs at the given Reynolds numbers."""
    import torch
    r = fine_ne // coarse_ne
    Pdev = torch.from_numpy(filter_matrix(pf, pc, r)).cuda()
    Xs, Ts, curves = [], [], {}
    for Re in Re_list:
        fine = SD(3, (fine_ne,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, pf, "compact", Physics(kind="ns", Re=Re), "f32")
        coarse = SD(3, (coarse_ne,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, pc, "compact",
                    Physics(kind="ns", Re=Re), "f64")
        fcurve = []

        def sample(t, U):
            _, mf = fine.closure_data(U.float(), features=False)
            Uc = filter_project(U, (coarse_ne,) * 3, r, pf, pc, Pdev)
            X, mc = coarse.closure_data(Uc)
            Xs.append(X)
            Ts.append(closure_targets(mf, mc, (coarse_ne,) * 3, r))
            fcurve.append(coarse.diagnostics(Uc, t))

        run_tgv(fine_ne, pf, Re, t_end, every, on_sample=sample)
        curves[Re] = fcurve
        fine.close()
        coarse.close()
    return torch.cat(Xs), torch.cat(Ts), curves


def train(X, T, steps=2000, lr=2e-3, seed=0, log_every=0):
    """Full-batch Adam training of the network on standardised features/targets."""
    mu_x, sg_x = colstats(X)
    mu_t, sg_t = colstats(T)
    Xb = standardise(X, mu_x, sg_x, bf16=True)
    Tn = standardise(T, mu_t, sg_t)
    net = MLP(init_params(seed), max_rows=X.shape[0])
    losses = []
    for k in range(steps):
        net.forward(Xb)
        loss = net.loss_backward(Tn)
        net.adam(lr=lr)
        if log_every and k % log_every == 0:
            losses.append((k, float(loss.item())))
    net.forward(Xb)
    losses.append((steps, float(net.loss_backward(Tn).item())))
    return net, (mu_x, sg_x, mu_t, sg_t), losses


def dissipation(rec, every):
    return tgv.dissipation(rec, every)


def evaluate(net, stats, coarse_ne, Re, t_end, every, reference, pc=3):
    """Dissipation-rate error (L2 over time, relative to the filtered fine run's curve) of
    the coarse run without and with the closure."""
    eps_ref = dissipation(reference, every)
    out = {}
    for name, cl in (("plain", None), ("closure", (net,) + tuple(stats))):
        rec = run_tgv(coarse_ne, pc, Re, t_end, every, closure=cl)
        if any(d["nonfinite"] for d in rec):
            out[name] = float("inf")
            continue
        eps = dissipation(rec, every)
        m = min(len(eps), len(eps_ref))
        out[name] = float(np.linalg.norm(eps[:m] - eps_ref[:m]) / np.linalg.norm(eps_ref[:m]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fine", type=int, default=64)
    ap.add_argument("--coarse", type=int, default=16)
    ap.add_argument("--re", type=float, nargs="+", default=[1600.0, 3000.0, 5000.0])
    ap.add_argument("--test-re", type=float, nargs="*", default=None)
    ap.add_argument("--holdout", type=float, default=None,
                    help="also train a second network without this Re (from the same fine data) "
                         "and evaluate it there")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--every", type=float, default=0.25)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=None, help="also write the JSON result to this file")
    a = ap.parse_args()
    import torch
    t0 = time.time()
    X, T, curves = training_data(a.fine, a.coarse, a.re, a.t_end, a.every)
    t1 = time.time()
    net, stats, losses = train(X, T, steps=a.steps, log_every=500)
    t2 = time.time()
    res = {}
    for Re in (a.test_re or a.re):
        if Re not in curves:
            _, _, c = training_data(a.fine, a.coarse, [Re], a.t_end, a.every)
            curves[Re] = c[Re]
        res[str(Re)] = evaluate(net, stats, a.coarse, Re, a.t_end, a.every, curves[Re])
    out = {"fine": "%d^3 p4" % a.fine, "coarse": "%d^3 p3" % a.coarse, "train_re": a.re,
           "samples": int(X.shape[0]), "losses": losses, "dissipation_rel_l2_error": res}
    if a.holdout is not None:
        # the samples of each Re are contiguous in X, T (training_data appends them in order)
        per = X.shape[0] // len(a.re)
        keep = torch.cat([torch.arange(i * per, (i + 1) * per, device=X.device)
                          for i, Re in enumerate(a.re) if Re != a.holdout])
        net_h, stats_h, losses_h = train(X[keep], T[keep], steps=a.steps, log_every=500)
        out["holdout"] = {"train_re": [Re for Re in a.re if Re != a.holdout], "test_re": a.holdout,
                          "losses": losses_h,
                          "dissipation_rel_l2_error": evaluate(net_h, stats_h, a.coarse, a.holdout, a.t_end,
                                                               a.every, curves[a.holdout])}
    out["seconds"] = {"data": t1 - t0, "train": t2 - t1, "eval": time.time() - t2}
    line = json.dumps(out)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
