"""Porous-medium (ZKB) runs with the interior penalty on the GPU (Sec. 4.3).

u_t = (u^m)_xx with m = 5 and C = 0.1 from the ZKB profile (Eq. zkb) at the time t0 at which
its support fills one element (the t0 formula of Sec. 4.3), on n_el equal elements of a
periodic interval of length 2 whose middle element is centred on x = 0, [-1 - h/2, 1 - h/2)
(the support reaches |x| = 0.39 at t = 1e-3; the paper gives neither the interval nor the
placement, and the profile must sit inside one element). Time stepping: RK4 in FP64 on the
GPU with dt = `safety` times RK4's real stability limit over the spectral radius of the
linearised operator, rho(B) m u_max^(m-1) / h^2 (rho(B) from the Bloch operator of the GPU
residual with this eta_IP; u_max of the exact profile at that time), so dt grows as
t^(2/3) as the profile spreads. The error is
the L2 norm over |x|^2 < 0.9 H(t) (the footnote of Sec. 4.3), Gauss quadrature, sampled at
log-spaced times.

    python -m paper_2608_09615_b300.pme --ne 100 200 --p 3 4 --eta 0 0.01 0.02 0.05 0.1 0.5 1.0

Only calls into the CUDA library advance the solution; the host evaluates the exact
profile and the error of the sampled states.
"""
import argparse
import json
import math

import numpy as np

from . import SD, Physics, inputs
from .eigen import RK4_REAL_LIMIT, spectral_radius


def zkb_t0(m, C, dx):
    """The t0 of Sec. 4.3: the ZKB support |x| <= sqrt(H(t)) equals dx / 2."""
    a1 = 1.0 / ((m - 1.0) + 2.0)
    return (C * 2.0 * m / (a1 * (m - 1.0)) * (2.0 / dx) ** 2) ** (-1.0 / (2.0 * a1))


def support_sq(m, C, t):
    """H(t): the 1D ZKB support is |x|^2 <= H."""
    a1 = 1.0 / ((m - 1.0) + 2.0)
    return 2.0 * m * C / (a1 * (m - 1.0)) * t ** (2.0 * a1)


def l2_error_masked(U, t, m, C, xs, ws, lo, h):
    """sqrt(sum_e (h/2) sum_i w_i (u - u_exact)^2) over the points with |x|^2 < 0.9 H(t)."""
    ne = U.shape[1]
    x = lo + (np.arange(ne)[:, None] + 0.5 + 0.5 * np.asarray(xs)[None, :]) * h
    ue = inputs.barenblatt(x, t, m, C)
    mask = x ** 2 < 0.9 * support_sq(m, C, t)
    w = 0.5 * h * np.asarray(ws)[None, :]
    return float(math.sqrt(np.sum(w * mask * (U[0] - ue) ** 2)))


def run(ne, p, scheme, eta_ip=0.0, m=5.0, C=0.1, t_end=1e-3, nsamples=40, length=2.0, safety=0.4):
    import torch
    h = length / ne
    lo = -0.5 * length - 0.5 * h
    hi = lo + length
    ctx = SD(1, (ne,), (lo,), (hi,), p, scheme, Physics(kind="pme", m_pme=m, eta_ip=eta_ip), "f64")
    xs, ws = ctx.points()
    t0 = zkb_t0(m, C, h)
    (x,) = inputs.coordinates(1, (ne,), (lo,), (hi,), p)
    U = torch.from_numpy(inputs.barenblatt(x, t0, m, C)[None].copy()).cuda()
    rho1 = spectral_radius(p, scheme, eta_ip, nth=91)          # h = 1, unit diffusivity
    alpha = 1.0 / ((m - 1.0) + 2.0)
    times = np.geomspace(max(t0 * 10.0, t_end * 1e-3), t_end, nsamples)
    t, steps, rec = t0, 0, []
    for ts in times:
        while t < ts * (1.0 - 1e-12):
            umax = t ** (-alpha) * C ** (1.0 / (m - 1.0))
            dt = safety * RK4_REAL_LIMIT * h * h / (rho1 * m * umax ** (m - 1.0))
            dt = min(dt, ts - t)
            ctx.rk_step(U, t, dt, "rk4")
            t += dt
            steps += 1
        rec.append((t, l2_error_masked(U.cpu().numpy(), t, m, C, xs, ws, lo, h)))
    ctx.close()
    return {"ne": ne, "p": p, "scheme": scheme, "eta_ip": eta_ip, "m": m, "C": C, "t0": t0, "steps": steps,
            "t": [r[0] for r in rec], "l2": [r[1] for r in rec]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ne", type=int, nargs="+", default=[100, 200])
    ap.add_argument("--p", type=int, nargs="+", default=[3, 4])
    ap.add_argument("--eta", type=float, nargs="+", default=[0.0, 0.01, 0.02, 0.05, 0.1, 0.5, 1.0])
    ap.add_argument("--t-end", type=float, default=1e-3)
    ap.add_argument("--samples", type=int, default=40)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = []
    for ne in a.ne:
        for p in a.p:
            for scheme in ("compact", "br1"):
                for eta in a.eta:
                    r = run(ne, p, scheme, eta, t_end=a.t_end, nsamples=a.samples)
                    r["l2_mean"] = float(np.mean(r["l2"]))
                    out.append(r)
                    print(json.dumps({k: r[k] for k in ("ne", "p", "scheme", "eta_ip", "steps", "l2_mean")}),
                          flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
