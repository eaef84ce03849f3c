"""Taylor-Green vortex runs on the GPU (Sec. 4.4): SSPRK(5,4) time stepping of the SD
residual from the Sec. 4.4 initial field, with the volume diagnostics sampled at a fixed
interval: kinetic energy (1/2 int u.u and 1/2 int rho u.u), enstrophy, conserved totals.
The kinetic-energy dissipation rate -dE_k/dt is taken by centred differences of the
samples.

    python -m paper_2608_09615_b300.tgv --ne 48 --p 4 --re 1600 --t-end 20 --every 0.1

The time step is cfl * h / ((p + 1)(u0 + c0)), with c0 = u0 / Ma the reference sound
speed, adjusted so that a whole number of steps fills each sampling interval. A run
stops early, and says so, when the state stops being finite.

With --wavy AMP the grid is the box's lattice with every node moved by the smooth periodic
field of inputs.wavy_lattice (amplitude AMP h): curved trilinear elements, the Taylor-Green
field evaluated at their solution points, and the time step scaled by 1 - 2 AMP (the
smallest node spacing).
"""
import argparse
import json
import math
import time

import numpy as np

from . import SD, Physics, inputs


def time_step(ne, p, Ma=0.1, u0=1.0, cfl=0.2, L=1.0):
    h = 2.0 * math.pi * L / ne
    return cfl * h / ((p + 1) * (u0 + u0 / Ma))


def run(ne, p, Re=1600.0, scheme="compact", t_end=20.0, every=0.1, precision="f32", cfl=0.2, Ma=0.1,
        rk="ssprk54", physics=None, closure=None, on_sample=None, perturb_seed=None, wavy=0.0):
    """Run and return a dict with the sample times, the diagnostics per sample, the time
    step, the wall time and the time at which the state stopped being finite (or None).
    wavy > 0: the curved grid of inputs.wavy_lattice with node displacement wavy * h."""
    import torch
    dt = time_step(ne, p, Ma, cfl=cfl) * (1.0 - 2.0 * wavy)
    steps_per = max(1, int(round(every / dt)))
    dt = every / steps_per
    phys = physics or Physics(kind="ns", Re=Re, Ma=Ma)
    if wavy > 0.0:
        nodes = inputs.wavy_lattice((ne,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, amp=wavy)
        ctx = SD.curvilinear(nodes, p, scheme, phys, precision)
        X = inputs.curvilinear_coordinates(nodes, p)
    else:
        ctx = SD(3, (ne,) * 3, (0.0,) * 3, (2 * math.pi,) * 3, p, scheme, phys, precision)
        X = None
    if closure is not None:
        ctx.closure_enable(*closure)
    U = torch.from_numpy(inputs.tgv_3d((ne,) * 3, p, Ma=Ma, perturb_seed=perturb_seed, X=X)).cuda()
    t = 0.0
    rec = [ctx.diagnostics(U, t, raise_nonfinite=False)]
    if on_sample:
        on_sample(t, U)
    blowup = None
    t0 = time.time()
    for k in range(int(round(t_end / every))):
        for _ in range(steps_per):
            ctx.rk_step(U, t, dt, rk)
            t += dt
        t = (k + 1) * every                    # no drift of the sample times
        d = ctx.diagnostics(U, t, raise_nonfinite=False)
        rec.append(d)
        if on_sample:
            on_sample(t, U)
        if d["nonfinite"]:
            blowup = t
            break
    torch.cuda.synchronize()
    wall = time.time() - t0
    ctx.close()
    return {"t": [d["t"] for d in rec], "diag": rec, "dt": dt, "wall_s": wall, "blowup": blowup,
            "steps": steps_per * (len(rec) - 1)}


def dissipation(rec, every):
    """-dE_k/dt (E_k = 1/2 int u.u per unit volume) by centred differences, at the interior
    sample times."""
    ke = np.array([d["ke"] / d["volume"] for d in rec])
    return -(ke[2:] - ke[:-2]) / (2.0 * every)


def summary(res, every):
    rec = res["diag"]
    ke = np.array([d["ke"] / d["volume"] for d in rec])
    ens = np.array([d["enstrophy"] / d["volume"] for d in rec])
    eps = dissipation(rec, every) if len(rec) > 2 else np.zeros(0)
    t = np.array(res["t"])
    out = {"dt": res["dt"], "steps": res["steps"], "wall_s": res["wall_s"], "blowup": res["blowup"],
           "ke0": float(ke[0]), "ke_end": float(ke[-1])}
    if eps.size and np.isfinite(eps).any():
        i = int(np.nanargmax(eps))
        out.update(eps_max=float(eps[i]), t_eps_max=float(t[1:-1][i]))
    if np.isfinite(ens).any():
        j = int(np.nanargmax(ens))
        out.update(ens_max=float(ens[j]), t_ens_max=float(t[j]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ne", type=int, default=48)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--re", type=float, default=1600.0)
    ap.add_argument("--scheme", nargs="+", default=["compact", "br1"])
    ap.add_argument("--t-end", type=float, default=20.0)
    ap.add_argument("--every", type=float, default=0.1)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--cfl", type=float, default=0.2)
    ap.add_argument("--ma", type=float, default=0.1)
    ap.add_argument("--wavy", type=float, default=0.0, metavar="AMP",
                    help="curved grid: nodes moved by AMP h (inputs.wavy_lattice)")
    ap.add_argument("--series", action="store_true", help="also print KE, enstrophy and dissipation series")
    a = ap.parse_args()
    for scheme in a.scheme:
        res = run(a.ne, a.p, a.re, scheme, a.t_end, a.every, a.precision, a.cfl, a.ma, wavy=a.wavy)
        line = {"ne": a.ne, "p": a.p, "Re": a.re, "Ma": a.ma, "scheme": scheme, "precision": a.precision,
                "cfl": a.cfl, "wavy": a.wavy}
        line.update(summary(res, a.every))
        if a.series:
            line["t"] = res["t"]
            line["ke"] = [d["ke"] / d["volume"] for d in res["diag"]]
            line["enstrophy"] = [d["enstrophy"] / d["volume"] for d in res["diag"]]
            line["dissipation"] = dissipation(res["diag"], a.every).tolist()
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
