#!/usr/bin/env python
"""Throughput benchmark of the SD residual on the Taylor-Green vortex (Re = 1600,
Ma = 0.1, Pr = 0.71, gamma = 1.4, periodic [0, 2 pi]^3, 48^3 hexahedra at p = 4, i.e.
240^3 solution points and 5 conserved variables), compact scheme, FP32 residual with FP64
Runge-Kutta accumulation.

One step = one SSPRK(5,4) time step: five residual evaluations (trace, gradient and
flux/divergence kernels) plus the FP64 stage updates, on a state that is already
resident in HBM; the kinetic-energy/enstrophy diagnostics run once per timed window
(their cadence in the run is every 0.1 time units, ~200 steps, so this over-counts them).
value = DOF-updates/s = 5 * (solution points) / (seconds per step), summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain numpy definition) on the host
cores, each step one SSPRK(5,4) step of a bounded sample of the same workload.
Under torchrun every rank runs an independent copy of the workload (weak scaling;
the residual has no data-path collective across independent problems).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2608_09615_b300 import inputs  # noqa: E402

METRIC = "SD residual DOF-updates/s (FP32 vs FP64) and % HBM roofline, TGV Re=1600, 1 B300"
UNIT = "DOF-updates/s"
NE, P = (48, 48, 48), 4
DT = 5e-4            # SSPRK(5,4) step; acoustic CFL ~0.4 at 48^3 p4, Ma = 0.1
STAGES = 5


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), float(mp.get("sm_max_mhz", 2032.0)), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, 2032.0, "fallback"


def residual_flops_per_element(n, nv=5, ng=9, dim=3):
    """Algorithmic FP32 flops per element of the NS residual (FMA = 2 flops), by the operation
    counts of the method's steps, each step counted once per element whichever kernel does
    it (work a kernel repeats, such as the flux kernel re-deriving the traces and v^S that
    the gradient kernel also forms, is not counted). One 1D sweep of length n costs 2n - 1.
      trace: the 2 dim face traces of every variable (step 1, interface rows);
      vs:    v^S of every variable along every direction (D sweep + two corrections);
      gfaces: the ng own interface gradient components of the 2 dim faces (compact
             correction included);
      face:  the dim faces owned by the element (its +d faces), each point once: averages of
             the state and gradient (2 (nv + ng)), viscous flux (~60) and Roe (~150) plus the
             combination (~25);
      interior: the solution and ng gradient components at the n - 1 interior flux points of
             every line and the flux there (~85);
      div:   the M divergence of all n + 1 flux points.
    Returns the per-step counts and their attribution to the kernels that perform them
    ("flux" = interior + div: the work of the flux/divergence kernel)."""
    npnt, nq, nf = n ** dim, n ** (dim - 1), 2 * dim
    sw = 2 * n - 1
    st = {"trace": nf * nv * nq * sw,
          "vs": nv * dim * npnt * (sw + 4),
          "gfaces": nf * ng * nq * (sw + 2),
          "face": dim * nq * (2 * (nv + ng) + 235),
          "interior": dim * (n - 1) * nq * ((nv + ng) * sw + 85),
          "div": dim * nv * npnt * (2 * (n + 1) - 1 + 2)}
    return {"trace": st["trace"], "grad": st["vs"] + st["gfaces"], "face": st["face"],
            "flux": st["interior"] + st["div"], "steps": st, "total": sum(st.values())}


def curv_flops_per_element(n, nv=5):
    """Algorithmic FP32 flops per element of the curved-grid NS residual kernels (FMA = 2
    flops; a 1D sweep of length n costs 2n - 1). Metric terms from the trilinear map: one
    row of S = 2 bilinear tangents (6 x 7 flops) and a cross product (9); J = 3 tangents,
    a cross and a dot (77).
    k_ctrace: the 6 face traces of every variable.
    k_cgrad: J^-1 at the solution points; per family the row of S and u^{F,C} at its flux
    points and the 3 nv derivative sums sum_f M (u S_m); the 6 faces' 3 nv own interface
    gradients (compact: one coefficient sum_i L J^-1 M and one row of S per face point).
    k_cface: the 3 faces owned by the element, per point: the row of S, unit normal, the
    penalty, averages, Roe along the normal (~180) and the full viscous flux (~110).
    k_cflux: J^-1; per family at the n - 1 interior flux points the extrapolated state and
    3 nv gradient components, the row of S and S . (F_c - F_v) (~140); the divergence of all
    n + 1 flux points; the J^-1 scaling."""
    npnt, nq, nfp = n ** 3, n ** 2, (n + 1) * n ** 2
    sw = 2 * n - 1
    row, jac = 51, 78
    trace = 6 * nv * nq * sw
    fam_grad = nfp * row + nfp * nv * sw + 2 * nv * nq + 3 * nv * npnt * (3 * (n + 1) + 1)
    grad = npnt * jac + 3 * fam_grad + 3 * nv * npnt + 6 * 3 * nv * nq * sw + 6 * nq * (3 * n + row) \
        + 6 * 3 * nv * nq * 3
    face = 3 * nq * (row + 10 + 6 * nv + 8 * nv + 180 + 110)
    fam_flux = (n - 1) * nq * (4 * nv * sw + row + 140) + nv * npnt * (2 * (n + 1))
    flux = npnt * jac + 3 * fam_flux + nv * npnt
    return {"trace": trace, "grad": grad, "face": face, "flux": flux}


# DRAM traffic of one k_line_flux launch at 48^3 p=4 (FP32, compact), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of that kernel), valid only while the kernel
# code (flux_sources_digest) hashes to the value recorded with it.
FLUX_TRAFFIC = {"ne": 48, "bytes": 804013056 + 251464448,
                "sources_sha256": "1ac4637e33b082623f91bdf5580b78002788772fbd56f851c4ca29f93184a6f7"}
FLUX_SOURCES = ("paper_2608_09615_b300/csrc/sd_line.cuh", "paper_2608_09615_b300/csrc/sd_kernels.cuh")


def code_digest(texts):
    """sha256 of C/CUDA source texts with comments, trailing blanks and blank lines removed
    (a change of the code changes it; a change of a comment does not)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for text in texts:
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()


def flux_sources_digest():
    """code_digest of the flux kernel's sources."""
    texts = []
    for f in FLUX_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), f)) as fh:
            texts.append(fh.read())
    return code_digest(texts)


def flux_traffic(ne):
    """Recorded per-launch DRAM bytes of k_line_flux for this grid, or None when the grid
    differs or the kernel code changed since the capture."""
    if flux_sources_digest() != FLUX_TRAFFIC["sources_sha256"] or tuple(ne) != (FLUX_TRAFFIC["ne"],) * 3:
        return None
    return FLUX_TRAFFIC["bytes"]


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() in ("active", "1", "yes"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself alone)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, npts, ms_per_step):
    """Whole-job DOF-updates/s: every rank advances its own copy of the workload by one
    SSPRK(5,4) step (STAGES residual evaluations) in ms_per_step (the slowest rank's)."""
    return world * STAGES * npts / (ms_per_step * 1e-3)


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_worker(args):
    """One SSPRK(5,4) step of the oracle on its own sample grid, in a worker process whose
    BLAS runs on one thread (all-cores baseline)."""
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = os.environ["MKL_NUM_THREADS"] = "1"
    sample_ne, seed = args
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass
    v, sec, npts = oracle_step_sample(sample_ne, 1, 0)
    return sec, npts


def oracle_all_cores(sample_ne, cores):
    """The oracle on every host core: `cores` worker processes (spawned, one BLAS thread
    each), each one SSPRK(5,4) step of its own sample grid of the workload; throughput =
    all workers' DOF-updates over the wall time of the pool."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [((2, 2, 2), k) for k in range(cores)])        # start-up, imports
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(sample_ne, k) for k in range(cores)])
        wall = time.perf_counter() - t0
    npts = sum(n for _, n in res)
    return STAGES * npts / wall, wall


def oracle_step_sample(sample_ne, steps, warmup):
    """SSPRK(5,4) steps of the FP64 oracle on a sample grid of the same workload."""
    from oracle.grid import Grid
    from oracle.physics import NavierStokes, NSParams
    from oracle.residual import residual
    from oracle.timestep import ssprk54_step
    g = Grid(3, sample_ne, (0.0,) * 3, (2 * math.pi,) * 3, P)
    phys = NavierStokes(NSParams())
    U = inputs.tgv_3d(sample_ne, P, perturb_seed=0)
    R = lambda V: residual(V, g, "compact", phys)  # noqa: E731
    for _ in range(warmup):
        U = ssprk54_step(R, U, DT)
    t0 = time.perf_counter()
    for _ in range(steps):
        U = ssprk54_step(R, U, DT)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    npts = int(np.prod(sample_ne)) * (P + 1) ** 3
    return STAGES * npts / dt, dt, npts


def workload_name(ne, scheme):
    """The workload both arms report: the Taylor-Green SSPRK(5,4) step of the benchmark."""
    npts = int(np.prod(ne)) * (P + 1) ** 3
    return ("TGV Re=1600 Ma=0.1 Pr=0.71, %dx%dx%d hex p=4 (%d DOF, 5 vars), %s scheme, Roe + Sutherland, "
            "FP32 residual, SSPRK(5,4) with FP64 state, dt=%g" % (tuple(ne) + (npts, scheme, DT)))


def run_reference(args, world):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = (8, 8, 8)
    value, sec, npts = oracle_step_sample(sample, args.steps, args.warmup)
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name((args.ne,) * 3, args.scheme),
                   "sample": "the FP64 oracle (numpy, host cores) on %dx%dx%d elements p=4 (%d DOF) of "
                             "that workload per step" % (sample + (npts,)),
                   "parallelism": "none (host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one SSPRK(5,4) step of the FP64 numpy oracle on a %dx%dx%d p=4 "
                                   "TGV sub-grid per step" % sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def residual_rate(sd, torch, dim, ne, p, scheme, phys, precision, U, reps=10, lo=0.0, hi=2 * math.pi):
    """ms per sd_residual call (CUDA events, after 2 warm-up calls) and DOF-updates/s."""
    lo, hi = (lo,) * dim, (hi,) * dim
    ctx = sd.SD(dim, ne, lo, hi, p, scheme, phys, precision)
    Ug = torch.from_numpy(np.ascontiguousarray(U)).to("cuda", ctx.dtype)
    R = torch.empty_like(Ug)
    for _ in range(2):
        ctx.residual(Ug, R)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.residual(Ug, R)
    e1.record()
    torch.cuda.synchronize()
    ok = bool(torch.isfinite(R).all())
    ctx.close()
    ms = e0.elapsed_time(e1) / reps
    npts = int(np.prod(ne)) * (p + 1) ** dim
    return {"ms": ms, "dof_per_s": npts / (ms * 1e-3), "dof": npts, "finite": ok}


def curvilinear_rate(sd, torch, ne, p, precision, fp32_peak, amp=0.15, reps=10):
    """The Taylor-Green residual on a curved grid: the 48^3 box with every node displaced
    by the smooth periodic field of inputs.wavy_lattice (amplitude 0.15 h). The state is
    the perturbed Taylor-Green field sampled at the uniform-grid positions (a smooth field;
    the time does not depend on the values). ms per sd_residual (CUDA events), per-kernel
    times from the context's profiling events, and the ALU roofline of the dominant kernel
    and of the whole residual against the algorithmic flops of curv_flops_per_element."""
    nodes = inputs.wavy_lattice(ne, (0.0,) * 3, (2 * math.pi,) * 3, amp=amp)
    ctx = sd.SD.curvilinear(nodes, p, "compact", sd.Physics(kind="ns"), precision)
    Ug = torch.from_numpy(inputs.tgv_3d(ne, p, perturb_seed=0)).to("cuda", ctx.dtype)
    R = torch.empty_like(Ug)
    for _ in range(2):
        ctx.residual(Ug, R)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.residual(Ug, R)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.profile(True)
    for _ in range(reps):
        ctx.residual(Ug, R)
    prof = ctx.profile_read()
    ctx.profile(False)
    ok = bool(torch.isfinite(R).all())
    ctx.close()
    kms = {k: prof[k][0] / max(prof[k][1], 1) for k in ("trace", "grad", "face", "flux_div")}
    fl = curv_flops_per_element(p + 1)
    fl["flux_div"] = fl.pop("flux")
    nelem = int(np.prod(ne))
    npts = nelem * (p + 1) ** 3
    top = max(kms, key=kms.get)
    names = {"trace": "k_ctrace", "grad": "k_cgrad", "face": "k_cface", "flux_div": "k_cflux"}
    ach = fl[top] * nelem / (kms[top] * 1e-3) / 1e12
    res = sum(fl.values()) * nelem / (sum(kms.values()) * 1e-3) / 1e12
    return {"workload": "TGV Re=1600 on %dx%dx%d wavy trilinear hexahedra (node displacement %.2f h), p=%d, "
                        "compact, %s residual" % (ne + (amp, p, precision.upper())),
            "ms": ms, "dof_per_s": npts / (ms * 1e-3), "finite": ok,
            "kernels_ms": kms, "flops_per_element": fl,
            "roofline": {"bound": "alu", "kernel": names[top], "achieved": ach, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": ach / fp32_peak,
                         "residual_alu_tflops": res, "residual_frac": res / fp32_peak}}


def other_configs(sd, torch):
    """Residual rates on the other workloads the method is run on: 3D heat (32^3, p = 3
    and 4, nu = 0.01), the Taylor-Green grid with the BR1 scheme, Taylor-Green Re = 5000 on
    64^3 p = 4, and the small 1D cases (heat 16 elements p = 3; porous medium m = 2,
    128 elements p = 4), whose times are launch latency."""
    out = {}
    heat = sd.Physics(kind="heat", nu=0.01)
    for p in (3, 4):
        U, _, _ = inputs.heat_modes_3d((32,) * 3, p, seed=0)
        for prec in ("f32", "f64"):
            out["heat3d_32_p%d_compact_%s" % (p, prec)] = residual_rate(sd, torch, 3, (32,) * 3, p, "compact",
                                                                          heat, prec, U)
    U = inputs.tgv_3d(NE, P, perturb_seed=0)
    out["tgv48_p4_re1600_br1_f32"] = residual_rate(sd, torch, 3, NE, P, "br1", sd.Physics(kind="ns"), "f32", U)
    del U
    U = inputs.tgv_3d((64,) * 3, P, perturb_seed=0)
    out["tgv64_p4_re5000_compact_f32"] = residual_rate(sd, torch, 3, (64,) * 3, P, "compact",
                                                       sd.Physics(kind="ns", Re=5000.0), "f32", U, reps=5)
    del U
    U = inputs.sin_1d(16, 3)
    out["heat1d_16_p3_compact_f64"] = residual_rate(sd, torch, 1, (16,), 3, "compact",
                                                    sd.Physics(kind="heat", nu=1.0), "f64", U, reps=100)
    U = inputs.barenblatt_1d(128, 4, m=2.0)
    out["pme1d_128_p4_compact_f64"] = residual_rate(sd, torch, 1, (128,), 4, "compact",
                                                    sd.Physics(kind="pme", m_pme=2.0), "f64", U, reps=100,
                                                    lo=-10.0, hi=10.0)
    return out


def residual_only(sd, torch, args, ne, lo, hi, phys):
    if args.wavy > 0:
        nodes = inputs.wavy_lattice(ne, lo, hi, amp=args.wavy)
        ctx = sd.SD.curvilinear(nodes, P, args.scheme, phys, args.precision)
    else:
        ctx = sd.SD(3, ne, lo, hi, P, args.scheme, phys, args.precision)
    npts = int(np.prod(ne)) * (P + 1) ** 3
    U = torch.from_numpy(inputs.tgv_3d(ne, P, perturb_seed=0)).to("cuda", ctx.dtype)
    R = torch.empty_like(U)
    ctx.residual(U, R)
    torch.cuda.synchronize()
    ctx.profile(True)
    for _ in range(args.residual_only):
        ctx.residual(U, R)
    prof = ctx.profile_read()
    ctx.close()
    out = {k: {"ms_per_launch": ms / max(n, 1), "launches": n} for k, (ms, n) in prof.items() if n}
    tot = sum(v["ms_per_launch"] for v in out.values())
    print(json.dumps({"grid": ne, "p": P, "precision": args.precision, "scheme": args.scheme, "wavy": args.wavy,
                      "kernels": out, "residual_ms": tot, "dof_per_s": npts / (tot * 1e-3)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", default="compact", choices=["compact", "br1"])
    ap.add_argument("--ne", type=int, default=NE[0])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=16, help="CPU baseline sample grid edge")
    ap.add_argument("--residual-only", type=int, default=0, metavar="K",
                    help="only evaluate K residuals (FP32 unless --precision f64) and print the "
                         "per-kernel CUDA-event times; the small command used for ncu captures")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--wavy", type=float, default=0.0, metavar="AMP",
                    help="with --residual-only: the curved grid whose nodes move by AMP h (wavy_lattice)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the residual rates of the other workloads")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, world)
        return

    import torch
    import paper_2608_09615_b300 as sd
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    ne = (args.ne,) * 3
    lo, hi = (0.0,) * 3, (2 * math.pi,) * 3
    phys = sd.Physics(kind="ns")
    if args.residual_only:
        residual_only(sd, torch, args, ne, lo, hi, phys)
        return
    ctx = sd.SD(3, ne, lo, hi, P, args.scheme, phys, "f32")
    npts = int(np.prod(ne)) * (P + 1) ** 3
    U0 = inputs.tgv_3d(ne, P, perturb_seed=rank)
    U64 = torch.from_numpy(U0).cuda()
    stream = torch.cuda.current_stream()
    t = 0.0
    for _ in range(args.warmup):
        ctx.rk_step(U64, t, DT, "ssprk54")
        t += DT
    ctx.diagnostics(U64, t)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ctx.profile(True)
    l0 = ctx.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    diag = ctx.diagnostics(U64, t)
    for _ in range(args.steps):
        ctx.rk_step(U64, t, DT, "ssprk54")
        t += DT
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count() - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    value = job_value(world, npts, ms)
    final = ctx.diagnostics(U64, t, raise_nonfinite=False)

    # per-kernel times of the step
    step_kms = {k: prof[k][0] / max(prof[k][1], 1) for k in prof}
    # roofline of the dominant kernel of the residual (k_line_flux), from live CUDA events on
    # the context's stream: standalone FP32 residuals of the current state
    hbm, smax, peak_kind = peaks()
    Ug32r = U64.float()
    R32r = torch.empty_like(Ug32r)
    for _ in range(2):
        ctx.residual(Ug32r, R32r)
    torch.cuda.synchronize()
    ctx.profile(True)
    for _ in range(max(5, args.steps)):
        ctx.residual(Ug32r, R32r)
    rprof = ctx.profile_read()
    ctx.profile(False)
    del Ug32r, R32r
    kms = {k: rprof[k][0] / max(rprof[k][1], 1) for k in rprof}
    flops = residual_flops_per_element(P + 1)
    nelem = int(np.prod(ne))
    flux_avg_ms = kms["flux_div"]
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_derived = nsm * 128 * 2 * smax * 1e6 / 1e12    # TFLOP/s at the maximum SM clock
    # measured FMA throughput (scalar and paired FMA), the roofline's denominator
    fp32_meas = {"scalar": sd.measure_fp32_peak(False), "paired_f32x2": sd.measure_fp32_peak(True)}
    fp32_peak = max(fp32_meas.values())
    achieved = flops["flux"] * nelem / (flux_avg_ms * 1e-3) / 1e12
    alg_bytes_res = 2 * 5 * npts * 4                    # read U, write R (FP32)
    res_ms = sum(kms[k] for k in ("trace", "grad", "face", "flux_div"))
    res_alu = flops["total"] * nelem / (res_ms * 1e-3) / 1e12

    # the two stage modes of FP32 contexts side by side (sd_set_rk_stages): FP32 increments
    # (the default, timed above) and FP64 stage states; a short window each, same state
    stage_modes = {}
    for mode in ("f32", "f64"):
        ctx.set_rk_stages(mode)
        for _ in range(2):
            ctx.rk_step(U64, t, DT, "ssprk54")
        torch.cuda.synchronize()
        e0m, e1m = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0m.record(stream)
        for _ in range(5):
            ctx.rk_step(U64, t, DT, "ssprk54")
        e1m.record(stream)
        torch.cuda.synchronize()
        stage_modes["%s_stages_ms_per_step" % mode] = e0m.elapsed_time(e1m) / 5
    ctx.set_rk_stages("f32")

    # standalone residual rates, FP32 and FP64
    Ug32 = U64.float()
    R32 = torch.empty_like(Ug32)
    for _ in range(3):
        ctx.residual(Ug32, R32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nrep = max(5, args.steps)
    e0.record(stream)
    for _ in range(nrep):
        ctx.residual(Ug32, R32)
    e1.record(stream)
    torch.cuda.synchronize()
    res32_ms = e0.elapsed_time(e1) / nrep

    # end to end through the host-buffer C-ABI call: pinned FP32 U in, R out
    Uh = Ug32.cpu().pin_memory()
    Rh = torch.empty_like(Uh).pin_memory()
    for _ in range(2):
        ctx.residual_host(Uh, Rh)
    nrep_e = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(nrep_e):
        ctx.residual_host(Uh, Rh)
    e2e_s = (time.perf_counter() - t0) / nrep_e
    ctx.close()
    del Ug32, R32

    ctx64 = sd.SD(3, ne, lo, hi, P, args.scheme, phys, "f64")
    R64 = torch.empty_like(U64)
    for _ in range(2):
        ctx64.residual(U64, R64)
    torch.cuda.synchronize()
    e0.record(stream)
    nrep64 = 3
    for _ in range(nrep64):
        ctx64.residual(U64, R64)
    e1.record(stream)
    torch.cuda.synchronize()
    res64_ms = e0.elapsed_time(e1) / nrep64
    ctx64.close()

    others = curv = None
    if rank == 0 and not args.no_other_configs:
        others = other_configs(sd, torch)
        curv = curvilinear_rate(sd, torch, ne, P, "f32", fp32_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = args.cpu_sample
        v1, sec, n_s = oracle_step_sample((s, s, s), 1, 0)
        ncores = os.cpu_count() or 1
        sa = max(4, s // 2)
        va, wall = oracle_all_cores((sa, sa, sa), ncores)
        cpu = {"value": va, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": "one SSPRK(5,4) step (5 residuals) of the FP64 numpy oracle per worker: %d spawned "
                         "workers (one BLAS thread each) on their own %dx%dx%d p=4 TGV sub-grids, %.1f s wall"
                         % (ncores, sa, sa, sa, wall),
               "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                               "sample": "one SSPRK(5,4) step of the oracle on a %dx%dx%d p=4 TGV sub-grid "
                                         "(%d DOF), %.1f s" % (s, s, s, n_s, sec)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(ne, args.scheme),
                       "step": "one SSPRK(5,4) step = 5 residuals + 5 stage updates (FP32 stage "
                               "increments, FP64 state update once per step); diagnostics (FP64 sums) "
                               "once per timed window",
                       "l2": "inputs larger than L2 (FP32 state %.0f MB, FP64 state %.0f MB)"
                             % (5 * npts * 4 / 1e6, 5 * npts * 8 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "kernel": "k_line_flux",
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": flux_traffic(ne),
                         "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "peak_source": "measured FP32 FMA throughput (sd_measure_fp32_peak, the larger "
                                        "of scalar and paired FMA): %s TFLOP/s; derived %d SM x 128 lanes "
                                        "x 2 x %.0f MHz = %.1f TFLOP/s"
                                        % ({k: round(v, 1) for k, v in fp32_meas.items()}, nsm, smax,
                                           fp32_derived),
                         "flops_per_element": flops["flux"],
                         "avg_launch_ms": flux_avg_ms,
                         "residual": {"ms": res_ms, "alu_tflops": res_alu, "alu_frac": res_alu / fp32_peak,
                                      "hbm_frac_of_%s" % peak_kind: alg_bytes_res / (res_ms * 1e-3) / 1e9 / hbm,
                                      "algorithmic_bytes": alg_bytes_res},
                         "hbm_peak_gbs": hbm},
            "kernels_ms": {"residual": {"trace": kms["trace"], "grad": kms["grad"], "face": kms["face"],
                                        "flux_div": flux_avg_ms},
                           "step_per_launch": step_kms,
                           "step_launches_per_window": {k: prof[k][1] for k in prof}},
            "rk_stage_modes": stage_modes,
            "residual_dof_per_s": {"f32": npts / (res32_ms * 1e-3), "f64": npts / (res64_ms * 1e-3),
                                   "f32_ms": res32_ms, "f64_ms": res64_ms},
            "other_configs_residual": others,
            "curvilinear": curv,
            "e2e": {"value": npts / e2e_s, "unit": UNIT, "call": "sd_residual_host (FP32)",
                    "h2d_bytes_per_step": 5 * npts * 4, "d2h_bytes_per_step": 5 * npts * 4},
            "gpu_launches": launches,
            "clocks": clk,
            "diagnostics": {"ke_over_vol": diag["ke"] / diag["volume"],
                            "enstrophy_over_vol": diag["enstrophy"] / diag["volume"],
                            "final_nonfinite": final["nonfinite"]},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
