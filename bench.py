#!/usr/bin/env python3
"""Benchmark of the D2Q37 thermal LB step on GB300 (one JSON line on rank 0).

Workload (default): a 2048 x 4096 Rayleigh-Taylor lattice (8,388,608 sites,
32 seeded interface modes, tau = 0.6, g = 1e-5, walls at T = 0.5 / 1.5),
float64 populations (two copies, 2 x 2.49 GB, far larger than L2).  One
"step" is one fused propagate + bc + collide launch over the whole lattice.

value        float64 MLUPS (million lattice-site updates per second), state
             resident in HBM, CUDA-event time over K steps.
fp32_store   the same lattice stored as float32 deviations f_l - w_l rho0.
adjoint      one adjoint step (recompute + transposed collide + push) over
             the same lattice, as a ratio to the forward step time.
e2e          the same metric through the C ABI with pinned HOST buffers:
             per step set_state(host) -> step -> get_state(host), three
             independent lattices on their own streams.
roofline     the fused float64 kernel against the FP64 FMA rate measured by
             the library's probe (the step is FP64-pipe bound).
cpu_baseline the float64 oracle (NumPy) on a bounded sample of the workload.

--impl reference times the oracle itself (the only reference this method
has) on the host cores, with the same metric and workload.
Under torchrun each rank steps its own replica lattice (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q37 MLUPS, FP64 vs FP32-store, and adjoint/forward step time ratio, 1 GB300"
WORKLOAD = "D2Q37 FP64 step, Rayleigh-Taylor 2048x4096, 32 modes, tau=0.6, g=1e-5"

# Float64 work of the fused step per site, counted stage by stage from the
# collide's formulation (an FMA counts 2 flops, the division 1/rho counts 1).
# The plain formulation (every sum and the per-pair polynomial in float64):
# moment sums 110, site fields 9, gravity shift and Hermite coefficients 30,
# per-shell terms 81, per-pair polynomial and relaxation 312: 542.
# The kernel forms the moment sums and evaluates the equilibrium polynomial at
# the 36 moving velocities exactly in fixed point on the integer pipe, and
# takes the equilibrium coefficients straight from the moment sums; the
# float64 work it keeps is: r^2 / rho, the shifted velocity, its squares and
# theta 16, the Hermite coefficients 19, the 15 monomial coefficients of the
# equilibrium 34, the eight shell factors rho omega w_j 8, one multiply and one
# FMA per population 111: 188.  ncu counts 131.2 FP64 instructions per site on
# this kernel (DFMA 62.0, DMUL 66.1, DADD 3.1: 193 flops, the 188 plus the
# Newton-Raphson step of 1/rho).
FP64_FLOP_PER_SITE = 542
FP64_PIPE_FLOP_PER_SITE = 188
FP64_INSTR_PER_SITE_NCU = 131.2
FP64_PIPE_FLOP_PER_SITE_NCU = 193.2
# DRAM bytes per site of the float64 step (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of one 2048 x 1024 launch, 1192.06 MB / 2097152 sites;
# traffic grows with the site count, so a full launch is scaled by sites).
FP64_TRAFFIC_BYTES_PER_SITE_NCU = 568.42
BYTES_PER_SITE_FP64 = 2 * 37 * 8
BYTES_PER_SITE_FP32 = 2 * 37 * 4
FP64_NOMINAL_TFLOPS = 1.25


def _hbm_peak():
    """HBM copy bandwidth measured on this GPU type (MEASURED_PEAKS.json)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json"
    except (OSError, ValueError, KeyError):
        return 6789.6, "fallback: earlier GB300 measurement"


HBM_GBS_MEASURED, HBM_PEAK_SOURCE = _hbm_peak()
SECTIONS = ("fp64", "fp32", "fp64df", "regularized", "observe", "adjoint", "e2e", "fp32_error", "rollout", "batch", "cpu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lx", type=int, default=2048)
    ap.add_argument("--ly", type=int, default=4096)
    ap.add_argument("--only", default="", help="comma list of sections: " + ",".join(SECTIONS))
    ap.add_argument("--e2e-lattices", type=int, default=3,
                    help="independent lattices (one stream each) in the end-to-end measurement")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--error-steps", type=int, default=1000)
    ap.add_argument("--rollout-steps", type=int, default=2000)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-lattices", type=int, default=64)
    ap.add_argument("--batch-tile", type=int, default=-1,
                    help="batch tile shape index (default: autotune over all shapes)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def rt_lattice(lx, ly, precision, rho0=None, **kw):
    import synth
    from paper_1703_00186_gb300.lbm import Lattice
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 32, 0)
    r0 = float(rho.mean()) if rho0 is None else rho0
    lat = Lattice(lx, ly, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb, precision=precision, rho0=r0, **kw)
    lat.init(rho, ux, uy, T)
    return lat, (rho, ux, uy, T)


def time_steps(lat, k, torch):
    """CUDA-event time (ms) of k fused steps on the lattice's stream."""
    s = lat.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    lat.step(k)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1)


def dist_max(v, torch, world):
    """Max of a host scalar over the ranks (the slowest replica sets the time)."""
    if world <= 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(torch, world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def _oracle_worker_init(core):
    """Spawned oracle worker: one BLAS / OpenMP thread (set before NumPy is
    imported), pinned to one host core when `core` is given."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    if core is not None:
        os.sched_setaffinity(0, {core})
    sys.path.insert(0, ROOT)


def _oracle_slab(args):
    """`steps` float64 oracle steps on columns [x0, x0 + width) of the
    workload's fields (the slab periodic in x); returns sites x steps."""
    lx, ly, x0, width, steps = args
    import synth
    from oracle import model as M
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 32, 0)
    cols = slice(x0, x0 + width)
    p = M.Params(width, ly, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
    f = M.init_state(rho[:, cols], ux[:, cols], uy[:, cols], T[:, cols])
    for _ in range(steps):
        f = M.step(f, p)
    return width * ly * steps


def _oracle_throughput(lx, ly, workers, width, steps, pin_one_core=False):
    """MLUPS of the oracle on `workers` spawned processes, each stepping its own
    column slab (independent slabs: the oracle's work split over host cores
    as the paper splits a lattice over nodes).  Spawned, never forked: the
    parent holds a CUDA context."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    core = sorted(os.sched_getaffinity(0))[0] if pin_one_core else None
    with ctx.Pool(workers, initializer=_oracle_worker_init, initargs=(core,)) as pool:
        pool.map(_oracle_slab, [(lx, ly, 0, 8, 1)] * workers)  # imports, first-touch
        jobs = [(lx, ly, (i * width) % max(1, lx - width + 1), width, steps) for i in range(workers)]
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_slab, jobs))
        dt = time.perf_counter() - t0
    return done / dt / 1e6, dt


def cpu_baseline(lx, ly, budget_s):
    """The float64 oracle (NumPy, as it stands) on the host cores: every core
    available to the process steps its own column slab of the workload in a
    spawned worker, and one worker alone on one core for comparison."""
    cores = len(os.sched_getaffinity(0))
    width = max(8, lx // cores)
    # size the steps so that one worker's share takes about budget_s / 2
    probe, dt = _oracle_throughput(lx, ly, 1, 32, 1, pin_one_core=True)
    steps = int(max(1, min(20, budget_s / 2 / max(width * ly / (probe * 1e6), 1e-6))))
    v_all, t_all = _oracle_throughput(lx, ly, cores, width, steps)
    v_one, t_one = _oracle_throughput(lx, ly, 1, width, steps, pin_one_core=True)
    return {"value": v_all, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{cores} spawned workers, each {steps} steps of its own {width}x{ly} column slab "
                      f"of the 2048x4096 RT lattice (periodic in x), NumPy float64, one thread each; "
                      f"{t_all:.1f} s",
            "one_core": {"value": v_one, "unit": "MLUPS", "cores": 1,
                         "sample": f"one worker pinned to one core, {steps} steps of a {width}x{ly} slab; "
                                   f"{t_one:.1f} s"},
            "scaling_all_over_one": v_all / v_one}


FP32_ARITHS = ("split", "fp64_terms", "fp64_collide")
FIELD_TOL = 1e-5


def _field_errors(a, b):
    """max |a - b| / max |b| for each of rho, ux, uy, T (b is the float64 run),
    the row of each maximum, and for the velocity also max |a - b| in units
    of the lattice sound speed (sqrt(T0) = 1), since max |u| of a nearly still
    fluid is a poor scale."""
    names = ("rho", "ux", "uy", "T")
    out = {}
    for n, x, y in zip(names, a, b):
        diff = (x - y).abs()
        d = diff.max().item()
        scale = y.abs().max().item()
        out[n] = d / scale if scale > 0 else d
        out[n + "_at_row"] = int(diff.amax(dim=1).argmax().item())
        if n in ("ux", "uy"):
            out[n + "_abs"] = d
            out[n + "_max"] = scale
    return out


def _verdict(rows):
    """Per-field pass/fail against the 1e-5 relative target, over every
    recorded step (the worst one)."""
    fin = [r for r in rows if r.get("finite", True) and "rho" in r]
    if len(fin) < len(rows):
        return {"finite": False}
    worst = {k: max(r[k] for r in fin) for k in ("rho", "ux", "uy", "T", "ux_abs", "uy_abs")}
    v = {k: {"worst": worst[k], "pass": worst[k] <= FIELD_TOL} for k in ("rho", "ux", "uy", "T")}
    v["u_abs"] = {"worst": max(worst["ux_abs"], worst["uy_abs"]),
                  "pass": max(worst["ux_abs"], worst["uy_abs"]) <= FIELD_TOL,
                  "unit": "lattice sound speed sqrt(T0) = 1"}
    return v


def fp32_error_study(lx, ly, steps, torch):
    """Field error of the float32-store path against the float64 path (which
    the tests pin to the oracle within 1e-12), every 100 steps, for the three
    arithmetics of the float32-store collide: "split" (the default),
    "fp64_terms" (float64 moment sums and temperature-dependent equilibrium
    terms) and "fp64_collide" (the float64 collide between decode and encode:
    the error of the float32 storage alone).  Two contrasts: a stable one
    (T = 0.75 / 1.25) and the workload's (T = 0.5 / 1.5, which plain BGK does
    not keep stable at tau = 0.6)."""
    import synth
    from paper_1703_00186_gb300.lbm import Lattice
    res = {}
    for label, delta in (("delta_0.5", 0.5), ("delta_1.0", 1.0)):
        rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 32, 0, delta=delta)
        r0 = float(rho.mean())
        kw = dict(tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
        a = Lattice(lx, ly, precision="fp64", **kw).init(rho, ux, uy, T)
        bs = {m: Lattice(lx, ly, precision="fp32", rho0=r0, fp32_arith=m, **kw).init(rho, ux, uy, T)
              for m in FP32_ARITHS}
        rows = {m: [] for m in FP32_ARITHS}
        a.step(1)
        for m, b in bs.items():
            b.step(1)
        ref = a.moments()
        for m, b in bs.items():
            rows[m].append({"step": 1, **_field_errors(b.moments(), ref)})
        done = 1
        while done < steps:
            k = min(100 - done % 100, steps - done)
            a.step(k)
            for b in bs.values():
                b.step(k)
            done += k
            fin_a = a.check_finite()
            ref = a.moments() if fin_a else None
            for m, b in bs.items():
                finite = fin_a and b.check_finite()
                row = {"step": done, "finite": finite}
                if finite:
                    row.update(_field_errors(b.moments(), ref))
                rows[m].append(row)
        entry = {"t_top": tt, "t_bottom": tb, "rho0": r0}
        for m in FP32_ARITHS:
            entry[m] = {"errors": rows[m], "verdict": _verdict(rows[m])}
        if delta == 0.5:
            # cost of each arithmetic: CUDA-event time of 20 steps (state in HBM)
            for m, b in bs.items():
                t_ms = time_steps(b, 20, torch)
                entry[m]["mlups"] = lx * ly * 20 / (t_ms * 1e-3) / 1e6
        res[label] = entry
        del a, bs
        torch.cuda.empty_cache()
    res["definition"] = ("max |fp32 - fp64| / max |fp64| per field on the 2048x4096 RT lattice, "
                         "tau = 0.6, g = 1e-5, 32 modes; *_abs: max |fp32 - fp64| of the velocity in units "
                         "of the sound speed; verdict: worst recorded step against 1e-5")
    return res


def rollout_study(steps, torch):
    """Checkpointed adjoint rollout on a 256 x 512 RT lattice: time of the
    forward rollout and of the backward sweep (recompute + adjoint steps),
    and the gradient against float64 central differences on 16 seeded
    directions; FP64, FP32-store and FP64_DF (double-float collide and
    cotangent sums), and the FP32-store rollout with float32 cotangents."""
    import numpy as np

    import synth
    from paper_1703_00186_gb300.adjoint import temperature_loss
    from paper_1703_00186_gb300.lbm import Lattice
    lx, ly, K, tau, g = 256, 512, 50, 0.8, 1e-4
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 4, 1)
    target = T + synth.smooth_field(lx, ly, 2, amp=0.05)
    dT0 = 0.01 * synth.smooth_field(lx, ly, 3, amp=1.0)
    dev = "cuda"
    rho_t, T_t, tgt = (torch.tensor(v, device=dev) for v in (rho, T, target))
    res = {"lattice": f"{lx}x{ly}", "steps": steps, "checkpoint_every": K, "tau": tau, "g": g}
    grads = {}
    fds, dirs = [], []
    # "fp32_f32cot": the FP32-store rollout with float32 cotangents and the
    # float32 adjoint (lbm_adjoint_step_f32)
    for name in ("fp64", "fp32", "fp64df", "fp32_f32cot"):
        prec = "fp32" if name == "fp32_f32cot" else name
        cot = torch.float32 if name == "fp32_f32cot" else torch.float64
        lat = Lattice(lx, ly, tau=tau, g=g, t_top=tt, t_bottom=tb, precision=prec, rho0=float(rho.mean()))
        d = torch.tensor(dT0, device=dev, requires_grad=True)
        temperature_loss(d, lat, rho_t, T_t, tgt, 4, 2, cotangent_dtype=cot).backward()  # warm-up
        d.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = temperature_loss(d, lat, rho_t, T_t, tgt, steps, K, cotangent_dtype=cot)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        grads[name] = d.grad.detach().cpu().numpy()
        res[name] = {"J": float(J.detach()), "forward_s": t1 - t0, "backward_s": t2 - t1,
                     "backward_over_forward": (t2 - t1) / (t1 - t0)}
        if name == "fp64":
            # float64 central differences of the float64 rollout on 16 seeded
            # directions: the check of every variant's gradient
            rng = np.random.default_rng(2024)
            eps = 1e-4
            for _ in range(16):
                v = rng.standard_normal(dT0.shape)
                with torch.no_grad():
                    jp = float(temperature_loss(torch.tensor(dT0 + eps * v, device=dev), lat, rho_t, T_t, tgt,
                                                steps, K))
                    jm = float(temperature_loss(torch.tensor(dT0 - eps * v, device=dev), lat, rho_t, T_t, tgt,
                                                steps, K))
                dirs.append(v)
                fds.append((jp - jm) / (2 * eps))
            res["fd_eps"] = eps
            res["fd_of"] = "float64 central differences of the float64 rollout, 16 seeded directions"
        errs = [abs(fd - float((grads[name] * v).sum())) / abs(fd) for fd, v in zip(fds, dirs)]
        res[name]["fd_max_rel_err_16_dirs"] = max(errs)
        res[name]["fd_pass_1e-6"] = max(errs) <= 1e-6
        del lat
        torch.cuda.empty_cache()
    g64 = grads["fp64"]
    for name in ("fp32", "fp64df", "fp32_f32cot"):
        res[name]["grad_rel_diff_vs_fp64"] = float(np.abs(grads[name] - g64).max() / np.abs(g64).max())
    res["fp64df"]["backward_over_fp64_forward"] = res["fp64df"]["backward_s"] / res["fp64"]["forward_s"]
    return res


def batch_study(steps, torch, lattices=64, tile=-1):
    """64 independent RT lattices of uneven sizes and parameters, FP32-store,
    autotuned launch candidate, `steps` steps as one CUDA-graph launch."""
    import synth
    from paper_1703_00186_gb300.batch import Batch
    specs = synth.batch_lattices(lattices, 7)
    flds, descs = [], []
    for sp in specs:
        rho, ux, uy, T, tt, tb = synth.rt_fields(sp.lx, sp.ly, 8, sp.seed, delta=sp.delta)
        flds.append((rho, ux, uy, T))
        descs.append(dict(lx=sp.lx, ly=sp.ly, tau=sp.tau, g=sp.g, t_top=tt, t_bottom=tb, rho0=float(rho.mean())))
    b = Batch(descs, precision="fp32")
    for i, f in enumerate(flds):
        b.init(i, *f)
    if tile < 0:
        best, times = b.autotune(steps=3)
    else:
        b.set_tile(tile)
        best, times = tile, []
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step(steps)          # capture the graph once (untimed) ...
    for i, f in enumerate(flds):
        b.init(i, *f)      # ... and start again from the initial state
    s = b.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    b.step(steps)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    finite = 0
    for i in range(len(b)):
        finite += int(bool(torch.isfinite(b.state(i)[:, 3:-3]).all()))
    # the same steps as one persistent cooperative launch (bounded grid barrier)
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step_persistent(2)
    torch.cuda.synchronize()
    e0.record(s)
    b.step_persistent(steps)
    e1.record(s)
    e1.synchronize()
    ms_p = e0.elapsed_time(e1)
    status_p = b.status()
    shapes = Batch.tile_shapes()
    labels = Batch.tile_labels()
    return {"lattices": len(b), "sites": b.sites, "steps": steps, "graph_launches": 1,
            "kernel_launches": steps * (len(b) if labels[best].startswith("per-lattice") else 1), "ms": ms, "mlups": b.sites * steps / (ms * 1e-3) / 1e6,
            "tile": shapes[best], "launch": labels[best],
            "autotune_ms_per_step": dict(zip(labels, times)),
            "persistent": {"ms": ms_p, "mlups": b.sites * steps / (ms_p * 1e-3) / 1e6, "status": status_p,
                           "what": "one cooperative launch, grid barrier between steps, 32x4 blocks x 8 rows"},
            "lattices_finite_after": finite,
            "state_bytes": 2 * 37 * 4 * sum(sp.lx * (sp.ly + 6) for sp in specs)}


def workload_config(lx, ly, world):
    """The `config` object of both arms' JSON lines (the same workload)."""
    return {"workload": WORKLOAD, "lx": lx, "ly": ly, "sites": lx * ly, "tau": 0.6, "g": 1e-5,
            "modes": 32, "seed": 0, "t_top": 0.5, "t_bottom": 1.5,
            "l2": "inputs larger than L2 (state 2 x %.2f GB)" % (37 * (ly + 6) * lx * 8 / 1e9),
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle arm: the float64 oracle on the host cores (every available
    core steps its own column slab), one line with impl = reference."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    width = max(8, args.lx // cores)
    _oracle_throughput(args.lx, args.ly, cores, width, max(1, min(args.warmup, 3)))  # warm-up
    v, dt = _oracle_throughput(args.lx, args.ly, cores, width, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.lx, args.ly, args.gpus),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"per step: {cores} spawned workers, each one step of its own "
                                       f"{width}x{args.ly} column slab of the RT lattice, NumPy float64, "
                                       f"one thread each"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1703_00186_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    barrier(torch, world)
    import ctypes

    from paper_1703_00186_gb300 import _lib as L
    lib = L.load()
    only = set(filter(None, args.only.split(","))) or set(SECTIONS)
    lx, ly, K, W = args.lx, args.ly, args.steps, args.warmup
    sites = lx * ly
    out = {}

    # float64 peak of this GPU (FMA probe)
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    rc = lib.lbm_probe_fma(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), 4096, 0,
                           ctypes.byref(tf), ctypes.byref(ms))
    fp64_peak = tf.value if rc == 0 else None
    # the same peak from unit counts and the clock: SMs x 2 FP64 FMAs per
    # clock x 2 flops x the SM clock sampled under load (max clock if none)
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    clocks = None
    if "fp64" in only:
        lat, _ = rt_lattice(lx, ly, "fp64")
        lat.step(W)
        sampler = ClockSampler(local)
        sampler.start()
        barrier(torch, world)
        t_ms = time_steps(lat, K, torch)
        barrier(torch, world)
        clocks = sampler.stop()
        t_ms = dist_max(t_ms, torch, world)
        finite = lat.check_finite()
        out["fp64"] = {"ms": t_ms, "mlups": world * sites * K / (t_ms * 1e-3) / 1e6, "finite": finite}
        del lat
        torch.cuda.empty_cache()
    if "fp32" in only:
        lat, _ = rt_lattice(lx, ly, "fp32")
        lat.step(W)
        barrier(torch, world)
        t_ms = dist_max(time_steps(lat, K, torch), torch, world)
        out["fp32"] = {"ms": t_ms, "mlups": world * sites * K / (t_ms * 1e-3) / 1e6,
                       "finite": lat.check_finite(), "loads": lat.step_path()}
        del lat
        torch.cuda.empty_cache()
        # the same step with its pull sources staged in shared memory by TMA
        lat, _ = rt_lattice(lx, ly, "fp32", tma_loads=True)
        lat.step(W)
        barrier(torch, world)
        t_tma = dist_max(time_steps(lat, K, torch), torch, world)
        out["fp32"]["mlups_tma_loads"] = world * sites * K / (t_tma * 1e-3) / 1e6
        out["fp32"]["tma_path"] = lat.step_path()
        del lat
        torch.cuda.empty_cache()
    if "fp64df" in only:
        lat, _ = rt_lattice(lx, ly, "fp64df")
        lat.step(W)
        barrier(torch, world)
        t_ms = dist_max(time_steps(lat, K, torch), torch, world)
        out["fp64df"] = {"ms": t_ms, "mlups": world * sites * K / (t_ms * 1e-3) / 1e6,
                         "finite": lat.check_finite()}
        del lat
        torch.cuda.empty_cache()
    if "regularized" in only:
        import synth
        from paper_1703_00186_gb300.lbm import Lattice
        rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 32, 0)
        lat = Lattice(lx, ly, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb, regularized=True).init(rho, ux, uy, T)
        lat.step(W)
        barrier(torch, world)
        t_ms = dist_max(time_steps(lat, K, torch), torch, world)
        out["regularized"] = {"ms": t_ms, "mlups": world * sites * K / (t_ms * 1e-3) / 1e6,
                              "finite": lat.check_finite()}
        del lat
        torch.cuda.empty_cache()
    if "observe" in only:
        lat, _ = rt_lattice(lx, ly, "fp64")
        lat.step(W)
        barrier(torch, world)
        s = lat.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ko = max(2, K // 5)
        lat.step_observe(2, 1)
        torch.cuda.synchronize()
        e0.record(s)
        lat.step_observe(ko, 1)
        e1.record(s)
        e1.synchronize()
        t_obs = dist_max(e0.elapsed_time(e1) / ko, torch, world)
        t_plain = dist_max(time_steps(lat, ko, torch) / ko, torch, world)
        out["observe"] = {"observing_step_ms": t_obs, "plain_step_ms": t_plain, "overhead": t_obs / t_plain - 1.0}
        del lat
        torch.cuda.empty_cache()
    if "adjoint" in only:
        def adjoint_times(precision, cot=torch.float64):
            lat, _ = rt_lattice(lx, ly, precision)
            lat.step(W)
            f_t = lat.state().clone()
            lam_a = lat.new_cotangent(0.0, dtype=cot).normal_()
            lam_b = lat.new_cotangent(0.0, dtype=cot)
            ka = max(3, K // 4)
            for _ in range(2):
                lat.adjoint_step(f_t, lam_a, lam_b)
            s = lat.stream
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            for i in range(ka):
                if i % 2 == 0:
                    lat.adjoint_step(f_t, lam_a, lam_b)
                else:
                    lat.adjoint_step(f_t, lam_b, lam_a)
            e1.record(s)
            e1.synchronize()
            ta = dist_max(e0.elapsed_time(e1) / ka, torch, world)
            tf_ms = dist_max(time_steps(lat, ka, torch) / ka, torch, world)
            del lat, f_t, lam_a, lam_b
            torch.cuda.empty_cache()
            return ta, tf_ms

        ta, tf_ms = adjoint_times("fp64")
        out["adjoint"] = {"adjoint_ms_per_step": ta, "forward_ms_per_step": tf_ms, "ratio": ta / tf_ms}
        # the LBM_FP64_DF mode: double-float forward collide and cotangent sums
        ta_df, tf_df = adjoint_times("fp64df")
        out["adjoint"]["fp64df"] = {"adjoint_ms_per_step": ta_df, "forward_ms_per_step": tf_df,
                                    "ratio": ta_df / tf_df, "ratio_vs_fp64_forward": ta_df / tf_ms}
        # FP32-store: float64 cotangents (double-float sums) and float32
        # cotangents (lbm_adjoint_step_f32)
        ta32, tf32 = adjoint_times("fp32")
        ta32f, _ = adjoint_times("fp32", torch.float32)
        out["adjoint"]["fp32"] = {"adjoint_ms_per_step": ta32, "forward_ms_per_step": tf32, "ratio": ta32 / tf32,
                                  "f32_cotangents": {"adjoint_ms_per_step": ta32f, "ratio": ta32f / tf32,
                                                     "hbm_gbs": 3 * 37 * 4 * sites / (ta32f * 1e-3) / 1e9}}
    if "e2e" in only:
        # Independent lattices, each on its own stream, each step of each
        # lattice through the C ABI from and to pinned host memory:
        # set_state(host) -> step(1) -> get_state(host).  The copy engines
        # move one lattice's state in while another's goes out or computes.
        streams = [torch.cuda.Stream() for _ in range(args.e2e_lattices)]
        lats = [rt_lattice(lx, ly, "fp64", stream=st)[0] for st in streams]
        host_in = [torch.empty(lats[0].shape, dtype=lats[0].dtype, pin_memory=True) for _ in lats]
        host_out = [torch.empty(lats[0].shape, dtype=lats[0].dtype, pin_memory=True) for _ in lats]
        for lat, h in zip(lats, host_in):
            lat.get_state(h)
        torch.cuda.synchronize()
        ke = max(3, min(K, 20))

        def e2e_round():
            for lat, hi, ho in zip(lats, host_in, host_out):
                lat.set_state(hi).step(1).get_state(ho)

        for _ in range(2):
            e2e_round()
        torch.cuda.synchronize()
        barrier(torch, world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        for st in streams[1:]:
            st.wait_event(e0)
        for _ in range(ke):
            e2e_round()
        for st in streams[1:]:
            eb = torch.cuda.Event()
            eb.record(st)
            streams[0].wait_event(eb)
        e1.record(streams[0])
        e1.synchronize()
        te = dist_max(e0.elapsed_time(e1), torch, world)
        out["e2e"] = {"value": world * len(lats) * sites * ke / (te * 1e-3) / 1e6, "unit": "MLUPS",
                      "h2d_bytes_per_step": lats[0].nbytes, "d2h_bytes_per_step": lats[0].nbytes,
                      "steps": ke * len(lats), "lattices": len(lats),
                      "path": "per lattice step: lbm_set_state(pinned host) + lbm_step(1) + "
                              "lbm_get_state(pinned host); independent lattices on their own streams"}
        del lats, host_in, host_out
        torch.cuda.empty_cache()
        # A simulation run through the public API: the initial fields come
        # from pinned host memory (lbm_init), every step is an observing step
        # whose row averages (the run's per-step result) are read back, and
        # the final moments go back to pinned host memory.
        import numpy as np
        lat, flds = rt_lattice(lx, ly, "fp64")
        host = [torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory() for v in flds]
        kr = max(3, K)
        obs_h = torch.empty((kr, 8, ly), dtype=torch.float64, pin_memory=True)
        mom_h = [torch.empty((ly, lx), dtype=torch.float64, pin_memory=True) for _ in range(4)]

        def sim_run():
            lat.init(*host)
            obs_h.copy_(lat.step_observe(kr, 1), non_blocking=True)
            for h, d in zip(mom_h, lat.moments()):
                h.copy_(d, non_blocking=True)

        sim_run()
        torch.cuda.synchronize()
        barrier(torch, world)
        s = lat.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sim_run()
        e1.record(s)
        e1.synchronize()
        tr = dist_max(e0.elapsed_time(e1), torch, world)
        out["e2e_run"] = {"value": world * sites * kr / (tr * 1e-3) / 1e6, "unit": "MLUPS", "steps": kr,
                          "h2d_bytes_per_step": 4 * 8 * sites / kr,
                          "d2h_bytes_per_step": 8 * 8 * ly + 4 * 8 * sites / kr,
                          "path": "lbm_init from pinned host fields, lbm_step_observe (row averages every "
                                  "step, read back), lbm_moments to pinned host memory"}
        del lat, host, obs_h, mom_h
        torch.cuda.empty_cache()
    if "fp32_error" in only:
        out["fp32_error"] = fp32_error_study(lx, ly, args.error_steps, torch)
        torch.cuda.empty_cache()
    if "rollout" in only:
        out["rollout"] = rollout_study(args.rollout_steps, torch)
        torch.cuda.empty_cache()
    if "batch" in only:
        out["batch"] = batch_study(args.batch_steps, torch, args.batch_lattices, args.batch_tile)
        torch.cuda.empty_cache()
    barrier(torch, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    res = {"metric": METRIC, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(lx, ly, world)}
    if "fp64" in out:
        f64 = out["fp64"]
        t_launch = f64["ms"] / K * 1e-3
        res["value"] = f64["mlups"]
        res["ms_per_step"] = f64["ms"] / K
        res["gpu_launches"] = K
        res["finite_after_timed_steps"] = f64["finite"]
        peak = fp64_peak if fp64_peak else FP64_NOMINAL_TFLOPS
        mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
        peak_units = {"sms": sms, "fp64_fma_per_clk_per_sm": 2, "sm_mhz": mhz,
                      "tflops": sms * 2 * 2 * mhz * 1e6 / 1e12}
        achieved = FP64_FLOP_PER_SITE * sites / t_launch / 1e12
        res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak,
                           "frac_note": "above 1 because the kernel forms the moment sums and evaluates the "
                                        "equilibrium polynomial exactly on the integer pipe, keeping "
                                        "fp64_pipe_flop_per_site of the formulation's 542 flops per site in "
                                        "float64; fp64_issue_frac is how busy the FP64 pipe is",
                           "traffic": FP64_TRAFFIC_BYTES_PER_SITE_NCU * sites,
                           "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                             "2048x1024 launch, scaled by sites",
                           "peak_source": ("measured FP64 FMA probe (lbm_probe_fma), this run" if fp64_peak
                                           else "nominal 1.25 TFLOP/s"),
                           "flop_per_site": FP64_FLOP_PER_SITE,
                           "fp64_pipe_flop_per_site": FP64_PIPE_FLOP_PER_SITE,
                           "fp64_pipe_flop_frac": FP64_PIPE_FLOP_PER_SITE * sites / t_launch / 1e12 / peak,
                           "fp64_instr_per_site_ncu": FP64_INSTR_PER_SITE_NCU,
                           "fp64_issue_frac": FP64_INSTR_PER_SITE_NCU * sites / t_launch / (peak * 1e12 / 2),
                           "fp64_pipe_flop_per_site_ncu": FP64_PIPE_FLOP_PER_SITE_NCU,
                           "peak_from_units": peak_units,
                           "algorithmic_bytes_per_launch": BYTES_PER_SITE_FP64 * sites,
                           "hbm_gbs": BYTES_PER_SITE_FP64 * sites / t_launch / 1e9,
                           "hbm_frac_of_measured": BYTES_PER_SITE_FP64 * sites / t_launch / 1e9 / HBM_GBS_MEASURED}
        res["clocks"] = clocks
    if "fp32" in out:
        f32 = out["fp32"]
        t_launch = f32["ms"] / K * 1e-3
        res["fp32_store"] = {"mlups": f32["mlups"], "ms_per_step": f32["ms"] / K,
                             "speedup_vs_fp64": (f32["mlups"] / out["fp64"]["mlups"]) if "fp64" in out else None,
                             "hbm_gbs": BYTES_PER_SITE_FP32 * sites / t_launch / 1e9,
                             "hbm_frac_of_measured": BYTES_PER_SITE_FP32 * sites / t_launch / 1e9 / HBM_GBS_MEASURED,
                             "hbm_peak_source": HBM_PEAK_SOURCE,
                             "loads": f32["loads"], "mlups_tma_loads": f32["mlups_tma_loads"],
                             "tma_path": f32["tma_path"],
                             "finite_after_timed_steps": f32["finite"]}
    if "fp64df" in out:
        d = out["fp64df"]
        t_launch = d["ms"] / K * 1e-3
        res["fp64_df"] = {"mlups": d["mlups"], "ms_per_step": d["ms"] / K,
                          "speedup_vs_fp64": (d["mlups"] / out["fp64"]["mlups"]) if "fp64" in out else None,
                          "hbm_gbs": BYTES_PER_SITE_FP64 * sites / t_launch / 1e9,
                          "hbm_frac_of_measured": BYTES_PER_SITE_FP64 * sites / t_launch / 1e9 / HBM_GBS_MEASURED,
                          "arithmetic": "double-float (two float32 words, ~48 bits) on the FP32 pipe; float64 storage",
                          "finite_after_timed_steps": d["finite"]}
    if "regularized" in out:
        d = out["regularized"]
        res["regularized"] = {"mlups": d["mlups"], "ms_per_step": d["ms"] / K,
                              "vs_fp64_bgk": (d["mlups"] / out["fp64"]["mlups"]) if "fp64" in out else None,
                              "collide": "float64, Hermite projection of order <= 4 before relaxing",
                              "finite_after_timed_steps": d["finite"]}
    if "observe" in out:
        res["observables"] = {**out["observe"], "quantities": 8,
                              "what": "row averages fused into the float64 step (every observing step)"}
    if "adjoint" in out:
        res["adjoint"] = out["adjoint"]
    if "e2e" in out:
        res["e2e"] = out["e2e"]
    if "e2e_run" in out:
        res["e2e_run"] = out["e2e_run"]
    for key in ("fp32_error", "rollout", "batch"):
        if key in out:
            res[key] = out[key]
    res["fp64_probe_tflops"] = fp64_peak
    if "cpu" in only:
        res["cpu_baseline"] = cpu_baseline(lx, ly, args.cpu_seconds)
    print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
