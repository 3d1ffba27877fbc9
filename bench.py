#!/usr/bin/env python
"""Benchmark of the fused D3Q19 BGK sparse-tile step on GB300.

Workload (default): periodic sphere-pack porous medium, 256^3 nodes, overlapping
solid spheres of radius 8 with uniform seeded centres (seed 161102445) until the
porosity first reaches 0.35; D3Q19 BGK with tau = 0.7, body force g_x = 1e-5 (Guo),
periodic faces, 4^3 tiles with all-solid tiles skipped; FP64 storage. A step is one
fused collide-and-stream launch over all kept tiles; the metric is MFLUPS, 10^6
non-solid node updates per second (Sec. 4.1 of the paper).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f64|f32|f16s]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

Under torchrun every rank runs its own replica of the workload (the path has no data
exchange between replicas); value = all ranks' node updates / the slowest rank's time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MFLUPS (10^6 non-solid node updates per second) of the fused D3Q19 BGK sparse-tile step"
WORKLOAD = ("porous sphere pack 256^3, radius 8, porosity 0.35, seed 161102445, D3Q19 BGK, "
            "tau 0.7, g_x 1e-5 (Guo), periodic, 4^3 tiles, all-solid tiles skipped")
BYTES_PER_VALUE = {"f64": 8, "f64n": 8, "f32": 4, "f16s": 2, "f16sr": 2}
DTYPE_NAME = {"f64": "f64 storage; FP64 moments and update, double-float (2xFP32) equilibrium and forcing",
              "f64n": "f64 storage, FP64 arithmetic throughout",
              "f32": "f32 (f - w shifted storage), f32 arithmetic",
              "f16s": "f16 (f - w shifted storage), f32 arithmetic",
              "f16sr": "f16 (f - w shifted storage, stochastic rounding), f32 arithmetic"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values of x (a timed-region duration); the replicas
    exchange nothing else."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mflups(nodes_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's node updates over the slowest rank's time."""
    return nodes_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def oracle_baseline(nt, steps_hint: int, budget_s: float, tau, g):
    """Time the FP64 oracle (as it stands) on the host cores on the full geometry."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    f = O.init(nt)
    B = f.copy()
    n = int(np.count_nonzero(nt))
    t0 = time.perf_counter()
    done = 0
    while done < steps_hint and (time.perf_counter() - t0) < budget_s:
        O.step(f, nt, 0b111, tau, g, nthreads=threads, out=B)
        f, B = B, f
        done += 1
    dt = time.perf_counter() - t0
    return {"value": n * done / dt / 1e6, "unit": "MFLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{done} full steps of the 256^3 porous workload ({n} non-solid nodes), "
                      f"dense FP64 oracle, OpenMP over z on {threads} threads, {dt:.1f} s"}


def oracle_baseline_serial(nt, budget_s: float, tau, g):
    """The same oracle on one host core: whole steps of the full workload until the
    budget is spent (at least one)."""
    from oracle import oracle as O
    f = O.init(nt)
    B = f.copy()
    n = int(np.count_nonzero(nt))
    t0 = time.perf_counter()
    done = 0
    while done == 0 or (time.perf_counter() - t0) < budget_s:
        O.step(f, nt, 0b111, tau, g, nthreads=1, out=B)
        f, B = B, f
        done += 1
    dt = time.perf_counter() - t0
    return {"value": n * done / dt / 1e6, "unit": "MFLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{done} full steps of the 256^3 porous workload ({n} non-solid nodes), "
                      f"dense FP64 oracle, serial, {dt:.1f} s"}


def _code_only(text: str) -> str:
    """C++/CUDA source with its comments, trailing blanks and empty lines removed (the
    library's sources hold no comment markers inside string literals)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def step_source_hash() -> str:
    """Hash of the CUDA library sources, comments left out; a stored DRAM traffic figure
    is valid only for the code it was captured with."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1611_02445_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            h.update(name.encode() + b"\0" + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def time_format(lbm, nt, dtype, tau, g, steps, warmup, stream):
    """A short timed run of one storage format on the benchmark workload (CUDA events on
    the launching stream around `steps` steps after `warmup`); MFLUPS and HBM fraction."""
    import torch
    L = lbm.Lattice(nt, dtype, 0b111, stream)
    info = L.info()
    L.set_params(tau, g)
    L.init_equilibrium()
    L.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mass, _ = L.reduce()
    L.close()
    assert np.isfinite(mass)
    n = info["n_nonsolid"]
    value = n * steps / (ms * 1e-3) / 1e6
    return value, ms / steps, n * 2 * 19 * BYTES_PER_VALUE[dtype] / (ms / steps * 1e-3) / 1e9


def run_reference(args, nt, tau, g):
    """--impl reference: the oracle on the host cores; each step is one oracle step on a
    z-slab sample of the workload, sized so the whole run ends in about two minutes."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    total = args.steps + args.warmup

    def slab(nz_s):
        s = np.ascontiguousarray(nt[:nz_s])
        return s, O.init(s)

    probe, fp = slab(16)
    Bp = fp.copy()
    t = time.perf_counter()
    O.step(fp, probe, 0b011, tau, g, nthreads=threads, out=Bp)
    t16 = max(time.perf_counter() - t, 1e-4)
    nz_s = int(max(4, min(256, 16 * (120.0 / total) / t16)) // 4 * 4)
    s, f = slab(nz_s)
    B = f.copy()
    n = int(np.count_nonzero(s))
    for _ in range(args.warmup):
        O.step(f, s, 0b011, tau, g, nthreads=threads, out=B)
        f, B = B, f
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(f, s, 0b011, tau, g, nthreads=threads, out=B)
        f, B = B, f
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e6
    sample = (f"z-slab 256x256x{nz_s} of the workload ({n} non-solid nodes; x, y periodic, z walls), "
              f"one dense FP64 oracle step per benchmark step, OpenMP over z on {threads} threads")
    # n_gpus is the N of the launch, as in the other arm; the oracle itself runs on the host
    # cores (cpu_baseline.cores)
    return {"metric": METRIC, "value": value, "unit": "MFLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "MFLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MFLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_adjoint_workload(args):
    """Adjoint workload: 128^3 sphere pack (radius 8, porosity 0.4, seed 161102448), FP32
    storage, tau 0.8, per-node x force 1e-5 + N(0, 1e-7) (seed 161102449), periodic;
    L = mean u_x over the plane x = 127 after T = 2000 steps from rest; checkpoints every
    100 steps. Reports the time of the forward alone and of forward + reverse sweep, and
    checks dL/dtau and one directional dL/dg against central differences (relative step
    1e-3) of the FP64 forward and against the FP64 adjoint."""
    import torch
    import __graft_entry__
    from paper_1611_02445_gb300 import inputs as I
    from paper_1611_02445_gb300 import lbm
    __graft_entry__.build()
    nt = I.sphere_pack(128, 8.0, 0.4, I.SEED_POROUS_128)
    gf = I.body_force_field(nt, 1e-5, 1e-7, I.SEED_FORCE_NOISE)
    T, K, plane, tau = args.adj_steps, 100, 127, 0.8

    def run(dtype, tau_, gf_, grads):
        with lbm.Lattice(nt, dtype, 0b111) as L:
            L.set_params(tau_, (0.0, 0.0, 0.0), gf_)
            L.init_equilibrium()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = L.adjoint(T, K, plane, grads)
            torch.cuda.synchronize()
            return out, time.perf_counter() - t0, L.info()

    run("f32", tau, gf, False)                      # warm-up
    (L32f, _, _), t_fwd, info = run("f32", tau, gf, False)
    (L32, dg32, dtau32), t_adj, _ = run("f32", tau, gf, True)
    (L64, dg64, dtau64), t_adj64, _ = run("f64", tau, gf, True)
    e = 1e-3
    fd_tau = (run("f64", tau * (1 + e), gf, False)[0][0] - run("f64", tau * (1 - e), gf, False)[0][0]) / (2 * e * tau)
    d = np.random.default_rng(0).standard_normal(nt.shape) * gf
    fd_g = (run("f64", tau, gf + e * d, False)[0][0] - run("f64", tau, gf - e * d, False)[0][0]) / (2 * e)
    m = nt != 0
    line = {"workload": "adjoint: sphere pack 128^3, porosity 0.4, FP32 storage, tau 0.8, g = 1e-5 + N(0,1e-7), "
                        f"L = mean u_x on x = 127 after T = {T}, checkpoints every {K}",
            "n_nonsolid": info["n_nonsolid"], "n_tiles": info["n_tiles"],
            "forward_s": t_fwd, "forward_plus_adjoint_s": t_adj, "ratio": t_adj / t_fwd,
            "f64_forward_plus_adjoint_s": t_adj64,
            "loss_f32": L32, "loss_f64": L64,
            "dL_dtau": {"f32_adjoint": dtau32, "f64_adjoint": dtau64, "f64_central_fd": fd_tau,
                        "rel_err_f64_vs_fd": abs(dtau64 - fd_tau) / abs(fd_tau),
                        "rel_err_f32_vs_f64": abs(dtau32 - dtau64) / abs(dtau64)},
            "dL_dg_directional": {"f64_adjoint": float((dg64 * d).sum()), "f32_adjoint": float((dg32 * d).sum()),
                                  "f64_central_fd": fd_g,
                                  "rel_err_f64_vs_fd": abs(float((dg64 * d).sum()) - fd_g) / abs(fd_g)},
            "dL_dg_f32_vs_f64_max_rel": float(np.abs(dg32[m] - dg64[m]).max() / np.abs(dg64).max())}
    print(json.dumps(line), flush=True)


def _timed_steps(L, n, stream):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    L.step(n)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def run_poiseuille(args):
    """Plane Poiseuille 32^3 (walls y = 0, 31; periodic x, z; tau 0.8; g_x 1e-6) for every
    storage format: MFLUPS over 1000 steps (CUDA-graph replay; the problem is launch-bound),
    the error of u_x against g/(2 nu) (y - 1/2)(30.5 - y) at 1000 steps (start-up, not
    steady) and at 12 000 steps, the relative mass drift, and, for the other formats, the
    velocity error against the FP64 run at 12 000 steps."""
    import torch
    import __graft_entry__
    from paper_1611_02445_gb300 import inputs as I
    from paper_1611_02445_gb300 import lbm
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    nt = I.poiseuille_channel(32, 32, 32)
    tau, g = 0.8, 1e-6
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, 31, dtype=np.float64)
    exact = g / (2 * nu) * (y - 0.5) * (30.5 - y)
    out = {"workload": "plane Poiseuille 32^3, walls y=0,31, periodic x,z, tau 0.8, g_x 1e-6"}
    u_end = {}
    for dtype in ("f64", "f64n", "f32", "f16s", "f16sr"):
        with lbm.Lattice(nt, dtype, 0b101, stream) as L:
            L.set_params(tau, (g, 0.0, 0.0))
            L.init_equilibrium()
            m0, _ = L.reduce()
            L.step(args.warmup)
            ms = _timed_steps(L, 1000, stream)
            n = L.info()["n_nonsolid"]
            res = {"mflups": n * 1000 / (ms * 1e-3) / 1e6, "ms_per_step": ms / 1000}
            L.init_equilibrium()
            for total in (1000, 12000):
                L.step(total - (0 if total == 1000 else 1000))
                rho, u = L.macroscopic()
                ux = u[0][:, 1:31, :]
                ex = np.broadcast_to(exact[None, :, None], ux.shape)
                res[f"l2_rel_err_{total}"] = float(np.sqrt(((ux - ex) ** 2).sum() / (ex ** 2).sum()))
            u_end[dtype] = u[0][:, 1:31, :]
            m1, _ = L.reduce()
            res["mass_drift_rel"] = abs(m1 - m0) / m0
            res["u_max_exact"] = float(g * 30 ** 2 / (8 * nu))
            out[dtype] = res
    ref = u_end["f64"]
    umax = float(np.abs(ref).max())
    for dtype in ("f64n", "f32", "f16s", "f16sr"):
        du = np.abs(u_end[dtype] - ref)
        out[dtype]["vs_f64_12000"] = {"max_err_over_umax": float(du.max() / umax),
                                      "l2_rel_err": float(np.sqrt((du ** 2).sum() / (ref ** 2).sum()))}
    print(json.dumps(out), flush=True)


def run_vessel(args):
    """Synthetic vessel tree 1024 x 512 x 512 (seed 161102446, root radius 24, ratio 0.79,
    6 generations, angles 25-45 deg), inlet u = 0.05 at x = 0, outlets at the leaf tips and
    box faces, tau 0.6, no body force, non-periodic: MFLUPS and bandwidth for FP64 and FP32
    storage over 5000 steps."""
    import torch
    import __graft_entry__
    from paper_1611_02445_gb300 import inputs as I
    from paper_1611_02445_gb300 import lbm
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    nt = I.vessel_tree()
    peaks, _ = load_peaks()
    out = {"workload": "vessel tree 1024x512x512, seed 161102446, tau 0.6, u_in 0.05, 4^3 tiles",
           "fluid_fraction": float(np.count_nonzero(nt) / nt.size)}
    for dtype in ("f64", "f32"):
        with lbm.Lattice(nt, dtype, 0, stream) as L:
            L.set_params(0.6, None, None, (0.05, 0.0, 0.0), 1.0)
            L.init_equilibrium()
            L.step(args.warmup)
            ms = _timed_steps(L, 5000, stream)
            info = L.info()
            mass, _ = L.reduce()
            n = info["n_nonsolid"]
            mfl = n * 5000 / (ms * 1e-3) / 1e6
            gbs = mfl * 1e6 * 2 * 19 * BYTES_PER_VALUE[dtype] / 1e9
            out[dtype] = {"mflups": mfl, "ms_per_step": ms / 5000, "n_nonsolid": n, "n_tiles": info["n_tiles"],
                          "eta_t": info["eta_t"], "algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / peaks["hbm_gbs"],
                          "mass_after": mass}
    print(json.dumps(out), flush=True)


def run_cavity(args):
    """Lid-driven cavity sweep (the dense cavity3D benchmark of Sec. 4.3, E3/E6): all-fluid
    N^3 boxes, N = 64 ... 384, walls on every face, the face z = N moving with u = (0.05, 0, 0)
    (moving-wall bounce-back), tau 0.6, quasi-compressible LBGK; MFLUPS and algorithmic
    GB/s for every storage format over args.steps steps (no tiles are skipped: eta_t = 1)."""
    import torch
    import __graft_entry__
    from paper_1611_02445_gb300 import lbm
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    peaks, _ = load_peaks()
    out = {"workload": "lid-driven cavity N^3, lid z = N at u = (0.05, 0, 0), tau 0.6, LBGK, "
                       f"{args.steps} timed steps after {args.warmup}", "hbm_peak_gbs": peaks["hbm_gbs"],
           "sizes": {}}
    for n in (64, 128, 192, 256, 320, 384):
        nt = np.ones((n, n, n), np.uint8)
        row = {}
        for dtype in ("f64", "f32", "f16s"):
            with lbm.Lattice(nt, dtype, 0, stream) as L:
                L.set_params(0.6)
                L.set_lid(5, (0.05, 0.0, 0.0))
                L.init_equilibrium()
                L.step(args.warmup)
                ms = _timed_steps(L, args.steps, stream)
                nodes = L.info()["n_nonsolid"]
            mflups = nodes * args.steps / (ms * 1e-3) / 1e6
            gbs = mflups * 1e6 * 2 * 19 * BYTES_PER_VALUE[dtype] / 1e9
            row[dtype] = {"mflups": mflups, "gbs": gbs, "frac": gbs / float(peaks["hbm_gbs"])}
        out["sizes"][str(n)] = row
    print(json.dumps(out), flush=True)


def run_precision(args):
    """Precision sweep: sphere pack 512^3 (radius 8, porosity 0.35, seed 161102447), tau 0.7,
    g_x 1e-5, periodic; FP64 vs FP32 vs FP16-shifted storage (round to nearest and stochastic
    rounding) after args.steps steps (20 000 for steady state): velocity error relative to
    u_max and permeability k = nu <u_x> / g_x (box average, solids counted as 0), against
    the FP64 run. On the 128^3 crop the same runs are compared with the FP64 oracle after
    2000 steps."""
    import torch
    import __graft_entry__
    from oracle import oracle as O
    from paper_1611_02445_gb300 import inputs as I
    from paper_1611_02445_gb300 import lbm
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    tau, g = 0.7, (1e-5, 0.0, 0.0)
    nu = (tau - 0.5) / 3.0

    def run(nt, dtype, steps):
        with lbm.Lattice(nt, dtype, 0b111, stream) as L:
            L.set_params(tau, g)
            L.init_equilibrium()
            ms = _timed_steps(L, steps, stream)
            rho, u = L.macroscopic()
            return u, L.info()["n_nonsolid"] * steps / (ms * 1e-3) / 1e6

    def compare(u, ref, solid):
        umax = float(np.abs(ref[0]).max())
        du = np.abs(u - ref)
        return {"max_err_over_umax": float(du.max() / umax),
                "l2_rel_err": float(np.sqrt((du ** 2).sum() / (ref ** 2).sum())),
                "perm_rel_err": float(abs(u[0].mean() - ref[0].mean()) / abs(ref[0].mean())),
                "u_max": umax}

    out = {"workload": f"precision sweep: sphere pack 512^3 (seed 161102447), tau 0.7, g_x 1e-5, {args.steps} steps"}
    nt = I.sphere_pack(512, 8.0, 0.35, I.SEED_POROUS_512)
    u64, m64 = run(nt, "f64", args.steps)
    out["f64"] = {"mflups": m64, "permeability": float(nu * u64[0].mean() / g[0])}
    for dt in ("f32", "f16s", "f16sr"):
        u, m = run(nt, dt, args.steps)
        out[dt] = dict(compare(u, u64, nt == 0), mflups=m, speedup_vs_f64=m / m64)
        del u
    del u64
    crop = I.crop(nt, 128)
    steps_c = 2000
    fo = O.run(O.init(crop), crop, steps_c, 0b111, tau, g, nthreads=os.cpu_count() or 1)
    _, uo = O.macroscopic(fo, crop, g)
    out["crop128_vs_oracle_2000_steps"] = {dt: compare(run(crop, dt, steps_c)[0], uo, crop == 0)
                                           for dt in ("f64", "f64n", "f32", "f16s", "f16sr")}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f64n", "f32", "f16s", "f16sr"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-formats", action="store_true", help="skip the other storage formats' timed runs")
    ap.add_argument("--kernel", default="full", choices=["full", "propagate", "rw"],
                    help="the fused step, or one of the paper's calibration kernels (propagation "
                         "only, read/write only)")
    ap.add_argument("--adjoint", action="store_true", help="run the adjoint workload instead")
    ap.add_argument("--model", default="bgk", choices=list(MODELS),
                    help="collision model: LBGK (Eq. 3, the benchmark), incompressible LBGK (Eq. 4), "
                         "MRT (Eq. 8) with either equilibrium")
    ap.add_argument("--workload", default="porous", choices=["porous", "poiseuille", "vessel", "precision", "cavity"],
                    help="porous is the benchmark line; the others print their own JSON line")
    ap.add_argument("--adj-steps", type=int, default=2000)
    ap.add_argument("--size", type=int, default=256,
                    help="edge of the cubic sphere pack (256 is the benchmark workload; smaller "
                         "sizes are for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.adjoint:
        run_adjoint_workload(args)
        return
    if args.workload != "porous":
        {"poiseuille": run_poiseuille, "vessel": run_vessel, "precision": run_precision,
         "cavity": run_cavity}[args.workload](args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1611_02445_gb300 import inputs as I
    tau, g = 0.7, (1e-5, 0.0, 0.0)

    if args.impl == "reference":
        if rank != 0:
            return
        nt = I.sphere_pack(256, 8.0, 0.35, I.SEED_POROUS_256)
        print(json.dumps(run_reference(args, nt, tau, g)), flush=True)
        return

    import torch
    import torch.distributed as dist
    import __graft_entry__
    from paper_1611_02445_gb300 import lbm

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    __graft_entry__.build()
    nt = I.sphere_pack(args.size, 8.0, 0.35, I.SEED_POROUS_256)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    L = lbm.Lattice(nt, args.dtype, 0b111, stream)
    info = L.info()
    L.set_params(tau, g)
    eq_m, coll_m = MODELS[args.model]
    if args.model != "bgk":
        L.set_model(eq_m, coll_m)
    L.init_equilibrium()
    n_nonsolid = info["n_nonsolid"]
    kind = {"full": lbm.KERNEL_FULL, "propagate": lbm.KERNEL_PROPAGATE, "rw": lbm.KERNEL_RW}[args.kernel]
    L.step_kernel(kind, args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # nvidia-smi samples every 200 ms, longer than a short timed region: the sampled
    # window also covers about a second of untimed steps right before it, under the same load
    ev0.record(stream)
    L.step_kernel(kind, 3)
    ev1.record(stream)
    torch.cuda.synchronize()
    soak = max(1, int(1000.0 / max(ev0.elapsed_time(ev1) / 3, 1e-3)))
    sampler = ClockSampler(local_rank)
    barrier()
    sampler.start()
    time.sleep(0.3)
    L.step_kernel(kind, soak)
    ev0.record(stream)
    L.step_kernel(kind, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world, dev)
    mass, _ = L.reduce()
    assert np.isfinite(mass)
    # the FP64 mass/momentum reduction over one population copy (host wall time of the
    # call, which waits for its result: an upper bound on the kernels' time)
    red_ms = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0r = time.perf_counter()
        L.reduce()
        red_ms.append((time.perf_counter() - t0r) * 1e3)
    red_ms = min(red_ms)
    if args.kernel != "full":
        args.no_e2e = True
    value = job_mflups(n_nonsolid, args.steps, world, ms_max)

    # roofline of the step kernel: algorithmic bytes B_node = 2 * 19 * n_d per non-solid
    # node update (Eq. 10) over the average launch duration
    nd = BYTES_PER_VALUE[args.dtype]
    launch_s = ms / args.steps * 1e-3
    alg_bytes = n_nonsolid * 2 * 19 * nd
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    achieved_gbs = alg_bytes / launch_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved_gbs / hbm_peak, "traffic": None,
            "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy)",
            "algorithmic_bytes_per_launch": alg_bytes}
    if args.dtype == "f64n":
        # FP64 arithmetic throughout bounds this kernel on GB300: FP64 FLOPs executed per
        # non-solid node update, counted with ncu (2 * dfma + dadd + dmul per node), over the
        # FP64 peak of 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz.
        flops_per_node = FP64_FLOPS_PER_NODE
        fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12
        achieved_tf = n_nonsolid * flops_per_node / launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": None,
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (probe measured 1.20)",
                "fp64_flops_per_node_update": flops_per_node,
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak}}
    full_size = args.kernel == "full" and args.model == "bgk" and args.size == 256
    captured = TRAFFIC_PER_LAUNCH_256.get(args.dtype) if full_size else None
    src_hash = step_source_hash()
    roof["sources"] = src_hash
    if captured is not None and TRAFFIC_PER_LAUNCH_256["sources"] == src_hash:
        roof["traffic"] = captured
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this launch (porous 256^3 "
                                  f"pack), mean of two captured launches, library sources {src_hash}")
        roof["traffic_per_node"] = captured / n_nonsolid
        roof["traffic_over_algorithmic"] = captured / alg_bytes
    elif captured is not None:
        roof["traffic_source"] = (f"null: captured for library sources {TRAFFIC_PER_LAUNCH_256['sources']}, "
                                  f"these are {src_hash}")

    line = {"metric": METRIC, "value": value, "unit": "MFLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD if args.size == 256 else WORKLOAD.replace("256^3", f"{args.size}^3"),
                       "kernel": {"full": "fused collide-and-stream step",
                                  "propagate": "calibration: propagation only (gather with bounce-back, store)",
                                  "rw": "calibration: read/write only (own values, no propagation)"}[args.kernel],
                       "storage": DTYPE_NAME[args.dtype] + (
                           " (the collision's form for a force along x, bit-identical to the general form)"
                           if args.dtype == "f64" and args.model == "bgk" and g[1] == 0.0 and g[2] == 0.0 else ""),
                       "n_nonsolid": n_nonsolid,
                       "collision_model": MODEL_NAME[args.model],
                       "n_tiles": info["n_tiles"], "eta_t": info["eta_t"],
                       "state_bytes": 2 * info["copy_bytes"],
                       "l2_policy": "inputs larger than L2 (two population copies of "
                                    f"{info['copy_bytes'] / 1e9:.2f} GB each vs 126 MB L2)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "gpu_launches": args.steps,
            "clocks": dict(clocks or {}, window=f"{soak} untimed steps right before the timed region, and the region"),
            "reduction": {"ms": red_ms, "bytes": info["copy_bytes"],
                          "gbs": info["copy_bytes"] / (red_ms * 1e-3) / 1e9,
                          "what": "lbm_reduce: FP64 mass and momentum over one copy, best of 5 calls, "
                                  "host wall time including the 32-byte result copy"}}

    # the other storage formats on the same workload, timed alike (the headline is f64)
    if args.kernel == "full" and args.model == "bgk" and not args.no_formats:
        L.close()
        fsteps = max(args.steps, 50)
        formats = {}
        for dt in ("f64n", "f32", "f16s"):
            if dt == args.dtype:
                continue
            v, ms_step, gbs = time_format(lbm, nt, dt, tau, g, fsteps, args.warmup, stream)
            entry = {"value": v, "ms_per_step": ms_step, "frac": gbs / hbm_peak, "speedup_over_headline": v / value,
                     "steps": fsteps}
            if dt == "f64n":
                tf = n_nonsolid * FP64_FLOPS_PER_NODE / (ms_step * 1e-3) / 1e12
                entry["fp64_alu"] = {"achieved_tflops": tf, "peak_tflops": 152 * 2 * 2 * 2.07e9 / 1e12,
                                     "frac": tf / (152 * 2 * 2 * 2.07e9 / 1e12)}
            formats[dt] = entry
        if args.dtype == "f64" and g[1] == 0.0 and g[2] == 0.0:
            # the headline takes the hybrid collision's form for a force along x; the same
            # workload with a small y force takes the general form
            g_yz = (g[0], 1e-9, 0.0)
            v, ms_step, gbs = time_format(lbm, nt, "f64", tau, g_yz, fsteps, args.warmup, stream)
            formats["f64_general_force"] = {"value": v, "ms_per_step": ms_step, "frac": gbs / hbm_peak,
                                            "speedup_over_headline": v / value, "steps": fsteps, "g": list(g_yz),
                                            "what": "FP64 hybrid storage with the general form of the collision "
                                                    "(a force with a y component)"}
        line["formats"] = {"headline": args.dtype, "unit": "MFLUPS", "frac_of": "measured hbm_gbs, algorithmic bytes",
                           "what": "the same workload and step with other storage formats, CUDA events around "
                                   f"{fsteps} steps after {args.warmup} warm-up steps", **formats}

    # end to end through the public API: host node types in, host results out
    if not args.no_e2e:
        L.close()
        pinned_nt = torch.from_numpy(nt.reshape(-1)).pin_memory()
        nz, ny, nx = nt.shape
        rho_h = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
        u_h = torch.empty((3, nz, ny, nx), dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        ctx = lbm.lbm_create(pinned_nt.numpy(), nx, ny, nz, 4, lbm.DTYPES[args.dtype], 0b111, stream)
        lbm.lbm_set_params(ctx, tau, g)
        if args.model != "bgk":
            lbm.lbm_set_model(ctx, eq_m, coll_m)
        lbm.lbm_init_equilibrium(ctx)
        lbm.lbm_step(ctx, args.steps)
        mass_e2e, _ = lbm.lbm_reduce(ctx)
        lbm.lbm_macroscopic(ctx, rho_h.numpy(), u_h.numpy(), out_f64=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lbm.lbm_destroy(ctx)
        dt = max_over_ranks(dt, world, dev)
        d2h = 4 * 8 + rho_h.numel() * 4 + u_h.numel() * 4
        line["e2e"] = {"value": n_nonsolid * args.steps * world / dt / 1e6, "unit": "MFLUPS",
                       "h2d_bytes_per_step": nt.size / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                       "includes": "lbm_create from pinned host node types (tile map on GPU), init, "
                                   f"{args.steps} steps, FP64 reduction and FP32 rho/u export to pinned host"}
    else:
        L.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # about 15 s of oracle steps on the host cores (a bounded sample of the workload)
        line["cpu_baseline"] = oracle_baseline(nt, 1000, 15.0, tau, g)
        line["cpu_baseline_serial"] = oracle_baseline_serial(nt, 5.0, tau, g)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Collision models: (equilibrium, collision) of lbm_set_model.
MODELS = {"bgk": (0, 0), "bgk-incompr": (1, 0), "mrt": (0, 1), "mrt-incompr": (1, 1)}
MODEL_NAME = {"bgk": "LBGK, quasi-compressible equilibrium (Eq. 3)",
              "bgk-incompr": "LBGK, incompressible equilibrium (Eq. 4, 6)",
              "mrt": "MRT (Eq. 8, d'Humieres et al. 2002 rates), quasi-compressible equilibrium",
              "mrt-incompr": "MRT (Eq. 8, d'Humieres et al. 2002 rates), incompressible equilibrium"}

# Executed FP64 FLOPs per non-solid node update of the all-FP64 step kernel: ncu counts
# of 2 * dfma + dadd + dmul over one launch on the 128^3 pack, divided by its 732 512 nodes.
FP64_FLOPS_PER_NODE = 331

# DRAM bytes (read + write) of one step launch on the porous 256^3 pack, from a one-pass
# ncu capture of this workload (dram__bytes_read.sum + dram__bytes_write.sum, the mean of
# two launches after three warm-up steps), with the hash (step_source_hash) of the library
# sources they were captured with; the bench reports them only while the sources match.
TRAFFIC_PER_LAUNCH_256 = {"sources": "2a89652ed962bf29",
                          "f64": 1194939136 + 855769856,
                          "f32": 685606912 + 416360448,
                          "f16s": 511596416 + 203400832}

if __name__ == "__main__":
    main()
