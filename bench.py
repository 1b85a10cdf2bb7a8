#!/usr/bin/env python
"""Benchmark: MRCM-OS-preconditioned GMRES solves on GB300.

One step = one complete solve of a synthetic problem whose inputs are already resident in HBM:
mrcm_factor_local (transmissibilities, informed spaces, local factors, basis functions, coupling
LU, Schwarz factors) followed by mrcm_gmres_solve from p0 = 0 to relative residual 1e-8.

Workloads (--workload):
  lognormal-2048 (default)  2048 x 2048 cells, log-normal permeability (variance 4, correlation
                            length 0.05), 64 x 64 subdomains of 32 x 32, oversampling 2, one
                            smoothing sweep, FP32 local factors and solves inside FP64 GMRES(30);
                            the same line also times the plain FP64 form of the same problem.
  channels-512              512 x 512 binary channel field (30 % fill, contrast 1e6), 16 x 16
                            subdomains of 32 x 32, oversampling 4, two sweeps, plain FP64, GMRES(30).
  qfs-64                    64 x 64 quarter-five-spot, 4 x 4 subdomains, oversampling 2, one sweep.
Every result is compared with the FP64 oracle's stored solution at sampled cells
(tests/golden/workloads_oracle.json, written by an oracle-only script).

Multi-GPU: one process per GPU (torchrun), each solving its own seeded problem (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and the max over ranks is
reported.

--impl reference times the FP64 CPU oracle on the host cores, one process per core, each step a
bounded sample of the same workload (rank 0 only).
"""

import argparse
import copy
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GMRES solves/s at rel. residual 1e-8"
UNIT = "solves/s"
NOMINAL_FP64_TFLOPS = 1.25      # GB300 dense FP64, recipe table (all SMs at 2070 MHz)
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA lanes x 2 flops x max SM clock
PROFILE_EVERY = 8   # timed steps: events around every 8th occurrence of the dominant phase
GOLDEN = os.path.join(ROOT, "tests", "golden", "workloads_oracle.json")
WORKLOADS = ("lognormal-2048", "channels-512", "qfs-64")
WINDOW = 256        # oracle sample of the 2048^2 workload: blocks of WINDOW^2 cells of its field


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrcm", choices=["mrcm", "reference"])
    ap.add_argument("--workload", default="lognormal-2048", choices=WORKLOADS)
    ap.add_argument("--prec", default=None, choices=["fp64", "fp32"],
                    help="local factors and solves (default: fp32 for lognormal-2048, else fp64)")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--smooth", default="additive", choices=["additive", "multiplicative"],
                    help="Schwarz sweeps: restricted additive (default) or multiplicative multicolour")
    ap.add_argument("--degree", type=int, default=0, choices=[0, 1],
                    help="interface-space degree: 0 piecewise constant (default), 1 piecewise linear")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="off: the library's built-in launch variants (for profiler runs, whose per-launch "
                         "overhead would mislead the autotuner's timings)")
    ap.add_argument("--no-fp64-form", action="store_true", help="mixed workloads: skip the FP64 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true", help="serving stream instead of the single-solve benchmark")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--inflight", type=int, default=8)
    ap.add_argument("--arena-gb", type=float, default=48.0)
    args = ap.parse_args(argv)
    if args.prec is None:
        args.prec = "fp32" if args.workload == "lognormal-2048" else "fp64"
    return args


def rank_seed(rank):
    """Each rank solves its own independent problem (weak scaling): seed 1 + rank."""
    return 1 + int(rank)


def aggregate(total_ms, steps, world, dist=None, device="cpu"):
    """Whole-job throughput: the slowest rank's timed region (MAX over ranks) bounds the job, and
    every rank solved `steps` problems.  Returns (solves/s over all ranks, max total ms)."""
    if world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def workload(args, rank=0, prec=None):
    from paper_2606_08883_gb300 import workloads as W
    prec = W.PREC_FP32 if (prec or args.prec) == "fp32" else W.PREC_FP64
    seed = rank_seed(rank)
    if args.workload == "lognormal-2048":
        prob, q = W.lognormal(2048, seed=seed, prec=prec)
    elif args.workload == "channels-512":
        prob, q = W.channels(512, seed=seed, prec=prec)
    else:
        prob, q = W.quarter_five_spot(64, seed=seed)
        q.local_prec = prec
    q.restart = args.restart
    q.max_iter = max(q.max_iter, 3 * args.restart)
    q.smooth_kind = 1 if getattr(args, "smooth", "additive") == "multiplicative" else 0
    q.iface_degree = int(getattr(args, "degree", 0))
    return prob, q


def workload_name(args):
    return {"lognormal-2048": "lognormal-2048x2048-var4-corr0.05", "channels-512": "channels-512x512-contrast1e6-fill0.30",
            "qfs-64": "quarter-five-spot-64x64-grf-var2-corr0.1"}[args.workload]


def config_dict(args, prob, q):
    return {"workload": workload_name(args), "cells": prob.cells,
            "subdomains": f"{-(-prob.n[0] // q.sub[0])}x{-(-prob.n[1] // q.sub[1])} of {q.sub[0]}x{q.sub[1]}",
            "oversample": q.oversample, "smooth_steps": q.smooth_steps, "alpha": q.alpha, "restart": q.restart,
            "tol_relative": q.tol, "local_prec": args.prec, "krylov_prec": "fp64",
            "refine_setup": int(getattr(q, "refine_setup", 0)),
            "smoothing": getattr(args, "smooth", "additive"), "iface_degree": int(getattr(args, "degree", 0)),
            "autotune": getattr(args, "autotune", "on"), "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single-gpu"}


def golden(args):
    """The oracle's stored result for the workload (seed 1), or None."""
    try:
        with open(GOLDEN) as fh:
            rec = json.load(fh)["results"].get(args.workload)
    except (OSError, ValueError, KeyError):
        return None
    if rec is None or rec.get("restart") != args.restart or args.smooth != "additive" or args.degree != 0:
        return None
    return rec


def err_vs_oracle(p, rec):
    """Relative L2 difference from the oracle's pressure over its stored sample of cells."""
    import numpy as np
    idx = np.asarray(rec["sample_cells"], dtype=np.int64)
    ref = np.asarray(rec["p_sample"])
    v = p.detach().cpu().numpy().ravel()[idx] if hasattr(p, "detach") else np.asarray(p).ravel()[idx]
    return float(np.linalg.norm(v - ref) / np.linalg.norm(ref))


# ----------------------------------------------------------------------------------- oracle
# One oracle solve per child process, on one core (BLAS threads 1): the whole workload, or one
# block of its field (the flow problem on that block, same cell size, subdomains, oversampling and
# smoothing).  Prints {setup_s, iter_s, iters, cells, converged}.
ORACLE_CHILD = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from paper_2606_08883_gb300 import workloads as W
from oracle.solve import build, solve
spec = json.loads({spec!r})
if spec["kind"] == "window":
    prob = W.flow_window(np.load(spec["path"]), spec["h"], "window")
    sub, l, s = tuple(spec["sub"]), spec["l"], spec["s"]
else:
    prob, q = {{"channels-512": lambda: W.channels(512, seed=1), "qfs-64": lambda: W.quarter_five_spot(64, seed=1)}}[spec["workload"]]()
    sub, l, s = q.sub, q.oversample, q.smooth_steps
t0 = time.perf_counter()
pre = build(prob.K, prob.h, prob.dim, prob.bc_kind, sub, l, s, 10.0, iface_degree=spec["degree"], smooth_kind=spec["kind_s"])
t1 = time.perf_counter()
p, info, _ = solve(prob.K, prob.h, prob.dim, prob.bc_kind, prob.bc_val, prob.f, sub=sub, l=l, smooth_steps=s, alpha=10.0,
                   tol=1e-8, restart=spec["restart"], max_iter=3 * spec["restart"] + 100, pre=pre)
t2 = time.perf_counter()
print(json.dumps({{"setup_s": t1 - t0, "iter_s": t2 - t1, "iters": info["iterations"], "cells": prob.cells,
                  "converged": info["status"] == 0}}))
"""


class OracleSampler:
    """Times the FP64 oracle on the host cores on a bounded sample of a workload: the whole
    problem when one oracle solve takes seconds (64^2, 512^2), else blocks of WINDOW^2 cells of the
    2048^2 field.  A block's time is converted to the whole workload by the cell ratio, with the
    GMRES part scaled by the oracle's own iteration count for the whole problem (stored golden
    value) over the block's: t = (n / n_block) (t_setup + t_gmres it / it_block)."""

    def __init__(self, args):
        self.args = args
        self.tmp = None
        self.paths = []
        self.rec = golden(args)

    def prepare(self):
        from paper_2606_08883_gb300 import workloads as W
        import numpy as np
        if self.args.workload != "lognormal-2048":
            return
        prob, q = workload(self.args, 0, "fp64")
        self.full_cells, self.q = prob.cells, q
        self.h = list(prob.h)
        self.tmp = tempfile.mkdtemp(prefix="mrcm_oracle_")
        K = prob.K[0]
        nb = K.shape[0] // WINDOW
        for bj in range(nb):
            for bi in range(nb):
                path = os.path.join(self.tmp, f"K_{bj}_{bi}.npy")
                np.save(path, K[None, bj * WINDOW:(bj + 1) * WINDOW, bi * WINDOW:(bi + 1) * WINDOW])
                self.paths.append(path)

    def _spec(self, i):
        a = self.args
        base = {"restart": a.restart, "degree": a.degree, "kind_s": 1 if a.smooth == "multiplicative" else 0}
        if a.workload == "lognormal-2048":
            return dict(base, kind="window", path=self.paths[i % len(self.paths)], h=self.h, sub=list(self.q.sub),
                        l=self.q.oversample, s=self.q.smooth_steps)
        return dict(base, kind="full", workload=a.workload)

    def run(self, procs):
        """procs concurrent oracle solves (distinct blocks where the sample is a block); returns
        (solves/s of the whole workload over all processes, wall seconds, per-process records)."""
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
        t0 = time.perf_counter()
        ps = [subprocess.Popen([sys.executable, "-c", ORACLE_CHILD.format(root=ROOT, spec=json.dumps(self._spec(i)))],
                               stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env) for i in range(procs)]
        recs = []
        for pr in ps:
            out, err = pr.communicate(timeout=1800)
            if pr.returncode != 0:
                raise RuntimeError("oracle sample failed: " + err[-1500:])
            recs.append(json.loads(out.strip().splitlines()[-1]))
        wall = time.perf_counter() - t0
        per = [self.full_time(r) for r in recs]
        return sum(1.0 / t for t in per), wall, recs

    def full_time(self, r):
        if self.args.workload != "lognormal-2048":
            return r["setup_s"] + r["iter_s"]
        it_full = self.rec["iterations"] if self.rec else r["iters"]
        return self.full_cells / r["cells"] * (r["setup_s"] + r["iter_s"] * it_full / max(r["iters"], 1))

    def describe(self, procs, recs):
        if self.args.workload != "lognormal-2048":
            return (f"{procs} concurrent full FP64 oracle solves of the workload (set-up + GMRES to 1e-8), one core "
                    f"each; iterations {recs[0]['iters']}")
        it_full = self.rec["iterations"] if self.rec else None
        return (f"{procs} concurrent FP64 oracle solves (set-up + GMRES to 1e-8), one core each, of distinct "
                f"{WINDOW}x{WINDOW}-cell blocks of the same 2048^2 field (same cell size, 32x32 subdomains, "
                f"oversampling 2, one sweep; p = 1 / 0 on the block's x faces); each converted to the whole "
                f"workload as (cells ratio {self.full_cells // recs[0]['cells']}) x (set-up + GMRES time x "
                f"{it_full} oracle iterations on the whole problem / {recs[0]['iters']} on the block)")

    def close(self):
        if self.tmp:
            import shutil
            shutil.rmtree(self.tmp, ignore_errors=True)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------- roofline
def krylov_model(n, iterations, restart):
    """Average algorithmic work of one Arnoldi step over a solve: at inner step j the step does the
    stencil (5 FMA per cell), j+1 basis coefficients and j Gram entries (dot products), ||A z||^2,
    w -= V h and ||w||^2: (3j + 9) n FMA; bytes: j+1 basis vectors read twice plus v_j, z, w."""
    js = [t % restart for t in range(max(int(iterations), 1))]
    fma = sum((3 * j + 9) * n for j in js) / len(js)
    nbytes = sum((2 * (j + 1) + 4) * 8 * n for j in js) / len(js)
    return 2 * fma, nbytes


def phase_model(prob, q, prec):
    """Algorithmic work per launch of each phase: (flops, bytes)."""
    S = (-(-prob.n[0] // q.sub[0])) * (-(-prob.n[1] // q.sub[1]))
    elt = 4 if prec == "fp32" else 8
    wl, hl = q.sub[0], q.sub[1]
    wo, ho = wl + 2 * q.oversample, hl + 2 * q.oversample

    def packed(w):
        return (w * (w + 1) // 2 + 3) // 4 * 4

    def factor(w, h):  # per line: Schur update + Cholesky + triangular inverse = w^3 / 2 FMA
        return S * h * w ** 3, S * h * packed(w) * elt

    def solve(w, h, nr, keep=0):
        # twisted solve: h - 1 eliminations, the middle line, and back substitution over the kept
        # lines (a restricted Schwarz solve keeps h - 2l of them); each step is one symmetric line
        # product of w^2 FMA per right-hand side.  Bytes: each line block and the couplings once,
        # the right-hand side and the result.
        m = h // 2
        products = (h - 1) + 1 + (m - keep) + (h - 1 - keep - m)
        return (S * products * 2 * w * w * nr,
                S * (h * packed(w) * elt + h * w * elt + 2 * w * h * 8 * nr))

    n = prob.cells
    schwarz = solve(wo, ho, 1, keep=q.oversample)
    # the particular solve runs on the extended box when l > 0 and keeps Omega plus one line per side
    particular = solve(wo, ho, 1, keep=q.oversample - 1) if q.oversample > 0 else solve(wl, hl, 1)
    if getattr(q, "smooth_kind", 0) == 1:  # multiplicative: one launch per colour, a quarter of the boxes each
        schwarz = (schwarz[0] / 4, schwarz[1] / 4)
    return {
        "factor_ohat_robin": factor(wo, ho), "factor_omega": factor(wl, hl), "factor_ohat_dirichlet": factor(wo, ho),
        "informed": solve(wo, ho, 4), "basis": solve(wl, hl, 4), "particular": particular,
        "schwarz": schwarz, "residual": (9 * n, 40 * n), "reconstruct": (8 * n, 56 * n),
    }


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu --set full
# capture of the kernel behind a phase, valid only while the kernel's source file is unchanged (its
# SHA-256 at capture time); see profiles/ for the capture commands.
NCU_TRAFFIC = {
    ("schwarz", "fp32"): (560.455936e6 + 26.21568e6, "paper_2606_08883_gb300/csrc/k_local.cu",
                          "90f92eb54507d866c4ceeca289bf9899587b21261f4891f4c94873720df18e60"),
    ("factor_ohat_robin", "fp32"): (76.70784e6 + 353.64608e6, "paper_2606_08883_gb300/csrc/k_local.cu",
                                    "90f92eb54507d866c4ceeca289bf9899587b21261f4891f4c94873720df18e60"),
}


# The Arnoldi step's traffic grows with the inner step j: (bytes, j) of the captured launch, scaled
# to the solve's average launch by the model's algorithmic bytes (krylov_model), in which the basis
# sweeps that make the traffic grow in proportion.
NCU_TRAFFIC_KRYLOV = (576.713984e6 + 62.34112e6, 5, "paper_2606_08883_gb300/csrc/k_krylov.cu",
                      "97bf265e4b30d16c4335a8ef6753b412892351f7adbec2e54e23ce2f20898f0f")


def krylov_traffic(n, iterations, restart):
    nbytes, jcap, src, sha = NCU_TRAFFIC_KRYLOV
    try:
        with open(os.path.join(ROOT, src), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != sha:
                return None
    except OSError:
        return None
    at_cap = (2 * (jcap + 1) + 4) * 8 * n
    return nbytes * krylov_model(n, iterations, restart)[1] / at_cap


def ncu_traffic(name, prec):
    entry = NCU_TRAFFIC.get((name, prec))
    if entry is None:
        return None
    nbytes, src, sha = entry
    try:
        with open(os.path.join(ROOT, src), "rb") as fh:
            cur = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    return nbytes if cur == sha else None


def fp64_peak(peaks):
    """(TFLOP/s, source) of the FP64 pipes: measured in this process when available."""
    if peaks.get("fp64_tflops"):
        return peaks["fp64_tflops"], ("measured in this process: register-operand FP64 FMA loop on every SM "
                                      "(mrcm_measure_fp64_peak)")
    return NOMINAL_FP64_TFLOPS, "nominal GB300 dense FP64 1.25 TFLOP/s at 2070 MHz"


def roofline(prof, prob, q, prec, peaks, iterations):
    """Roofline of the phase with the largest event-timed share (the dominant kernel)."""
    model = phase_model(prob, q, prec)
    model["krylov"] = krylov_model(prob.cells, iterations, q.restart)   # FP64 in both precisions
    cands = {k: v for k, v in prof.items() if k in model and v[1] > 0}
    if not cands:
        return None, None
    name = max(cands, key=lambda k: cands[k][0])
    ms, launches = cands[name]
    per_launch_s = ms / 1e3 / launches
    flops, nbytes = model[name]
    p64, p64_src = fp64_peak(peaks)
    if name == "krylov":
        achieved = flops / per_launch_s / 1e12
        return name, {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s",
                      "frac": achieved / p64, "traffic": krylov_traffic(prob.cells, iterations, q.restart),
                      "kernel": "k_arnoldi_ls",
                      "launch_ms": per_launch_s * 1e3, "algorithmic_flops_per_launch": flops,
                      "algorithmic_bytes_per_launch": nbytes, "peak_source": p64_src}
    if name in ("residual", "reconstruct") or (prec == "fp32" and name in ("schwarz", "particular")):
        achieved = nbytes / per_launch_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return name, {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                      "traffic": ncu_traffic(name, prec), "kernel": name, "launch_ms": per_launch_s * 1e3,
                      "algorithmic_bytes_per_launch": nbytes, "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)"}
    fp32_alu = prec == "fp32" and name.startswith("factor")
    peak = NOMINAL_FP32_TFLOPS if fp32_alu else p64
    achieved = flops / per_launch_s / 1e12
    return name, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                  "traffic": ncu_traffic(name, prec), "kernel": name, "launch_ms": per_launch_s * 1e3,
                  "algorithmic_flops_per_launch": flops,
                  "peak_source": "nominal FP32 FMA lanes x 2 x 2070 MHz x 152 SMs" if fp32_alu else p64_src}


def dominant_phase(prof, prob, q, prec, iterations):
    """The modelled phase with the largest event-timed share of a fully profiled step (None when
    nothing was recorded)."""
    model = phase_model(prob, q, prec)
    model["krylov"] = krylov_model(prob.cells, iterations, q.restart)
    cands = {k: v for k, v in prof.items() if k in model and v[1] > 0}
    return max(cands, key=lambda k: cands[k][0]) if cands else None


def phase_rooflines(prof, prob, q, prec, peaks, iterations):
    """Every modelled phase against its bound, from the event-timed launch durations: the local
    factorisations and FP64 solves and the Arnoldi step against the FP64 (or FP32) pipe, the FP32
    solves, the residual, the reconstruction and the dense coupling product against HBM."""
    model = phase_model(prob, q, prec)
    model["krylov"] = krylov_model(prob.cells, iterations, q.restart)
    mx, my = -(-prob.n[0] // q.sub[0]), -(-prob.n[1] // q.sub[1])
    nc = 2 * (mx * (my - 1) + my * (mx - 1))
    nc *= 1 + getattr(q, "iface_degree", 0)
    if nc <= 4096:  # one product with the explicit G^-1 per apply
        model["coarse_solve"] = (2 * nc * nc, 8 * nc * nc)
    out = {}
    for name, (flops, nbytes) in model.items():
        ms, launches = prof.get(name, (0.0, 0))
        if launches <= 0 or ms <= 0.0:
            continue
        per = ms / 1e3 / launches
        mem = name in ("residual", "reconstruct", "coarse_solve") or (
            prec == "fp32" and name in ("schwarz", "particular", "informed", "basis"))
        if mem:
            peak = peaks.get("hbm_gbs", 6800.0)
            ach = nbytes / per / 1e9
            out[name] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 3), "launch_ms": round(per * 1e3, 4)}
        else:
            peak = NOMINAL_FP32_TFLOPS if (prec == "fp32" and name.startswith("factor")) else fp64_peak(peaks)[0]
            ach = flops / per / 1e12
            out[name] = {"bound": "alu", "achieved": round(ach, 4), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(ach / peak, 3), "launch_ms": round(per * 1e3, 4)}
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}



# ----------------------------------------------------------------------------------- arms
def reference_arm(args):
    """The FP64 oracle on the host cores: every step runs one oracle process per core at once on
    the bounded sample (OracleSampler); value = the whole-workload solves/s of all processes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    sampler = OracleSampler(args)
    sampler.prepare()
    try:
        rates, walls, recs = [], [], None
        for step in range(args.warmup + args.steps):
            rate, wall, recs = sampler.run(cores)
            if step >= args.warmup:
                rates.append(rate)
                walls.append(wall)
        desc = sampler.describe(cores, recs)
    finally:
        sampler.close()
    v = statistics.median(rates)
    prob, q = workload(args, 0, "fp64")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(args, prob, q),
            "sample_wall_s_median": statistics.median(walls),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args):
    """The oracle on the host cores, before any CUDA call: one process alone, then one per core at
    once (OracleSampler)."""
    sampler = OracleSampler(args)
    try:
        sampler.prepare()
        r1, _, recs1 = sampler.run(1)
        cores = host_cores()
        rn, wall_n, recs_n = sampler.run(cores)
        return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sampler.describe(cores, recs_n),
                "one_core": {"value": r1, "unit": UNIT, "cores": 1, "sample": sampler.describe(1, recs1),
                             "setup_s": recs1[0]["setup_s"], "gmres_s": recs1[0]["iter_s"],
                             "iterations": recs1[0]["iters"], "cells": recs1[0]["cells"]},
                "wall_s": wall_n}
    except Exception as exc:  # reported, never silently replaced
        return {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": "failed: " + str(exc)[:300]}
    finally:
        sampler.close()


def timed_solves(solver, steps, warmup, stream, dev, flush, barrier, profile_dominant=None):
    """Warm-up then `steps` timed solves (set-up + GMRES), CUDA events on the launching stream with
    a synchronize on both sides; returns (times ms, iterations, last p, last info)."""
    import torch
    p, info = None, None
    for _ in range(warmup):
        solver.factor()
        p, info = solver.solve()
    torch.cuda.synchronize(dev)
    times, iters = [], []
    for _ in range(steps):
        flush.fill_(1)
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.factor()
        p, info = solver.solve()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        times.append(e0.elapsed_time(e1))
        iters.append(info["iterations"])
    return times, iters, p, info


def mrcm_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)   # before any CUDA call: the oracle runs in its own processes
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2606_08883_gb300 import mrcm
    if getattr(args, "autotune", "on") == "off":
        mrcm.autotune(0)
    stream = torch.cuda.current_stream(dev)
    peaks = load_peaks()
    peaks["fp64_tflops"] = mrcm.measure_fp64_peak(stream)
    prob, q = workload(args, rank)
    solver = mrcm.Solver(prob, q, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up; the last warm-up step is fully profiled to find the dominant phase
    info = None
    for i in range(args.warmup):
        if i == args.warmup - 1:
            solver.profile(True)  # grow the profiler's event pool outside the timed region
        solver.factor()
        p, info = solver.solve()
    torch.cuda.synchronize(dev)
    # the timed region records events only around every PROFILE_EVERY-th occurrence of the dominant
    # phase (the one the roofline reports); the per-phase breakdown comes from one fully profiled
    # step after it, so the timed steps carry no other instrumentation
    warm = solver.profile_read(reset=True) if args.warmup > 0 else {}
    dom_phase = dominant_phase(warm, prob, q, args.prec, info["iterations"] if info else 1)
    solver.profile(True, phases=[dom_phase] if dom_phase else None, every=PROFILE_EVERY if dom_phase else 1)
    solver.profile_read(reset=True)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{gpu_id}" if gpu_id is not None else local)
    clocks.start()
    launches0 = mrcm.mrcm_launch_count()
    times, iters, p, info = timed_solves(solver, args.steps, 0, stream, dev, flush, barrier)
    launches = mrcm.mrcm_launch_count() - launches0
    clk = clocks.stop()
    prof = solver.profile_read(reset=True)
    solver.profile(True)
    solver.factor()
    p, info = solver.solve()
    prof_all = solver.profile_read(reset=True)
    solver.profile(False)
    value, total_ms = aggregate(sum(times), args.steps, world, dist, dev)
    rec = golden(args) if rank == 0 else None
    err = err_vs_oracle(p, rec) if rec else None
    # set-up / solve split from one step without events
    torch.cuda.synchronize(dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    solver.factor()
    e[1].record(stream)
    solver.solve()
    e[2].record(stream)
    torch.cuda.synchronize(dev)
    setup_ms, solve_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    # end to end through the C ABI with host buffers (K in, p out, pinned)
    e2e = None
    if not args.no_e2e:
        K_host = torch.as_tensor(prob.K.ravel()).pin_memory()
        p_host = torch.empty(prob.cells, dtype=torch.float64).pin_memory()
        solver.solve_host(K_host, p_host)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            solver.solve_host(K_host, p_host)
        torch.cuda.synchronize(dev)
        barrier()
        e2e_value, _ = aggregate(1e3 * (time.perf_counter() - t0), args.steps, world, dist, dev)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * prob.cells,
               "d2h_bytes_per_step": 8 * prob.cells}
    solver.close()
    # the mixed form without the refinement of its set-up solves, and the plain FP64 form of the
    # same problem (mixed workloads): same timing, fewer steps
    unrefined_form = None
    if args.prec == "fp32" and not args.no_fp64_form and q.refine_setup:
        probr, qr = workload(args, rank)
        qr.refine_setup = 0
        sr = mrcm.Solver(probr, qr, device=dev)
        kr = max(1, min(args.steps, 5))
        tr, itr, pr, infor = timed_solves(sr, kr, max(1, min(args.warmup, 2)), stream, dev, flush, barrier)
        vr, totr = aggregate(sum(tr), kr, world, dist, dev)
        unrefined_form = {"value": vr, "unit": UNIT, "steps": kr, "ms_per_step": totr / kr,
                          "iterations": int(statistics.median(itr)), "rel_res": infor["rel_res"],
                          "err_vs_oracle": err_vs_oracle(pr, rec) if rec else None,
                          "what": "FP32 set-up solves not refined (refine_setup = 0)"}
        sr.close()
    fp64_form = None
    if args.prec == "fp32" and not args.no_fp64_form:
        prob64, q64 = workload(args, rank, "fp64")
        s64 = mrcm.Solver(prob64, q64, device=dev)
        k64 = max(1, min(args.steps, 5))
        t64, it64, p64, info64 = timed_solves(s64, k64, max(1, min(args.warmup, 2)), stream, dev, flush, barrier)
        v64, tot64 = aggregate(sum(t64), k64, world, dist, dev)
        fp64_form = {"value": v64, "unit": UNIT, "steps": k64, "ms_per_step": tot64 / k64,
                     "iterations": int(statistics.median(it64)), "rel_res": info64["rel_res"],
                     "err_vs_oracle": err_vs_oracle(p64, rec) if rec else None,
                     "mixed_over_fp64": value / v64}
        s64.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    dom, roof = roofline(prof, prob, q, args.prec, peaks, statistics.median(iters))
    per_phase = phase_rooflines(prof_all, prob, q, args.prec, peaks, statistics.median(iters))
    lat = sorted(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.prec == "fp32" else "f64", "data": "synthetic", "config": config_dict(args, prob, q),
        "mcells_per_s": value * prob.cells / 1e6, "iterations": int(statistics.median(iters)),
        "rel_res": info["rel_res"],
        "oracle": ({"iterations": rec["iterations"], "err_vs_oracle": err, "sample_cells": len(rec["sample_cells"]),
                    "source": "tests/golden/workloads_oracle.json (FP64 oracle, seed 1)"} if rec else None),
        "fp64_form": fp64_form, "unrefined_form": unrefined_form,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "setup_ms": setup_ms, "solve_ms": solve_ms,
        "phases_ms_per_step": {k: round(v[0], 4) for k, v in prof_all.items()},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "fp64_peak_tflops_measured": peaks["fp64_tflops"],
        "autotuned": autotune_summary(), "phase_rooflines": per_phase,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def autotune_summary():
    """The launch variants the library's autotuner chose during the warm-up (identical results)."""
    from paper_2606_08883_gb300 import mrcm
    out = []
    for e in mrcm.autotune_table():
        k = e["key"]
        if e["kind"] == 0:
            shape = f"local solve fp{8 * k[0]} mode {k[1]} x{k[2]} rhs, {k[3]}x{k[4]} boxes x{k[5]}"
        else:
            shape = f"coupling LU n={k[0]} kl={k[1]} ku={k[2]}"
        out.append(f"{shape}: variant {e['choice'] + 1} of {e['ncand']}, {e['best_us']:.1f} us")
    return out


def serve_arm(args):
    """Serving stream: requests with grids drawn from 128^2..1024^2, log-normal fields (variance
    U[1, 5], correlation length 0.1, seed = 1000 + id), 32 x 32 subdomains, oversampling 2, one
    sweep, FP32 local solves, FP64 GMRES(30).  First the mix back to back (capacity), then Poisson
    arrivals at 0.8 x capacity (seed 7) for latency percentiles."""
    import numpy as np
    import torch
    from paper_2606_08883_gb300 import mrcm, workloads as W
    rng = np.random.default_rng(7)
    sizes = rng.choice([128, 256, 512, 1024], size=args.requests)
    reqs = []
    for i, N in enumerate(sizes):
        var = float(np.random.default_rng(1000 + i).uniform(1.0, 5.0))
        prob, q = W.lognormal(int(N), seed=1000 + i, variance=var, corr=0.1, sub=32, oversample=2, smooth_steps=1,
                              prec=W.PREC_FP32)
        q.restart = args.restart
        q.max_iter = max(q.max_iter, 3 * args.restart)
        reqs.append((prob, q))
    torch.cuda.set_device(0)
    srv = mrcm.Server(int(args.arena_gb * (1 << 30)), max_inflight=args.inflight)

    def run(arrivals):
        t0 = time.perf_counter()
        pending, done, k = {}, {}, 0
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while k < len(reqs) and arrivals[k] <= now:
                pending[srv.submit(*reqs[k])] = k
                k += 1
            for t in list(pending):
                r = srv.poll(t)
                if r is not None:
                    done[pending.pop(t)] = r
            time.sleep(0.0005)
        return time.perf_counter() - t0, done

    # warm-up: one request of each size through the server (module loading, first-touch costs)
    for N in sorted(set(int(v) for v in sizes)):
        i = int(np.nonzero(sizes == N)[0][0])
        t = srv.submit(*reqs[i])
        while srv.poll(t) is None:
            time.sleep(0.001)
    makespan, done = run([0.0] * len(reqs))
    capacity = len(reqs) / makespan
    gaps = rng.exponential(1.0 / (0.8 * capacity), size=len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    wall, done2 = run(list(arrivals))
    lat = sorted(r[2]["latency_ms"] for r in done2.values())
    ok = sum(1 for r in done2.values() if r[0] == mrcm.MRCM_OK)
    cells = sum(p.cells for p, _ in reqs)
    line = {"metric": "serving solves/s and latency (Poisson arrivals at 0.8 x capacity)",
            "value": len(reqs) / wall, "unit": "solves/s", "n_gpus": 1, "requests": len(reqs),
            "capacity_solves_per_s": capacity, "mcells_per_s": cells / wall / 1e6,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
            "converged": ok, "iterations_median": float(np.median([r[2]["iterations"] for r in done2.values()])),
            "max_inflight": args.inflight, "arena_gb": args.arena_gb, "arena_peak_gb": srv.stats()["arena_peak"] / 2 ** 30,
            "dtype": "f32 local / f64 Krylov", "data": "synthetic",
            "config": {"workload": "serving-lognormal-128..1024", "subdomain": "32x32", "oversample": 2,
                       "smooth_steps": 1, "restart": args.restart}}
    srv.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.serve:
        serve_arm(args)
    else:
        mrcm_arm(args)


if __name__ == "__main__":
    main()
