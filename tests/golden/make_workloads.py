"""Writes tests/golden/workloads_oracle.json: the FP64 oracle on the benchmark workloads (the
quarter-five-spot 64 x 64, the 512 x 512 channel field and the 2048 x 2048 log-normal field, each
with its stated subdomains, oversampling, smoothing steps and GMRES(30) to relative 1e-8): GMRES
iterations, final relative residual, ||b||, and the pressure at a seeded sample of 1024 cells, so
that a GPU result can be compared with the oracle where a full oracle solve is too slow to repeat
in a test or a benchmark run.

Calls only oracle/ and the input generators.  Run from the repository root (about a minute and 6 GB of
memory, most of it the 2048 x 2048 solve):
    python tests/golden/make_workloads.py
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2606_08883_gb300 import workloads as W  # noqa: E402

SAMPLE = 1024      # cells sampled per workload
SAMPLE_SEED = 20260


def sample_cells(n_cells):
    if n_cells <= SAMPLE:
        return np.arange(n_cells)
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n_cells, size=SAMPLE, replace=False))


def run(name, prob, q):
    t0 = time.time()
    p, info, _ = oracle.solve(prob.K, prob.h, prob.dim, prob.bc_kind, prob.bc_val, prob.f, sub=q.sub, l=q.oversample,
                              smooth_steps=q.smooth_steps, alpha=q.alpha, tol=q.tol, tol_relative=bool(q.tol_relative),
                              restart=q.restart, max_iter=q.max_iter, iface_degree=q.iface_degree,
                              smooth_kind=q.smooth_kind)
    idx = sample_cells(prob.cells)
    rec = {"workload": prob.name, "cells": prob.cells, "sub": list(q.sub), "oversample": q.oversample,
           "smooth_steps": q.smooth_steps, "restart": q.restart, "tol": q.tol, "iterations": info["iterations"],
           "rel_res": info["rel_res"], "abs_res": info["abs_res"], "b_norm": float(np.linalg.norm(info["b"])),
           "p_norm": float(np.linalg.norm(p)), "sample_cells": idx.tolist(), "p_sample": p.ravel()[idx].tolist(),
           "oracle_s": time.time() - t0}
    print(name, info["iterations"], f"{info['rel_res']:.2e}", f"{rec['oracle_s']:.1f}s", flush=True)
    return rec


def main():
    out = {"generator": "tests/golden/make_workloads.py (FP64 oracle, per-step Givens check)", "results": {}}
    prob, q = W.quarter_five_spot(64, 1)
    out["results"]["qfs-64"] = run("qfs-64", prob, q)
    prob, q = W.channels(512, 1)
    out["results"]["channels-512"] = run("channels-512", prob, q)
    prob, q = W.lognormal(2048, 1)
    q.local_prec = W.PREC_FP64
    out["results"]["lognormal-2048"] = run("lognormal-2048", prob, q)
    with open(os.path.join(HERE, "workloads_oracle.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
