"""Host bookkeeping of bench.py on CPU: the dominant phase comes from a fully profiled step, and the
roofline's mean launch duration is a phase's event time over its recorded launches, so sampling
every n-th launch of the phase leaves it unchanged."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2606_08883_gb300 import workloads as W  # noqa: E402

PHASES = ("assemble", "factor_ohat_robin", "informed", "factor_omega", "basis", "coarse_factor",
          "factor_ohat_dirichlet", "particular", "coarse_solve", "reconstruct", "residual", "schwarz", "krylov", "stage")


def _case():
    prob, q = W.channels(64, seed=1, sub=16, oversample=2, smooth_steps=2)
    return prob, q


def _prof(**entries):
    out = {name: (0.0, 0) for name in PHASES}
    out.update(entries)
    return out


def test_dominant_phase_is_the_largest_modelled_share():
    prob, q = _case()
    prof = _prof(schwarz=(3.0, 30), krylov=(2.0, 15), particular=(1.0, 15), coarse_factor=(5.0, 2))
    # coarse_factor has no work model, so it is never the roofline's kernel
    assert bench.dominant_phase(prof, prob, q, "fp64", 15) == "schwarz"
    assert bench.dominant_phase(_prof(), prob, q, "fp64", 15) is None


def test_roofline_mean_launch_from_sampled_events():
    prob, q = _case()
    peaks = {"hbm_gbs": 6680.0}
    flops = bench.phase_model(prob, q, "fp64")["schwarz"][0]
    # every launch recorded: 40 launches in 4 ms; every 8th recorded: 5 launches in 0.5 ms
    full = bench.roofline(_prof(schwarz=(4.0, 40)), prob, q, "fp64", peaks, 15)
    sampled = bench.roofline(_prof(schwarz=(0.5, 5)), prob, q, "fp64", peaks, 15)
    for name, roof in (full, sampled):
        assert name == "schwarz"
        assert roof["launch_ms"] == pytest.approx(0.1)
        assert roof["achieved"] == pytest.approx(flops / 1e-4 / 1e12)
        assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
        assert roof["unit"] == "TFLOP/s" and roof["bound"] == "alu"
    assert bench.PROFILE_EVERY >= 1


def test_phase_rooflines_cover_every_profiled_modelled_phase():
    prob, q = _case()
    prof = _prof(schwarz=(1.0, 10), particular=(0.5, 5), reconstruct=(0.1, 5), factor_omega=(1.5, 1))
    out = bench.phase_rooflines(prof, prob, q, "fp64", {"hbm_gbs": 6680.0}, 15)
    assert set(out) == {"schwarz", "particular", "reconstruct", "factor_omega"}
    assert out["reconstruct"]["bound"] == "hbm" and out["schwarz"]["bound"] == "alu"
    assert out["factor_omega"]["launch_ms"] == pytest.approx(1.5)


def test_default_line_is_the_2048_mixed_workload():
    args = bench.parse([])
    assert (args.workload, args.prec, args.restart) == ("lognormal-2048", "fp32", 30)
    prob, q = bench.workload(args)
    assert prob.n[:2] == (2048, 2048) and tuple(q.sub[:2]) == (32, 32)
    assert (q.oversample, q.smooth_steps, q.local_prec) == (2, 1, W.PREC_FP32)
    assert bench.config_dict(args, prob, q)["subdomains"] == "64x64 of 32x32"
    prob64, q64 = bench.workload(args, prec="fp64")
    assert q64.local_prec == W.PREC_FP64 and prob64.name == prob.name
    assert bench.parse(["--workload", "channels-512"]).prec == "fp64"


def test_block_sample_converted_by_cells_and_oracle_iterations():
    # t = (n / n_block) (t_setup + t_gmres it / it_block)
    args = bench.parse([])
    s = bench.OracleSampler(args)
    s.full_cells = 2048 * 2048
    s.rec = {"iterations": 10}
    r = {"setup_s": 0.5, "iter_s": 1.3, "iters": 13, "cells": 256 * 256}
    assert s.full_time(r) == pytest.approx(64 * (0.5 + 1.3 * 10 / 13))
    full = bench.OracleSampler(bench.parse(["--workload", "channels-512"]))
    assert full.full_time(r) == pytest.approx(1.8)   # a full-size sample is not scaled


def test_error_against_the_stored_oracle_samples():
    import numpy as np
    rec = {"sample_cells": [0, 5, 9], "p_sample": [1.0, 2.0, 2.0]}
    p = np.zeros(10)
    p[[0, 5, 9]] = [1.0, 2.0, 2.0 + 3e-9]
    assert bench.err_vs_oracle(p, rec) == pytest.approx(1e-9)
    args = bench.parse([])
    rec = bench.golden(args)
    assert rec is not None and rec["iterations"] > 0 and len(rec["sample_cells"]) == len(rec["p_sample"]) == 1024
    assert bench.golden(bench.parse(["--restart", "20"])) is None   # another configuration: no stored value


def test_particular_solve_modelled_on_the_extended_box():
    prob, q = _case()   # oversampling 2: 20 x 20 extended boxes, Omega plus one line per side kept
    m = bench.phase_model(prob, q, "fp64")
    w = q.sub[0] + 2 * q.oversample
    S = (prob.n[0] // q.sub[0]) * (prob.n[1] // q.sub[1])
    products = (w - 1) + 1 + (w // 2 - (q.oversample - 1)) + (w - 1 - (q.oversample - 1) - w // 2)
    assert m["particular"][0] == S * products * 2 * w * w


def test_krylov_roofline_traffic_scaled_from_the_captured_step(monkeypatch):
    """The Arnoldi step's ncu traffic was taken at one inner step j; the line reports it scaled to
    the solve's average step by the model's algorithmic bytes, and drops it (None) once the
    kernel's source file no longer matches the capture."""
    prob, q = _case()
    n, iters = prob.cells, 10
    nbytes, jcap = bench.NCU_TRAFFIC_KRYLOV[0], bench.NCU_TRAFFIC_KRYLOV[1]
    want = nbytes * bench.krylov_model(n, iters, q.restart)[1] / ((2 * (jcap + 1) + 4) * 8 * n)
    assert bench.krylov_traffic(n, iters, q.restart) == pytest.approx(want)
    # a solve of jcap + 1 steps (j = 0..jcap) averages below the captured step, so its traffic is smaller
    assert bench.krylov_traffic(n, jcap + 1, q.restart) < nbytes * 1.0001
    name, roof = bench.roofline(_prof(krylov=(2.0, 10)), prob, q, "fp64", {"hbm_gbs": 6680.0}, iters)
    assert name == "krylov" and roof["kernel"] == "k_arnoldi_ls"
    assert roof["traffic"] == pytest.approx(want)
    stale = (nbytes, jcap, bench.NCU_TRAFFIC_KRYLOV[2], "0" * 64)
    monkeypatch.setattr(bench, "NCU_TRAFFIC_KRYLOV", stale)
    assert bench.krylov_traffic(n, iters, q.restart) is None


def test_ncu_traffic_follows_the_source_hash(monkeypatch):
    entry = bench.NCU_TRAFFIC[("schwarz", "fp32")]
    assert bench.ncu_traffic("schwarz", "fp32") in (entry[0], None)
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("schwarz", "fp32"), (entry[0], entry[1], "0" * 64))
    assert bench.ncu_traffic("schwarz", "fp32") is None
    assert bench.ncu_traffic("no such phase", "fp32") is None
