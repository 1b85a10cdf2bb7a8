"""Request server (continuous batching) on the GPU: results are the same alone and in the mix,
admission respects the arena, cancellation and oversize requests are reported."""

import time

import numpy as np
import pytest

from paper_2606_08883_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrcm():
    from paper_2606_08883_gb300 import mrcm as m
    return m


def _mix():
    out = []
    for seed in (1, 2):
        out.append(W.quarter_five_spot(64, seed=seed))
    for seed, prec in ((3, W.PREC_FP64), (4, W.PREC_FP32)):
        prob, q = W.lognormal(128, seed=seed, variance=2.0, corr=0.1, sub=32, oversample=2, smooth_steps=1, prec=prec)
        out.append((prob, q))
    prob, q = W.channels(128, seed=5, sub=32, oversample=4, smooth_steps=2)
    out.append((prob, q))
    prob, q = W.lognormal(96, seed=6, variance=1.0, corr=0.1, sub=16, oversample=2, smooth_steps=1, prec=W.PREC_FP64)
    out.append((prob, q))
    # the variants: a diagonal permeability tensor, piecewise-linear interface spaces, a grid the
    # subdomain size does not divide, multiplicative smoothing
    out.append((W.random_problem((96, 64, 1), seed=21, contrast=1e3, tensor=True),
                W.Params(sub=(16, 16, 1), oversample=2, smooth_steps=2, restart=30)))
    prob, q = W.channels(128, seed=7, sub=32, oversample=4, smooth_steps=2)
    q.iface_degree = 1
    out.append((prob, q))
    out.append((W.random_problem((100, 70, 1), seed=22, contrast=1e3),
                W.Params(sub=(32, 32, 1), oversample=2, smooth_steps=1, restart=30)))
    prob, q = W.quarter_five_spot(64, seed=8)
    q.smooth_kind = 1
    out.append((prob, q))
    return out


def _wait(srv, tickets, timeout=300.0):
    results = {}
    t0 = time.time()
    while len(results) < len(tickets):
        for t in tickets:
            if t in results:
                continue
            r = srv.poll(t, history_cap=512)
            if r is not None:
                results[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.002)
    return results


def test_results_identical_alone_and_in_the_mix(mrcm):
    mix = _mix()
    srv = mrcm.Server(2 << 30, max_inflight=4)
    tickets = [srv.submit(p, q) for (p, q) in mix]
    results = _wait(srv, tickets)
    st = srv.stats()
    bad = [(prob.name, results[t][2].get("error")) for t, (prob, q) in zip(tickets, mix) if results[t][0] != mrcm.MRCM_OK]
    assert st["completed"] == len(mix) and st["failed"] == 0 and len(st["latency_ms"]) == len(mix), bad
    assert 0 < st["arena_peak"] <= 2 << 30
    srv.close()
    for t, (prob, q) in zip(tickets, mix):
        rc, p_served, info = results[t]
        assert rc == mrcm.MRCM_OK, (prob.name, rc)
        s = mrcm.Solver(prob, q)
        s.factor()
        p_alone, info_alone = s.solve(history_cap=512)
        assert info["iterations"] == info_alone["iterations"], prob.name
        assert np.array_equal(p_served, p_alone.cpu().numpy()), prob.name
        assert info["history"] == info_alone["history"][:len(info["history"])]
        assert info["rel_res"] <= q.tol and info["latency_ms"] >= info["queue_ms"] >= 0.0
        s.close()


def test_admission_by_footprint_and_cancel(mrcm):
    prob, q = W.quarter_five_spot(64, seed=7)
    need = mrcm.footprint(prob, q)
    # room for exactly one request at a time: they run one after another
    srv = mrcm.Server(need + 4 * (1 << 20), max_inflight=4)
    tickets = [srv.submit(prob, q) for _ in range(3)]
    results = _wait(srv, tickets)
    st = srv.stats()
    assert st["completed"] == 3 and st["arena_peak"] <= need + 4 * (1 << 20)
    ps = [results[t][1] for t in tickets]
    assert all(np.array_equal(ps[0], x) for x in ps[1:])
    # a request that can never fit is refused at submission
    big, bq = W.channels(256, seed=1)
    with pytest.raises(mrcm.MRCMError) as ei:
        srv.submit(big, bq)
    assert ei.value.status == mrcm.MRCM_ERR_OOM
    # a queued request cancelled before admission finishes at once as cancelled
    a = srv.submit(prob, q)
    b = srv.submit(prob, q)
    srv.cancel(b)
    res = _wait(srv, [a, b])
    assert res[a][0] == mrcm.MRCM_OK
    assert res[b][0] == mrcm.MRCM_ERR_CANCELLED
    srv.close()


def test_cancel_a_running_request(mrcm):
    # a solve whose tolerance is out of reach runs until it is cancelled; the cancel is seen at the
    # next GMRES step, the request finishes as cancelled with the steps it ran, its arena block is
    # released (the stream idle first) and the server goes on serving
    prob, q = W.lognormal(512, seed=9, variance=2.0, corr=0.1, sub=32, oversample=2, smooth_steps=1, prec=W.PREC_FP64)
    q.tol, q.max_iter = 1e-15, 20000
    srv = mrcm.Server(2 << 30, max_inflight=2)
    t = srv.submit(prob, q)
    t0 = time.time()
    while srv.stats()["running"] == 0:
        assert time.time() - t0 < 60.0
        time.sleep(0.002)
    time.sleep(0.5)   # past the set-up, inside GMRES
    assert srv.poll(t) is None
    srv.cancel(t)
    res = _wait(srv, [t], timeout=60.0)
    rc, _p, info = res[t]
    assert rc == mrcm.MRCM_ERR_CANCELLED
    assert 0 < info["iterations"] < q.max_iter
    small, sq = W.quarter_five_spot(64, seed=3)
    t2 = srv.submit(small, sq)
    r2 = _wait(srv, [t2])
    assert r2[t2][0] == mrcm.MRCM_OK
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 1 and st["running"] == 0
    srv.close()


def test_mixed_sizes_under_load_all_converge(mrcm):
    # many requests of different sizes in flight at once: every kernel's launch limits are set once
    # per process (workers launch the same kernels with different shared-memory sizes from several
    # threads), so every request converges as it does alone
    reqs = []
    for i in range(32):
        N = (128, 256, 512, 192)[i % 4]
        prob, q = W.lognormal(N, seed=500 + i, variance=1.0 + (i % 5), corr=0.1, sub=32, oversample=2,
                              smooth_steps=1, prec=W.PREC_FP32 if i % 2 else W.PREC_FP64)
        reqs.append((prob, q))
    srv = mrcm.Server(8 << 30, max_inflight=8)
    tickets = [srv.submit(p, q) for p, q in reqs]
    res = {}
    t0 = time.time()
    while len(res) < len(tickets) and time.time() - t0 < 300:
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.001)
    srv.close()
    assert len(res) == len(tickets)
    assert all(r[0] == mrcm.MRCM_OK for r in res.values()), [(t, r[0]) for t, r in res.items() if r[0] != mrcm.MRCM_OK]
    assert all(r[2]["iterations"] <= 20 for r in res.values())
