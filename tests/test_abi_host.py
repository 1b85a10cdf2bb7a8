"""C-ABI library checks that need no GPU: it loads, exports every symbol include/mrcm.h declares,
and its host planner (MRCM-OS step 1) matches the oracle's integer tables bit for bit.  No compute
entry point is called here."""

import os
import re

import numpy as np
import pytest

from oracle.partition import Partition
from paper_2606_08883_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_08883_gb300 import build
    build.build()
    from paper_2606_08883_gb300 import mrcm
    return mrcm


def _declared():
    src = open(os.path.join(ROOT, "include", "mrcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrcm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib._lib, name), name
        assert name in lib.EXPORTED, name


@pytest.mark.parametrize("n,sub,l", [((24, 16, 1), (8, 8, 1), 2), ((64, 64, 1), (16, 16, 1), 4),
                                     ((40, 24, 1), (8, 12, 1), 7), ((10, 10, 1), (10, 10, 1), 0),
                                     ((12, 8, 4), (4, 4, 2), 1), ((61, 45, 1), (16, 12, 1), 3),
                                     ((50, 37, 1), (16, 12, 1), 0), ((40, 20, 1), (16, 32, 1), 2),
                                     ((14, 11, 6), (4, 3, 4), 1)])
def test_plan_export_matches_oracle_bit_exactly(lib, n, sub, l):
    dim = 3 if n[2] > 1 else 2
    prob = W.random_problem(n, dim=dim, seed=0)
    q = W.Params(sub=sub, oversample=l)
    got = lib.plan_export(prob, q)
    want = Partition(dim, n, sub, l).export()
    assert got.dtype == want.dtype and np.array_equal(got, want)


@pytest.mark.parametrize("bad", [dict(sub=(5, 8, 1), oversample=4), dict(sub=(0, 8, 1)), dict(oversample=8), dict(oversample=-1), dict(alpha=0.0),
                                 dict(tol=-1.0), dict(restart=0), dict(max_iter=0), dict(local_prec=7),
                                 dict(smooth_kind=2), dict(iface_degree=2), dict(iface_degree=-1)])
def test_invalid_parameters_rejected(lib, bad):
    prob = W.random_problem((24, 16, 1), seed=0)
    kw = dict(sub=(8, 8, 1), oversample=2)
    kw.update(bad)
    with pytest.raises(lib.MRCMError) as ei:
        lib.plan_export(prob, W.Params(**kw))
    assert ei.value.status == lib.MRCM_ERR_INVALID_ARG


def test_pure_neumann_rejected_and_3d_unsupported(lib):
    prob = W.random_problem((16, 16, 1), seed=0, bc_kind=[1, 1, 1, 1, 1, 1])
    with pytest.raises(lib.MRCMError) as ei:
        lib.footprint(prob, W.Params(sub=(8, 8, 1)))
    assert ei.value.status == lib.MRCM_ERR_INVALID_ARG
    prob3 = W.random_problem((8, 8, 4), dim=3, seed=0)
    with pytest.raises(lib.MRCMError) as ei:
        lib.footprint(prob3, W.Params(sub=(4, 4, 2), oversample=1))
    assert ei.value.status == lib.MRCM_ERR_UNSUPPORTED


def test_footprint_grows_with_restart_and_smoothing(lib):
    prob, params = W.channels(128, sub=32)
    a = lib.footprint(prob, params)
    params.restart += 40
    b = lib.footprint(prob, params)
    assert b > a and a % 256 == 0 and b % 256 == 0
    params.smooth_steps = 0
    c = lib.footprint(prob, params)
    assert c < b


def test_piecewise_linear_sides_need_two_faces(lib):
    # 37 = 3 * 12 + 1: the last row of subdomains is one cell high, so its -x / +x Robin sides have
    # one face and the linear side function vanishes there
    prob = W.random_problem((50, 37, 1), seed=0)
    lib.plan_export(prob, W.Params(sub=(16, 12, 1), oversample=0))
    with pytest.raises(lib.MRCMError) as ei:
        lib.plan_export(prob, W.Params(sub=(16, 12, 1), oversample=0, iface_degree=1))
    assert ei.value.status == lib.MRCM_ERR_INVALID_ARG


def test_plan_export_matches_oracle_on_random_partitions(lib):
    # random grids, subdomain sizes (dividing or not) and oversampling widths: the host planner's
    # integer tables equal the oracle's bit for bit, and both reject the same invalid inputs
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(nx=st.integers(1, 40), ny=st.integers(1, 40), sx=st.integers(1, 16), sy=st.integers(1, 16),
               l=st.integers(0, 6))
    def check(nx, ny, sx, sy, l):
        prob = W.random_problem((nx, ny, 1), seed=0)
        q = W.Params(sub=(sx, sy, 1), oversample=l)
        try:
            want = Partition(2, (nx, ny, 1), (sx, sy, 1), l).export()
        except ValueError:
            with pytest.raises(lib.MRCMError) as ei:
                lib.plan_export(prob, q)
            assert ei.value.status == lib.MRCM_ERR_INVALID_ARG
            return
        got = lib.plan_export(prob, q)
        assert got.dtype == want.dtype and np.array_equal(got, want)

    check()


def test_plan_export_matches_oracle_on_random_3d_partitions(lib):
    # the same comparison on random 3-D grids: boxes, oversampled boxes, Robin sides, interface
    # tables and banded coupling rows for six sides per subdomain
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=100, deadline=None)
    @hyp.given(nx=st.integers(1, 12), ny=st.integers(1, 12), nz=st.integers(2, 10), sx=st.integers(1, 6),
               sy=st.integers(1, 6), sz=st.integers(1, 6), l=st.integers(0, 3))
    def check(nx, ny, nz, sx, sy, sz, l):
        prob = W.random_problem((nx, ny, nz), dim=3, seed=0)
        q = W.Params(sub=(sx, sy, sz), oversample=l)
        try:
            want = Partition(3, (nx, ny, nz), (sx, sy, sz), l).export()
        except ValueError:
            with pytest.raises(lib.MRCMError) as ei:
                lib.plan_export(prob, q)
            assert ei.value.status == lib.MRCM_ERR_INVALID_ARG
            return
        got = lib.plan_export(prob, q)
        assert got.dtype == want.dtype and np.array_equal(got, want)

    check()
