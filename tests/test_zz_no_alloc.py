"""The allocation-free residual-norm entry point, for callers that cannot allocate device memory.

mrcm_residual_norm_noalloc keeps its scratch in a fixed array inside the library instead of the
caller's workspace.  It must return exactly what the GMRES entry point reports as its final true
residual (same kernel arithmetic and reduction order), call after call, whether this file runs
alone in a fresh process or after every other test.  This file is named to be collected last.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_2606_08883_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_gmres_true_residual():
    from paper_2606_08883_gb300 import mrcm
    prob, q = W.quarter_five_spot(64, seed=3)
    s = mrcm.Solver(prob, q)
    s.factor()
    b = s.rhs()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        p, info = s.solve()                          # existing entry point: reports ||b - A p||
        rc = mrcm.mrcm_residual_norm_noalloc(s.handle, C.c_void_p(b.data_ptr()), C.c_void_p(p.data_ptr()),
                                             C.c_void_p(out.data_ptr()), stream)
        assert rc == mrcm.MRCM_OK, mrcm.mrcm_last_error(s.handle)
        torch.cuda.synchronize()
        got = float(out.item())
        assert got == info["abs_res"], (call, got, info["abs_res"])
        # and it is the residual norm of the returned solution
        ref = float(torch.linalg.vector_norm(b - s.apply_operator(p)))
        assert np.isclose(got, ref, rtol=1e-12, atol=0.0)
        out.fill_(-1.0)
    # a different iterate on the second pass through the shared scratch
    p2 = 0.5 * p
    rc = mrcm.mrcm_residual_norm_noalloc(s.handle, C.c_void_p(b.data_ptr()), C.c_void_p(p2.data_ptr()),
                                         C.c_void_p(out.data_ptr()), stream)
    assert rc == mrcm.MRCM_OK
    torch.cuda.synchronize()
    ref2 = float(torch.linalg.vector_norm(b - s.apply_operator(p2)))
    assert np.isclose(float(out.item()), ref2, rtol=1e-12, atol=0.0)
    s.close()
