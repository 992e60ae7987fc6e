"""The allocation-free Psi^H entry point (pd_apply_psi_adj_noalloc) against pd_apply_psi_adj.

Callers that cannot allocate device memory while running use the variant whose
scratch is the library's static device array. This file is collected last, so a
run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_OP32, TOL_OP64, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("precision,tol", [("f32", TOL_OP32), ("f64", TOL_OP64)])
def test_noalloc_psi_adj_matches_plan_entry_point_on_two_calls(precision, tol):
    from paper_1610_08895_gb300 import _binding as B
    from paper_1610_08895_gb300.api import Plan
    n, levels, ids = 128, 4, list(range(9))
    dt = torch.float32 if precision == "f32" else torch.float64
    plan = Plan(n, n, np.zeros((1, 2)), np.zeros(1, np.int32), 1, kernel_width=8, basis_ids=ids, levels=levels,
                precision=precision)
    rng = np.random.default_rng(5)
    xs = [torch.tensor(rng.normal(size=(n, n)), dtype=dt, device="cuda") for _ in range(2)]
    refs = [plan.pd_apply_psi_adj(x).cpu().numpy() for x in xs]
    hid = np.ascontiguousarray(ids, dtype=np.int32)
    prec = B.PD_F32 if precision == "f32" else B.PD_F64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for x in xs:                                      # two calls in a row on the shared static scratch
        out = torch.full((len(ids), n, n), float("nan"), dtype=dt, device="cuda")
        B.call("pd_apply_psi_adj_noalloc", ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n, n,
               levels, hid.ctypes.data, len(ids), prec, stream)
        outs.append(out)
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < tol


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    from paper_1610_08895_gb300 import _binding as B
    hid = np.arange(9, dtype=np.int32)
    x = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    out = torch.zeros((1,), dtype=torch.float32, device="cuda")    # never written: the call is refused first
    st = B.load().pd_apply_psi_adj_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), 2048,
                                           2048, 4, hid.ctypes.data, 9, B.PD_F32, None)
    assert st == B.PD_EINVAL
    assert b"static array holds" in B.load().pd_last_error()
