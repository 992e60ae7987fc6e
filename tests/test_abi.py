"""The C-ABI library builds, loads without a GPU and exports every symbol include/pd.h declares."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1610_08895_gb300 import _binding
    return _binding.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1610_08895_gb300 import _binding
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_binding.exported_symbols()) == names


def test_host_only_entry_points_work_without_gpu(lib):
    from oracle import wavelets as W
    from paper_1610_08895_gb300.api import daubechies_filter
    # the library derives db1..db8 with its own root finder; they agree with the oracle's
    for k in range(1, 9):
        assert np.max(np.abs(daubechies_filter(k) - W.daubechies_lowpass(k))) < 1e-13
    h = np.zeros(2)
    assert lib.pd_daubechies_filter(9, h.ctypes.data) == 1            # PD_EINVAL
    assert b"1..8" in lib.pd_last_error()
    assert lib.pd_plan_create(None, ctypes.byref(ctypes.c_void_p())) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1610_08895_gb300 import _binding
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(_binding.ExtensionMissing):
        _binding.load()


def test_plan_descriptions_are_refused_before_any_device_work(lib):
    """Invalid or unsupported plan descriptions return a status and a message without
    touching a GPU (this runs on machines that have none)."""
    from paper_1610_08895_gb300 import _binding as B
    m = 16
    uv = np.zeros((m, 2))
    blk = np.zeros(m, np.int32)
    ids = np.array([0, 1], np.int32)
    bad_ids = np.array([0, 9], np.int32)
    dde = np.zeros((m, 3, 3, 2))

    def create(**over):
        kw = dict(nx=64, ny=64, osf=2, nvis=m, uv=uv.ctypes.data, nblocks=1, block_of_vis=blk.ctypes.data,
                  kernel_width=8, kb_beta=0.0, nbases=2, basis_ids=ids.ctypes.data, levels=2,
                  precision=B.PD_F32, tile=0)
        kw.update(over)
        d = B.PdPlanDesc(**kw)
        h = ctypes.c_void_p()
        st = lib.pd_plan_create(ctypes.byref(d), ctypes.byref(h))
        return st, lib.pd_last_error()

    cases = [
        (dict(nx=48), 1, b"powers of two"),
        (dict(ny=8), 1, b"powers of two"),
        (dict(osf=3), 1, b"oversampling"),
        (dict(nx=8192, ny=8192, precision=B.PD_F64), 6, b"FP64"),
        (dict(kernel_width=7), 1, b"kernel_width"),
        (dict(nblocks=0), 1, b"nblocks"),
        (dict(basis_ids=bad_ids.ctypes.data), 1, b"basis ids"),
        (dict(levels=7, nx=16, ny=16), 1, b"levels"),
        (dict(tile=4), 1, b"tile"),
        (dict(precision=7), 1, b"precision"),
        (dict(g_mode=2), 1, b"g_mode"),
        (dict(g_mode=B.PD_G_CSR, kernel_width=10), 6, b"CSR"),
        (dict(dde_width=3, dde_kernels=dde.ctypes.data), 1, b"PD_G_CSR"),
        (dict(g_mode=B.PD_G_CSR, dde_width=2, dde_kernels=dde.ctypes.data), 1, b"odd"),
        (dict(g_mode=B.PD_G_CSR, dde_width=3), 1, b"dde_kernels"),
        (dict(g_mode=B.PD_G_CSR, dde_width=3, dde_kernels=dde.ctypes.data), 6, b"<= 8"),
    ]
    for over, status, text in cases:
        st, msg = create(**over)
        assert st == status, (over, st, msg)
        assert text in msg, (over, msg)


def test_reweighting_rule_refuses_bad_arguments_without_gpu(lib):
    x = np.zeros(4)
    assert lib.pd_sara_weights(None, x.ctypes.data, ctypes.c_double(0.1), x.ctypes.data, None) == 1
    assert b"pd_sara_weights" in lib.pd_last_error()
