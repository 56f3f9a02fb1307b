"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/*.h (no compute calls: CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1902_09046_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"#[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{]*\)\s*;", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not build.up_to_date():
        try:
            build.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    return ctypes.CDLL(build.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"abc_prior_predictive", "abc_select", "pvalue_sweep"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTED)


def test_exports_are_extern_c(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in syms, name


def test_host_side_calls_without_gpu(lib):
    lib.ppabc_abi_version.restype = ctypes.c_int
    assert lib.ppabc_abi_version() == 1
    lib.abc_select_workspace_bytes.restype = ctypes.c_size_t
    lib.abc_select_workspace_bytes.argtypes = [ctypes.c_uint64]
    small = lib.abc_select_workspace_bytes(1)
    big = lib.abc_select_workspace_bytes(1 << 24)
    assert small > 0 and big > small and big % 256 == 0


def test_invalid_arguments_fail_before_any_launch(lib):
    b = binding.load_library()
    m = binding.OUModel.from_dict({"lo": (0.1, -2, 0.1), "hi": (2, 2, 1), "x0": 0.0, "dt": 0.01,
                                   "n_steps": 5, "n_obs": 10})  # fewer steps than observations
    y = (ctypes.c_double * 10)(*([0.0] * 10))
    rc = b.abc_prior_predictive(ctypes.byref(m), y, 10, 0, 1, 0, None, None, ctypes.c_void_p(16), None)
    assert rc == binding.PPABC_EINVAL
    assert b"n_steps" in b.ppabc_last_error()
    # k > n is rejected
    rc = b.abc_select(ctypes.c_void_p(16), 4, 5, 0.0, None, 0, 0, 0, ctypes.c_void_p(16), None, None,
                      0, ctypes.c_void_p(16), None, None, ctypes.c_void_p(256), 1 << 20, None)
    assert rc == binding.PPABC_EINVAL
    # undersized workspace
    rc = b.abc_select(ctypes.c_void_p(16), 4, 2, 0.0, None, 0, 0, 0, ctypes.c_void_p(16), None, None,
                      0, ctypes.c_void_p(16), None, None, ctypes.c_void_p(256), 8, None)
    assert rc == binding.PPABC_ENOMEM
    # p-value sweep: zero data sets
    rc = b.pvalue_sweep(ctypes.c_void_p(16), 4, 50, 0, 0, 1.0, 2, ctypes.c_void_p(16), None, None, None)
    assert rc == binding.PPABC_EINVAL
    # p-value sweep: data-set range past 2^32
    rc = b.pvalue_sweep(ctypes.c_void_p(16), 4, 50, 10, (1 << 32) - 5, 1.0, 2, ctypes.c_void_p(16),
                        None, None, None)
    assert rc == binding.PPABC_EINVAL


def test_no_device_is_reported_as_error_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    b = binding.load_library()
    rc = b.ppabc_device_check()
    assert rc in (binding.PPABC_ECUDA, binding.PPABC_ENODEV)


def test_merge_entry_points_validate_before_any_launch(lib):
    """abc_select_candidates / abc_merge_candidates (the exchange step of a
    sample-sharded job) reject every malformed call on the host, before the
    device is touched; the pointers below are aligned dummies that the calls
    never dereference."""
    b = binding.load_library()
    P = ctypes.c_void_p
    a = P(1 << 12)
    EINVAL, ENOMEM = binding.PPABC_EINVAL, binding.PPABC_ENOMEM
    cand = b.abc_select_candidates
    assert cand(None, 10, 0, None, None, 0, None, None, None, None) == binding.PPABC_OK  # nothing to record
    assert cand(a, 4, 0, a, a, 5, a, a, a, None) == EINVAL  # more candidates than samples
    assert b"count" in b.ppabc_last_error()
    assert cand(a, 1 << 32, 0, a, a, 5, a, a, a, None) == EINVAL  # n must fit 32 bits
    assert cand(None, 10, 0, a, a, 5, a, a, a, None) == EINVAL  # NULL distances
    assert cand(a, 10, 0, a, a, 5, a, None, a, None) == EINVAL  # NULL index output
    assert cand(a, 10, 0, a, P((1 << 12) + 8), 5, a, a, a, None) == EINVAL  # records not 16-byte aligned
    assert cand(a, 10, (1 << 32) - 5, a, a, 5, a, a, a, None) == EINVAL  # global indices past 2^32
    assert b"sample_base" in b.ppabc_last_error()

    ws = b.abc_merge_workspace_bytes
    assert ws(1, 1) > 0 and ws(1000, 10) % 256 == 0
    assert ws(1 << 20, 100) > ws(1000, 100) and ws(1000, 900) >= ws(1000, 10)
    need = ws(100, 10)
    merge = b.abc_merge_candidates
    wsp = P(1 << 16)
    assert merge(a, a, a, 100, 0, a, a, a, None, None, wsp, need, None) == EINVAL  # k = 0
    assert merge(a, a, a, 100, 101, a, a, a, None, None, wsp, need, None) == EINVAL  # k > m
    assert b"k must be" in b.ppabc_last_error()
    assert merge(a, a, a, 1 << 32, 10, a, a, a, None, None, wsp, need, None) == EINVAL  # m must fit 32 bits
    assert merge(a, None, a, 100, 10, a, a, a, None, None, wsp, need, None) == EINVAL  # NULL global indices
    assert merge(a, a, a, 100, 10, a, a, None, None, None, wsp, need, None) == EINVAL  # NULL count output
    assert merge(a, a, a, 100, 10, a, P((1 << 12) + 4), a, None, None, wsp, need, None) == EINVAL  # rec_out
    assert merge(a, a, a, 100, 10, a, a, a, None, None, wsp, need - 1, None) == ENOMEM  # workspace too small
    assert merge(a, a, a, 100, 10, a, a, a, None, None, None, need, None) == ENOMEM  # no workspace
    assert merge(a, a, a, 100, 10, a, a, a, None, None, P((1 << 16) + 128), need, None) == EINVAL  # alignment
    assert b"256-byte" in b.ppabc_last_error()


def test_device_info_without_gpu(lib):
    import torch
    b = binding.load_library()
    assert b.ppabc_device_info(None, None) == binding.PPABC_EINVAL
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sm, clk = ctypes.c_int(-1), ctypes.c_int(-1)
    assert b.ppabc_device_info(ctypes.byref(sm), ctypes.byref(clk)) in (binding.PPABC_ECUDA, binding.PPABC_ENODEV)
    with pytest.raises(RuntimeError):
        binding.device_info()
