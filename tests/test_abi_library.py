"""The C-ABI boundary without a GPU: libvlasov builds for sm_103a, loads,
and exports exactly the entry points that include/vlasov.h declares (each
bound in the Python layer with the same name); the host-only calls
(workspace sizing, descriptor validation, error text) answer correctly.
No call here launches a kernel."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2109_06743_gb300 import abi
from paper_2109_06743_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "vlasov.h")


def declared():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\([^;{]*\)\s*;", src, flags=re.M)


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2109_06743_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    return abi.lib()


def test_header_declarations_are_exported_and_bound(lib):
    names = declared()
    assert len(names) >= 20 and len(set(names)) == len(names)
    assert set(names) == set(abi.EXPORTED)
    for n in names:
        assert getattr(lib, n) is not None
    nm = shutil.which("nm")
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", abi.LIB_PATH], capture_output=True, text=True).stdout
        text = {line.split()[-1] for line in out.splitlines() if " T " in line}
        public = {t for t in text if not t.startswith("_")}
        # no undeclared C entry points (C++ symbols are mangled and start with _)
        assert public == set(names), public ^ set(names)


def test_workspace_sizing_and_validation_on_host(lib):
    cfg = W.harris(nx=16, ny=8, nv=8, lx=3.2, ly=1.6)
    d = abi.make_desc(cfg)
    nb = abi.vlasov_work_bytes(d)
    nc = cfg.ncell
    # at least the shear tables (20 doubles per cell) and two fits of 10
    # parameters per cell
    assert nb >= nc * 20 * 8 + 2 * nc * 10 * 8
    bad = abi.make_desc(cfg)
    bad.nx = 0
    assert abi.vlasov_work_bytes(bad) == 0
    assert b"nx" in lib.vl_last_error(None)
    bad = abi.make_desc(cfg)
    bad.precision = 16
    assert abi.vlasov_work_bytes(bad) == 0
    bad = abi.make_desc(cfg)
    bad.vmin[0][1] = bad.vmin[0][1] * 0.5  # walls need a box symmetric in v_y
    assert abi.vlasov_work_bytes(bad) == 0
    assert isinstance(lib.vl_last_error(None), bytes)


def test_host_only_calls_reject_a_missing_context(lib):
    """moment_fit_wide is host-only: without a context it returns VL_EINVAL
    (1) and launches nothing."""
    assert lib.moment_fit_wide(None, 0, 1) == 1


def test_static_pass_refuses_bad_pointers_before_any_launch(lib):
    """pfc_advect_v_static checks its raw pointers on the host: a pointer not
    aligned to its element size (f) or to 8 bytes (E and B, moments), or
    moments that overlap f, return VL_EINVAL (1) before the scratch address
    is looked up or anything is launched (the addresses here are never
    dereferenced)."""
    cfg = W.harris(nx=4, ny=4, nv=8, lx=0.8, ly=0.8, precision=32)
    d = abi.make_desc(cfg)
    D = abi.ctypes.byref(d)
    V = 8 ** 3
    base = 1 << 40
    eb = base + (1 << 30)
    mom = base + (2 << 30)
    cases = [
        (base + 2, eb, mom, b"f_dev is not aligned"),
        (base, eb + 4, mom, b"eb_dev is not 8-byte aligned"),
        (base, eb, mom + 4, b"mom_out is not 8-byte aligned"),
        (base, eb, base + 8 * V * 4, b"mom_out overlaps f_dev"),
    ]
    for f, e, m, msg in cases:
        assert lib.pfc_advect_v_static(D, 0, f, e, 16, 0.01, m, None) == abi.VL_EINVAL
        assert msg in lib.vl_last_error(None), lib.vl_last_error(None)
    d64 = abi.make_desc(cfg)
    d64.precision = 64
    assert lib.pfc_advect_v_static(abi.ctypes.byref(d64), 0, base + 4, eb, 16, 0.01, None, None) == abi.VL_EINVAL
    assert b"f_dev is not aligned" in lib.vl_last_error(None)


def test_sync_status_rejects_a_missing_context(lib):
    assert lib.vl_sync_status(None, None) == abi.VL_EINVAL


def test_fma_peak_rejects_bad_arguments_on_the_host(lib):
    """vl_fma_peak refuses a precision other than 32 or 64, missing pointers
    and a misaligned sink before any device work (no GPU needed)."""
    import ctypes
    out = ctypes.c_double(-1.0)
    sink = ctypes.c_void_p(4096)
    assert lib.vl_fma_peak(48, ctypes.byref(out), sink, None) == abi.VL_EINVAL
    assert b"precision" in lib.vl_last_error(None)
    assert lib.vl_fma_peak(32, None, sink, None) == abi.VL_EINVAL
    assert lib.vl_fma_peak(64, ctypes.byref(out), None, None) == abi.VL_EINVAL
    assert lib.vl_fma_peak(32, ctypes.byref(out), ctypes.c_void_p(4100), None) == abi.VL_EINVAL
    assert b"aligned" in lib.vl_last_error(None)
