"""The C-ABI library builds, loads and exports every function include/xdrop.h declares;
host-side argument handling that needs no GPU."""
import ctypes

import numpy as np
import pytest

from paper_2304_08662_gb300 import xdrop


def test_header_declares_the_boundary():
    names = xdrop.header_symbols()
    for required in ("xd_create", "xd_submit_batch", "xd_poll", "xd_destroy", "xd_last_error",
                     "xd_run_device", "xd_reserve", "xd_device_status", "xd_get_stats", "xd_version",
                     "xd_autotune"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = xdrop.lib()
    for name in xdrop.header_symbols():
        assert hasattr(L, name), name


def _exported_xd_symbols(path):
    """Global function names starting with xd_ that the library's dynamic symbol table
    defines (nm -D on this project's own build)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    names = set()
    for ln in out.splitlines():
        parts = ln.split()
        if len(parts) == 3 and parts[1] == "T" and parts[2].startswith("xd_"):
            names.add(parts[2])
    return names


def test_every_exported_symbol_is_declared():
    from paper_2304_08662_gb300 import build
    exported = _exported_xd_symbols(build.build())
    assert exported, "no xd_ symbols exported"
    missing = sorted(exported - set(xdrop.header_symbols()))
    assert not missing, f"exported but not declared in include/xdrop.h: {missing}"


def test_struct_layouts_match_header():
    assert ctypes.sizeof(xdrop.xd_batch) == 96
    assert xdrop.RESULT_DTYPE.itemsize == 56
    assert xdrop.SIDE_DTYPE.itemsize == 24
    assert xdrop.PAIR_DTYPE.itemsize == 20


def test_version_and_null_arguments():
    assert "sm_103a" in xdrop.xd_version()
    L = xdrop.lib()
    assert L.xd_create(None, None) == xdrop.XD_EINVAL
    assert L.xd_poll(None, 1, None, 0) == xdrop.XD_EINVAL
    assert L.xd_destroy(None) == xdrop.XD_EINVAL


def test_create_without_gpu_reports_edevice():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(xdrop.XdError) as e:
        xdrop.xd_create(0)
    assert e.value.status == xdrop.XD_EDEVICE
