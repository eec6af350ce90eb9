"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and exports every
function include/kpdhg.h declares; the ctypes structs match the header's layout."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kpdhg.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1902_09657_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("kp_plan_create", "kp_plan_set_trajectory", "kp_plan_set_maps", "kp_make_preconditioner",
               "kp_sense_forward", "kp_sense_adjoint", "kp_max_eig", "kp_pdhg_solve", "kp_plan_destroy"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.kp_status_string(0) == b"KP_OK"
    assert lib.kp_status_string(1) == b"KP_EINVAL"


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1902_09657_gb300 import _lib
    assert lib.kp_plan_create(None, None, None) == _lib.KP_EINVAL
    assert lib.kp_plan_destroy(None) == _lib.KP_OK
    assert lib.kp_sense_forward(None, None, None, 0, None) == _lib.KP_EINVAL
    prm = _lib.KpParams()
    prm.ndim = 4
    h = ctypes.c_void_p()
    assert lib.kp_plan_create(ctypes.byref(h), ctypes.byref(prm), None) == _lib.KP_EINVAL
    assert b"ndim" in lib.kp_last_error()


def test_struct_layout_matches_header():
    from paper_1902_09657_gb300 import _lib
    # kp_params: int, (pad), int64[3], int, (pad), int64, float, int, int, (pad) -> 64 bytes
    assert ctypes.sizeof(_lib.KpParams) == 64
    assert _lib.KpParams.nsamples.offset == 40
    assert ctypes.sizeof(_lib.KpStats) == 8 + 5 * 8 + 12 * 8


def test_sources_use_blackwell_target():
    from paper_1902_09657_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_release_bounds_report_without_gpu(lib):
    """The release build has no bounds checks: its report is empty and touches no device."""
    from paper_1902_09657_gb300 import _lib
    ck, n, site, idx = ctypes.c_int(7), ctypes.c_uint32(7), ctypes.c_uint32(7), ctypes.c_int64(7)
    assert lib.kp_bounds_report(ctypes.byref(ck), ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx)) == _lib.KP_OK
    assert (ck.value, n.value, site.value, idx.value) == (0, 0, 0, 0)
    assert lib.kp_bounds_report(None, None, None, None) == _lib.KP_OK


def test_checked_build_flag_and_library_choice():
    """`_build --checked` compiles with -DKP_CHECKED into its own library and object folder;
    KPDHG_CHECKED=1 makes the binding load that library."""
    import subprocess
    import sys
    from paper_1902_09657_gb300 import _build
    assert _build.LIB_CHECKED != _build.LIB and _build.BUILD_CHECKED != _build.BUILD
    code = "from paper_1902_09657_gb300 import _lib; print(_lib.LIB_PATH)"
    env = dict(__import__("os").environ, KPDHG_CHECKED="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True).stdout
    assert out.strip().endswith("libkpdhg_checked.so")


def test_checked_build_compiles_and_exports_the_same_symbols():
    """The bounds-checked variant (-DKP_CHECKED) builds for sm_103a without a GPU and exports
    every symbol the header declares (the checks only add code inside the kernels)."""
    from paper_1902_09657_gb300 import _build
    path = _build.build(checked=True)
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
