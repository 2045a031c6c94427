"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every function include/sor.h declares; the
ctypes structures match the C layout; argument checking fails cleanly."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1401_0763_gb300 import _build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sor.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return capi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sor_[a-z_0-9]+)\s*\(", text)) - {"sor_alloc_fn", "sor_free_fn"})


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert "sor_solve" in names and "sor_batch_submit" in names and "sor_poll" in names
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (sor_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    assert set(capi.EXPORTED) == set(names)


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sor.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(sor_params), sizeof(sor_result), sizeof(sor_stats),'
                   ' offsetof(sor_params, omega), offsetof(sor_result, final_maxdelta)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(capi.sor_params), ctypes.sizeof(capi.sor_result), ctypes.sizeof(capi.sor_stats),
            capi.sor_params.omega.offset, capi.sor_result.final_maxdelta.offset]
    assert [int(x) for x in got] == want


def test_status_strings_and_omega(lib):
    assert capi.status_string(capi.SOR_OK) == "ok"
    assert capi.status_string(capi.SOR_ERR_BUDGET).startswith("over")
    assert capi.sor_omega_opt(256) == pytest.approx(1.9758476503, abs=1e-10)
    assert capi.sor_omega_opt(4096) == pytest.approx(1.9984675689, abs=1e-10)
    assert capi.sor_omega_opt(0) == 0.0


def test_null_arguments_rejected_without_device(lib):
    P = ctypes.POINTER
    assert lib.sor_create(None, 0, 0, None, capi._alloc_fn(), capi._free_fn(), None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_solve(None, None, None, None, None, None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_solve3d(None, None, None, None, None, None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_solve9(None, None, None, None, None, None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_diag_flow_wait(None, 10, 0, None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_diag_fp64_rate(None, 0, None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_destroy(None) == capi.SOR_ERR_INVALID_ARG
    assert lib.sor_poll(None, 1, None) == capi.SOR_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    st = lib.sor_create(ctypes.byref(h), 0, 0, None, capi._alloc_fn(), capi._free_fn(), None)
    import torch
    if not torch.cuda.is_available():
        assert st in (capi.SOR_ERR_CUDA, capi.SOR_ERR_INVALID_ARG) and not h.value
    else:
        assert st == capi.SOR_OK
        lib.sor_destroy(h)
    del P


def test_debug_build_exports_the_same_symbols():
    """The debug variant (device-side index checks) builds for sm_103a and
    exports every function the header declares."""
    lib = _build.build(debug=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (sor_\w+)", out))
    assert set(declared_functions()) <= exported
