"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/pd.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^PD_API\s+(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, re.M)
    return names


def test_library_exports_every_declared_symbol(built_lib):
    names = _declared()
    assert "pd_step" in names and "mlmc_estimate" in names and len(names) >= 20
    L = ctypes.CDLL(built_lib.lib_path())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(built_lib):
    assert set(_declared()) <= set(built_lib._SIGS)


def test_version_string(built_lib):
    assert b"sm_103a" in built_lib.lib().pd_version()


def test_argument_errors_need_no_gpu(built_lib):
    """Host-side validation rejects bad arguments before any CUDA call."""
    L = built_lib.lib()
    g = built_lib.Grid(0, 1, 1, 1e-3, 3.01, 0, 0, 0)
    nb = ctypes.c_int64(0)
    assert L.pd_build_neighbours(ctypes.byref(g), None, None, 0, ctypes.byref(nb), None) == built_lib.PD_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    L.pd_last_error(buf, 256)
    assert b"positive" in buf.value
    V = (ctypes.c_double * 2)(1.0, 1.0)
    Cst = (ctypes.c_double * 2)(1.0, 4.0)
    N = (ctypes.c_int64 * 2)()
    assert L.pd_mlmc_allocation(2, V, Cst, ctypes.c_double(0.125), N) == 0
    # N_l = floor(eps^-2 (sum sqrt(V C)) sqrt(V/C)) = floor(64 * 3 * [1, 0.5])
    assert list(N) == [192, 96]
