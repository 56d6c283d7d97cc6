"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/godec.h declares (no compute calls here)."""
import ctypes

import paper_1309_0302_gb300 as g


def test_library_exports_header_symbols():
    lib = g.library()
    syms = g.header_symbols()
    assert "godec_init" in syms and "godec_iterate" in syms and "godec_solve" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert missing == []


def test_status_strings_and_bad_args_without_gpu():
    lib = g.library()
    assert lib.godec_status_string(0) == b"ok"
    assert lib.godec_status_string(4) == b"non-finite values"
    # argument validation runs before any CUDA call
    h = ctypes.c_void_p()
    p = g._binding.GodecParams(m=10, n=10, ldx=12, r=0, q=0, k=5, tol=1e-7, max_iter=5)
    assert lib.godec_init(ctypes.byref(h), ctypes.byref(p), None, None, None) == 1
    assert b"r must satisfy" in lib.godec_last_error(None)
    p = g._binding.GodecParams(m=10, n=10, ldx=10, r=2, q=0, k=5, tol=1e-7, max_iter=5)
    assert lib.godec_init(ctypes.byref(h), ctypes.byref(p), None, None, None) == 1   # ldx*4 % 16
    assert h.value is None
