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
    # the two first-projection flags exclude each other
    p = g._binding.GodecParams(m=10, n=12, ldx=12, r=2, q=0, k=5, tol=1e-7, max_iter=5,
                               flags=g.FLAG_SPARSE_FIRST | g.FLAG_DENSE_FIRST)
    assert lib.godec_init(ctypes.byref(h), ctypes.byref(p), None, None, None) == 1
    assert b"exclude each other" in lib.godec_last_error(None)


def _header_arity():
    """Parameter count of every function prototype in include/godec.h."""
    import re
    txt = open(g._binding.HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(godec_\w+)\s*\(([^;{]*?)\)\s*;", txt):
        args = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes signature the binding declares has the header prototype's number of
    parameters (a drift would pass arguments in the wrong slots on the GPU)."""
    lib = g.library()
    arity = _header_arity()
    checked = 0
    for name in g.header_symbols():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue                       # not used by the binding
        assert len(f.argtypes) == arity[name], name
        checked += 1
    assert checked >= 20


def _header_struct(name):
    """(type, field) pairs of `typedef struct name { ... } name;` in include/godec.h."""
    import re
    txt = open(g._binding.HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), txt, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        typ, names = decl.split(" ", 1)
        out += [(typ, n.strip()) for n in names.split(",")]
    return out


def test_binding_structs_match_the_header():
    """GodecParams, GodecInfo and GrebsmoParams have the header's fields, in order, with the same widths
    (a drift would shift every later field)."""
    import ctypes as C
    width = {"int32_t": 4, "int64_t": 8, "double": 8}
    for hname, cls in (("godec_params", g._binding.GodecParams), ("godec_info", g._binding.GodecInfo),
                       ("godec_grebsmo_params", g._binding.GrebsmoParams)):
        fields = _header_struct(hname)
        assert [f for _, f in fields] == [f for f, _ in cls._fields_], hname
        assert [width[t] for t, _ in fields] == [C.sizeof(t) for _, t in cls._fields_], hname
