"""The C-ABI library builds, loads without a GPU, and exports every function include/pocketgs.h
declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pgs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["pgs_create", "pgs_destroy", "pgs_render", "pgs_backward", "pgs_step",
                 "pgs_status", "pgs_strerror"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2601_17354_gb300 import _lib
    L = _lib.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.EXPORTED) <= set(declared_functions())


def test_error_strings_without_a_gpu():
    from paper_2601_17354_gb300 import _lib
    L = _lib.lib()
    assert L.pgs_strerror(_lib.PGS_ERR_CAPACITY).decode().startswith("more")
    assert L.pgs_strerror(12345).decode() == "unknown error"


def test_invalid_arguments_are_rejected_on_the_host():
    from paper_2601_17354_gb300 import _lib
    L = _lib.lib()
    out = ctypes.c_void_p(123)
    for tile in (12, 64, 0):  # tile edges other than 8, 16, 32 are refused before any CUDA call
        cfg = _lib.PgsConfig(tile, 0, 0, 0.9, 0.999, 1e-15, (ctypes.c_float * 6)(*[1e-3] * 6))
        assert L.pgs_create(ctypes.byref(out), ctypes.byref(cfg), None) == _lib.PGS_ERR_INVALID_ARG
    assert out.value is None
    assert L.pgs_render(None, None, None, None) == _lib.PGS_ERR_INVALID_ARG
    assert L.pgs_status(None, None) == _lib.PGS_ERR_INVALID_ARG
    L.pgs_destroy(None)


def declared_arity():
    """Number of parameters of every function include/pocketgs.h declares."""
    arity = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
            for m in re.finditer(r"\b(pgs_[a-z0-9_]+)\s*\(([^;{)]*)\)\s*;", src):
                params = " ".join(m.group(2).split())
                arity[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return arity


def test_binding_signatures_match_the_header():
    """The ctypes binding marshals every declared function with as many arguments as the header
    gives it (a drifted signature would pass garbage through the ABI)."""
    from paper_2601_17354_gb300 import _lib
    L = _lib.lib()
    arity = declared_arity()
    assert set(arity) == set(declared_functions())
    wrong = {n: (k, len(getattr(L, n).argtypes or ())) for n, k in arity.items()
             if getattr(L, n).argtypes is None or len(getattr(L, n).argtypes) != k}
    assert not wrong, wrong
