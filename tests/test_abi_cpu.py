"""The C ABI library builds, loads without a GPU and exports every declared symbol."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "atsfft.h")).read()
    return sorted(set(re.findall(r"\b(atsfft_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_02461_gb300 import build

    return ctypes.CDLL(build())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "atsfft_exec" in names and "atsfft_plan" in names and "atsfft_exec_2d" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_1908_02461_gb300._lib as L

    assert sorted(L.EXPORTED) == _declared()


def test_host_only_calls(lib):
    import paper_1908_02461_gb300 as A

    p = A.atsfft_default_params()
    assert p.delta1 == 0.02 and p.delta2 == 0.05 and p.eps1 == 0.5 and p.eps2 == 1.0
    assert p.loops_loc == 7 and p.loops_est == 7 and p.tie_eta == 0.01
    assert A.atsfft_status_string(0) == "ok"
    assert "capacity" in A.atsfft_status_string(6)
    # argument checks happen before any device call
    st, h = A.atsfft_plan(1, (1000,), 0, None, 0)
    assert st == A.E_INVALID_ARG and h is None
    st, h = A.atsfft_plan(3, (1024,), 0, None, 0)
    assert st == A.E_INVALID_ARG
    bad = A.params(eps1=0.25)
    st, h = A.atsfft_plan(1, (1 << 14,), 0, bad, 0)
    assert st == A.E_INVALID_ARG
    assert A.atsfft_exec(None, 0, 0, 0, 0, 0, 0, 0, None) == A.E_INVALID_ARG


def test_product_package_never_imports_oracle():
    """The product path shares no code with the oracle and never loads it."""
    pkg = os.path.join(ROOT, "paper_1908_02461_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "atsfft_oracle", "orc_"):
                    assert bad not in txt, (f, bad)


def _prototypes():
    """name -> list of parameter declarations, from the header's function prototypes."""
    txt = open(os.path.join(ROOT, "include", "atsfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)   # comments out
    protos = {}
    for m in re.finditer(r"\b(atsfft_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
        params = [p.strip() for p in m.group(2).split(",")]
        protos[m.group(1)] = [] if params == ["void"] else params
    return protos


def _ctype_class(decl):
    """The ctypes argument class a C parameter declaration needs."""
    if "*" in decl or re.match(r"(const\s+)?atsfft_(plan|batch)_t\b", decl):
        return "pointer"
    if re.match(r"(const\s+)?uint64_t\b", decl):
        return "u64"
    if re.match(r"(const\s+)?int64_t\b", decl):
        return "i64"
    if re.match(r"(const\s+)?(int|int32_t|atsfft_status)\b", decl):
        return "i32"
    raise AssertionError(f"unclassified parameter {decl!r}")


def test_binding_argument_lists_match_the_prototypes():
    """Every ctypes argtypes list has the prototype's length and, position by position,
    the same kind of argument (pointer, 32-bit int, signed or unsigned 64-bit int): a
    mismatch would hand the library garbage without any error."""
    import ctypes as C

    import paper_1908_02461_gb300._lib as L

    lib = L.load()
    protos = _prototypes()
    assert set(protos) == set(L.EXPORTED)
    kinds = {C.c_void_p: "pointer", C.c_char_p: "pointer", C.c_int64: "i64",
             C.c_uint64: "u64", C.c_int: "i32", C.c_int32: "i32"}
    for name, params in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, name
        assert len(argtypes) == len(params), (name, len(argtypes), len(params))
        for a, decl in zip(argtypes, params):
            got = "pointer" if hasattr(a, "_type_") and issubclass(a, C._Pointer) else kinds.get(a)
            assert got == _ctype_class(decl), (name, decl, a)


def test_binding_return_types_match_the_prototypes():
    import ctypes as C

    import paper_1908_02461_gb300._lib as L

    lib = L.load()
    txt = re.sub(r"/\*.*?\*/", " ", open(os.path.join(ROOT, "include", "atsfft.h")).read(),
                 flags=re.S)
    want = {"atsfft_status": C.c_int, "void": None, "const char *": C.c_char_p}
    found = re.findall(r"^(atsfft_status|void|const char \*)\s*(atsfft_[a-z0-9_]+)\s*\(", txt,
                       flags=re.M)
    assert {nm for _, nm in found} == set(L.EXPORTED)
    for ret, name in found:
        assert getattr(lib, name).restype is want[ret], (name, ret)
