"""CPU checks of the C-ABI library: it builds, loads and exports every entry point
that include/dae.h declares; calls that need no GPU behave."""
import ctypes
import os
import re

import pytest

from paper_2102_11026_gb300 import dae

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dae_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = dae.lib()
    syms = declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in sorted(syms) if not hasattr(L, s)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert not [s for s in syms if not hasattr(dae, s)]


def test_version_and_status_strings():
    assert dae.dae_version() >= 10000
    assert dae.dae_status_string(0) == "DAE_OK"
    assert dae.dae_status_string(-7) == "DAE_ERR_INVERTED"


def test_default_newton_opts():
    o = dae.dae_default_newton_opts()
    assert o.max_iter == 5 and o.max_halvings == 8
    assert o.h_cs == 2.0 ** -20 and o.tol == 1e-8


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(dae.DaeError) as e:
        dae.dae_create(0)
    assert e.value.status == -2


def test_null_arguments_are_rejected():
    L = dae.lib()
    assert L.dae_destroy(None) == -1
    assert L.dae_free_decoder(None) == -1
    assert L.dae_free_mesh(None) == -1
    assert L.dae_sync(None) == -1


def test_every_entry_point_rejects_null_handles():
    """Every call that takes a context, decoder, mesh or trainer handle returns
    DAE_ERR_INVALID_ARG for NULL handles and NULL arrays (no dereference, no GPU)."""
    import ctypes
    L = dae.lib()
    skip = {"dae_version", "dae_status_string", "dae_default_newton_opts", "dae_last_error"}
    ints = (ctypes.c_int, ctypes.c_uint, ctypes.c_long, ctypes.c_longlong, ctypes.c_size_t)
    checked = 0
    for name, (argtypes, _) in dae.SIGNATURES.items():
        if name in skip:
            continue
        vals = [0 if a in ints else 0.0 if a in (ctypes.c_double, ctypes.c_float) else None
                for a in argtypes]
        assert getattr(L, name)(*vals) == -1, name
        checked += 1
    assert checked >= 25
    assert L.dae_last_error(None) == b"null context"


# ----------------------------------------------------------------------------
# The binding's ctypes signatures and structures against the header's prototypes:
# a parameter count, an operand kind or a field out of step would pass arguments or
# read reports wrongly without any error, so both are read from include/dae.h.

def _header_source():
    src = open(os.path.join(ROOT, "include", "dae.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


_SCALARS = {"int": ctypes.c_int, "dae_status": ctypes.c_int, "dae_prec": ctypes.c_int,
            "dae_act": ctypes.c_int, "dae_material": ctypes.c_int, "unsigned": ctypes.c_uint,
            "double": ctypes.c_double, "float": ctypes.c_float, "long long": ctypes.c_longlong,
            "size_t": ctypes.c_size_t}


def _c_type(decl):
    """Type part of a parameter declaration 'const float* const* W' -> 'const float* const*'."""
    decl = " ".join(decl.split())
    m = re.match(r"^(.*?)\s*\b([A-Za-z_]\w*)$", decl)
    t = m.group(1) if m and m.group(1) else decl
    return t


def _is_pointer_ctype(t):
    return (t in (ctypes.c_void_p, ctypes.c_char_p) or
            (isinstance(t, type) and issubclass(t, ctypes._Pointer)))


def _same_scalar(t, expected):
    floats = (ctypes.c_float, ctypes.c_double)
    return (ctypes.sizeof(t) == ctypes.sizeof(expected) and
            (t in floats) == (expected in floats))


def header_prototypes():
    out = {}
    for ret, name, params in re.findall(
            r"([A-Za-z_][\w \*]*?)\b(dae_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", _header_source(), flags=re.S):
        p = params.strip()
        out[name] = (" ".join(ret.split()), [] if p in ("", "void") else
                     [_c_type(x) for x in p.split(",")])
    return out


def test_binding_signatures_match_the_header():
    protos = header_prototypes()
    assert len(protos) >= 30
    assert set(protos) == set(dae.SIGNATURES), set(protos) ^ set(dae.SIGNATURES)
    for name, (ret, params) in protos.items():
        args, res = dae.SIGNATURES[name]
        assert len(args) == len(params), (name, params, args)
        for i, (ct, a) in enumerate(zip(params, args)):
            if "*" in ct:
                assert _is_pointer_ctype(a), (name, i, ct, a)
            else:
                base = " ".join(w for w in ct.split() if w != "const")
                assert base in _SCALARS, (name, i, ct)
                assert not _is_pointer_ctype(a) and _same_scalar(a, _SCALARS[base]), (name, i, ct, a)
        if ret == "void":
            assert res is None, name
        elif "*" in ret:
            assert res is ctypes.c_char_p, (name, ret, res)
        else:
            assert res is not None and _same_scalar(res, _SCALARS[ret]), (name, ret, res)


def header_structs():
    out = {}
    for body, name in re.findall(r"typedef struct\s*\w*\s*\{(.*?)\}\s*(\w+)\s*;", _header_source(),
                                 flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if decl:
                t = _c_type(decl)
                fields.append((decl[len(t):].strip(), t))
        out[name] = fields
    return out


def test_binding_structs_match_the_header():
    structs = header_structs()
    mirrors = {"dae_newton_opts": dae.dae_newton_opts, "dae_newton_report": dae.dae_newton_report,
               "dae_system": dae.dae_system}
    assert set(mirrors) <= set(structs), set(structs)
    for name, cls in mirrors.items():
        fields = structs[name]
        assert [f for f, _ in fields] == [f for f, _ in cls._fields_], name
        for (fname, ct), (_, t) in zip(fields, cls._fields_):
            if "*" in ct:
                assert _is_pointer_ctype(t), (name, fname, ct, t)
            else:
                base = " ".join(w for w in ct.split() if w != "const")
                assert _same_scalar(t, _SCALARS[base]), (name, fname, ct, t)
