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
