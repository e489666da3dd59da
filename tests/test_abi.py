"""The C-ABI library loads and exports every entry point include/slm.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(slm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("slm_node_split", "slm_grow_level", "slm_train_tree", "slm_predict",
                     "slm_evaluate_swarm", "slm_create", "slm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2208_07023_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2208_07023_gb300 import binding
    L = binding.lib()
    for n in declared_functions():
        assert getattr(L, n).argtypes is not None, n


def test_status_strings_without_gpu():
    from paper_2208_07023_gb300 import binding
    L = binding.lib()
    assert L.slm_status_string(0) == b"ok"
    assert L.slm_status_string(1) == b"invalid argument"


def test_params_struct_layout_matches_header():
    from paper_2208_07023_gb300 import binding
    # int32 x 17 (+ padding to 8) then uint64 seed; the library asserts the
    # same size and offset at compile time
    assert ctypes.sizeof(binding.slm_params) == 17 * 4 + 4 + 8
    assert binding.slm_params.seed.offset == 72 and binding.slm_params.apso.offset == 64
    assert ctypes.sizeof(binding.slm_eval) == 56
    assert ctypes.sizeof(binding.slm_split) == 56 + 16
