"""The C ABI library: builds for sm_103a, loads, exports every entry point
declared in include/tgp.h, and rejects bad arguments on the host before any
device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2501_17168_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tgp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tgp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tgp_eval_forward", "tgp_fitness_mse", "tgp_validate", "tgp_workspace_size",
              "tgp_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_declares_every_header_symbol():
    assert set(_declared()) <= set(_lib.declared_symbols())


def test_status_strings(lib):
    assert lib.tgp_status_string(0) == b"TGP_OK"
    assert lib.tgp_status_string(3) == b"TGP_ERR_WORKSPACE"
    assert b"sm_103a" in lib.tgp_version()


def test_host_argument_checks_need_no_device(lib):
    P = ctypes.POINTER
    pop = _lib.tgp_population(None, None, None, 4, 8, 8)      # null arrays with pop > 0
    data = _lib.tgp_data(None, 0, 1, 1)
    assert lib.tgp_fitness_mse(ctypes.byref(pop), ctypes.byref(data), None, 1, None, None, None, 0,
                               None) == _lib.TGP_ERR_INVALID_ARG
    pop = _lib.tgp_population(None, None, None, 0, 2000, 2000)  # max_len beyond the limit
    assert lib.tgp_eval_forward(ctypes.byref(pop), ctypes.byref(data), 1, None, None, None, 0,
                                None) == _lib.TGP_ERR_INVALID_ARG
    pop = _lib.tgp_population(None, None, None, 0, 8, 4)        # ld < max_len
    assert lib.tgp_workspace_size(ctypes.byref(pop), None, 1, None) == 0
    pop = _lib.tgp_population(None, None, None, 0, 8, 8)
    assert lib.tgp_validate(ctypes.byref(pop), 0, 1, None, None, 0, None) == _lib.TGP_ERR_INVALID_ARG
    assert lib.tgp_validate(ctypes.byref(pop), 1, 99, None, None, 0, None) == _lib.TGP_ERR_INVALID_ARG
