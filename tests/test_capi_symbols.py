"""The C-ABI library builds for sm_103a, loads, and exports every entry point the header
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

from paper_2602_16797_gb300 import build as libbuild
from paper_2602_16797_gb300 import rlobpcg as rl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rlobpcg_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    assert os.path.exists(path)
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    d = _declared()
    for must in ["rlobpcg_plan", "rlobpcg_solve", "rlobpcg_plan_destroy", "rlobpcg_default_opts",
                 "rlobpcg_status_string", "rlobpcg_sketch", "rlobpcg_gram", "rlobpcg_factor", "rlobpcg_tsqr"]:
        assert must in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) <= set(rl.declared_symbols())


def test_host_only_calls(lib):
    rl.load()
    o = rl.rlobpcg_default_opts()
    assert o.zeta == 8 and o.use_stagnation == 1 and o.tau < 0 and o.sketch_prec == rl.RLOBPCG_SKETCH_F64
    assert rl.rlobpcg_status_string(rl.RLOBPCG_ERR_INVALID_ARG) == "invalid argument"
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert rl.load().rlobpcg_plan(ctypes.byref(h), 100, 10, 4, 0, None, None) == rl.RLOBPCG_ERR_INVALID_ARG  # 3b > n
    assert rl.load().rlobpcg_plan(ctypes.byref(h), 5, 10, 1, 0, None, None) == rl.RLOBPCG_ERR_INVALID_ARG    # n > m
    assert rl.load().rlobpcg_plan(ctypes.byref(h), 100, 10, 1, 7, None, None) == rl.RLOBPCG_ERR_INVALID_ARG  # dtype
    assert rl.load().rlobpcg_sketch(None, 10, 10, 10, 0, 8, 8, 0, 0, None, None) == rl.RLOBPCG_ERR_INVALID_ARG
    assert rl.load().rlobpcg_gram(None, 10, 10, 10, 0, None, 1, 1, None, 1, None, 1, None, 0, None) == rl.RLOBPCG_ERR_INVALID_ARG
    # the asynchronous solve's entry points check their arguments before starting a thread
    assert rl.load().rlobpcg_solve_wait(None) == rl.RLOBPCG_ERR_INVALID_ARG
    assert rl.load().rlobpcg_solve_async(None, None, 0, -1.0, None, None, None, None, None) == rl.RLOBPCG_ERR_INVALID_ARG
