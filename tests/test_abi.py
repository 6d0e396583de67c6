"""The C ABI library builds, loads and exports every entry point declared in
include/*.h; host-side argument and configuration checks run without a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_7808_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sr_fmg_create", "sr_fmg_solve", "sr_fmg_destroy", "sr_fmg_solve_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_1406_7808_gb300 import srfmg
    src = open(srfmg.__file__).read()
    missing = [n for n in declared_functions() if n not in src]
    assert not missing, missing


def test_config_struct_layout(lib):
    from paper_1406_7808_gb300 import srfmg
    c = srfmg.Config()
    lib.sr_fmg_default_config(ctypes.byref(c), 64)
    assert (c.n, c.seg, c.K, c.alpha, c.nu1, c.nu2) == (64, 0, 0, 1, 2, 2)
    assert abs(c.cheb_lo - 1.0 / 6.0) < 1e-15 and c.cheb_hi == 1.0
    assert (c.A, c.B, c.use_J, c.precision) == (8, 0, 0, 0)


def _create(lib, **kw):
    from paper_1406_7808_gb300 import srfmg
    c = srfmg.Config()
    lib.sr_fmg_default_config(ctypes.byref(c), kw.pop("n"))
    for k, v in kw.items():
        if k == "J":
            c.use_J = 1
            for i, x in enumerate(v):
                c.J[i] = x
        elif k == "len":
            for i, x in enumerate(v):
                c.len[i] = x
        else:
            setattr(c, k, v)
    h = ctypes.c_void_p()
    lib.sr_fmg_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(srfmg.Config)]
    st = lib.sr_fmg_create(ctypes.byref(h), ctypes.byref(c))
    return st, h


@pytest.mark.parametrize("kw,expected", [
    (dict(n=20), -2),                                   # 20 -> 10 -> 5 never reaches 2 or 3
    (dict(n=64, n_coarse=5), -2),
    (dict(n=64, n_coarse=32), -2),                      # coarsest grid larger than supported
    (dict(n=1024, len=(2, 1, 1)), -2),                  # 2^31 cells: beyond 32-bit cell indices
    (dict(n=64, n_coarse=16, len=(4, 1, 1)), -2),       # 64 x 16 x 16 coarsest cells: too many
    (dict(n=64, seg=24, K=2), -1),                      # seg does not divide n
    (dict(n=64, seg=16, K=5), -1),                      # seg not divisible by 2^K
    (dict(n=64, seg=16, K=2, J=[4, 3]), -1),            # odd buffer
    (dict(n=64, seg=16, K=2, J=[2, 8]), -1),            # J_1 < J_2 / 2
    (dict(n=64, alpha=-1), -1),
    (dict(n=64, cheb_lo=0.5, cheb_hi=0.4), -1),
    (dict(n=64, precision=7), -1),
])
def test_invalid_configurations_rejected_on_host(lib, kw, expected):
    st, h = _create(lib, **kw)
    assert st == expected
    assert not h.value


def test_null_arguments(lib):
    lib.sr_fmg_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.sr_fmg_create(None, None) == -1
    lib.sr_fmg_solve.argtypes = [ctypes.c_void_p] * 4
    assert lib.sr_fmg_solve(None, None, None, None) == -1
    lib.sr_fmg_destroy.argtypes = [ctypes.c_void_p]
    assert lib.sr_fmg_destroy(None) == 0


def test_status_strings(lib):
    lib.sr_fmg_status_string.restype = ctypes.c_char_p
    assert lib.sr_fmg_status_string(0) == b"ok"
    assert b"not finite" in lib.sr_fmg_status_string(-6)
    assert lib.sr_fmg_status_string(-99) == b"unknown status"


def test_buffer_schedule_matches_oracle(oracle_mod):
    from paper_1406_7808_gb300 import srfmg
    for A, B, K in [(4, 1, 3), (8, 0, 5), (2, 3, 4), (7, 2, 6)]:
        assert srfmg.buffer_schedule(A, B, K) == oracle_mod.buffer_schedule(A, B, K)
