"""The C-ABI library builds, loads and exports what include/percol.h declares;
host-side argument validation works without a GPU (no compute call)."""
from __future__ import annotations

import os
import re
import subprocess

import pytest

import paper_1401_2130_gb300 as pc
from paper_1401_2130_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "percol.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return pc.load()


def declared_symbols() -> set[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(pc_[a-z_0-9]+)\s*\(", text))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for need in ("pc_lattice_info", "pc_occupancy", "pc_inspect", "pc_inspect_occupancy",
                 "pc_shutdown", "pc_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pc.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pc_[a-z_0-9]+)\b", out))
    missing = declared_symbols() - exported
    assert not missing, missing
    for name in declared_symbols():
        assert hasattr(lib, name)
    # the binding covers the same names
    assert declared_symbols() <= set(pc.SIGNATURES)


def test_lattice_info(lib):
    assert pc.pc_lattice_info(0, 1) == (1, 1)
    assert pc.pc_lattice_info(4, 16) == (61, 976)
    assert pc.pc_lattice_info(8, 64) == (217, 13888)
    assert pc.pc_lattice_info(64, 4096) == (12481, 51122176)
    assert pc.pc_lattice_info(46, 400)[1] == 2_594_800


@pytest.mark.parametrize("W,L", [(-1, 4), (256, 4), (4, 0), (4, 1 << 24)])
def test_lattice_argument_errors(lib, W, L):
    with pytest.raises(pc.PercolError) as e:
        pc.pc_lattice_info(W, L)
    assert e.value.status == pc.PC_ERR_ARG


def test_inspect_argument_errors_without_gpu(lib):
    import ctypes
    v = (ctypes.c_uint8 * 4)()
    bad = [
        dict(W=4, L=16, p=-0.1, b=0, n=4),
        dict(W=4, L=16, p=1.5, b=0, n=4),
        dict(W=4, L=16, p=float("nan"), b=0, n=4),
        dict(W=4, L=16, p=0.2, b=-1, n=4),
        dict(W=4, L=16, p=0.2, b=0, n=-4),
        dict(W=4, L=16, p=0.2, b=2**32 - 2, n=4),
        dict(W=-3, L=16, p=0.2, b=0, n=4),
    ]
    for a in bad:
        st = lib.pc_inspect(a["W"], a["L"], a["p"], 1, a["b"], a["n"], ctypes.addressof(v),
                            None, None, None, None, None, 0, None)
        assert st == pc.PC_ERR_ARG, a
        assert lib.pc_last_error()
    # NULL verdicts with n > 0, and Pi with device outputs
    assert lib.pc_inspect(4, 16, 0.2, 1, 0, 4, None, None, None, None, None, None, 0, None) \
        == pc.PC_ERR_ARG
    pi = ctypes.c_double()
    assert lib.pc_inspect(4, 16, 0.2, 1, 0, 4, ctypes.addressof(v), None, None, None, None,
                          ctypes.addressof(pi), pc.PC_OUT_DEVICE, None) == pc.PC_ERR_ARG
    # both solvers forced, and flag bits the call does not define
    for flags in (pc.PC_MODE_RESIDENT | pc.PC_MODE_STREAM, pc.PC_ASYNC, 0x4, 0x100, 1 << 30):
        assert lib.pc_inspect(4, 16, 0.2, 1, 0, 4, ctypes.addressof(v), None, None, None, None,
                              None, flags, None) == pc.PC_ERR_ARG, flags
        assert lib.pc_inspect_occupancy(4, 16, ctypes.addressof(v), 4, ctypes.addressof(v), None,
                                        None, None, None, None, flags, None) == pc.PC_ERR_ARG, flags


def test_lazy_mass_argument_errors_without_gpu(lib):
    import ctypes
    fh = (ctypes.c_int32 * 4)()
    m = (ctypes.c_float * 4)()
    o = (ctypes.c_float * 4)()
    a = [ctypes.addressof(fh), ctypes.addressof(m)]
    for hold in (-0.1, 1.0, 1.5, float("nan")):
        assert lib.pc_lazy_mass(*a, 4, hold, ctypes.addressof(o), 0, None) == pc.PC_ERR_ARG, hold
    assert lib.pc_lazy_mass(*a, -1, 0.5, ctypes.addressof(o), 0, None) == pc.PC_ERR_ARG
    assert lib.pc_lazy_mass(None, a[1], 4, 0.5, ctypes.addressof(o), 0, None) == pc.PC_ERR_ARG
    assert lib.pc_lazy_mass(*a, 4, 0.5, None, 0, None) == pc.PC_ERR_ARG
    assert lib.pc_lazy_mass(*a, 4, 0.5, ctypes.addressof(o), pc.PC_BITS_ONLY, None) == pc.PC_ERR_ARG
    assert lib.pc_lazy_mass(None, None, 0, 0.5, None, 0, None) == pc.PC_OK  # nothing to do


def test_batch_argument_errors_without_gpu(lib):
    import ctypes
    v = (ctypes.c_uint8 * 4)()
    good = pc.PcQuery(W=4, L=16, p=0.2, seed=1, config_begin=0, n_configs=4,
                      verdicts=ctypes.addressof(v))
    for flags in (pc.PC_MODE_STREAM, 0x4, 1 << 30):
        assert lib.pc_batch_run(ctypes.addressof(good), 1, None, flags, None) == pc.PC_ERR_ARG, flags
    # PC_ASYNC needs device outputs and no host summaries
    assert lib.pc_batch_run(ctypes.addressof(good), 1, None, pc.PC_ASYNC, None) == pc.PC_ERR_ARG
    for q in (dict(W=256), dict(L=0), dict(p=1.01), dict(n_configs=-1), dict(config_begin=2**32),
              dict(verdicts=None)):
        bad = pc.PcQuery(**{**dict(W=4, L=16, p=0.2, seed=1, config_begin=0, n_configs=4,
                                   verdicts=ctypes.addressof(v)), **q})
        assert lib.pc_batch_run(ctypes.addressof(bad), 1, None, 0, None) == pc.PC_ERR_ARG, q
    assert lib.pc_batch_run(None, 3, None, 0, None) == pc.PC_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    import importlib
    mod = importlib.import_module("paper_1401_2130_gb300")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(ImportError):
            mod.load(str(tmp_path / "nope.so"))
    finally:
        mod._lib = saved


def test_binding_constants_equal_the_header():
    """Every PC_* flag and status the header defines has the same value in
    the Python binding (the binding only marshals: a drifted constant would
    send the wrong flag through the ABI)."""
    import re
    text = open(os.path.join(ROOT, "include", "percol.h")).read()
    defs = dict(re.findall(r"#define (PC_[A-Z0-9_]+) \(?(-?(?:0x[0-9a-fA-F]+|\d+))\)?", text))
    assert {"PC_OK", "PC_ERR_ARG", "PC_OUT_DEVICE", "PC_MODE_STREAM", "PC_BITS_ONLY", "PC_VERDICT_FIRST",
            "PC_ASYNC"} <= set(defs)
    for name, value in defs.items():
        if hasattr(pc, name):
            assert getattr(pc, name) == int(value, 0), name
