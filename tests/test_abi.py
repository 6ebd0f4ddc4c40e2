"""The C-ABI library builds, loads and exports every symbol of include/trg.h.

CPU only: no compute call is made; host-side logic (status strings, config
defaults, argument rejection without a GPU) is checked.
"""
import ctypes
import os
import re

import pytest

from paper_2306_00358_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "trg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trg_[a-z_0-9]+)\s*\(", text)) - {"trg_alloc_fn", "trg_free_fn"})


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = _lib.load()
    assert lib is not None


def test_every_declared_symbol_is_exported_and_bound():
    lib = _lib.load()
    declared = _declared_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in trg.h but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no binding"


def test_header_declares_all_bound_symbols():
    declared = set(_declared_symbols())
    assert set(_lib.SIGNATURES) <= declared


def test_status_strings_and_defaults():
    lib = _lib.load()
    assert lib.trg_status_string(0) == b"ok"
    assert lib.trg_status_string(4) == b"numerical failure"
    assert lib.trg_status_string(99) == b"unknown status"
    cfg = _lib.trg_config()
    assert lib.trg_config_default(ctypes.byref(cfg)) == 0
    assert cfg.precision == _lib.TRG_FP64
    assert cfg.split_slices == 4
    assert cfg.oversample == 24
    assert cfg.eig_tol == 1e-12
    # the fields after the first ones land where the C struct has them
    assert (cfg.mma_pairs, cfg.fused_slices, cfg.fp64_max_dd, cfg.env_slices, cfg.autotune) == (1, 1, 16, 0, 1)
    assert cfg.split_from_step == 0 and cfg.workspace_bytes == 0
    assert lib.trg_config_default(None) == _lib.TRG_EINVAL


def test_null_context_is_rejected():
    lib = _lib.load()
    assert lib.trg_coarse_grain(None, 16, 1) == _lib.TRG_EINVAL
    assert lib.trg_init_tensor(None, 0, 0.44, 0.0, 2) == _lib.TRG_EINVAL
    assert lib.trg_destroy(None) == _lib.TRG_OK
    assert lib.trg_launch_count(None) == 0


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.trg_create(ctypes.byref(h), 0, None)
    assert st != _lib.TRG_OK
    assert not h.value
