"""The accuracy gate of the Ising coupling grid (beta_c, 0.40, 0.48 x h 0,
1e-3; 40 half-steps = 2^20 x 2^20 sites, the lattice of Sec. 3.2) at bond
dimensions 32, 48 and 64.

* Dcut 32: the GPU against the oracle (tests/golden/oracle_solves_dcut32.json,
  written by tests/golden/make_golden.py --dcut32 from the oracle alone):
  FP64 path |df| <= 1e-10 and kept spectra to 1e-9 lambda_1; split path
  |df| <= 1e-9.
* Dcut 48 and 64: the oracle's 2304^2 and 4096^2 Jacobi solves per half-step
  are out of reach of a test (hours), so the split path is held to the FP64
  GPU path on the same solve, |f_split - f_fp64| <= 1e-9; the FP64 path is
  itself pinned to the oracle at Dcut <= 32.  The Dcut-64 FP64 solve takes
  about four and a half minutes (marked slow).
* XY model (the O(2) case of Sec. 3.3, multiplet-preserving cuts) at
  beta 1.0 and 1.1, Dcut 32, 30 half-steps: the GPU against the oracle
  (tests/golden/oracle_solves_xy32.json, make_golden.py --xy32), the same
  bounds as the Ising grid; the split path only where the oracle's
  multiplet cuts are resolved at split precision (beta 1.1; at beta 1.0
  near-degenerate levels sit within 2^-20 of the threshold).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2306_00358_gb300 import Solver

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN32 = json.load(open(os.path.join(HERE, "golden", "oracle_solves_dcut32.json")))
GOLDEN_XY32 = json.load(open(os.path.join(HERE, "golden", "oracle_solves_xy32.json")))
BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))

F_TOL_FP64 = 1e-10
F_TOL_SPLIT = 1e-9
SPEC_TOL = 1e-9
GAP_PINNED = 1e-6
# the split configuration the headline numbers are measured with
SPLIT = {"precision": "split", "split_slices": 4}


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _solve(model, beta, h, dcut, nsteps, spectra=False, **cfg):
    with Solver(0, **cfg) as s:
        s.init_tensor(model, beta, h)
        s.coarse_grain(dcut, nsteps)
        f, _ = s.free_energy()
        sp = [s.spectrum(k) for k in range(1, nsteps + 1)] if spectra else None
        dims = s.state()[1:3]
    return f, sp, list(dims)


def test_dcut32_golden_covers_the_grid():
    assert len(GOLDEN32) == 6
    for g in GOLDEN32.values():
        assert g["dcut"] == 32 and g["nsteps"] == 40 and g["model"] == "ising"


def test_xy32_golden_covers_two_couplings():
    assert sorted(g["beta"] for g in GOLDEN_XY32.values()) == [1.0, 1.1]
    for g in GOLDEN_XY32.values():
        assert g["model"] == "xy" and g["dcut"] == 32 and g["trunc"] == "multiplet"


def _fp64_against(g):
    f, spectra, dims = _solve(g["model"], g["beta"], g["h"], g["dcut"], g["nsteps"], spectra=True,
                              precision="fp64", trunc=g["trunc"], eig_tol=1e-13)
    assert dims == g["steps"][-1]["dims"]
    assert abs(f - g["f"]) <= F_TOL_FP64, (f, g["f"])
    compared = 0
    prev_gap = 1.0
    for st, lam in zip(g["steps"], spectra):
        if not st["truncated"]:
            assert lam.size == 0
            continue
        ref = np.array(st["kept"])
        assert lam.size == ref.size
        # after a cut with a tiny gap the kept vectors are fixed only to about
        # residual / gap and later spectra inherit that (f stays pinned)
        if compared and prev_gap < GAP_PINNED:
            break
        prev_gap = st["gap"]
        compared += 1
        assert np.abs(lam / lam[0] - ref / ref[0]).max() <= SPEC_TOL, st["step"]
    assert compared >= 1


def _split_against(g):
    f, _, dims = _solve(g["model"], g["beta"], g["h"], g["dcut"], g["nsteps"], trunc=g["trunc"], **SPLIT)
    assert dims == g["steps"][-1]["dims"]
    assert abs(f - g["f"]) <= F_TOL_SPLIT, (f, g["f"])


@pytest.mark.parametrize("name", sorted(GOLDEN32))
def test_dcut32_fp64_matches_oracle(torch, name):
    _fp64_against(GOLDEN32[name])


@pytest.mark.parametrize("name", sorted(GOLDEN32))
def test_dcut32_split_matches_oracle(torch, name):
    _split_against(GOLDEN32[name])


@pytest.mark.parametrize("name", sorted(GOLDEN_XY32))
def test_xy32_fp64_matches_oracle(torch, name):
    _fp64_against(GOLDEN_XY32[name])


def _multiplet_decisions_resolved_in_split(g, lo=1e-11, hi=5e-6):
    """Split products separate exactly degenerate eigenvalues by up to
    ~2^-20 lambda_1 (S = 4), so the multiplet rule treats relative gaps below
    that as degenerate.  A solve whose oracle spectra hold a gap (at a cut
    or between kept values) between FP64 noise and a few times that bound
    has cuts the split path may take differently, each correctly for its
    own spectrum; f then differs by the truncation, not by arithmetic."""
    for st in g["steps"]:
        if not st["truncated"]:
            continue
        k = st["kept"]
        gaps = [st["gap"]] + [(k[i] - k[i + 1]) / k[0] for i in range(len(k) - 1)]
        if any(lo < x < hi for x in gaps):
            return False
    return True


def test_xy32_golden_has_a_split_resolved_case():
    assert any(_multiplet_decisions_resolved_in_split(g) for g in GOLDEN_XY32.values())


@pytest.mark.parametrize("name", sorted(GOLDEN_XY32))
def test_xy32_split_matches_oracle(torch, name):
    g = GOLDEN_XY32[name]
    if not _multiplet_decisions_resolved_in_split(g):
        pytest.skip("near-degenerate levels within split precision of the multiplet threshold")
    _split_against(g)


@pytest.mark.slow
@pytest.mark.parametrize("dcut,beta,h", [(48, BETA_C, 1e-3), (48, BETA_C, 0.0), (64, BETA_C, 1e-3)])
def test_split_matches_fp64_at_large_dcut(torch, dcut, beta, h):
    f64, _, d64 = _solve("ising", beta, h, dcut, 40, precision="fp64")
    fs, _, ds = _solve("ising", beta, h, dcut, 40, **SPLIT)
    assert d64 == ds == [dcut, dcut]
    assert abs(fs - f64) <= F_TOL_SPLIT, (fs, f64, abs(fs - f64))
