"""The cubic-lattice blocking on the GPU against the 3D oracle.

* Untruncated steps (1, 2, 3: the 1x1x2, 2x1x2 and 2x2x2 tori) equal exact
  enumeration, FP64 to 1e-12 and split to 1e-9 in ln Z.
* Truncated solves equal the oracle: f to 1e-10 (FP64); ln Z / V to 1e-9
  (split: the 2D gate of 1e-9 on f at beta ~ 0.44 is ~4e-10 on ln Z / V,
  and f = -(ln Z / V) / beta magnifies an error by 1 / beta = 4.5 at the
  cubic lattice's beta_c = 0.2217, so the gate is put on ln Z / V); the
  kept spectra of both isometries, as lambda_i / lambda_1, to 1e-9 (FP64;
  the split path's spectra are reported, not gated).
* Unsupported models and bad arguments are reported.
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg3d
from paper_2306_00358_gb300 import Solver, _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-9)])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_untruncated_matches_enumeration(torch, precision, tol, nsteps):
    beta, h = 0.3, 0.1
    lx, ly, lz = hotrg3d.block3d(nsteps)
    with Solver(0, precision=precision) as s:
        _, lnz = s.solve3d(beta, h, 10 ** 6, nsteps)
    ref = exact.ising3d_lnz_exact(lx, ly, lz, beta, h)
    assert abs(lnz * lx * ly * lz - ref) <= tol * max(1.0, abs(ref))


# (beta, h, Dcut, steps, truncation); at Dcut 8 the y isometry of step 2
# meets an exactly degenerate pair at the cut (relative gap 2.5e-17), which
# the multiplet rule keeps whole; the other cuts have relative gaps >= 1.5e-4
CASES = [(0.2216544, 0.0, 4, 8, "paper"), (0.2, 0.05, 6, 7, "paper"), (0.3, 0.0, 5, 6, "paper"),
         (0.2216544, 0.0, 8, 6, "multiplet")]


@pytest.mark.parametrize("beta,h,dcut,nsteps,trunc", CASES)
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_truncated_matches_oracle(torch, beta, h, dcut, nsteps, trunc, precision):
    ref = hotrg3d.solve3d(hotrg3d.ising3d_tensor(beta, h), beta, dcut, nsteps, trunc=trunc)
    with Solver(0, precision=precision, trunc=trunc) as s:
        f, lnz = s.solve3d(beta, h, dcut, nsteps)
        spectra = [s.spectrum(k) for k in range(1, 2 * nsteps + 1)]
    if precision == "fp64":
        assert abs(f - ref.f) <= 1e-10, (f, ref.f)
    else:
        assert abs(lnz - ref.lnz_per_site) <= 1e-9, (lnz, ref.lnz_per_site)
    if precision == "fp64":
        for k, (rx, ry) in enumerate(ref.spectra):
            for got, want in ((spectra[2 * k], rx), (spectra[2 * k + 1], ry)):
                assert got.shape == want.shape
                if want.size:
                    assert np.abs(got / got[0] - want / want[0]).max() <= 1e-9


def test_errors(torch):
    with Solver(0) as s:
        f = _lib.load()
        import ctypes
        out = ctypes.c_double()
        assert f.trg_solve3d(s._h, _lib.TRG_XY, 1.0, 0.0, 4, 2, ctypes.byref(out), None) == _lib.TRG_ENOTSUP
        assert f.trg_solve3d(s._h, _lib.TRG_ISING, 0.0, 0.0, 4, 2, ctypes.byref(out), None) == _lib.TRG_EINVAL
        assert f.trg_solve3d(s._h, _lib.TRG_ISING, 0.3, 0.0, 0, 2, ctypes.byref(out), None) == _lib.TRG_EINVAL
        assert f.trg_solve3d(s._h, _lib.TRG_ISING, 0.3, 0.0, 4, 2, None, None) == _lib.TRG_EINVAL
        # the context stays usable
        fv, _ = s.solve3d(0.3, 0.0, 4, 3)
        assert math.isfinite(fv)
