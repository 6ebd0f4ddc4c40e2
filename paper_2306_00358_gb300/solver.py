"""Python face of libtrg: the same calls as include/trg.h, marshalled.

PyTorch supplies device memory (the context's allocations go through its
caching allocator) and the CUDA stream; every step of the HOTRG path runs in
the library's own kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import TRGError, check  # noqa: F401  (re-exported)

_MODELS = {"ising": _lib.TRG_ISING, "xy": _lib.TRG_XY, "potts": _lib.TRG_POTTS}
_PREC = {"fp64": _lib.TRG_FP64, "split": _lib.TRG_SPLIT_BF16, "split_bf16": _lib.TRG_SPLIT_BF16}
_TRUNC = {"paper": _lib.TRG_TRUNC_PAPER, "multiplet": _lib.TRG_TRUNC_MULTIPLET}


def _torch():
    import torch
    return torch


def default_config(**kw) -> _lib.trg_config:
    lib = _lib.load()
    cfg = _lib.trg_config()
    check(lib.trg_config_default(ctypes.byref(cfg)))
    if "precision" in kw:
        p = kw.pop("precision")
        cfg.precision = _PREC[p] if isinstance(p, str) else int(p)
    if "trunc" in kw:
        t = kw.pop("trunc")
        cfg.trunc = _TRUNC[t] if isinstance(t, str) else int(t)
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k!r}")
        setattr(cfg, k, v)
    return cfg


class _TorchAllocator:
    """Routes libtrg's device allocations through torch's caching allocator."""

    def __init__(self, device: int):
        torch = _torch()
        self.device = device
        self._torch = torch

        def alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:
                return None

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = _lib.ALLOC_FN(alloc)
        self.free = _lib.FREE_FN(free)


class Solver:
    """One HOTRG solve on one GPU (a libtrg context)."""

    def __init__(self, device: int = 0, stream=None, torch_alloc: bool = True, **config):
        torch = _torch()
        self._lib = _lib.load()
        self.device = int(device)
        cfg = default_config(**config)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.trg_create(ctypes.byref(h), self.device, ctypes.byref(cfg)), None, "trg_create")
        self._h = h
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(self.device)
            check(self._lib.trg_set_allocator(h, self._alloc.alloc, self._alloc.free, None), h,
                  "trg_set_allocator")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.set_stream(stream)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._lib.trg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st, what):
        check(st, self._h, what)

    def set_stream(self, stream):
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        self._check(self._lib.trg_set_stream(self._h, ctypes.c_void_p(raw)), "trg_set_stream")

    def set_wait_limit(self, acc_wait_ns: int = 0):
        """Limit of the split products' accumulator wait (0 = 2 s); see trg_set_wait_limit."""
        self._check(self._lib.trg_set_wait_limit(self._h, int(acc_wait_ns)), "trg_set_wait_limit")

    def set_precision(self, precision, split_slices: int = 4, split_from_step: int = 0):
        p = _PREC[precision] if isinstance(precision, str) else int(precision)
        self._check(self._lib.trg_set_precision(self._h, p, split_slices, split_from_step), "trg_set_precision")

    # -- the solve
    def init_tensor(self, model: str, beta: float, h: float = 0.0, d0: int | None = None):
        m = _MODELS[model.lower()]
        if d0 is None:
            d0 = {_lib.TRG_ISING: 2, _lib.TRG_XY: 9, _lib.TRG_POTTS: 3}[m]
        self._check(self._lib.trg_init_tensor(self._h, m, float(beta), float(h), int(d0)), "trg_init_tensor")

    def init_tensor_raw(self, t: np.ndarray, beta: float):
        t = np.ascontiguousarray(t, dtype=np.float64)
        if t.ndim != 4 or t.shape[0] != t.shape[2] or t.shape[1] != t.shape[3]:
            raise ValueError("tensor of shape (Dx, Dy, Dx, Dy) expected")
        self._check(self._lib.trg_init_tensor_raw(self._h, t.ctypes.data_as(_lib.P_double), t.shape[0],
                                                  t.shape[1], float(beta)), "trg_init_tensor_raw")

    def init_impure(self, t_imp: np.ndarray | None = None):
        """Insert the model's observable (Ising s, XY cos theta, Potts [s=0]),
        or the given impure tensor, to be blocked alongside the pure one."""
        if t_imp is None:
            self._check(self._lib.trg_init_impure(self._h), "trg_init_impure")
            return
        t_imp = np.ascontiguousarray(t_imp, dtype=np.float64)
        self._check(self._lib.trg_init_impure_raw(self._h, t_imp.ctypes.data_as(_lib.P_double)),
                    "trg_init_impure_raw")

    def expectation(self) -> float:
        """<O> = Tr T_imp / Tr T of the current tensors."""
        v = ctypes.c_double()
        self._check(self._lib.trg_expectation(self._h, ctypes.byref(v)), "trg_expectation")
        return v.value

    def coarse_grain(self, dcut: int, nsteps: int):
        self._check(self._lib.trg_coarse_grain(self._h, int(dcut), int(nsteps)), "trg_coarse_grain")

    def free_energy(self):
        f = ctypes.c_double()
        lnz = ctypes.c_double()
        self._check(self._lib.trg_free_energy(self._h, ctypes.byref(f), ctypes.byref(lnz)), "trg_free_energy")
        return f.value, lnz.value

    # -- one half-step split over ranks (the caller exchanges the slabs)
    def shard_extent(self) -> int:
        nj = ctypes.c_int()
        self._check(self._lib.trg_shard_extent(self._h, ctypes.byref(nj)), "trg_shard_extent")
        return nj.value

    def shard_begin(self, dcut: int, j_begin: int, j_end: int, slab) -> int:
        """Environment, isometry and the output rows j_begin <= j < j_end into
        `slab` (CUDA float64, at least (j_end - j_begin) Dn^2 nj elements);
        returns Dn."""
        _require(slab, 1)
        dn = ctypes.c_int()
        self._check(self._lib.trg_shard_begin(self._h, int(dcut), int(j_begin), int(j_end), slab.data_ptr(),
                                              slab.numel(), ctypes.byref(dn)), "trg_shard_begin")
        return dn.value

    def shard_finish(self, gathered, j_rows: int):
        """Place the gathered output (rows j of Dn^2 nj elements) and close the half-step."""
        _require(gathered, 1)
        self._check(self._lib.trg_shard_finish(self._h, gathered.data_ptr(), int(j_rows)), "trg_shard_finish")

    def solve3d(self, beta: float, h: float, dcut: int, nsteps: int, model: str = "ising"):
        """A whole cubic-lattice solve (steps z, x, y, ...): returns (f, ln Z / V)."""
        f = ctypes.c_double()
        lnz = ctypes.c_double()
        self._check(self._lib.trg_solve3d(self._h, _MODELS[model.lower()], float(beta), float(h), int(dcut),
                                          int(nsteps), ctypes.byref(f), ctypes.byref(lnz)), "trg_solve3d")
        return f.value, lnz.value

    def spectrum(self, step: int) -> np.ndarray:
        n = ctypes.c_int()
        self._check(self._lib.trg_get_spectrum(self._h, int(step), None, 0, ctypes.byref(n)), "trg_get_spectrum")
        out = np.zeros(n.value)
        if n.value:
            self._check(self._lib.trg_get_spectrum(self._h, int(step), out.ctypes.data_as(_lib.P_double),
                                                   n.value, ctypes.byref(n)), "trg_get_spectrum")
        return out

    def state(self):
        s, dx, dy = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ln = ctypes.c_double()
        self._check(self._lib.trg_get_state(self._h, ctypes.byref(s), ctypes.byref(dx), ctypes.byref(dy),
                                            ctypes.byref(ln)), "trg_get_state")
        return s.value, dx.value, dy.value, ln.value

    def tensor(self) -> np.ndarray:
        _, dx, dy, _ = self.state()
        out = np.empty((dx, dy, dx, dy))
        self._check(self._lib.trg_get_tensor(self._h, out.ctypes.data_as(_lib.P_double), out.size),
                    "trg_get_tensor")
        return out

    def launch_count(self) -> int:
        return int(self._lib.trg_launch_count(self._h))

    def counters(self) -> dict:
        arr = (_lib.c_uint64 * 7)()
        self._check(self._lib.trg_get_counters(self._h, arr, 7), "trg_get_counters")
        names = ("subspace_iterations", "rayleigh_ritz", "jacobi_sweeps_fp32", "jacobi_sweeps_fp64",
                 "cholqr_repairs", "cholqr_single_pass", "shapes_tuned")
        return {k: int(v) for k, v in zip(names, arr)}

    def profile(self, on: bool = True):
        self._check(self._lib.trg_profile_enable(self._h, 1 if on else 0), "trg_profile_enable")

    def phase_stats(self) -> dict:
        out = {}
        for i, name in enumerate(_lib.PHASES):
            st = _lib.trg_phase_stats()
            self._check(self._lib.trg_profile_read(self._h, i, ctypes.byref(st)), "trg_profile_read")
            out[name] = {"ms": st.ms, "calls": int(st.calls), "flops": st.flops, "mma_flops": st.mma_flops}
        return out

    # -- components on device tensors (torch CUDA float64, contiguous)
    def gemm(self, a, b):
        torch = _torch()
        _require(a, 2)
        _require(b, 2)
        m, k = a.shape
        k2, n = b.shape
        if k != k2:
            raise ValueError("inner dimensions differ")
        c = torch.empty((m, n), dtype=torch.float64, device=a.device)
        self._check(self._lib.trg_gemm(self._h, m, n, k, a.data_ptr(), k, b.data_ptr(), n, c.data_ptr(), n),
                    "trg_gemm")
        return c

    def environment(self, t):
        torch = _torch()
        _require(t, 4)
        dx, dy = t.shape[0], t.shape[1]
        m = torch.empty((dx * dx, dx * dx), dtype=torch.float64, device=t.device)
        self._check(self._lib.trg_environment(self._h, t.data_ptr(), dx, dy, m.data_ptr()), "trg_environment")
        return m

    def isometry(self, m, dcut: int):
        torch = _torch()
        _require(m, 2)
        n = m.shape[0]
        dmax = min(n, int(dcut))
        u = torch.empty((n, dmax), dtype=torch.float64, device=m.device)
        lam = np.zeros(dmax)
        dn = ctypes.c_int()
        self._check(self._lib.trg_isometry(self._h, m.data_ptr(), n, int(dcut), u.data_ptr(),
                                           lam.ctypes.data_as(_lib.P_double), ctypes.byref(dn)), "trg_isometry")
        return u[:, :dn.value], (lam[:dn.value] if dn.value < n else None), dn.value

    def contract(self, t, u):
        torch = _torch()
        _require(t, 4)
        dx, dy = t.shape[0], t.shape[1]
        dn = u.shape[-1]
        if u.numel() != dx * dx * dn:
            raise ValueError("isometry shape does not match the tensor")
        u = u.contiguous()
        out = torch.empty((dn, dy, dn, dy), dtype=torch.float64, device=t.device)
        self._check(self._lib.trg_contract(self._h, t.data_ptr(), u.data_ptr(), dx, dy, dn, out.data_ptr()),
                    "trg_contract")
        return out


def _require(x, ndim):
    torch = _torch()
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
            and x.ndim == ndim):
        raise TypeError(f"contiguous CUDA float64 tensor of rank {ndim} expected")


def free_energy(model: str, beta: float, h: float, dcut: int, nsteps: int, d0: int | None = None,
                device: int = 0, **config):
    """Convenience one-shot solve: returns (f, ln Z / V)."""
    with Solver(device, **config) as s:
        s.init_tensor(model, beta, h, d0)
        s.coarse_grain(dcut, nsteps)
        return s.free_energy()
