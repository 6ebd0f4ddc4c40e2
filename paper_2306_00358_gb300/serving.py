"""Python face of the solve engine (trg_batch_run, trg_serve_*): marshalling only.

The scheduler, its worker slots and every solve run inside libtrg.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import check

_MODELS = {"ising": _lib.TRG_ISING, "xy": _lib.TRG_XY, "potts": _lib.TRG_POTTS}
_PREC = {"fp64": _lib.TRG_FP64, "split": _lib.TRG_SPLIT_BF16}
_TRUNC = {"paper": _lib.TRG_TRUNC_PAPER, "multiplet": _lib.TRG_TRUNC_MULTIPLET}


@dataclass
class Spec:
    model: str = "ising"
    beta: float = 0.44
    h: float = 0.0
    d0: int | None = None
    dcut: int = 16
    nsteps: int = 40
    precision: str = "split"
    slices: int = 4
    trunc: str = "paper"
    seed: int = 0

    def c(self) -> _lib.trg_solve_spec:
        m = _MODELS[self.model]
        d0 = self.d0 if self.d0 is not None else {_lib.TRG_ISING: 2, _lib.TRG_XY: 9, _lib.TRG_POTTS: 3}[m]
        return _lib.trg_solve_spec(m, float(self.beta), float(self.h), int(d0), int(self.dcut), int(self.nsteps),
                                   _PREC[self.precision], int(self.slices), _TRUNC[self.trunc], int(self.seed))


def _result(r: _lib.trg_solve_result) -> dict:
    return {"status": r.status, "f": r.f, "lnz_per_site": r.lnz_per_site, "seconds_queued": r.seconds_queued,
            "seconds_run": r.seconds_run, "slot": r.slot}


_POLICIES = {"fifo": _lib.TRG_SERVE_FIFO, "shortest": _lib.TRG_SERVE_SHORTEST_FIRST}


def server_config(slots=8, hbm_budget_bytes=150 << 30, workspace_bytes=1 << 30, dry_run=False,
                  dry_run_seconds_per_step=1e-3, policy="fifo", max_wait_s=60.0) -> _lib.trg_server_config:
    """policy "fifo" (arrival order) or "shortest" (least estimated work first,
    unless the oldest request has waited max_wait_s)."""
    return _lib.trg_server_config(int(slots), int(hbm_budget_bytes), int(workspace_bytes), 1 if dry_run else 0,
                                  float(dry_run_seconds_per_step), _POLICIES[policy], float(max_wait_s))


def solve_bytes(spec: Spec, workspace_bytes: int = 0) -> int:
    lib = _lib.load()
    sp = spec.c()
    return int(lib.trg_solve_bytes(ctypes.byref(sp), int(workspace_bytes)))


class Server:
    """Continuous-batching solve server on one GPU (trg_serve_*)."""

    def __init__(self, device: int = 0, **cfg):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        c = server_config(**cfg)
        check(self._lib.trg_serve_create(ctypes.byref(h), int(device), ctypes.byref(c)), None, "trg_serve_create")
        self._h = h

    def submit(self, spec: Spec) -> int:
        t = ctypes.c_uint64()
        sp = spec.c()
        check(self._lib.trg_serve_submit(self._h, ctypes.byref(sp), ctypes.byref(t)), None, "trg_serve_submit")
        return int(t.value)

    def poll(self, ticket: int):
        r = _lib.trg_solve_result()
        st = self._lib.trg_serve_poll(self._h, int(ticket), ctypes.byref(r))
        if st == _lib.TRG_EAGAIN:
            return None
        check(st, None, "trg_serve_poll")
        return _result(r)

    def wait(self, ticket: int, timeout: float = -1.0):
        r = _lib.trg_solve_result()
        check(self._lib.trg_serve_wait(self._h, int(ticket), float(timeout), ctypes.byref(r)), None,
              "trg_serve_wait")
        return _result(r)

    def cancel(self, ticket: int) -> int:
        return self._lib.trg_serve_cancel(self._h, int(ticket))

    def stats(self) -> dict:
        s = _lib.trg_serve_stats()
        check(self._lib.trg_serve_get_stats(self._h, ctypes.byref(s)), None, "trg_serve_get_stats")
        return {k: getattr(s, k) for k, _ in _lib.trg_serve_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.trg_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_run(specs, device: int = 0, **cfg):
    """Run independent solves concurrently (trg_batch_run); returns results in order."""
    lib = _lib.load()
    n = len(specs)
    arr = (_lib.trg_solve_spec * n)(*[s.c() for s in specs])
    res = (_lib.trg_solve_result * n)()
    c = server_config(**cfg)
    lib.trg_batch_run(int(device), arr, n, ctypes.byref(c), res)
    return [_result(r) for r in res]
