"""Scheduler of the solve engine (trg_serve_*, trg_batch_run), host only.

Dry-run mode: the worker slots sleep for a duration shaped like each solve
instead of touching the GPU, so admission, FIFO order, the HBM budget,
cancellation, failure reporting and the statistics are checked on the CPU.
Failures are injected on the host (a spec with the dry-run failure seed).
"""
import time

import pytest

from paper_2306_00358_gb300 import _lib
from paper_2306_00358_gb300 import serving as sv

DRY = dict(dry_run=True, dry_run_seconds_per_step=2e-4)


def test_estimate_grows_with_dcut():
    small = sv.solve_bytes(sv.Spec(dcut=16))
    big = sv.solve_bytes(sv.Spec(dcut=64))
    xy = sv.solve_bytes(sv.Spec(model="xy", dcut=64))
    assert 0 < small < big
    assert xy >= big * 0.9


def test_all_requests_complete_and_stats():
    with sv.Server(slots=4, hbm_budget_bytes=1 << 40, **DRY) as s:
        tickets = [s.submit(sv.Spec(dcut=d, nsteps=20)) for d in (16, 24, 32, 16, 48, 24, 16, 32)]
        res = [s.wait(t) for t in tickets]
        st = s.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["completed"] == 8 and st["failed"] == 0 and st["queued"] == 0 and st["running"] == 0
    assert 0 < st["p50_latency_s"] <= st["p99_latency_s"] <= st["max_latency_s"]
    assert st["solves_per_s"] > 0
    assert {r["slot"] for r in res} <= {0, 1, 2, 3}


def test_budget_is_never_exceeded():
    per = sv.solve_bytes(sv.Spec(dcut=32))
    budget = int(per * 2.5)            # room for two at a time
    with sv.Server(slots=8, hbm_budget_bytes=budget, **DRY) as s:
        tickets = [s.submit(sv.Spec(dcut=32, nsteps=10)) for _ in range(10)]
        running_max = 0
        while any(s.poll(t) is None for t in tickets):
            running_max = max(running_max, s.stats()["running"])
            time.sleep(0.002)
        st = s.stats()
    assert st["peak_bytes"] <= budget
    assert running_max <= 2
    assert st["completed"] == 10


def test_fifo_order_with_one_slot():
    with sv.Server(slots=1, hbm_budget_bytes=1 << 40, **DRY) as s:
        tickets = [s.submit(sv.Spec(dcut=16, nsteps=5)) for _ in range(6)]
        res = [s.wait(t) for t in tickets]
    starts = [r["seconds_queued"] for r in res]
    assert starts == sorted(starts)   # later submissions never start earlier


def test_oversized_request_is_rejected():
    with sv.Server(slots=2, hbm_budget_bytes=1 << 30, **DRY) as s:
        with pytest.raises(_lib.TRGError) as e:
            s.submit(sv.Spec(dcut=96))
        assert e.value.status == _lib.TRG_ENOMEM


def test_invalid_spec_is_rejected():
    with sv.Server(slots=2, hbm_budget_bytes=1 << 40, **DRY) as s:
        for bad in (sv.Spec(beta=-1.0), sv.Spec(dcut=0), sv.Spec(model="xy", d0=8),
                    sv.Spec(slices=7), sv.Spec(nsteps=-1)):
            with pytest.raises(_lib.TRGError) as e:
                s.submit(bad)
            assert e.value.status == _lib.TRG_EINVAL


def test_cancel_queued_request():
    with sv.Server(slots=1, hbm_budget_bytes=1 << 40, **DRY) as s:
        first = s.submit(sv.Spec(dcut=32, nsteps=40))
        second = s.submit(sv.Spec(dcut=16, nsteps=5))
        time.sleep(0.01)                             # the first one is running
        assert s.cancel(second) == _lib.TRG_OK
        assert s.cancel(first) == _lib.TRG_ESTATE    # already started
        with pytest.raises(_lib.TRGError) as e:
            s.wait(second)
        assert e.value.status == _lib.TRG_ECANCELED
        assert s.wait(first)["status"] == 0
        assert s.stats()["cancelled"] == 1


def test_failed_solve_is_reported_and_server_continues():
    with sv.Server(slots=2, hbm_budget_bytes=1 << 40, **DRY) as s:
        bad = s.submit(sv.Spec(dcut=16, nsteps=5, seed=_lib.TRG_DRY_RUN_FAIL_SEED))
        good = s.submit(sv.Spec(dcut=16, nsteps=5))
        assert s.wait(bad)["status"] == _lib.TRG_ENUMERIC
        assert s.wait(good)["status"] == 0
        st = s.stats()
    assert st["failed"] == 1 and st["completed"] == 1


def test_wait_timeout():
    with sv.Server(slots=1, hbm_budget_bytes=1 << 40, **DRY) as s:
        t = s.submit(sv.Spec(dcut=64, nsteps=40))
        with pytest.raises(_lib.TRGError) as e:
            s.wait(t, timeout=0.001)
        assert e.value.status == _lib.TRG_ETIMEOUT
        s.wait(t)


def test_slots_run_concurrently():
    n, per_step, steps = 8, 2e-4, 40
    with sv.Server(slots=8, hbm_budget_bytes=1 << 40, dry_run=True, dry_run_seconds_per_step=per_step) as s:
        t0 = time.perf_counter()
        tickets = [s.submit(sv.Spec(dcut=16, nsteps=steps)) for _ in range(n)]
        for t in tickets:
            s.wait(t)
        wall = time.perf_counter() - t0
    serial = n * per_step * steps
    assert wall < 0.6 * serial


def test_batch_run_returns_in_order():
    specs = [sv.Spec(dcut=16, nsteps=3 + i) for i in range(5)]
    res = sv.batch_run(specs, slots=3, hbm_budget_bytes=1 << 40, **DRY)
    assert [r["status"] for r in res] == [0] * 5


def _finish_order(policy, **extra):
    # one slot, busy with a blocker while a long and three short requests queue
    with sv.Server(slots=1, hbm_budget_bytes=1 << 40, policy=policy, **DRY, **extra) as s:
        # the blocker sleeps 0.2 s, far longer than the submissions below take
        blocker = s.submit(sv.Spec(dcut=32, nsteps=250))
        time.sleep(0.005)
        long_t = s.submit(sv.Spec(dcut=48, nsteps=40))
        shorts = [s.submit(sv.Spec(dcut=16, nsteps=5)) for _ in range(3)]
        s.wait(blocker)
        res = {t: s.wait(t) for t in [long_t] + shorts}
    end = {t: r["seconds_queued"] + r["seconds_run"] for t, r in res.items()}
    return long_t, shorts, end


def test_shortest_first_lets_short_requests_pass():
    long_t, shorts, end = _finish_order("shortest")
    assert all(end[t] < end[long_t] for t in shorts)
    long_t, shorts, end = _finish_order("fifo")
    assert all(end[t] > end[long_t] for t in shorts)


def test_shortest_first_does_not_starve_a_long_request():
    # with max_wait_s = 0 the oldest request always goes first: FIFO again
    long_t, shorts, end = _finish_order("shortest", max_wait_s=0.0)
    assert all(end[t] > end[long_t] for t in shorts)


def test_bad_policy_is_rejected():
    c = sv.server_config(**DRY)
    c.policy = 7
    lib = _lib.load()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.trg_serve_create(ctypes.byref(h), 0, ctypes.byref(c)) == _lib.TRG_EINVAL
