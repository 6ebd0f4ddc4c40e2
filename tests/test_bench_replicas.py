"""The multi-GPU path of bench.py (replicas, no exchange) on CPU ranks.

Two gloo ranks take the bookkeeping the GPU run uses under torchrun: each
rank's coupling, the max over ranks of the timed region, the whole-job
seconds per half-step, and the reference arm that only rank 0 runs.
"""
import importlib.util
import os
import socket

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
BENCH = os.path.join(os.path.dirname(HERE), "bench.py")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", BENCH)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = 100.0 + 50.0 * rank                  # rank 1 is the slower one
    ms_max = b.max_over_ranks(ms, world, device="cpu")
    out.put((rank, b.replica_beta(rank), ms_max, b.seconds_per_half_step(ms_max, 10, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, beta0, max0, v0), (r1, beta1, max1, v1) = res
    assert max0 == max1 == 150.0
    # 2 ranks x 10 half-steps in 150 ms of the slowest rank
    assert v0 == v1 == pytest.approx(0.150 / 20)
    assert beta0 != beta1 and abs(beta1 / beta0 - 1.0 - 1e-4) < 1e-12


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(12.5, 1) == 12.5
    assert b.seconds_per_half_step(100.0, 10, 1) == pytest.approx(0.01)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(b, "oracle_half_step_sample", lambda: called.append(1) or (1.0, "x"))

    class A:
        steps, warmup, gpus = 1, 1, 2
    b.run_reference(A())
    assert called == [] and capsys.readouterr().out == ""
