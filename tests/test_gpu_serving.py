"""Batched and served solves on the GPU: each result is the same alone and in
a mix (bit for bit: same kernels, no shared buffers), requests that arrive
while others run start before those finish, and the mixed results agree with
the oracle where a golden value exists."""
import json
import os
import time

import pytest

from paper_2306_00358_gb300 import Solver
from paper_2306_00358_gb300 import serving as sv

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "oracle_solves.json")))


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _alone(spec: sv.Spec):
    with Solver(0, precision=spec.precision, split_slices=spec.slices, trunc=spec.trunc,
                workspace_bytes=1 << 30) as s:
        s.init_tensor(spec.model, spec.beta, spec.h, spec.d0)
        s.coarse_grain(spec.dcut, spec.nsteps)
        return s.free_energy()[0]


MIX = [
    sv.Spec(model="ising", beta=0.44, dcut=16, nsteps=40),
    sv.Spec(model="ising", beta=0.40, h=1e-2, dcut=24, nsteps=31),
    sv.Spec(model="ising", beta=0.48, dcut=12, nsteps=20, precision="fp64"),
    sv.Spec(model="xy", beta=1.0, dcut=12, nsteps=12, trunc="multiplet"),
    sv.Spec(model="ising", beta=0.4406868, h=1e-3, dcut=32, nsteps=26),
    sv.Spec(model="xy", beta=1.1, h=0.05, d0=9, dcut=20, nsteps=8, trunc="multiplet", precision="fp64"),
]


def test_batch_results_equal_alone(torch):
    res = sv.batch_run(MIX, slots=4, hbm_budget_bytes=100 << 30, workspace_bytes=1 << 30)
    for spec, r in zip(MIX, res):
        assert r["status"] == 0
        assert r["f"] == _alone(spec), spec


def test_batch_matches_oracle_golden(torch):
    g1 = GOLDEN["ising_b0.44_d16_n40"]
    g2 = GOLDEN["xy_b1.1_d20_h0.05_n8"]
    res = sv.batch_run([MIX[0], MIX[5]], slots=2, hbm_budget_bytes=100 << 30)
    assert abs(res[0]["f"] - g1["f"]) <= 1e-9      # split, 4 slices
    assert abs(res[1]["f"] - g2["f"]) <= 1e-10     # FP64


def test_served_requests_overlap_and_match(torch):
    long_spec = sv.Spec(model="ising", beta=0.4406868, dcut=48, nsteps=30)
    short = [sv.Spec(model="ising", beta=0.40 + 0.01 * i, dcut=16, nsteps=20) for i in range(4)]
    with sv.Server(0, slots=4, hbm_budget_bytes=100 << 30) as s:
        t_long = s.submit(long_spec)
        time.sleep(0.2)                       # the long solve is on the GPU now
        t_short = [s.submit(x) for x in short]
        r_short = [s.wait(t) for t in t_short]
        r_long = s.wait(t_long)
        st = s.stats()
    assert st["completed"] == 5 and st["failed"] == 0
    # the short requests were admitted while the long one was running
    assert all(r["seconds_queued"] < r_long["seconds_run"] for r in r_short)
    for spec, r in zip(short, r_short):
        assert r["f"] == _alone(spec)
    assert r_long["f"] == _alone(long_spec)
