"""Write the oracle's expected values for the GPU parity tests.

Calls only the oracle (oracle/), never the CUDA library.  Run from the
repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact, hotrg, models  # noqa: E402

CASES = [
    # name, model, beta, h, dcut, nsteps, trunc
    ("ising_b0.44_d16_n40", "ising", 0.44, 0.0, 16, 40, "paper"),
    ("ising_bc_d16_h1e-3_n40", "ising", exact.BETA_C, 1e-3, 16, 40, "paper"),
    ("ising_b0.48_d10_n21", "ising", 0.48, 0.0, 10, 21, "paper"),
    ("xy_b1.0_d12_n12", "xy", 1.0, 0.0, 12, 12, "multiplet"),
    ("xy_b1.1_d20_h0.05_n8", "xy", 1.1, 0.05, 20, 8, "multiplet"),
    ("potts_bc_d12_n30", "potts", math.log(1 + math.sqrt(3)), 0.0, 12, 30, "multiplet"),
]


def run(name, model, beta, h, dcut, nsteps, trunc):
    t0 = models.initial_tensor(model, beta, h)
    s = hotrg.solve(t0, beta, dcut, nsteps, trunc=trunc, keep_full_spectra=True)
    steps = []
    for k, (kept, full) in enumerate(zip(s.spectra, s.full_spectra), start=1):
        n = full.shape[0]
        dn = kept.shape[0]
        truncated = dn < n
        gap = float((full[dn - 1] - full[dn]) / full[0]) if truncated else None
        steps.append({"step": k, "n": int(n), "dn": int(dn), "truncated": bool(truncated),
                      "kept": [float(x) for x in kept] if truncated else [], "gap": gap,
                      "dims": list(s.dims[k - 1])})
    rec = {"name": name, "model": model, "beta": beta, "h": h, "dcut": dcut, "nsteps": nsteps,
           "trunc": trunc, "f": s.f, "lnz_per_site": s.lnz_per_site, "steps": steps,
           "source": "oracle/hotrg.py solve() (CPU FP64, cyclic Jacobi)"}
    if model == "ising" and h == 0.0:
        rec["f_onsager"] = exact.onsager_free_energy(beta)
    return rec


EXPECTATION_CASES = [
    # name, model, beta, h, dcut, nsteps, trunc: impure tensor of the model's observable
    ("ising_bc_d16_h1e-3_n20", "ising", exact.BETA_C, 1e-3, 16, 20, "paper"),
    ("ising_b0.6_d16_h1e-10_n40", "ising", 0.6, 1e-10, 16, 40, "paper"),
    ("xy_b1.0_d12_h0.05_n12", "xy", 1.0, 0.05, 12, 12, "multiplet"),
    ("potts_b1.0_d12_h0.02_n16", "potts", 1.0, 0.02, 12, 16, "multiplet"),
]


def expectations():
    """oracle_expectations.json: <O> = Tr T_imp / Tr T of truncated solves and
    of untruncated small tori (with the enumerated value beside it)."""
    out = {"solves": {}, "tori": {}}
    for (name, model, beta, h, dcut, nsteps, trunc) in EXPECTATION_CASES:
        print("oracle (impure):", name, flush=True)
        s = hotrg.solve(models.initial_tensor(model, beta, h), beta, dcut, nsteps, trunc=trunc,
                        impure=models.impure_tensor(model, beta, h))
        out["solves"][name] = {"model": model, "beta": beta, "h": h, "dcut": dcut, "nsteps": nsteps, "trunc": trunc,
                               "expectation": s.expectation, "f": s.f,
                               "source": "oracle/hotrg.py solve(impure=...) (CPU FP64)"}
    for nsteps in (2, 3, 4):
        w, hh = exact.hotrg_block(nsteps)
        out["tori"][f"ising_b0.44_h0.01_n{nsteps}"] = {
            "model": "ising", "beta": 0.44, "h": 0.01, "nsteps": nsteps,
            "expectation": exact.ising_magnetization_exact(w, hh, 0.44, 0.01)}
    for nsteps in (1, 2):
        w, hh = exact.hotrg_block(nsteps)
        out["tori"][f"xy_b0.9_h0.1_n{nsteps}"] = {
            "model": "xy", "beta": 0.9, "h": 0.1, "nsteps": nsteps,
            "expectation": exact.xy_cos_exact(w, hh, 0.9, 0.1, 9)}
    for nsteps in (2, 3):
        w, hh = exact.hotrg_block(nsteps)
        out["tori"][f"potts_b0.8_h0.05_n{nsteps}"] = {
            "model": "potts", "beta": 0.8, "h": 0.05, "nsteps": nsteps,
            "expectation": exact.potts_fraction0_exact(w, hh, 0.8, 0.05, 3)}
    with open(os.path.join(HERE, "oracle_expectations.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote oracle_expectations.json")


# The Ising coupling grid at Dcut 32 (beta_c, 0.40, 0.48 x h 0, 1e-3; 40
# half-steps): the sizes of the split-versus-FP64 accuracy gate at its
# smallest bond dimension.  Each solve runs the oracle's cyclic Jacobi on
# matrices up to 1024 x 1024, tens of minutes of CPU per solve, so they run
# as separate processes and are written to their own file.
DCUT32_CASES = [
    (f"ising_{bn}_d32_h{h:g}_n40", "ising", b, h, 32, 40, "paper")
    for (bn, b) in (("bc", exact.BETA_C), ("b0.40", 0.40), ("b0.48", 0.48))
    for h in (0.0, 1e-3)
]


# The truncated XY model (D0 = 9, charges |n| <= 4) at Dcut 32, 30 half-steps
# (the lattice of the XY runs), multiplet truncation: the oracle's 1024 x 1024
# Jacobi solves make each of these tens of CPU-minutes too.
XY32_CASES = [(f"xy_b{b:g}_d32_n30", "xy", b, 0.0, 32, 30, "multiplet") for b in (1.0, 1.1)]


def _run_case(case):
    return case[0], run(*case)


def dcut32(names=None, cases_all=None, fname="oracle_solves_dcut32.json"):
    """oracle_solves_dcut32.json: the Dcut-32 coupling grid (or the named
    subset of it), one process per solve."""
    import multiprocessing as mp
    cases = [c for c in (cases_all or DCUT32_CASES) if not names or c[0] in names]
    path = os.path.join(HERE, fname)
    out = json.load(open(path)) if os.path.exists(path) else {}
    with mp.get_context("spawn").Pool(len(cases)) as pool:
        for name, rec in pool.imap_unordered(_run_case, cases):
            print("oracle done:", name, rec["f"], flush=True)
            out[name] = rec
            with open(path, "w") as fh:
                json.dump(dict(sorted(out.items())), fh, indent=1)
    print("wrote", fname)


def main():
    if "--expectations" in sys.argv:
        expectations()
        return
    if "--dcut32" in sys.argv:
        dcut32([a for a in sys.argv[1:] if not a.startswith("--")])
        return
    if "--xy32" in sys.argv:
        dcut32([a for a in sys.argv[1:] if not a.startswith("--")], XY32_CASES, "oracle_solves_xy32.json")
        return
    expectations()
    out = {}
    for case in CASES:
        print("oracle:", case[0], flush=True)
        out[case[0]] = run(*case)
    with open(os.path.join(HERE, "oracle_solves.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    # exact partition functions of small tori (no truncation)
    ex = {}
    for (beta, h) in [(0.44, 0.0), (0.44, 0.01), (0.3, -0.25)]:
        for nsteps in (2, 3, 4):
            w, hh = exact.hotrg_block(nsteps)
            ex[f"ising_b{beta}_h{h}_n{nsteps}"] = {"model": "ising", "beta": beta, "h": h, "nsteps": nsteps,
                                                   "width": w, "height": hh,
                                                   "lnz": exact.ising_lnz_exact(w, hh, beta, h)}
    for (beta, h) in [(1.0, 0.0), (0.8, 0.05)]:
        for nsteps in (2, 3):
            w, hh = exact.hotrg_block(nsteps)
            ex[f"potts_b{beta}_h{h}_n{nsteps}"] = {"model": "potts", "beta": beta, "h": h, "nsteps": nsteps,
                                                   "width": w, "height": hh,
                                                   "lnz": exact.potts_lnz_exact(w, hh, beta, h, 3)}
    for (beta, h) in [(1.0, 0.0), (0.9, 0.1)]:
        for nsteps in (1, 2):
            w, hh = exact.hotrg_block(nsteps)
            ex[f"xy_b{beta}_h{h}_n{nsteps}"] = {"model": "xy", "beta": beta, "h": h, "nsteps": nsteps,
                                                "width": w, "height": hh,
                                                "lnz": exact.xy_lnz_exact(w, hh, beta, h, 9)}
    with open(os.path.join(HERE, "exact_tori.json"), "w") as fh:
        json.dump(ex, fh, indent=1)
    print("wrote oracle_solves.json, exact_tori.json")


if __name__ == "__main__":
    main()
