"""CPU FP64 oracle for the HOTRG coarse-graining path.

ORACLE / TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously
correct restatement of the method (Sec. 2 of the paper: environment, SVD
isometry, U.T.T.U contraction, normalisation, periodic trace) and of exact
results that pin it (Onsager's free energy, brute-force partition functions).
Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it.  It shares no code with the CUDA library and never imports it.

Parity status of each function is stated in its module docstring; every
function here is pinned by a test under tests/ against an exact result.
"""
