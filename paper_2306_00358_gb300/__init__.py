"""GB300-native HOTRG coarse-graining (arXiv:2306.00358, Sec. 2) behind a C ABI.

``include/trg.h`` is the boundary; ``libtrg.so`` (built from ``csrc/`` for
sm_103a) does all the work; this package only marshals arguments.
"""
from .solver import Solver, TRGError, default_config, free_energy  # noqa: F401

__all__ = ["Solver", "TRGError", "default_config", "free_energy"]
