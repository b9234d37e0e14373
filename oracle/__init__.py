"""FP64 CPU oracle for the APMGSRN hot path.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA
library is checked against: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and imports nothing from it.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` to
something other than itself (closed forms, invariants stated in the paper,
brute force at high precision on tiny inputs, central finite differences,
published known-answer vectors).
"""
from . import apmgsrn, render, sampler  # noqa: F401
