"""FP64 Matching Pursuit oracle — test infrastructure only.

Imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py``; never by the product library.
"""
from .mp_oracle import (STOP_CONVERGED, STOP_MAX_ITERS, STOP_ZERO_Y, follow, mp,  # noqa: F401
                        reconstruction_error, support_score)
