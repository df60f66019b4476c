"""Counter-based SplitMix64 and the initial-value rule (oracle side).

The paper starts compression from "randomly initialized parameters"
(Sec. 2.1, Algorithm 1) and says the FDM is "initialized randomly"
(Sec. 3.2). It gives no distribution. The reading used here:

* Value ``idx`` of tensor ``tid`` comes from the SplitMix64 stream seeded
  with ``seed + G * tid * 2**32``: output number ``idx + 1`` of that stream,
  i.e. ``mix(seed + G * (tid * 2**32 + idx + 1))`` with G = 0x9E3779B97F4A7C15.
  SplitMix64 is the generator of Steele, Lea and Flood (OOPSLA 2014).
* The top 24 bits ``k`` of that output give w = (2k + 1 - 2**24) / 2**24,
  which lies in (-1, 1) and is exact in FP32.
* The value is the FP32 product fl32(fl32(bound) * w). So every initial value
  is an FP32 number, and any implementation that follows this rule
  reproduces it bit for bit.

Parity: pinned by the published SplitMix64 outputs for seed 0 and by the
distribution's moments (tests/test_oracle_rng.py).
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, tid: int, idx: np.ndarray) -> np.ndarray:
    """Outputs ``idx + 1`` of the SplitMix64 stream of tensor ``tid``."""
    idx = np.asarray(idx, dtype=np.uint64)
    base = np.uint64((seed + GOLDEN * (tid << 32)) & MASK64)
    with np.errstate(over="ignore"):
        z = base + np.uint64(GOLDEN) * (idx + np.uint64(1))
        return _mix(z)


def init_values(seed: int, tid: int, n: int, bound: float, start: int = 0) -> np.ndarray:
    """``n`` initial values of tensor ``tid``, uniform in (-bound, bound), FP32.

    Returned as float64 holding the FP32 values exactly.
    """
    idx = np.arange(start, start + n, dtype=np.uint64)
    k = (splitmix64(seed, tid, idx) >> np.uint64(40)).astype(np.int64)
    w = ((2 * k + 1 - (1 << 24)).astype(np.float64) / float(1 << 24)).astype(np.float32)
    b32 = np.float32(bound)
    return (b32 * w).astype(np.float32).astype(np.float64)
