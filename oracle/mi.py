"""Mutual information for the Information Flow Refinement analysis (Sec. 3.1.1).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the library's estimator.

Sec. 3.1.1 measures I(S; S + X^(k)) between an MBRB's skip input S and its
fused output with Kraskov's k-nearest-neighbour estimator,

    I(Z; Y) ~ psi(v) + psi(c) - (1/c) sum_i ( psi(c_z(i) + 1) + psi(c_y(i) + 1) ),

v neighbours, c samples, and compares branch counts by the ratio
IFR_{k1 -> k2} = I^(k1) / I^(k2). Read as Kraskov, Stoegbauer and
Grassberger's first algorithm (2004): the distance in the joint space (z, y)
is the larger of the two max-norm distances; eps(i) is the v-th smallest
joint distance from sample i to the other samples; c_z(i) and c_y(i) count
the other samples strictly closer than eps(i) in z alone and in y alone.

Distances, the v-th neighbour and the counts are taken in FP32 (|a - b| and
max are exact in FP32 once the operands are FP32), so a GPU estimator given
the same FP32 samples must reproduce the counts exactly; the digamma sum is
FP64 (scipy).

Parity: pinned by a brute-force loop on a tiny input, the closed form
-(1/2) ln(1 - rho^2) per pair of jointly Gaussian coordinates, and zero for
independent samples (tests/test_oracle_mi.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import digamma


def _maxnorm_rows(A: np.ndarray, rows: slice) -> np.ndarray:
    """FP32 max-norm distances from the samples in ``rows`` to every sample."""
    return np.abs(A[rows, None, :] - A[None, :, :]).max(axis=2)


def ksg_counts(Z: np.ndarray, Y: np.ndarray, k: int, block: int = 32):
    """eps (FP32), c_z and c_y for every sample (see the module docstring)."""
    Z = np.ascontiguousarray(Z, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    N = Z.shape[0]
    assert Y.shape[0] == N and 1 <= k < N
    eps = np.empty(N, np.float32)
    cz = np.empty(N, np.int64)
    cy = np.empty(N, np.int64)
    for i0 in range(0, N, block):
        rows = slice(i0, min(N, i0 + block))
        dz = _maxnorm_rows(Z, rows)
        dy = _maxnorm_rows(Y, rows)
        d = np.maximum(dz, dy)
        for r, i in enumerate(range(rows.start, rows.stop)):
            others = np.delete(np.arange(N), i)
            e = np.partition(d[r, others], k - 1)[k - 1]
            eps[i] = e
            cz[i] = int((dz[r, others] < e).sum())
            cy[i] = int((dy[r, others] < e).sum())
    return eps, cz, cy


def ksg_mi(Z: np.ndarray, Y: np.ndarray, k: int = 3) -> float:
    """Kraskov's estimate of I(Z; Y) in nats."""
    N = Z.shape[0]
    _, cz, cy = ksg_counts(Z, Y, k)
    return float(digamma(k) + digamma(N) - np.mean(digamma(cz + 1.0) + digamma(cy + 1.0)))


def ifr(i_k1: float, i_k2: float) -> float:
    """IFR_{k1 -> k2} = I^(k1) / I^(k2)."""
    return i_k1 / i_k2
