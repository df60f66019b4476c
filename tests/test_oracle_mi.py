"""Pins for the oracle's Kraskov mutual-information estimator (CPU only)."""
import math

import numpy as np
import pytest

from oracle.mi import ifr, ksg_counts, ksg_mi


def test_counts_match_a_brute_force_loop():
    rng = np.random.default_rng(3)
    Z = rng.normal(size=(9, 2)).astype(np.float32)
    Y = rng.normal(size=(9, 3)).astype(np.float32)
    k = 2
    eps, cz, cy = ksg_counts(Z, Y, k)
    for i in range(9):
        dist = []
        for j in range(9):
            if j == i:
                continue
            a = max(abs(float(Z[i, t]) - float(Z[j, t])) for t in range(2))
            b = max(abs(float(Y[i, t]) - float(Y[j, t])) for t in range(3))
            dist.append((max(a, b), a, b))
        e = sorted(x[0] for x in dist)[k - 1]
        assert math.isclose(float(eps[i]), e, rel_tol=1e-6)
        assert cz[i] == sum(1 for _, a, _ in dist if a < eps[i])
        assert cy[i] == sum(1 for _, _, b in dist if b < eps[i])


@pytest.mark.parametrize("rho,dims", [(0.9, 1), (0.6, 1), (0.8, 2)])
def test_gaussian_closed_form(rho, dims):
    """Jointly Gaussian pairs (z_t, y_t), t < dims, correlation rho each:
    I = -(dims / 2) ln(1 - rho^2)."""
    rng = np.random.default_rng(int(rho * 10) + dims)
    N = 2500
    z = rng.normal(size=(N, dims))
    y = rho * z + math.sqrt(1 - rho * rho) * rng.normal(size=(N, dims))
    exact = -0.5 * dims * math.log(1 - rho * rho)
    est = ksg_mi(z, y, k=3)
    assert abs(est - exact) < 0.05 * dims + 0.02, (est, exact)


def test_independent_samples_have_no_information():
    rng = np.random.default_rng(11)
    est = ksg_mi(rng.uniform(size=(2500, 2)), rng.normal(size=(2500, 3)), k=3)
    assert abs(est) < 0.03


def test_ifr_is_the_ratio():
    assert ifr(0.8, 0.4) == 2.0
