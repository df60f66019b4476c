"""Kraskov mutual information of Sec. 3.1.1 on the GPU vs the oracle (needs a GPU).

The estimator's decisions (max-norm distances, the k-th neighbour, strict
counts) are exact functions of the FP32 samples, so the per-sample counts
must equal the oracle's bit for bit; the FP64 digamma sums agree to 1e-9.
Cases: random samples, samples with ties, jointly Gaussian samples (also
against the closed form), and a model's MBRB skip input and fused output.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
from oracle.mi import ksg_counts, ksg_mi  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu(Z, Y, k):
    z = torch.from_numpy(np.ascontiguousarray(Z, np.float32)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(Y, np.float32)).cuda()
    n = Z.shape[0]
    cz = torch.zeros(n, dtype=torch.int32, device="cuda")
    cy = torch.zeros(n, dtype=torch.int32, device="cuda")
    mi = edpc.ksg_mi(z.data_ptr(), y.data_ptr(), n, Z.shape[1], Y.shape[1], k, cz.data_ptr(), cy.data_ptr())
    return mi, cz.cpu().numpy(), cy.cpu().numpy()


@pytest.mark.parametrize("n,dz,dy,k,ties", [(300, 37, 50, 3, False), (64, 1, 1, 1, False), (257, 5, 3, 63, False),
                                            (200, 4, 6, 4, True)])
def test_counts_match_oracle(n, dz, dy, k, ties):
    rng = np.random.default_rng(n + k)
    Z = rng.normal(size=(n, dz)).astype(np.float32)
    Y = (0.5 * Z[:, :1] + rng.normal(size=(n, dy))).astype(np.float32)
    if ties:
        Z = np.round(Z * 2).astype(np.float32)
        Y = np.round(Y * 2).astype(np.float32)
    mi, cz, cy = _gpu(Z, Y, k)
    _, oz, oy = ksg_counts(Z, Y, k)
    assert np.array_equal(cz, oz) and np.array_equal(cy, oy)
    assert abs(mi - ksg_mi(Z, Y, k)) < 1e-9


def test_gaussian_closed_form():
    rng = np.random.default_rng(1)
    n, rho = 2000, 0.9
    z = rng.normal(size=(n, 1))
    y = rho * z + math.sqrt(1 - rho * rho) * rng.normal(size=(n, 1))
    mi, _, _ = _gpu(z, y, 3)
    assert abs(mi + 0.5 * math.log(1 - rho * rho)) < 0.05


def test_block_features_of_a_model():
    dims = dict(context=8, embed_dim=16, latent=64, hidden=64, blocks=2, branches=2, lr=1e-3, seed=4)
    b = 256
    m = edpc.Model(edpc.make_cfg(precision=edpc.EDPC_BF16, **dims), b)
    rng = np.random.default_rng(2)
    for _ in range(3):
        m.train_step(rng.integers(0, 256, size=(b, 8)).astype(np.uint8), rng.integers(0, 256, size=b).astype(np.uint8),
                     np.ones(b, np.uint8))
    m.forward(rng.integers(0, 256, size=(b, 8)).astype(np.uint8))
    for blk in range(2):
        s, so = m.block_io(blk)
        mi, cz, cy = _gpu(s, so, 3)
        _, oz, oy = ksg_counts(s, so, 3)
        assert np.array_equal(cz, oz) and np.array_equal(cy, oy)
    m.close()
