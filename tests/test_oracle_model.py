"""Pins for the oracle's model, adjoint and Adam (CPU only)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import softmax as sp_softmax
from scipy.stats import norm

from oracle.model import (ADAM_EPS, Config, Model, gelu, gelu_grad, param_layout,
                          softmax)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_cfg(**kw):
    base = dict(context=3, embed_dim=4, latent=6, hidden=5, blocks=2, branches=2, lr=1e-3, seed=17)
    base.update(kw)
    return Config(**base)


def _perm_matrix(n, perm):
    """M with M[j, perm[j]] = 1."""
    M = np.zeros((n, n))
    M[np.arange(n), perm] = 1.0
    return M


# ---- forward: special cases with closed forms -------------------------------------

def test_forward_orientation_with_permutations():
    """Identity MBRBs and permutation LTE/FDM weights make z a known shuffle of h0.

    With non-involutive permutations, any transposed operand (W vs W^T, x'U vs
    Ux'), any wrong embedding order, or a residual that skips X changes z.
    """
    cfg = small_cfg(context=2, embed_dim=4, latent=8, hidden=4, blocks=2)
    F = cfg.F
    m = Model(cfg, streams=3)
    for j in range(cfg.blocks):
        m.P[f"blk{j}.Wo"][:] = 0.0
        m.P[f"blk{j}.co"][:] = 0.0
    p1 = np.array([1, 2, 3, 4, 5, 6, 7, 0])
    p2 = np.array([3, 0, 6, 1, 7, 2, 4, 5])
    p3 = np.array([5, 3, 0, 7, 1, 6, 2, 4])
    m.P["lte.W1"][:] = _perm_matrix(F, p1)      # X'[j] = X[p1[j]]
    m.P["lte.b1"][:] = 0
    U = np.zeros((F, F))
    U[np.arange(F), p2] = 1.0                   # y[p2[i]] = x'[i]
    m.U[:] = U
    m.P["lte.W2"][:] = _perm_matrix(F, p3)      # X''[j] = y[p3[j]]
    m.P["lte.b2"][:] = 0
    m.P["head.W"][:] = 0
    m.P["head.W"][:F, :] = np.eye(F)
    m.P["head.b"][:] = 0
    ctx = np.array([[7, 200], [0, 255], [31, 31]])
    z, _ = m.forward(ctx)
    inv2 = np.argsort(p2)
    for s in range(3):
        h0 = np.concatenate([m.P["E"][ctx[s, 0]], m.P["E"][ctx[s, 1]]])
        xp = h0[p1]
        y = np.empty(F)
        y[p2] = xp
        want = y[p3]
        assert np.array_equal(z[s, :F], want)
        assert np.all(z[s, F:] == 0)
        # the same map written as one index chain
        assert np.array_equal(want, h0[p1[inv2[p3]]])


def test_mbrb_identity_and_residual():
    cfg = small_cfg()
    m = Model(cfg, 2)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(2, cfg.F))
    m.P["blk0.Wo"][:] = 0
    m.P["blk0.co"][:] = 0
    cache = {"blocks": [None] * cfg.blocks}
    assert np.array_equal(m._mbrb_fwd(0, X, cache), X)


def test_mbrb_layernorm_is_per_row_affine_invariant():
    cfg = small_cfg(hidden=7)
    m = Model(cfg, 2)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(4, cfg.F)) * 3
    a = np.array([[0.5], [2.0], [7.0], [1.3]])
    c = np.array([[1.0], [-4.0], [0.25], [10.0]])
    cache = {"blocks": [None] * cfg.blocks}
    d1 = m._mbrb_fwd(0, X, cache) - X
    Y = a * X + c
    d2 = m._mbrb_fwd(0, Y, cache) - Y
    np.testing.assert_allclose(d1, d2, rtol=0, atol=1e-5)
    xhat = cache["blocks"][0]["xhat"]
    np.testing.assert_allclose(xhat.mean(1), 0, atol=1e-12)
    v = Y.var(1)
    np.testing.assert_allclose(xhat.var(1), v / (v + 1e-5), rtol=1e-12)


def test_mbrb_branch_product_reduces_to_single_path():
    """W_2 = 0, c_2 = s makes X_fused = s * X_1; s = 0 leaves only co."""
    cfg = small_cfg()
    m = Model(cfg, 2)
    H = cfg.hidden
    rng = np.random.default_rng(2)
    X = rng.normal(size=(3, cfg.F))
    m.P["blk0.W"][H:, :] = 0
    m.P["blk0.c"][H:] = 0.0
    cache = {"blocks": [None] * cfg.blocks}
    out0 = m._mbrb_fwd(0, X, cache)
    np.testing.assert_array_equal(out0, X + m.P["blk0.co"])
    m.P["blk0.c"][H:] = 1.0
    out1 = m._mbrb_fwd(0, X, cache)
    x1 = cache["blocks"][0]["Xs"][0]
    # single-path FFN: GELU(X1) Wo^T + co + X, GELU as x * Phi(x)
    want = (x1 * norm.cdf(x1)) @ m.P["blk0.Wo"].T + m.P["blk0.co"] + X
    np.testing.assert_allclose(out1, want, rtol=1e-12, atol=1e-12)


def test_gelu_against_normal_cdf():
    x = np.linspace(-8, 8, 1001)
    np.testing.assert_allclose(gelu(x), x * norm.cdf(x), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gelu_grad(x), norm.cdf(x) + x * norm.pdf(x), rtol=1e-12, atol=1e-14)


def test_softmax_against_scipy():
    z = np.random.default_rng(3).normal(size=(5, 256)) * 10
    np.testing.assert_allclose(softmax(z), sp_softmax(z, axis=1), rtol=1e-12)


def test_fdm_is_per_stream():
    cfg = small_cfg()
    m = Model(cfg, 4)
    ctx = np.random.default_rng(4).integers(0, 256, size=(4, cfg.context))
    z0, _ = m.forward(ctx)
    m.U[2] += 0.3
    z1, _ = m.forward(ctx)
    changed = np.any(z0 != z1, axis=1)
    assert list(changed) == [False, False, True, False]


def test_forward_on_row_subset_matches_full():
    cfg = small_cfg()
    m = Model(cfg, 5)
    ctx = np.random.default_rng(5).integers(0, 256, size=(5, cfg.context))
    z, _ = m.forward(ctx)
    zs, _ = m.forward(ctx[[1, 4]], rows=[1, 4])
    np.testing.assert_array_equal(zs, z[[1, 4]])


# ---- paper numbers that fix the LTE / FDM reading -----------------------------------

def test_lte_flop_reduction_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))["lte_flop_reduction_pct"]
    F = 256
    cfg = Config(context=16, embed_dim=16, latent=F // g["r"], hidden=128, blocks=2)
    shapes = {n: s for n, s, _ in param_layout(cfg)}
    Fp = cfg.latent
    with_lte = shapes["lte.W1"][0] * shapes["lte.W1"][1] + Fp * Fp + shapes["lte.W2"][0] * shapes["lte.W2"][1]
    without = F * F  # per-instance F x F FDM, no projection
    red = 100 * (1 - with_lte / without)
    assert abs(red - g["value"]) < 0.02


def test_without_lte_orientation_with_permutations():
    """w/o LTE: with identity MBRBs and a permutation FDM, z is h0 shuffled by
    the FDM alone (no projection touches it), so y = x U fixes the orientation."""
    cfg = small_cfg(context=2, embed_dim=4, latent=0, hidden=4, blocks=2)
    F = cfg.F
    m = Model(cfg, streams=2)
    assert m.U.shape == (2, F, F) and not any(n.startswith("lte.") for n, _, _ in m.layout)
    for j in range(cfg.blocks):
        m.P[f"blk{j}.Wo"][:] = 0.0
        m.P[f"blk{j}.co"][:] = 0.0
    p2 = np.array([3, 0, 6, 1, 7, 2, 4, 5])
    U = np.zeros((F, F))
    U[np.arange(F), p2] = 1.0                   # y[p2[i]] = x[i]
    m.U[:] = U
    m.U[1] = 2.0 * U                            # the second stream's FDM is its own
    m.P["head.W"][:] = 0
    m.P["head.W"][:F, :] = np.eye(F)
    m.P["head.b"][:] = 0
    ctx = np.array([[7, 200], [0, 255]])
    z, _ = m.forward(ctx)
    for s in range(2):
        h0 = m.P["E"][ctx[s]].reshape(F)
        y = np.zeros(F)
        y[p2] = h0
        assert np.allclose(z[s, :F], (1.0 + s) * y, atol=1e-12)


def test_without_lte_parameter_gap_matches_table4():
    """The oracle's two models differ by b (F^2 - F'^2) FDM entries less the LTE's
    own 2 F F' + F' + F; Table 4 prints 2.93e8 vs 4.15e7 at batch 4096 (F = 256,
    F' = 64 inferred)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))["table4_params"]
    b = g["batch"]
    kw = dict(context=16, embed_dim=16, hidden=128, blocks=2)
    count = lambda cfg: sum(int(np.prod(sh)) for _, sh, _ in param_layout(cfg)) + b * cfg.fdm_dim ** 2  # noqa: E731
    gap = count(Config(latent=0, **kw)) - count(Config(latent=64, **kw))
    assert gap == b * (256 * 256 - 64 * 64) - (2 * 256 * 64 + 64 + 256)
    printed = g["without_lte"] - g["edpc"]
    assert abs(gap - printed) / printed < 0.005


def test_table4_parameter_gap_is_per_stream_fdm():
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))["table4_params"]
    F, Fp, b = 256, 64, g["batch"]
    gap = b * (F * F - Fp * Fp)
    printed = g["without_lte"] - g["edpc"]
    # printed to 3 significant digits
    assert abs(gap - printed) / printed < 0.005


# ---- adjoint vs central finite differences -------------------------------------------

def _fd_check(m, ctx, targets, rows, n_coords=25, h=1e-5, seed=0):
    p, g, dU, _ = m.grad_step(ctx, targets, rows)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for name, shape, _ in m.layout:
        flat = m.P[name].reshape(-1)
        gflat = g[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(n_coords, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = m.loss(ctx, targets, rows)
            flat[i] = old - h
            lm = m.loss(ctx, targets, rows)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            err = abs(fd - gflat[i]) / max(1e-6, abs(fd) + abs(gflat[i]))
            worst = max(worst, err if abs(fd - gflat[i]) > 1e-9 else 0.0)
    for r_, s in enumerate(rows):
        for _ in range(8):
            i, j = rng.integers(0, m.cfg.fdm_dim, size=2)
            old = m.U[s, i, j]
            m.U[s, i, j] = old + h
            lp = m.loss(ctx, targets, rows)
            m.U[s, i, j] = old - h
            lm = m.loss(ctx, targets, rows)
            m.U[s, i, j] = old
            fd = (lp - lm) / (2 * h)
            err = abs(fd - dU[r_, i, j]) / max(1e-6, abs(fd) + abs(dU[r_, i, j]))
            worst = max(worst, err if abs(fd - dU[r_, i, j]) > 1e-9 else 0.0)
    return worst


@pytest.mark.parametrize("branches,blocks,latent", [(2, 2, 6), (3, 2, 6), (2, 4, 6), (1, 3, 6), (2, 2, 0), (3, 3, 0)])
def test_adjoint_matches_finite_differences(branches, blocks, latent):
    # latent = 0: the "w/o LTE" variant (per-stream F x F FDM, no projections)
    cfg = small_cfg(branches=branches, blocks=blocks, latent=latent)
    m = Model(cfg, 4)
    rng = np.random.default_rng(branches * 10 + blocks)
    # move away from the initial point so LN gamma/beta and Adam state are generic
    for _ in range(3):
        ctx = rng.integers(0, 256, size=(4, cfg.context))
        tg = rng.integers(0, 256, size=4)
        _, g, dU, _ = m.grad_step(ctx, tg)
        m.adam(g, dU)
    for name in m.P:
        m.P[name] = m.P[name] + rng.normal(scale=0.05, size=m.P[name].shape)
    rows = np.array([0, 2, 3])
    ctx = rng.integers(0, 256, size=(3, cfg.context))
    ctx[1, 0] = ctx[0, 1]  # a repeated byte exercises the embedding scatter-add
    tg = rng.integers(0, 256, size=3)
    assert _fd_check(m, ctx, tg, rows) < 1e-5


# ---- Adam closed forms ------------------------------------------------------------------

def test_adam_first_steps_closed_form():
    cfg = small_cfg()
    m = Model(cfg, 3)
    rng = np.random.default_rng(6)
    g = {k: rng.normal(size=v.shape) for k, v in m.P.items()}
    dU = rng.normal(size=(2,) + m.U.shape[1:])
    p0 = {k: v.copy() for k, v in m.P.items()}
    U0 = m.U.copy()
    m.adam(g, dU, rows=[0, 2])
    # Step 1 with bias correction: m_hat = g, v_hat = g^2.
    for k in m.P:
        np.testing.assert_allclose(m.P[k], p0[k] - cfg.lr * g[k] / (np.abs(g[k]) + ADAM_EPS), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m.U[[0, 2]], U0[[0, 2]] - cfg.lr * dU / (np.abs(dU) + ADAM_EPS), atol=1e-15)
    # The inactive stream's FDM and moments are untouched.
    assert np.array_equal(m.U[1], U0[1]) and not m.mU[1].any() and not m.vU[1].any()
    # Step 2 with the same gradient: m_hat = g, v_hat = g^2 again.
    p1 = {k: v.copy() for k, v in m.P.items()}
    m.adam(g, dU, rows=[0, 2])
    for k in m.P:
        np.testing.assert_allclose(m.P[k], p1[k] - cfg.lr * g[k] / (np.abs(g[k]) + ADAM_EPS), rtol=0, atol=1e-14)


def test_flat_layout_roundtrip():
    cfg = small_cfg()
    m = Model(cfg, 2)
    v = m.flat()
    total = sum(math.prod(s) for _, s, _ in m.layout)
    assert v.size == total
    m2 = Model(small_cfg(seed=99), 2)
    m2.set_flat(v)
    assert np.array_equal(m2.flat(), v)
