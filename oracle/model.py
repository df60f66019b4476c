"""FP64 probability model, its analytic adjoint, and Adam (oracle side).

Model(x_{i-t..i-1}) of Algorithm 1 (Sec. 2.1, Eq. 1), as read from Sec. 3:

  h0     = concat_k E[x_{i-K+k}], k = 0..K-1 (oldest byte first)       [embedding]
  X      = MBRB_j(X) for the n//2 "Local" blocks                       [Sec. 3.1.2]
  X'     = X W1^T + b1                                  (Eq. 14)       [LTE down]
  y_s    = x'_s U_s, per stream s                       (Eq. 15)       [FDM, bmm]
  X      = Y W2^T + b2                                  (Eq. 16)       [LTE up]
  X      = MBRB_j(X) for the n - n//2 "Global" blocks                  [Sec. 3.1.2]
  z      = X Wh^T + bh;   p = softmax(z)                               [256-way head]

  MBRB (Eqs. 9-13): X0 = LN(X); X_i = X0 W_i^T + c_i (i = 1..k);
  Xf = X_1 * ... * X_k; G = GELU(Xf); out = G Wo^T + co + X.

  Variant "w/o LTE" (ablation of Table 4 and Sec. 4.4.3; latent = 0): no
  projections; the per-stream FDM is F x F and acts on X itself,
  y_s = x_s U_s and X = Y. Its parameter count exceeds the LTE model's by
  b (F^2 - F'^2) - (2 F F' + F' + F), the reading of Table 4's gap.

Readings where the paper is silent or ambiguous:
  * Layer order (Fig. 3 is missing): embedding, Local MBRBs, LTE, Global
    MBRBs, head. There is no residual around the LTE and no final norm.
  * The byte embedding is a 256 x D table, concatenated over the K context
    bytes, so F = K * D.
  * Eq. 14 writes W1 X with X in R^{b x F}; read as X' = X W1^T + b1 (and
    Eq. 16 likewise). Eq. 15's bmm(X', U) is read as y_s = x'_s U_s with
    x'_s a row vector, so y_s[j] = sum_i x'_s[i] U_s[i, j].
  * LN: biased variance, eps = 1e-5, affine gamma = 1, beta = 0 at start.
  * GELU: the exact erf form.
  * Loss: mean cross-entropy over the streams active at this step.
  * Adam (Sec. 4.1, lr 1e-3): beta = (0.9, 0.999), eps = 1e-8, bias
    correction, no weight decay, no clipping. One global step counter.
    A stream that is not active at a step leaves its FDM and the FDM's
    moments unchanged.
  * Initial values: uniform, from the counter-based rule in ``rng``.
    Linear weights and biases use bound 1/sqrt(fan_in). E uses sqrt(3)
    (unit variance). U uses sqrt(3/F') (variance 1/F'). LN gamma = 1, beta = 0.

Parity: forward pinned by special cases that reduce to library routines
(tests/test_oracle_model.py): permutation weights fix the orientation of
each Linear and of the bmm; LN against its moments; GELU against the
normal CDF; softmax against scipy; stream independence of the FDM.
The adjoint is pinned by FP64 central finite differences. Adam is pinned by
its closed-form first and second steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf

from .rng import init_values

LN_EPS = 1e-5
ADAM_B1 = 0.9
ADAM_B2 = 0.999
ADAM_EPS = 1e-8
FDM_TID = 1023
SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


@dataclass(frozen=True)
class Config:
    context: int = 16      # K: history bytes (t in Algorithm 1)
    embed_dim: int = 16    # D
    latent: int = 128      # F' = F / r; 0: no LTE (the FDM is F x F, Table 4's "w/o LTE")
    hidden: int = 128      # H: MBRB branch width
    blocks: int = 2        # n: Local blocks n//2, Global blocks n - n//2
    branches: int = 2      # k: MBRB branches
    lr: float = 1e-3
    seed: int = 0

    @property
    def F(self) -> int:
        return self.context * self.embed_dim

    @property
    def n_local(self) -> int:
        return self.blocks // 2

    @property
    def lte(self) -> bool:
        return self.latent > 0

    @property
    def fdm_dim(self) -> int:
        # side of each stream's FDM: F' with the LTE, F without it
        return self.latent if self.lte else self.F


def param_layout(cfg: Config):
    """Canonical order of the shared parameters: list of (name, shape, init).

    init is ("uniform", bound) or ("const", value). The tensor id used by
    the initial-value rule is the position in this list. This order is also
    the flat layout exchanged with the library's state export.
    """
    F, H, Fp, D, k = cfg.F, cfg.hidden, cfg.latent, cfg.embed_dim, cfg.branches
    inv = lambda n: 1.0 / math.sqrt(float(n))  # noqa: E731
    out = [("E", (256, D), ("uniform", math.sqrt(3.0)))]
    for j in range(cfg.blocks):
        out += [
            (f"blk{j}.ln_g", (F,), ("const", 1.0)),
            (f"blk{j}.ln_b", (F,), ("const", 0.0)),
            (f"blk{j}.W", (k * H, F), ("uniform", inv(F))),
            (f"blk{j}.c", (k * H,), ("uniform", inv(F))),
            (f"blk{j}.Wo", (F, H), ("uniform", inv(H))),
            (f"blk{j}.co", (F,), ("uniform", inv(H))),
        ]
    if cfg.lte:
        out += [
            ("lte.W1", (Fp, F), ("uniform", inv(F))),
            ("lte.b1", (Fp,), ("uniform", inv(F))),
            ("lte.W2", (F, Fp), ("uniform", inv(Fp))),
            ("lte.b2", (F,), ("uniform", inv(Fp))),
        ]
    out += [
        ("head.W", (256, F), ("uniform", inv(F))),
        ("head.b", (256,), ("uniform", inv(F))),
    ]
    return out


def fdm_bound(cfg: Config) -> float:
    return math.sqrt(3.0 / float(cfg.fdm_dim))


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def softmax(z):
    z = z - z.max(axis=-1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=-1, keepdims=True)


class Model:
    """Parameters, FDM, Adam state, and the forward/adjoint of one step."""

    def __init__(self, cfg: Config, streams: int):
        self.cfg = cfg
        self.b = streams
        self.layout = param_layout(cfg)
        self.P = {}
        for tid, (name, shape, (kind, val)) in enumerate(self.layout):
            size = int(np.prod(shape))
            if kind == "const":
                self.P[name] = np.full(shape, float(val))
            else:
                self.P[name] = init_values(cfg.seed, tid, size, val).reshape(shape)
        Fp = cfg.fdm_dim
        self.U = init_values(cfg.seed, FDM_TID, streams * Fp * Fp, fdm_bound(cfg)).reshape(streams, Fp, Fp)
        self.m = {k: np.zeros_like(v) for k, v in self.P.items()}
        self.v = {k: np.zeros_like(v) for k, v in self.P.items()}
        self.mU = np.zeros_like(self.U)
        self.vU = np.zeros_like(self.U)
        self.t = 0

    # ---- canonical flat layout -------------------------------------------------
    def flat(self, which: str = "P") -> np.ndarray:
        d = {"P": self.P, "m": self.m, "v": self.v}[which]
        return np.concatenate([d[name].ravel() for name, _, _ in self.layout])

    def set_flat(self, vec: np.ndarray, which: str = "P") -> None:
        d = {"P": self.P, "m": self.m, "v": self.v}[which]
        o = 0
        for name, shape, _ in self.layout:
            n = int(np.prod(shape))
            d[name] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(shape).copy()
            o += n
        assert o == vec.size

    @staticmethod
    def flat_grads(layout, grads) -> np.ndarray:
        return np.concatenate([grads[name].ravel() for name, _, _ in layout])

    # ---- forward -----------------------------------------------------------------
    def _mbrb_fwd(self, j, X, cache):
        P, H, k = self.P, self.cfg.hidden, self.cfg.branches
        mu = X.mean(axis=1, keepdims=True)
        var = ((X - mu) ** 2).mean(axis=1, keepdims=True)
        rstd = 1.0 / np.sqrt(var + LN_EPS)
        xhat = (X - mu) * rstd
        X0 = xhat * P[f"blk{j}.ln_g"] + P[f"blk{j}.ln_b"]          # Eq. 9
        A = X0 @ P[f"blk{j}.W"].T + P[f"blk{j}.c"]                 # Eq. 10, all k paths
        Xs = [A[:, i * H:(i + 1) * H] for i in range(k)]
        Xf = Xs[0].copy()
        for i in range(1, k):
            Xf = Xf * Xs[i]                                        # Eq. 11
        G = gelu(Xf)                                               # Eq. 12
        out = G @ P[f"blk{j}.Wo"].T + P[f"blk{j}.co"] + X          # Eq. 13
        cache["blocks"][j] = dict(xhat=xhat, rstd=rstd, X0=X0, Xs=Xs, Xf=Xf, G=G)
        return out

    def forward(self, ctx: np.ndarray, rows=None):
        """Logits z (len(rows), 256) for contexts ``ctx`` (len(rows), K) of streams ``rows``."""
        cfg, P = self.cfg, self.P
        rows = np.arange(self.b) if rows is None else np.asarray(rows)
        ctx = np.asarray(ctx, dtype=np.int64)
        b = ctx.shape[0]
        cache = {"ctx": ctx, "rows": rows, "blocks": [None] * cfg.blocks}
        X = P["E"][ctx].reshape(b, cfg.F)
        for j in range(cfg.n_local):
            X = self._mbrb_fwd(j, X, cache)
        cache["lte_in"] = X
        Xp = X @ P["lte.W1"].T + P["lte.b1"] if cfg.lte else X     # Eq. 14 (w/o LTE: X itself)
        Us = self.U[rows]
        Y = np.matmul(Xp[:, None, :], Us)[:, 0, :]                 # Eq. 15
        cache["Xp"], cache["Y"], cache["Us"] = Xp, Y, Us
        X = Y @ P["lte.W2"].T + P["lte.b2"] if cfg.lte else Y      # Eq. 16 (w/o LTE: Y itself)
        for j in range(cfg.n_local, cfg.blocks):
            X = self._mbrb_fwd(j, X, cache)
        cache["head_in"] = X
        z = X @ P["head.W"].T + P["head.b"]
        return z, cache

    # ---- adjoint -----------------------------------------------------------------
    def _mbrb_bwd(self, j, dOut, cache, g):
        P, k = self.P, self.cfg.branches
        c = cache["blocks"][j]
        g[f"blk{j}.Wo"] = dOut.T @ c["G"]
        g[f"blk{j}.co"] = dOut.sum(axis=0)
        dG = dOut @ P[f"blk{j}.Wo"]
        dXf = dG * gelu_grad(c["Xf"])
        parts = []
        for i in range(k):
            other = np.ones_like(dXf)
            for l2 in range(k):
                if l2 != i:
                    other = other * c["Xs"][l2]
            parts.append(dXf * other)
        dA = np.concatenate(parts, axis=1)
        g[f"blk{j}.W"] = dA.T @ c["X0"]
        g[f"blk{j}.c"] = dA.sum(axis=0)
        dX0 = dA @ P[f"blk{j}.W"]
        g[f"blk{j}.ln_g"] = (dX0 * c["xhat"]).sum(axis=0)
        g[f"blk{j}.ln_b"] = dX0.sum(axis=0)
        dxh = dX0 * P[f"blk{j}.ln_g"]
        dX = c["rstd"] * (dxh - dxh.mean(axis=1, keepdims=True)
                          - c["xhat"] * (dxh * c["xhat"]).mean(axis=1, keepdims=True))
        return dOut + dX

    def backward(self, cache, dz):
        """Gradients of sum_s dz[s] . z[s] w.r.t. all parameters.

        Returns (grads by name, dU for the FDMs of ``cache['rows']``).
        """
        cfg, P = self.cfg, self.P
        g = {}
        g["head.W"] = dz.T @ cache["head_in"]
        g["head.b"] = dz.sum(axis=0)
        dX = dz @ P["head.W"]
        for j in reversed(range(cfg.n_local, cfg.blocks)):
            dX = self._mbrb_bwd(j, dX, cache, g)
        if cfg.lte:
            g["lte.W2"] = dX.T @ cache["Y"]
            g["lte.b2"] = dX.sum(axis=0)
            dY = dX @ P["lte.W2"]
        else:
            dY = dX
        dU = cache["Xp"][:, :, None] * dY[:, None, :]
        dXp = np.matmul(cache["Us"], dY[:, :, None])[:, :, 0]
        if cfg.lte:
            g["lte.W1"] = dXp.T @ cache["lte_in"]
            g["lte.b1"] = dXp.sum(axis=0)
            dX = dXp @ P["lte.W1"]
        else:
            dX = dXp
        for j in reversed(range(cfg.n_local)):
            dX = self._mbrb_bwd(j, dX, cache, g)
        dh = dX.reshape(dX.shape[0], cfg.context, cfg.embed_dim)
        dE = np.zeros_like(P["E"])
        np.add.at(dE, cache["ctx"], dh)
        g["E"] = dE
        return g, dU

    # ---- loss, gradient of one step ------------------------------------------------
    def loss(self, ctx, targets, rows=None) -> float:
        z, _ = self.forward(ctx, rows)
        p = softmax(z)
        return float(-np.log(p[np.arange(len(targets)), targets]).mean())

    def grad_step(self, ctx, targets, rows=None):
        """Probabilities and gradients of the mean cross-entropy (Eq. 2)."""
        z, cache = self.forward(ctx, rows)
        p = softmax(z)
        dz = p.copy()
        dz[np.arange(len(targets)), targets] -= 1.0
        dz /= len(targets)
        g, dU = self.backward(cache, dz)
        return p, g, dU, cache

    # ---- Adam ----------------------------------------------------------------------
    def adam(self, grads, dU, rows=None):
        """One Adam step on all shared parameters and on the FDMs of ``rows``."""
        cfg = self.cfg
        self.t += 1
        bc1 = 1.0 - ADAM_B1 ** self.t
        bc2 = 1.0 - ADAM_B2 ** self.t
        for name, _, _ in self.layout:
            gr = grads[name]
            m = self.m[name] = ADAM_B1 * self.m[name] + (1.0 - ADAM_B1) * gr
            v = self.v[name] = ADAM_B2 * self.v[name] + (1.0 - ADAM_B2) * gr * gr
            self.P[name] = self.P[name] - cfg.lr * (m / bc1) / (np.sqrt(v / bc2) + ADAM_EPS)
        rows = np.arange(self.b) if rows is None else np.asarray(rows)
        mU = ADAM_B1 * self.mU[rows] + (1.0 - ADAM_B1) * dU
        vU = ADAM_B2 * self.vU[rows] + (1.0 - ADAM_B2) * dU * dU
        self.U[rows] = self.U[rows] - cfg.lr * (mU / bc1) / (np.sqrt(vU / bc2) + ADAM_EPS)
        self.mU[rows] = mU
        self.vU[rows] = vU
