"""The 1 GiB workload's model at its full launch size (needs a GPU).

4096 streams, K = 64, D = 16 (F = 1024), F' = 512, 6 MBRBs of hidden 512, two
branches: the state is 10.8 M shared parameters plus 4096 FDMs of 512 x 512
(12.9 GB of FP32 state with the Adam moments). The oracle cannot hold 4096
FP64 FDMs in a test, so the checks sample streams:

  * forward: every stream's logits depend only on its own context and FDM, so
    sampled streams' logits are compared with the oracle's one by one;
  * adjoint: with only the sampled streams active, the shared gradient is the
    mean over those streams alone (Q11/Q12 masking), which the oracle computes
    exactly; the sampled FDM gradients are compared and every inactive
    stream's FDM gradient must be exactly zero;
  * round trip: a 4096-stream prefix of the mix through compress/decompress.

Tolerances as in the other parity tests: FP32 logits 1e-4 of max |z|,
gradients 1e-3 per tensor; BF16 3e-2 and 6e-2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.model import Config, Model as OModel, softmax  # noqa: E402

pytestmark = pytest.mark.gpu

DIMS = dict(context=64, embed_dim=16, latent=512, hidden=512, blocks=6, branches=2, lr=1e-3, seed=3)
B = 4096


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


@pytest.mark.parametrize("prec,tz,tg", [(edpc.EDPC_FP32, 1e-4, 1e-3), (edpc.EDPC_BF16, 3e-2, 6e-2)],
                         ids=["fp32", "bf16"])
def test_full_launch_sampled_streams_against_oracle(prec, tz, tg):
    c = edpc.make_cfg(precision=prec, **DIMS)
    o = Config(**DIMS)
    K, Fp = o.context, o.latent
    m = edpc.Model(c, B)
    rng = np.random.default_rng(41)
    # one update of every stream moves all tensors off their initial values
    m.train_step(rng.integers(0, 256, size=(B, K)).astype(np.uint8),
                 rng.integers(0, 256, size=B).astype(np.uint8), np.ones(B, np.uint8))
    st = m.get_state(which=("P", "U"))
    assert st["t"] == 1
    sample = np.unique(np.concatenate([[0, 1, B // 2 - 1, B - 1], rng.choice(B, size=6, replace=False)]))
    U = st["U"].reshape(B, Fp, Fp)
    om = OModel(o, len(sample))
    om.set_flat(st["P"].astype(np.float64))
    om.U = U[sample].astype(np.float64)
    del st, U

    ctx = rng.integers(0, 256, size=(B, K)).astype(np.uint8)
    z, _ = m.forward(ctx)
    zo, cache = om.forward(ctx[sample].astype(np.int64))
    assert np.abs(z[sample] - zo).max() <= tz * np.abs(zo).max()

    tgt = rng.integers(0, 256, size=B).astype(np.uint8)
    active = np.zeros(B, np.uint8)
    active[sample] = 1
    g, gu = m.backward(ctx, tgt, active)
    po = softmax(zo)
    dz = po.copy()
    dz[np.arange(len(sample)), tgt[sample]] -= 1
    dz /= len(sample)
    go, dUo = om.backward(cache, dz)
    gf = OModel.flat_grads(om.layout, go)
    off = 0
    for name, shape, _ in om.layout:
        n = int(np.prod(shape))
        ref = gf[off:off + n]
        if np.linalg.norm(ref) > 1e-12:
            assert _rel(g[off:off + n], ref) <= tg, (name, _rel(g[off:off + n], ref))
        off += n
    gu = gu.reshape(B, Fp * Fp)
    assert _rel(gu[sample].reshape(-1, Fp, Fp), dUo) <= tg
    inactive = np.ones(B, bool)
    inactive[sample] = False
    assert not np.any(gu[inactive])
    m.close()


def test_prefix_roundtrip_bf16():
    """The first 160 bytes of each of 4096 streams of the multimedia mix (640 KiB)
    through the full-size model: 96 coded model steps after the 64-byte prefix."""
    x = synth.multimedia_mix(B * 160, 20250723)
    c = edpc.make_cfg(streams=B, precision=edpc.EDPC_BF16, **DIMS)
    bits = edpc.compress(x, c)
    _, n, b = edpc.peek(bits)
    assert (n, b) == (x.size, B)
    assert np.array_equal(edpc.decompress(bits), x)
