"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

Exactness where the computation is integer (quantizer given the same FP32 p,
range coder given the same symbols, initial values); float tolerances where
it is floating point:
  * FP32 forward logits: max |dz| <= 1e-4 * max |z| (FP32 sums of <= 2048 terms).
  * FP32 gradients: per tensor ||g - g_ref|| <= 1e-3 ||g_ref|| (the benchmark spec's bound).
  * BF16 (8-bit mantissa operands, FP32 accumulation): logits within 3e-2
    relative; gradients within 6e-2 relative per tensor.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402
from oracle.coder import RangeEncoder, quantize_cdf  # noqa: E402
from oracle.compress import oracle_compress  # noqa: E402
from oracle.model import ADAM_B1, ADAM_B2, ADAM_EPS, Config, Model as OModel, softmax  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cfgs(**kw):
    keys = ("context", "embed_dim", "latent", "hidden", "blocks", "branches", "lr", "seed")
    o = Config(**{k: kw[k] for k in keys if k in kw})
    c = edpc.make_cfg(**kw)
    return c, o


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


# ---- integer-exact kernels ---------------------------------------------------------------

def test_cdf_quantize_exact():
    rng = np.random.default_rng(0)
    p = np.concatenate([
        rng.dirichlet(np.full(256, 0.05), size=300),
        rng.dirichlet(np.full(256, 3.0), size=300),
        softmax(rng.normal(size=(300, 256)) * 6),
        np.eye(256)[:50],
        np.full((5, 256), 1 / 256),
    ]).astype(np.float32)
    rows = p.shape[0]
    pd = torch.from_numpy(p).cuda()
    fd = torch.empty((rows, 256), dtype=torch.int32, device="cuda")
    cd = torch.empty((rows, 257), dtype=torch.int32, device="cuda")
    edpc.cdf_quantize(pd.data_ptr(), rows, fd.data_ptr(), cd.data_ptr())
    f, cum = quantize_cdf(p)
    assert np.array_equal(fd.cpu().numpy().astype(np.int64), f)
    assert np.array_equal(cd.cpu().numpy().astype(np.int64), cum)


@pytest.mark.parametrize("streams,nsym", [(1, 1), (37, 500), (256, 3000)])
def test_range_encode_exact(streams, nsym):
    rng = np.random.default_rng(streams)
    sym = np.empty((nsym, streams), dtype=np.uint32)
    pairs = [[] for _ in range(streams)]
    for t in range(nsym):
        p = rng.dirichlet(np.full(256, 0.03), size=streams).astype(np.float32)
        f, cum = quantize_cdf(p)
        for s in range(streams):
            if rng.random() < 0.05:
                sym[t, s] = 0xFFFFFFFF
                continue
            # mostly likely symbols, sometimes the top of the CDF (carry paths)
            x = int(np.argmax(f[s])) if rng.random() < 0.6 else int(rng.integers(0, 256))
            if rng.random() < 0.1:
                x = 255
            sym[t, s] = int(cum[s, x]) | ((int(f[s, x]) - 1) << 16)
            pairs[s].append((int(cum[s, x]), int(f[s, x])))
    cap = 2 * nsym + 64
    sd = torch.from_numpy(sym.view(np.int32)).cuda()
    out = torch.zeros(streams * cap, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(streams, dtype=torch.int32, device="cuda")
    edpc.range_encode(sd.data_ptr(), nsym, streams, out.data_ptr(), cap, ln.data_ptr())
    out = out.cpu().numpy()
    ln = ln.cpu().numpy()
    for s in range(streams):
        e = RangeEncoder()
        for c, f in pairs[s]:
            e.encode(c, f)
        ref = e.finish()
        got = bytes(out[s * cap:s * cap + ln[s]])
        assert got == ref, s


# ---- model: initial state, forward, adjoint, Adam ------------------------------------------

SMALL = dict(context=5, embed_dim=8, latent=72, hidden=40, blocks=3, branches=2, lr=1e-3, seed=11)


def test_initial_state_is_bit_identical():
    c, o = cfgs(**SMALL)
    b = 7
    m = edpc.Model(c, b)
    st = m.get_state()
    om = OModel(o, b)
    assert np.array_equal(st["P"], om.flat().astype(np.float32))
    assert np.array_equal(st["U"], om.U.reshape(-1).astype(np.float32))
    assert not st["M"].any() and not st["Uv"].any()


def _state_after_steps(m, om, b, K, steps, rng):
    for _ in range(steps):
        ctx = rng.integers(0, 256, size=(b, K)).astype(np.uint8)
        tg = rng.integers(0, 256, size=b).astype(np.uint8)
        m.train_step(ctx, tg, np.ones(b, np.uint8))
    st = m.get_state()
    om.set_flat(st["P"].astype(np.float64))
    om.U = st["U"].astype(np.float64).reshape(om.U.shape).copy()
    return st


@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("dims,b", [(SMALL, 7), (dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2,
                                                       branches=2, lr=1e-3, seed=1), 4),
                                    (dict(context=8, embed_dim=16, latent=136, hidden=200, blocks=2, branches=3,
                                          lr=1e-3, seed=5), 130)])
def test_forward_and_gradient_parity(prec, dims, b):
    c, o = cfgs(precision=prec, **dims)
    m = edpc.Model(c, b)
    om = OModel(o, b)
    rng = np.random.default_rng(b)
    _state_after_steps(m, om, b, o.context, 3, rng)
    ctx = rng.integers(0, 256, size=(b, o.context)).astype(np.uint8)
    ctx[1 % b, 0] = ctx[0, -1]
    z, p = m.forward(ctx)
    zo, cache = om.forward(ctx.astype(np.int64))
    tol_z = 1e-4 if prec == edpc.EDPC_FP32 else 3e-2
    assert np.abs(z - zo).max() <= tol_z * np.abs(zo).max()
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    active = np.ones(b, np.uint8)
    active[-1] = 0 if b > 2 else 1
    g, gu = m.backward(ctx, tg, active)
    rows = np.nonzero(active)[0]
    po = softmax(zo[rows])
    dz = po.copy()
    dz[np.arange(len(rows)), tg[rows]] -= 1
    dz /= len(rows)
    _, cache = om.forward(ctx[rows].astype(np.int64), rows)
    go, dUo = om.backward(cache, dz)
    tol = 1e-3 if prec == edpc.EDPC_FP32 else 6e-2
    o_flat = OModel.flat_grads(om.layout, go)
    off = 0
    for name, shape, _ in om.layout:
        n = int(np.prod(shape))
        ref = o_flat[off:off + n]
        if np.linalg.norm(ref) > 1e-12:
            assert _rel(g[off:off + n], ref) <= tol, (name, _rel(g[off:off + n], ref))
            if prec == edpc.EDPC_FP32:
                # element by element: |dg| <= 1e-3 max|g_ref| (+ a floor far below FP32 noise of O(1) terms)
                err = np.abs(g[off:off + n] - ref).max()
                assert err <= 1e-3 * np.abs(ref).max() + 1e-9, (name, err, np.abs(ref).max())
        off += n
    gu = gu.reshape(b, o.latent, o.latent)
    assert _rel(gu[rows], dUo) <= tol
    if prec == edpc.EDPC_FP32:
        assert np.abs(gu[rows] - dUo).max() <= 1e-3 * np.abs(dUo).max() + 1e-9
    assert not gu[active == 0].any()


def test_gradient_against_central_differences():
    """GPU FP32 adjoint vs FP64 central differences (h = 1e-4) of the oracle loss
    at the GPU's own state, on a 256-byte input (b = 4, K = 16: 48 model steps per
    stream have been taken when the check runs)."""
    dims = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=2)
    c, o = cfgs(**dims)
    b, K = 4, 16
    x = synth.markov_bytes(256, 1, 0.1, 3)
    m = edpc.Model(c, b)
    om = OModel(o, b)
    streams = x.reshape(b, 64)
    for i in range(K, 63):
        m.train_step(streams[:, i - K:i].copy(), streams[:, i].copy(), np.ones(b, np.uint8))
    st = m.get_state()
    om.set_flat(st["P"].astype(np.float64))
    om.U = st["U"].astype(np.float64).reshape(om.U.shape).copy()
    ctx = streams[:, 63 - K:63].copy()
    tg = streams[:, 63].copy()
    g, gu = m.backward(ctx, tg, np.ones(b, np.uint8))
    rng = np.random.default_rng(0)
    flat = om.flat()
    h = 1e-4
    idx = rng.choice(flat.size, size=300, replace=False)
    fd = np.empty(idx.size)
    for k, i in enumerate(idx):
        v = flat.copy()
        v[i] = flat[i] + h
        om.set_flat(v)
        lp = om.loss(ctx.astype(np.int64), tg.astype(np.int64))
        v[i] = flat[i] - h
        om.set_flat(v)
        lm = om.loss(ctx.astype(np.int64), tg.astype(np.int64))
        fd[k] = (lp - lm) / (2 * h)
    om.set_flat(flat)
    big = np.abs(fd) > 1e-5
    assert big.sum() > 50
    assert _rel(g[idx][big], fd[big]) <= 1e-3


@pytest.mark.parametrize("prec,flags", [(edpc.EDPC_FP32, 0), (edpc.EDPC_BF16, 0), (edpc.EDPC_FP8E4M3, 0),
                                        (edpc.EDPC_BF16, edpc.EDPC_FLAG_OVERLAP_FDM)],
                         ids=["fp32", "bf16", "fp8", "bf16-overlap"])
@pytest.mark.parametrize("dims", [SMALL, dict(SMALL, latent=128), dict(SMALL, latent=256, hidden=64)],
                         ids=["latent72", "latent128", "latent256"])
def test_adam_kernel_matches_closed_form_update(prec, flags, dims):
    """One Adam step of every parameter, the FDMs included (with the overlap flag
    the FDM update is the separate persistent kernel on its own stream), against
    the closed form applied to the gradient the library reports at the same state."""
    c, o = cfgs(precision=prec, flags=flags, **dims)
    b = 5
    m = edpc.Model(c, b)
    rng = np.random.default_rng(4)
    K = o.context
    for _ in range(2):
        m.train_step(rng.integers(0, 256, size=(b, K)).astype(np.uint8), rng.integers(0, 256, size=b).astype(np.uint8),
                     np.ones(b, np.uint8))
    before = m.get_state()
    ctx = rng.integers(0, 256, size=(b, K)).astype(np.uint8)
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    act = np.array([1, 0, 1, 1, 1], np.uint8)
    g, gu = m.backward(ctx, tg, act)
    m.train_step(ctx, tg, act)
    after = m.get_state()
    t = after["t"]
    bc1, bc2 = 1 - ADAM_B1 ** t, 1 - ADAM_B2 ** t

    def adam(p, mm, vv, gg):
        mm = ADAM_B1 * mm + (1 - ADAM_B1) * gg
        vv = ADAM_B2 * vv + (1 - ADAM_B2) * gg * gg
        return p - o.lr * (mm / bc1) / (np.sqrt(vv / bc2) + ADAM_EPS), mm, vv

    P, M, V = adam(before["P"].astype(np.float64), before["M"].astype(np.float64), before["V"].astype(np.float64),
                   g.astype(np.float64))
    np.testing.assert_allclose(after["P"], P, rtol=0, atol=2e-6)
    # The kernel holds beta1 and 1 - beta1 in FP32 (1 - 0.9f = 0.10000002), so
    # each term of m carries a relative error of a few FP32 ulps; bound the
    # error by the size of the terms, not of their (possibly cancelling) sum.
    scale = 0.9 * np.abs(before["M"].astype(np.float64)) + 0.1 * np.abs(g.astype(np.float64))
    assert np.all(np.abs(after["M"] - M) <= 4e-7 * scale + 1e-20)
    U, Um, Uv = adam(before["U"].astype(np.float64), before["Um"].astype(np.float64),
                     before["Uv"].astype(np.float64), gu.astype(np.float64))
    sh = (b, o.latent * o.latent)
    live = act.astype(bool)
    np.testing.assert_allclose(after["U"].reshape(sh)[live], U.reshape(sh)[live], rtol=0, atol=2e-6)
    assert np.array_equal(after["U"].reshape(sh)[~live], before["U"].reshape(sh)[~live])
    assert np.array_equal(after["Uv"].reshape(sh)[~live], before["Uv"].reshape(sh)[~live])


# ---- end to end -----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [edpc.EDPC_FP32, edpc.EDPC_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("n,b,K", [(0, 4, 4), (1, 4, 4), (7, 4, 4), (9, 3, 2), (1000, 7, 8), (4099, 16, 16),
                                   (20000, 64, 8)])
def test_roundtrip_edge_cases(prec, n, b, K):
    x = np.random.default_rng(n).integers(0, 256, size=n).astype(np.uint8)
    if n > 100:
        x[: n // 3] = synth.markov_bytes(n // 3, 1, 0.05, n)
    c = edpc.make_cfg(streams=b, context=K, embed_dim=8, latent=64, hidden=64, blocks=2, precision=prec, seed=9)
    bits = edpc.compress(x, c)
    y = edpc.decompress(bits)
    assert np.array_equal(x, y)


@pytest.mark.parametrize("flags", [0, edpc.EDPC_FLAG_NO_PIPELINE, edpc.EDPC_FLAG_NO_GRAPH])
def test_small_workload_matches_oracle_bits_per_byte(flags):
    g = json.load(open(os.path.join(GOLDEN, "oracle_c0.json")))
    tab = synth.markov_table(2, 0.1, g["data_seed"])
    x = synth.markov_bytes(g["n"], 2, 0.1, g["data_seed"], table=tab)
    assert bytes(x[:64]).hex() == g["input_sha_prefix"]
    c = edpc.make_cfg(streams=g["streams"], flags=flags, **g["cfg"])
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)
    _, n, b = edpc.peek(bits)
    payload = len(bits) - (88 + 4 * b + 4)
    bpb = 8 * payload / n
    # the FP32 GPU trajectory and the FP64 oracle's differ only by rounding
    assert abs(bpb - g["bits_per_byte"]) <= 0.005 * g["bits_per_byte"], (bpb, g["bits_per_byte"])


def test_pipeline_and_graph_do_not_change_the_bitstream():
    x = synth.markov_bytes(30000, 1, 0.05, 1)
    outs = []
    for flags in (0, edpc.EDPC_FLAG_NO_PIPELINE, edpc.EDPC_FLAG_NO_GRAPH):
        c = edpc.make_cfg(streams=8, context=8, embed_dim=8, latent=64, hidden=64, flags=flags)
        outs.append(edpc.compress(x, c))
    assert outs[0] == outs[1] == outs[2]


def test_session_steps_match_one_shot():
    x = synth.markov_bytes(40000, 1, 0.05, 2)
    c = edpc.make_cfg(streams=8, context=8, embed_dim=8, latent=64, hidden=64)
    one = edpc.compress(x, c)
    with edpc.Encoder(c, x) as e:
        total = e.remaining()
        done = 0
        for k in (1, 63, 64, 65, 200, 1):
            done += e.run(k, sync=bool(k % 2))
        assert e.remaining() == total - done
        assert e.finish() == one


def test_device_input_and_output():
    x = synth.markov_bytes(50000, 1, 0.05, 3)
    c = edpc.make_cfg(streams=16, context=8, embed_dim=8, latent=64, hidden=64, precision=edpc.EDPC_BF16)
    xd = torch.from_numpy(x).cuda()
    with edpc.Encoder(c, device_ptr=xd.data_ptr(), length=x.size) as e:
        bits = e.finish()
    assert bits == edpc.compress(x, c)
    yd = torch.zeros(x.size, dtype=torch.uint8, device="cuda")
    with edpc.Decoder(bits, out_device_ptr=yd.data_ptr()) as d:
        d.finish(to_host=False)
    assert np.array_equal(yd.cpu().numpy(), x)


def test_corruption_is_detected():
    x = synth.markov_bytes(20000, 1, 0.05, 4)
    c = edpc.make_cfg(streams=4, context=8, embed_dim=8, latent=64, hidden=64)
    bits = bytearray(edpc.compress(x, c))
    hdr = 88 + 4 * 4 + 4
    bad = bytearray(bits)
    bad[hdr + 100] ^= 0x10
    with pytest.raises(edpc.EdpcError) as e:
        edpc.decompress(bytes(bad))
    assert e.value.code == 3
    with pytest.raises(edpc.EdpcError) as e:
        edpc.decompress(bytes(bits[:-3]))
    assert e.value.code == 3
    bad = bytearray(bits)
    bad[20] ^= 1
    with pytest.raises(edpc.EdpcError) as e:
        edpc.decompress(bytes(bad))
    assert e.value.code == 3


def test_large_config_dims_sampled_against_oracle():
    """The 64 MiB multimedia configuration's model (512 streams, K = 32, F' = 256,
    4 MBRBs of hidden 256) in BF16 and FP32 at one state: all logits and the
    gradients of every shared tensor, against the FP64 oracle."""
    dims = dict(context=32, embed_dim=16, latent=256, hidden=256, blocks=4, branches=2, lr=1e-3, seed=1)
    b = 512
    for prec, tz, tg_ in ((edpc.EDPC_FP32, 1e-4, 1e-3), (edpc.EDPC_BF16, 3e-2, 6e-2)):
        c, o = cfgs(precision=prec, **dims)
        m = edpc.Model(c, b)
        om = OModel(o, b)
        rng = np.random.default_rng(7)
        _state_after_steps(m, om, b, 32, 2, rng)
        ctx = rng.integers(0, 256, size=(b, 32)).astype(np.uint8)
        z, _ = m.forward(ctx)
        zo, cache = om.forward(ctx.astype(np.int64))
        assert np.abs(z - zo).max() <= tz * np.abs(zo).max()
        tgt = rng.integers(0, 256, size=b).astype(np.uint8)
        g, gu = m.backward(ctx, tgt, np.ones(b, np.uint8))
        po = softmax(zo)
        dz = po.copy()
        dz[np.arange(b), tgt] -= 1
        dz /= b
        go, dUo = om.backward(cache, dz)
        gf = OModel.flat_grads(om.layout, go)
        off = 0
        for name, shape, _ in om.layout:  # tensor by tensor
            n = int(np.prod(shape))
            ref = gf[off:off + n]
            if np.linalg.norm(ref) > 1e-12:
                assert _rel(g[off:off + n], ref) <= tg_, (prec, name)
                if prec == edpc.EDPC_FP32:
                    err = np.abs(g[off:off + n] - ref).max()
                    assert err <= 1e-3 * np.abs(ref).max() + 1e-9, (name, err)
            off += n
        sample = rng.choice(b, size=16, replace=False)
        assert _rel(gu.reshape(b, 256, 256)[sample], dUo[sample]) <= tg_
        if prec == edpc.EDPC_FP32:
            d = gu.reshape(b, 256, 256)[sample] - dUo[sample]
            assert np.abs(d).max() <= 1e-3 * np.abs(dUo[sample]).max() + 1e-9
        m.close()


def test_multimedia_roundtrip_bf16():
    """A 4 MiB slice of the multimedia mix through the 512-stream BF16 model."""
    x = synth.multimedia_mix(4 * synth.MIB, 20250719)
    c = edpc.make_cfg(streams=512, context=32, embed_dim=16, latent=256, hidden=256, blocks=4,
                      precision=edpc.EDPC_BF16, seed=1)
    bits = edpc.compress(x, c)
    assert np.array_equal(edpc.decompress(bits), x)


def test_autograd_function_matches_oracle():
    """The adjoint kernels behind torch.autograd.Function: gradients of the mean
    cross-entropy w.r.t. the shared parameters and the FDM, against the oracle."""
    from paper_2507_18969_gb300.autograd import step_loss
    dims = dict(context=16, embed_dim=16, latent=128, hidden=128, blocks=2, branches=2, lr=1e-3, seed=4)
    c, o = cfgs(**dims)
    b = 4
    m = edpc.Model(c, b)
    om = OModel(o, b)
    rng = np.random.default_rng(21)
    st = _state_after_steps(m, om, b, o.context, 4, rng)
    shared = torch.tensor(st["P"], requires_grad=True)
    fdm = torch.tensor(st["U"], requires_grad=True)
    ctx = rng.integers(0, 256, size=(b, o.context)).astype(np.uint8)
    tg = rng.integers(0, 256, size=b).astype(np.uint8)
    act = np.ones(b, np.uint8)
    loss = step_loss(shared, fdm, m, ctx, tg, act)
    gs, gf = torch.autograd.grad(loss, [shared, fdm])
    lo = om.loss(ctx.astype(np.int64), tg.astype(np.int64))
    assert abs(float(loss.detach()) - lo) <= 1e-5 * max(1.0, abs(lo))
    _, go, dUo, _ = om.grad_step(ctx.astype(np.int64), tg.astype(np.int64))
    assert _rel(gs.numpy(), OModel.flat_grads(om.layout, go)) <= 1e-3
    assert _rel(gf.numpy().reshape(b, 128, 128), dUo) <= 1e-3
