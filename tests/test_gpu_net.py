"""The warm start's conv1d network on the GPU (BF16 tensor cores, FP32 accumulation)
against the oracle in mirrored mode (bf16 rounding of weights, layer inputs and
fed-back output gradients at the same points; binary64 accumulation).

Layer by layer (gsr_net_layer_forward / _backward) both sides see identical
bf16 operands and only the FP32 (GPU) vs FP64 (oracle) summation differs: each
element is within k 2^-23 of its sum of |terms| (k = the number of terms; one
unit of binary32 rounding or truncation per addition), and
each tensor within 1e-4 relative in the 2-norm. Through the whole network a
bf16 rounding tie flipped by that difference moves one activation by one bf16
ulp (2^-8 relative), which propagates; the whole-network checks (2e-3 forward,
1e-2 gradients) are smoke checks of the composition.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2308_00778_gb300 as g

pytestmark = pytest.mark.gpu


def _random_params(rng):
    ps = []
    for ci, co in zip(oracle.NET_CHANNELS[:-1], oracle.NET_CHANNELS[1:]):
        ps.append((rng.standard_normal((co, ci, 5)) * np.sqrt(2.0 / (5 * ci)), rng.standard_normal(co) * 0.1))
    return ps


def _flat(ps):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in ps]).astype(np.float32)


def _unflat(v):
    ps, off = [], 0
    for ci, co in zip(oracle.NET_CHANNELS[:-1], oracle.NET_CHANNELS[1:]):
        W = v[off:off + co * ci * 5].reshape(co, ci, 5)
        off += co * ci * 5
        b = v[off:off + co]
        off += co
        ps.append((W.astype(np.float64), b.astype(np.float64)))
    return ps


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("shape", [(1, 64), (2, 200), (3, 77)])
def test_forward_vs_mirrored_oracle(shape):
    rng = np.random.default_rng(1)
    ps = _random_params(rng)
    flat = _flat(ps)
    ps = _unflat(flat)  # the fp32 values the GPU holds
    net = g.Net()
    net.set_params(flat)
    x = rng.standard_normal(shape + (6,)).astype(np.float32)
    out = torch.zeros(shape + (3,), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(x, device="cuda"), out)
    torch.cuda.synchronize()
    y, _ = oracle.net_forward(ps, x.astype(np.float64), mirrored=True)
    assert _rel(out.cpu().numpy(), y) <= 2e-3
    np.testing.assert_array_equal(net.get_params(), flat)
    net.close()


@pytest.mark.parametrize("shape", [(1, 64), (2, 131)])
def test_gradients_vs_mirrored_oracle(shape):
    rng = np.random.default_rng(2)
    flat = _flat(_random_params(rng))
    ps = _unflat(flat)
    net = g.Net()
    net.set_params(flat)
    x = rng.standard_normal(shape + (6,)).astype(np.float32)
    t = rng.standard_normal(shape + (3,)).astype(np.float32)
    grads, loss = net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    y, acts = oracle.net_forward(ps, x.astype(np.float64), mirrored=True)
    loss_ref, dy = oracle.mse(y, t.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=2e-3)
    ref = oracle.net_backward(ps, acts, dy, mirrored=True)
    gl = _unflat(grads)
    for layer, ((dW, db), (rW, rb)) in enumerate(zip(gl, ref)):
        assert _rel(dW, rW) <= 1e-2, (layer, _rel(dW, rW))
        assert _rel(db, rb) <= 1e-2, (layer, _rel(db, rb))
    # the gradient query leaves the parameters and the optimiser untouched
    np.testing.assert_array_equal(net.get_params(), flat)
    net.close()


LAYERS = list(zip(oracle.NET_CHANNELS[:-1], oracle.NET_CHANNELS[1:]))


@pytest.mark.parametrize("layer", range(6))
def test_layer_forward_backward_vs_mirrored_oracle(layer):
    """One layer at a time on identical bf16 operands: forward (before the ReLU), din, dW and db."""
    rng = np.random.default_rng(20 + layer)
    flat = _flat(_random_params(rng))
    ps = _unflat(flat)
    net = g.Net()
    net.set_params(flat)
    cin, cout = LAYERS[layer]
    B, L = 2, 300  # three 128-position CTAs of the convolution, the last one ragged
    x = rng.standard_normal((B, L, cin)).astype(np.float32)
    if layer > 0:
        x = np.maximum(x, 0.0)  # the output of the previous layer's ReLU
    dout = (rng.standard_normal((B, L, cout)) * 1e-2).astype(np.float32)
    xd, dd = torch.tensor(x, device="cuda"), torch.tensor(dout, device="cuda")
    out = torch.zeros((B, L, cout), dtype=torch.float32, device="cuda")
    din = torch.zeros((B, L, cin), dtype=torch.float32, device="cuda")
    dW = torch.zeros((cout, cin, 5), dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    net.layer_forward(layer, xd, out)
    net.layer_backward(layer, xd, dd, din, dW, db)
    torch.cuda.synchronize()
    W, bias = ps[layer]
    x64, d64 = x.astype(np.float64), dout.astype(np.float64)
    # the tensor cores' fp32 accumulation may truncate instead of rounding: 2^-23 per addition
    u = 2.0 ** -23
    # forward: K = 5 cin products and the bias per element
    ref = oracle.conv_fwd(x64, W, bias, relu=False, mirrored=True)
    mag = oracle.conv_fwd(np.abs(x64), np.abs(W), np.abs(bias), relu=False, mirrored=True)
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= (5 * cin + 1) * u * mag + 1e-30), layer
    assert _rel(got, ref) <= 1e-4
    # backward: din has 5 cout products per element, dW B*L, db B*L unrounded terms
    rin, rW, rb = oracle.conv_bwd(x64, d64, W, mirrored=True)
    min_, mW, mb = oracle.conv_bwd(np.abs(x64), np.abs(d64), np.abs(W), mirrored=True)
    gin, gW, gb = (t.cpu().numpy().astype(np.float64) for t in (din, dW, db))
    assert np.all(np.abs(gin - rin) <= 5 * cout * u * min_ + 1e-30), layer
    assert np.all(np.abs(gW - rW) <= (B * L + 64) * u * mW + 1e-30), layer
    assert np.all(np.abs(gb - rb) <= B * L * u * mb + 1e-30), layer
    for a, r in ((gin, rin), (gW, rW), (gb, rb)):
        assert _rel(a, r) <= 1e-4, layer
    # the layer calls leave the parameters untouched
    np.testing.assert_array_equal(net.get_params(), flat)
    net.close()


def test_adam_three_steps_match_oracle():
    """Three Adam steps with caller gradients spanning 1e-6..1 in magnitude, against the oracle's
    binary64 Adam; the GPU keeps the moments and weights in binary32, so each parameter is within a few
    2^-24 of its value plus lr times the binary32 error of the update direction."""
    rng = np.random.default_rng(3)
    flat = _flat(_random_params(rng))
    net = g.Net()
    net.set_params(flat)
    n = flat.size
    w = flat.astype(np.float64)
    m = np.zeros(n)
    v = np.zeros(n)
    lr = 1e-3
    for step in range(1, 4):
        mag = 10.0 ** rng.uniform(-6, 0, n)
        gr = (mag * rng.choice([-1.0, 1.0], n)).astype(np.float32)
        net.apply_gradients(gr, lr)
        oracle.adam(w, m, v, gr.astype(np.float64), lr, step=step)
        got = net.get_params().astype(np.float64)
        tol = 4 * 2.0 ** -24 * np.abs(w) + lr * 1e-5
        assert np.all(np.abs(got - w) <= tol), (step, np.max(np.abs(got - w) - tol))
    net.close()


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(3)
    flat = _flat(_random_params(rng))
    net = g.Net()
    net.set_params(flat)
    x = torch.tensor(rng.standard_normal((2, 100, 6)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.standard_normal((2, 100, 3)).astype(np.float32), device="cuda")
    grads, _ = net.gradients(x, t)
    lr = 1e-3
    net.train_step(x, t, lr)
    w = flat.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    oracle.adam(w, m, v, grads.astype(np.float64), lr, step=1)
    got = net.get_params().astype(np.float64)
    # first Adam step moves every parameter by lr * g / (|g| + eps): sign-like, so compare the updates
    upd_gpu = got - flat
    upd_ref = w - flat
    big = np.abs(grads) > 1e-3  # where |g| >> eps the update is lr * sign(g) on both sides
    np.testing.assert_allclose(upd_gpu[big], upd_ref[big], rtol=1e-3, atol=1e-7)
    net.close()


def test_training_reduces_loss():
    """A short run on a smooth regression task: the loss falls by 10x."""
    rng = np.random.default_rng(4)
    flat = _flat(_random_params(rng))
    net = g.Net()
    net.set_params(flat)
    L = 256
    k = np.arange(L)
    xs, ts = [], []
    for _ in range(8):
        f = rng.uniform(0.01, 0.05, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        clean = np.stack([np.sin(2 * np.pi * f[a] * k + ph[a]) for a in range(3)], axis=1)
        noisy = clean + 0.3 * rng.standard_normal(clean.shape)
        xs.append(np.concatenate([noisy, np.zeros((L, 3))], axis=1))
        ts.append(clean - noisy)  # the residual the network must predict
    x = torch.tensor(np.array(xs, dtype=np.float32), device="cuda")
    t = torch.tensor(np.array(ts, dtype=np.float32), device="cuda")
    first = net.train_step(x, t, 2e-3)
    for _ in range(300):
        last = net.train_step(x, t, 2e-3)
    assert last < 0.1 * first, (first, last)
    net.close()


def test_save_load_roundtrip(tmp_path):
    rng = np.random.default_rng(5)
    flat = _flat(_random_params(rng))
    net = g.Net()
    net.set_params(flat)
    net.save(tmp_path / "w.bin")
    net2 = g.Net()
    net2.load(tmp_path / "w.bin")
    np.testing.assert_array_equal(net2.get_params(), flat)
    (tmp_path / "bad.bin").write_bytes(b"not weights")
    with pytest.raises(g.GsrError):
        net2.load(tmp_path / "bad.bin")
    net.close()
    net2.close()


def test_tensor_core_wait_gives_up_and_the_context_stays_usable():
    """The tensor-core kernels' bounded wait run out on purpose (an mbarrier nothing arrives on, 20 ms):
    the kernel reports the timeout, releases its TMEM and ends; a network forward on the same device
    afterwards is correct (it allocates TMEM again)."""
    timed_out, ms = g.tc_wait_check(0, 20.0)
    assert timed_out == 1
    assert 20.0 <= ms < 1000.0, ms
    rng = np.random.default_rng(9)
    flat = _flat(_random_params(rng))
    ps = _unflat(flat)
    net = g.Net()
    net.set_params(flat)
    x = rng.standard_normal((1, 300, 6)).astype(np.float32)
    out = torch.zeros((1, 300, 3), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(x, device="cuda"), out)
    torch.cuda.synchronize()
    y, _ = oracle.net_forward(ps, x.astype(np.float64), mirrored=True)
    assert _rel(out.cpu().numpy(), y) <= 2e-3
    net.close()


@pytest.mark.parametrize("L", [1, 2, 5, 129])
def test_layer_products_at_short_and_ragged_lengths(L):
    """The convolution products where the zero padding and the tile edges meet: sequences of 1, 2
    and 5 positions (every tap reaches past an end) and 129 (one position into a second tile of 128);
    forward, din, dW and db of a 64 -> 64 layer against the oracle at the per-layer bounds."""
    layer = 2
    rng = np.random.default_rng(40 + L)
    flat = _flat(_random_params(rng))
    ps = _unflat(flat)
    net = g.Net()
    net.set_params(flat)
    cin, cout = LAYERS[layer]
    B = 3
    x = np.maximum(rng.standard_normal((B, L, cin)), 0.0).astype(np.float32)
    dout = (rng.standard_normal((B, L, cout)) * 1e-2).astype(np.float32)
    xd, dd = torch.tensor(x, device="cuda"), torch.tensor(dout, device="cuda")
    out = torch.zeros((B, L, cout), dtype=torch.float32, device="cuda")
    din = torch.zeros((B, L, cin), dtype=torch.float32, device="cuda")
    dW = torch.zeros((cout, cin, 5), dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    net.layer_forward(layer, xd, out)
    net.layer_backward(layer, xd, dd, din, dW, db)
    torch.cuda.synchronize()
    W, bias = ps[layer]
    x64, d64 = x.astype(np.float64), dout.astype(np.float64)
    u = 2.0 ** -23
    ref = oracle.conv_fwd(x64, W, bias, relu=False, mirrored=True)
    mag = oracle.conv_fwd(np.abs(x64), np.abs(W), np.abs(bias), relu=False, mirrored=True)
    assert np.all(np.abs(out.cpu().numpy().astype(np.float64) - ref) <= (5 * cin + 1) * u * mag + 1e-30)
    rin, rW, rb = oracle.conv_bwd(x64, d64, W, mirrored=True)
    min_, mW, mb = oracle.conv_bwd(np.abs(x64), np.abs(d64), np.abs(W), mirrored=True)
    gin, gW, gb = (t.cpu().numpy().astype(np.float64) for t in (din, dW, db))
    assert np.all(np.abs(gin - rin) <= 5 * cout * u * min_ + 1e-30)
    assert np.all(np.abs(gW - rW) <= (B * L + 64) * u * mW + 1e-30)
    assert np.all(np.abs(gb - rb) <= B * L * u * mb + 1e-30)
    net.close()
