"""The warm start's conv1d network on the GPU (BF16 tensor cores, FP32 accumulation)
against the oracle in mirrored mode (bf16 rounding of weights, layer inputs and
fed-back output gradients at the same points; binary64 accumulation).

Both sides see identical bf16 operands; only the FP32 (GPU) vs FP64 (oracle)
summation differs, so per tensor |gpu - ref| / |ref| is ~1e-6. A bf16 rounding
tie flipped by that difference moves one activation by one bf16 ulp (2^-8
relative), which propagates; the bars (2e-3 forward, 1e-2 gradients, per
tensor in the 2-norm) leave room for a few such flips and still catch a wrong
tap, channel, sign or layout.
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
