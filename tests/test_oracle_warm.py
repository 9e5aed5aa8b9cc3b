"""Pins of the warm-start oracle (oracle/warm.c and its composition in oracle/__init__.py).

* conv1d forward against a direct numpy evaluation of the definition;
* conv1d / network gradients against central finite differences;
* bfloat16 rounding against hand-computed ties and carries;
* MSE and Adam against closed forms;
* the per-star 5x5 astrometric solve (n_astro x n_astro for section variants)
  against numpy least squares per star;
* the Jacobi features against an explicit dense evaluation.
"""
import numpy as np
import pytest

import gsrgen
import oracle
from conftest import dense_matrix


def _conv_numpy(x, W, b):
    nb, L, cin = x.shape
    cout = W.shape[0]
    xp = np.zeros((nb, L + 4, cin))
    xp[:, 2:L + 2] = x
    out = np.zeros((nb, L, cout)) + b
    for t in range(5):
        out += np.einsum("bpc,oc->bpo", xp[:, t:t + L], W[:, :, t])
    return out


def test_conv_forward_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 37, 6))
    W = rng.standard_normal((9, 6, 5))
    b = rng.standard_normal(9)
    np.testing.assert_allclose(oracle.conv_fwd(x, W, b, relu=False), _conv_numpy(x, W, b), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.conv_fwd(x, W, b, relu=True), np.maximum(_conv_numpy(x, W, b), 0), atol=1e-13)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 11, 4))
    W = rng.standard_normal((5, 4, 5))
    b = rng.standard_normal(5)
    dout = rng.standard_normal((2, 11, 5))  # loss = sum(dout * conv(x))
    din, dW, db = oracle.conv_bwd(x, dout, W)
    h = 1e-6

    def loss(x_, W_, b_):
        return float(np.sum(dout * oracle.conv_fwd(x_, W_, b_, relu=False)))

    for idx in [(0, 3, 1), (1, 0, 0), (1, 10, 3), (0, 5, 2)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (loss(x + e, W, b) - loss(x - e, W, b)) / (2 * h)
        assert din[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0), (4, 3, 4), (2, 1, 2)]:
        e = np.zeros_like(W)
        e[idx] = h
        fd = (loss(x, W + e, b) - loss(x, W - e, b)) / (2 * h)
        assert dW[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    np.testing.assert_allclose(db, dout.sum(axis=(0, 1)), rtol=1e-13)


def _params(rng, chans=oracle.NET_CHANNELS):
    return [(rng.standard_normal((co, ci, 5)) * np.sqrt(2.0 / (5 * ci)), rng.standard_normal(co) * 0.1)
            for ci, co in zip(chans[:-1], chans[1:])]


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(2)
    chans = [6, 8, 8, 8, 8, 8, 3]
    params = _params(rng, chans)
    x = rng.standard_normal((2, 13, 6))
    t = rng.standard_normal((2, 13, 3))

    def loss_of(ps):
        y, _ = oracle.net_forward(ps, x)
        return oracle.mse(y, t)[0]

    y, acts = oracle.net_forward(params, x)
    loss, dy = oracle.mse(y, t)
    grads = oracle.net_backward(params, acts, dy)
    h = 1e-6
    for layer, idx in [(0, (3, 2, 1)), (2, (1, 7, 4)), (5, (2, 0, 3)), (3, (5, 5, 0))]:
        W, b = params[layer]
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        pp = list(params)
        pp[layer] = (Wp, b)
        pm = list(params)
        pm[layer] = (Wm, b)
        fd = (loss_of(pp) - loss_of(pm)) / (2 * h)
        assert grads[layer][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    W, b = params[4]
    bp, bm = b.copy(), b.copy()
    bp[3] += h
    bm[3] -= h
    pp, pm = list(params), list(params)
    pp[4], pm[4] = (W, bp), (W, bm)
    assert grads[4][1][3] == pytest.approx((loss_of(pp) - loss_of(pm)) / (2 * h), rel=1e-5, abs=1e-9)


def test_bf16_rounding():
    assert oracle.bf16(1.0) == 1.0
    assert oracle.bf16(1 + 2 ** -8) == 1.0                  # tie: round to even
    assert oracle.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6      # tie: round to even (up)
    assert oracle.bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7
    assert oracle.bf16(-3.0) == -3.0
    assert oracle.bf16(0.0) == 0.0
    assert oracle.bf16(2 - 2 ** -9) == 2.0                   # carry into the exponent
    # the mirrored convolution uses exactly these roundings
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 9, 3))
    W = rng.standard_normal((2, 3, 5))
    b = rng.standard_normal(2)
    xr = np.vectorize(oracle.bf16)(x)
    Wr = np.vectorize(oracle.bf16)(W)
    np.testing.assert_allclose(oracle.conv_fwd(x, W, b, False, mirrored=True), _conv_numpy(xr, Wr, b), rtol=1e-13,
                               atol=1e-13)


def test_mse_and_adam_closed_forms():
    y = np.array([1.0, 2.0, -1.0, 0.5])
    t = np.array([0.0, 2.5, -1.0, 1.5])
    loss, g = oracle.mse(y, t)
    assert loss == pytest.approx(np.mean((y - t) ** 2))
    np.testing.assert_allclose(g, 2 * (y - t) / 4)
    w = np.array([1.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    gr = np.array([0.3, -4.0, 1e-3])
    lr, eps = 0.01, 1e-8
    oracle.adam(w, m, v, gr, lr, eps=eps, step=1)
    # first step: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    np.testing.assert_allclose(w, np.array([1.0, -2.0, 0.5]) - lr * gr / (np.abs(gr) + eps), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * gr)
    np.testing.assert_allclose(v, 0.001 * gr ** 2)


@pytest.mark.parametrize("sections", [(5, 6, 1), (3, 4, 2), (1, 0, 5)])
def test_astro_solve_vs_lstsq_per_star(sections):
    na, ni, ng = sections
    cfg = gsrgen.make_cfg(11, 40, (6, 80), 30, 12, n_astro=na, n_ipr=ni, n_glob=ng)
    h = gsrgen.generate(cfg)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    x = np.zeros(s.n_cols)
    a0 = s.blocks()["att"][0]
    x[a0:] = h.x_true[a0:] + 0.1  # some non-astrometric start
    rest = x[a0:].copy()
    assert oracle.astro_solve(s, b, x) == 0
    D = dense_matrix(h.star_ptr, h.A, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob, na, ni)
    r = b - D[:, a0:] @ rest
    for st in range(cfg.n_stars):
        r0, r1 = h.star_ptr[st], h.star_ptr[st + 1]
        ref = np.linalg.lstsq(D[r0:r1, na * st:na * st + na], r[r0:r1], rcond=None)[0]
        np.testing.assert_allclose(x[na * st:na * st + na], ref, rtol=1e-8, atol=1e-10)
    assert np.all(x[a0:] == rest)  # non-astrometric parts untouched


def test_jacobi_features_dense():
    cfg = gsrgen.make_cfg(12, 30, 40, 10, 8)
    h = gsrgen.generate(cfg)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    f, scale = oracle.jacobi_features(s, b)
    D = dense_matrix(h.star_ptr, h.A, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    a0, a1 = s.blocks()["att"]
    colsq = (D[:, a0:a1] ** 2).sum(axis=0)
    jac = (D[:, a0:a1].T @ b) / colsq
    np.testing.assert_allclose(scale, np.sqrt(np.mean(jac ** 2)), rtol=1e-12)
    for ax in range(3):
        np.testing.assert_allclose(f[:, ax] * scale, jac[ax * 10:(ax + 1) * 10], rtol=1e-11)
        lg = np.log(colsq) - np.log(colsq).mean()
        np.testing.assert_allclose(f[:, 3 + ax], lg[ax * 10:(ax + 1) * 10], rtol=1e-11, atol=1e-12)


def _bf16_torch(a):
    """Round to bfloat16 (nearest even) with torch's own conversion, independent of the oracle's."""
    import torch

    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _conv_bwd_numpy(x, dout, W):
    """din, dW, db of one layer (kernel 5, zero padding 2) written as shifted products."""
    nb, L, cin = x.shape
    xp = np.zeros((nb, L + 4, cin))
    xp[:, 2:L + 2] = x
    dW = np.zeros_like(W)
    dinp = np.zeros((nb, L + 4, cin))
    for t in range(5):
        # out[p] takes in[p + t - 2] = xp[p + t] through W[:, :, t]
        dW[:, :, t] = np.einsum("bpo,bpc->oc", dout, xp[:, t:t + L])
        dinp[:, t:t + L] += np.einsum("bpo,oc->bpc", dout, W[:, :, t])
    return dinp[:, 2:L + 2], dW, dout.sum(axis=(0, 1))


def test_mirrored_conv_backward_rounding_points():
    """The mirrored backward rounds the output gradient, the layer input and the weights to bfloat16 in the
    products (the points where the GPU stores bfloat16 operands) and sums the bias gradient from the
    unrounded output gradient; an independent restatement with torch's bfloat16 conversion agrees, and
    moving any one rounding point changes the result by far more than the tolerance."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, 23, 6))
    W = rng.standard_normal((7, 6, 5))
    dout = rng.standard_normal((2, 23, 7))
    din, dW, db = oracle.conv_bwd(x, dout, W, mirrored=True)
    rin, rW, rb = _conv_bwd_numpy(_bf16_torch(x), _bf16_torch(dout), _bf16_torch(W))
    np.testing.assert_allclose(din, rin, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dW, rW, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(db, dout.sum(axis=(0, 1)), rtol=1e-13)
    # each rounding point matters: leaving one out moves the result by ~2^-9 relative
    for alt in (_conv_bwd_numpy(x, _bf16_torch(dout), _bf16_torch(W)),
                _conv_bwd_numpy(_bf16_torch(x), dout, _bf16_torch(W)),
                _conv_bwd_numpy(_bf16_torch(x), _bf16_torch(dout), W)):
        moved = max(np.abs(alt[0] - din).max() / np.abs(din).max(), np.abs(alt[1] - dW).max() / np.abs(dW).max())
        assert moved > 1e-5
    # the bias gradient is not taken from the rounded dout
    assert np.abs(_bf16_torch(dout).sum(axis=(0, 1)) - db).max() > 1e-6


def test_adam_later_steps_closed_form():
    """Adam over three steps with changing gradients against the unrolled moments
    m_t = (1 - b1) sum_k b1^(t-k) g_k, v_t = (1 - b2) sum_k b2^(t-k) g_k^2 and the bias corrections
    1 - b^t of each step (the recursive form in the oracle must reproduce them at t = 2, 3)."""
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 0.01
    w0 = np.array([1.0, -2.0, 0.5, 3.0])
    gs = [np.array([0.3, -4.0, 1e-3, 1e-6]), np.array([-0.1, -2.0, 2e-3, 1.0]),
          np.array([0.25, 1.0, -5e-4, 1e-6])]
    w, m, v = w0.copy(), np.zeros(4), np.zeros(4)
    ref = w0.copy()
    for t in range(1, 4):
        oracle.adam(w, m, v, gs[t - 1], lr, b1=b1, b2=b2, eps=eps, step=t)
        mt = (1 - b1) * sum(b1 ** (t - k) * gs[k - 1] for k in range(1, t + 1))
        vt = (1 - b2) * sum(b2 ** (t - k) * gs[k - 1] ** 2 for k in range(1, t + 1))
        ref = ref - lr * (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
        np.testing.assert_allclose(m, mt, rtol=1e-13)
        np.testing.assert_allclose(v, vt, rtol=1e-13)
        np.testing.assert_allclose(w, ref, rtol=1e-13, atol=1e-15)
    # a stale bias correction (step 1's at step 3) would move the last update visibly
    w2, m2, v2 = w0.copy(), np.zeros(4), np.zeros(4)
    for t in range(1, 4):
        oracle.adam(w2, m2, v2, gs[t - 1], lr, b1=b1, b2=b2, eps=eps, step=1 if t == 3 else t)
    assert np.abs(w2 - ref).max() > 1e-4
