"""The device twin of the input generator writes the same bits as the host generator."""
import numpy as np
import pytest
import torch

import gsrgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
def test_device_generator_bit_identical(fp32):
    cfg = gsrgen.make_cfg(13, 700, (1, 260), 3000, 500, att_kind=1)
    h = gsrgen.generate(cfg, fp32=fp32)
    sp = h.star_ptr
    n = int(sp[-1])
    stride = n + 3
    dt = torch.float32 if fp32 else torch.float64
    vals = torch.zeros(24 * stride, dtype=dt, device="cuda")
    knot = torch.zeros(n, dtype=torch.int32, device="cuda")
    ins = torch.zeros(6 * stride, dtype=torch.int32, device="cuda")
    spd = torch.tensor(sp, device="cuda")
    s0, s1 = 100, 600
    r0, r1 = int(sp[s0]), int(sp[s1])
    gsrgen.dev_rows(cfg, spd, sp, s0, s1, vals, stride, knot, ins)
    torch.cuda.synchronize()
    m = r1 - r0
    V = vals.view(24, stride)[:, :m].cpu().numpy().T
    want = h.A32[r0:r1] if fp32 else h.A[r0:r1]
    assert np.array_equal(V, want)
    assert np.array_equal(knot[:m].cpu().numpy(), h.knot[r0:r1])
    assert np.array_equal(ins.view(6, stride)[:, :m].cpu().numpy().T, h.instr[r0:r1])
    xt = torch.zeros(cfg.ncols(), dtype=torch.float64, device="cuda")
    gsrgen.dev_xtrue(cfg, xt)
    eps = torch.zeros(n, dtype=torch.float64, device="cuda")
    gsrgen.dev_noise(cfg, eps)
    torch.cuda.synchronize()
    assert np.array_equal(xt.cpu().numpy(), h.x_true)
    assert np.array_equal(eps.cpu().numpy(), h.eps)
