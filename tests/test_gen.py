"""The seeded input generator: determinism, structure and distributions."""
import math

import numpy as np

import gsrgen


def test_deterministic_and_chunk_independent():
    cfg = gsrgen.make_cfg(11, 30, (20, 40), 16, 9)
    a = gsrgen.generate(cfg)
    b = gsrgen.generate(cfg)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.knot, b.knot) and np.array_equal(a.instr, b.instr)
    assert np.array_equal(a.x_true, b.x_true) and np.array_equal(a.eps, b.eps)
    sp = a.star_ptr
    A2, k2, i2 = gsrgen.rows(cfg, sp, 7, 19)
    r0, r1 = sp[7], sp[19]
    assert np.array_equal(A2, a.A[r0:r1]) and np.array_equal(k2, a.knot[r0:r1]) and np.array_equal(i2, a.instr[r0:r1])
    assert np.array_equal(gsrgen.xtrue(cfg, 10, 25), a.x_true[10:35])
    assert np.array_equal(gsrgen.noise(cfg, 5, 50), a.eps[5:55])


def test_structure():
    cfg = gsrgen.make_cfg(3, 50, (10, 60), 40, 12, att_kind=1)
    h = gsrgen.generate(cfg)
    obs = np.diff(h.star_ptr)
    assert obs.min() >= 10 and obs.max() <= 60 and len(set(obs.tolist())) > 5
    assert h.knot.min() >= 0 and h.knot.max() <= cfg.n_dfa - 4
    for s in range(cfg.n_stars):
        k = h.knot[h.star_ptr[s]:h.star_ptr[s + 1]]
        assert np.all(np.diff(k) >= 0), "knots must be sorted within a star"
    assert h.instr.min() >= 0 and h.instr.max() < cfg.n_instr
    assert all(len(set(r.tolist())) == 6 for r in h.instr)
    assert h.x_true.shape == (cfg.ncols(),)


def test_fp32_rounding_and_glob0():
    cfg = gsrgen.make_cfg(4, 5, 10, 8, 6, n_glob=0)
    h = gsrgen.generate(cfg, fp32=True)
    assert np.array_equal(h.A, h.A32.astype(np.float64))
    assert np.all(h.A[:, 23] == 0.0)
    h64 = gsrgen.generate(cfg)
    assert np.array_equal(h64.A.astype(np.float32), h.A32)


def test_distributions():
    cfg = gsrgen.make_cfg(9, 400, 100, 100, 60, noise_sigma=1e-3)
    h = gsrgen.generate(cfg)
    v = h.A.ravel()
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01
    kurt = ((v - v.mean()) ** 4).mean() / v.var() ** 2
    assert abs(kurt - 3.0) < 0.05
    assert abs(h.eps.std() - 1e-3) < 2e-5
    # knots spread over the whole range: uniform observation times
    hist = np.bincount(h.knot, minlength=cfg.n_dfa - 3)
    assert hist.min() > 0.5 * hist.mean()


def test_series_helpers_match_libm():
    L = gsrgen._load_host()
    for u in np.concatenate([np.geomspace(1e-16, 1.0, 500), np.linspace(0.01, 1.0, 500)]):
        assert abs(L.gsrgen_host_ln(float(u)) - math.log(u)) <= 2e-15 * max(1.0, abs(math.log(u)))
    for u in np.linspace(0.0, 1.0, 2000, endpoint=False):
        assert abs(L.gsrgen_host_cos_turn(float(u)) - math.cos(2 * math.pi * u)) <= 2e-15


def test_sinusoid_attitude_is_smooth():
    cfg = gsrgen.make_cfg(1, 10, 10, 3000, 20, att_kind=1)
    x = gsrgen.xtrue(cfg)
    att = x[50:50 + 3000]
    # sum of 8 sinusoids of <= 10 cycles per 1000 knots: neighbouring knots differ little
    assert np.abs(np.diff(att)).max() < 0.2 and att.std() > 0.2


def test_section_variants_share_the_standard_draws():
    """Compact rows of a section variant hold the same draws as the standard slots they stand for
    (Sec. 2: 0..5 astrometric, 12 attitude, 0..6 instrumental, the global section); the instrumental
    columns are a prefix of the standard row's; globals past the first have draws of their own."""
    std = gsrgen.make_cfg(13, 9, (3, 17), 11, 8)
    h = gsrgen.generate(std)
    for na, ni, ng in [(3, 4, 2), (0, 6, 1), (5, 0, 0), (2, 1, 5), (5, 6, 3)]:
        cfg = gsrgen.make_cfg(13, 9, (3, 17), 11, 8, n_glob=ng, n_astro=na, n_ipr=ni)
        v = gsrgen.generate(cfg)
        assert v.A.shape == (h.n_rows, na + 12 + ni + ng) and v.instr.shape == (h.n_rows, ni)
        assert np.array_equal(v.star_ptr, h.star_ptr) and np.array_equal(v.knot, h.knot)
        assert np.array_equal(v.A[:, :na], h.A[:, :na])
        assert np.array_equal(v.A[:, na:na + 12], h.A[:, 5:17])
        assert np.array_equal(v.A[:, na + 12:na + 12 + ni], h.A[:, 17:17 + ni])
        assert np.array_equal(v.instr, h.instr[:, :ni])
        g = v.A[:, na + 12 + ni:]
        if ng:
            assert np.array_equal(g[:, 0], h.A[:, 23])
            assert all(len(set(r.tolist())) == ng for r in g)  # distinct draws
        assert v.x_true.shape == (cfg.ncols(),) and cfg.ncols() == na * 9 + 33 + 8 + ng
    # a section variant with fewer instrumental unknowns than the standard row's six
    small = gsrgen.generate(gsrgen.make_cfg(2, 6, 10, 9, 3, n_ipr=3, n_glob=0))
    assert all(sorted(r.tolist()) == [0, 1, 2] for r in small.instr)
