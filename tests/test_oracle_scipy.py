"""The oracle's LSQR against an independent implementation of the same published algorithm
(Paige and Saunders 1982; Alg. 1 runs it on the column-scaled system): scipy.sparse.linalg.lsqr
on the explicit matrix of small generated systems. Without the column preconditioner the
iterates, the stop code and iteration count, the norm and condition estimates and the variance
estimates agree; with it, the oracle's x equals scipy's solution of A diag(p) y = b mapped back
(x = p y, p_j = 1 / |A_:,j|). A plausible slip in the oracle's recurrences (a rotation, the phi or
rho update, the damping term, the w or x update, a stopping test) changes the iterates or the
estimates well beyond the 1e-9 bars used here."""
import numpy as np
import pytest

import gsrgen
import oracle
from conftest import dense_matrix

scipy_linalg = pytest.importorskip("scipy.sparse.linalg")

CASES = {
    "tiny": gsrgen.make_cfg(7, 20, 30, 12, 8),
    "ragged": gsrgen.make_cfg(21, 40, (3, 25), 16, 10),
    "no_global": gsrgen.make_cfg(22, 30, (5, 20), 10, 7, n_glob=0),
}


def _system(name):
    cfg = CASES[name]
    h = gsrgen.generate(cfg)
    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    D = dense_matrix(h.star_ptr, h.A, h.knot, h.instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    return s, b, D


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("damp", [0.0, 0.3])
@pytest.mark.parametrize("itn", [5, 17])
def test_unpreconditioned_iterates_and_estimates_match_scipy(name, damp, itn):
    s, b, D = _system(name)
    x, info, var = oracle.lsqr(s, b, itn, 0.0, 0.0, 0.0, damp, precond=False, want_var=True)
    ref = scipy_linalg.lsqr(D, b, damp=damp, atol=0.0, btol=0.0, conlim=0.0, iter_lim=itn, calc_var=True)
    xr, istop, itr, r1, r2, anorm, acond, arnorm, xnorm, varr = ref[:10]
    assert info["itn"] == itr and info["istop"] == istop
    assert _rel(x, xr) <= 1e-9
    for mine, theirs in ((info["r1norm"], r1), (info["r2norm"], r2), (info["anorm"], anorm),
                         (info["acond"], acond), (info["arnorm"], arnorm), (info["xnorm"], xnorm)):
        assert abs(mine - theirs) <= 1e-9 * max(abs(theirs), 1e-300), (mine, theirs)
    assert _rel(var, varr) <= 1e-9


@pytest.mark.parametrize("name", sorted(CASES))
def test_preconditioned_solution_is_scipys_on_the_scaled_columns(name):
    s, b, D = _system(name)
    norms = np.linalg.norm(D, axis=0)
    p = np.where(norms > 0.0, 1.0 / np.where(norms > 0.0, norms, 1.0), 0.0)
    for itn in (4, 12):
        x, info = oracle.lsqr(s, b, itn, 0.0, 0.0, 0.0, 0.1, precond=True)
        ref = scipy_linalg.lsqr(D * p, b, damp=0.1, atol=0.0, btol=0.0, conlim=0.0, iter_lim=itn)
        assert info["itn"] == ref[2]
        assert _rel(x, p * ref[0]) <= 1e-9
