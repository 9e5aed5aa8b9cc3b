"""Shared test set-up: import paths, the gpu marker, and the host-side builds.

Tests marked ``gpu`` need a CUDA device and the sm_103a library; everything
else runs on the CPU (oracle pins, generator checks, host logic, ABI symbols).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _host_libs():
    """The oracle and the host generator are plain C: build them if missing."""
    import gsrgen.build
    import oracle.build

    if not os.path.exists(os.path.join(ROOT, "oracle", "liboracle.so")):
        oracle.build.build()
    if not os.path.exists(os.path.join(ROOT, "gsrgen", "libgsrgen_host.so")):
        gsrgen.build.build_host()
    yield


def dense_matrix(star_ptr, A, knot, instr, n_dfa, n_instr, n_glob, n_astro=5, n_ipr=6):
    """Explicit dense A (tiny systems only), placed entry by entry from the
    paper's storage (Sec. 2): a row holds n_astro astrometric coefficients
    (columns n_astro*star + j), 3 x 4 attitude coefficients (columns
    n_astro*n_stars + axis*n_dfa + knot + j), n_ipr instrumental ones (their
    stored columns) and n_glob global ones, in that order along the row."""
    import numpy as np

    n_stars = len(star_ptr) - 1
    n = int(star_ptr[-1])
    c = n_astro * n_stars + 3 * n_dfa + n_instr + n_glob
    a0 = n_astro * n_stars
    i0 = a0 + 3 * n_dfa
    g0 = i0 + n_instr
    D = np.zeros((n, c))
    for s in range(n_stars):
        for r in range(star_ptr[s], star_ptr[s + 1]):
            k = 0
            for j in range(n_astro):
                D[r, n_astro * s + j] += A[r, k]
                k += 1
            for ax in range(3):
                for j in range(4):
                    D[r, a0 + ax * n_dfa + knot[r] + j] += A[r, k]
                    k += 1
            for j in range(n_ipr):
                D[r, i0 + instr[r, j]] += A[r, k]
                k += 1
            for j in range(n_glob):
                D[r, g0 + j] += A[r, k]
                k += 1
    return D
