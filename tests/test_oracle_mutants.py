"""The oracle pins catch plausible mistakes.

Each case copies oracle/*.c to a temporary directory, plants one mistake (a
dropped term, a wrong sign, a transposed index, a skipped damping rotation, a
wrong norm), builds it there, and runs the pin tests against that library:
they must fail. The real oracle is never modified.
"""
import glob
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "sign of rhobar": ("rhobar = -cs * alpha;", "rhobar = cs * alpha;"),
    "dropped global term": ("for (int j = 0; j < s->n_glob; ++j) sum = sum + a[k + j] * x[glob0 + j];", ";"),
    "no damping rotation": ("const double sn1 = damp / rhobar1;", "const double sn1 = 0.0;"),
    "attitude knot off by one": ("const int64_t k2 = att0 + (int64_t)ax * s->n_dfa + s->knot[i];\n"
                                 "                for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) x[k2 + j2]",
                                 "const int64_t k2 = att0 + (int64_t)ax * s->n_dfa + s->knot[i] + 1;\n"
                                 "                for (int j2 = 0; j2 < N_PAR_AXIS; ++j2, ++k) x[k2 + j2 - 1 + (j2 == 0)]"),
    "norm without sqrt": ("return m * sqrt(ssq);", "return m * ssq;"),
    "w update sign": ("const double t2 = -theta / rho;", "const double t2 = theta / rho;"),
    "preconditioner not inverted": ("p[j] = (p[j] > 0.0) ? 1.0 / sqrt(p[j]) : 1.0;",
                                    "p[j] = (p[j] > 0.0) ? sqrt(p[j]) : 1.0;"),
    # section variants: mistakes invisible on the standard 24-coefficient row
    "astrometric stride fixed at five": ("const int64_t offset_astro = (int64_t)na * star;",
                                         "const int64_t offset_astro = (int64_t)5 * star;"),
    "instrumental row stride fixed at six": ("sum = sum + a[k] * x[instr0 + s->instr[i * ni + j]];",
                                             "sum = sum + a[k] * x[instr0 + s->instr[i * 6 + j]];"),
    "second global reads the first": ("x[glob0 + j] = x[glob0 + j] + a[k + j] * yi;",
                                      "x[glob0 + j] = x[glob0 + j] + a[k] * yi;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        shutil.copy(f, tmp_path)
    src = (tmp_path / "oracle.c").read_text()
    assert old in src, f"mutation site for '{name}' not found"
    (tmp_path / "oracle.c").write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle_mutant.so"
    srcs = sorted(str(p) for p in tmp_path.glob("*.c"))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(lib), *srcs, "-lm"],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")], env=env, capture_output=True, text=True,
                       cwd=ROOT)
    assert r.returncode != 0, f"pins did not catch mutant '{name}'"
