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

# mistakes in the warm-start oracle (oracle/warm.c), caught by tests/test_oracle_warm.py
WARM_MUTANTS = {
    "adam bias correction of step 1": ("const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);",
                                       "const double c1 = 1.0 - pow(b1, 1), c2 = 1.0 - pow(b2, step);"),
    "adam second moment without square": ("(1.0 - b2) * g[i] * g[i];", "(1.0 - b2) * fabs(g[i]);"),
    "mirrored backward skips the dout rounding": ("const double g = rnd(dout[(b * L + p) * cout + co], mirrored);",
                                                  "const double g = dout[(b * L + p) * cout + co];"),
    "mirrored backward rounds the bias gradient": ("dbias[co] = dbias[co] + dout[(b * L + p) * cout + co];",
                                                   "dbias[co] = dbias[co] + rnd(dout[(b * L + p) * cout + co], "
                                                   "mirrored);"),
    "forward tap reversed": ("const int64_t q = p + t - 2;\n                    if (q < 0 || q >= L) continue;\n"
                             "                    for (int ci = 0; ci < cin; ++ci)\n                        s = s",
                             "const int64_t q = p - t + 2;\n                    if (q < 0 || q >= L) continue;\n"
                             "                    for (int ci = 0; ci < cin; ++ci)\n                        s = s"),
}


def _run_pins_on_mutant(tmp_path, fname, old, new, test_file):
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        shutil.copy(f, tmp_path)
    src = (tmp_path / fname).read_text()
    assert old in src, f"mutation site not found: {old!r}"
    (tmp_path / fname).write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle_mutant.so"
    srcs = sorted(str(p) for p in tmp_path.glob("*.c"))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(lib), *srcs, "-lm"],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", test_file)], env=env, capture_output=True, text=True, cwd=ROOT)
    return r.returncode


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    assert _run_pins_on_mutant(tmp_path, "oracle.c", old, new, "test_oracle.py") != 0, \
        f"pins did not catch mutant '{name}'"


@pytest.mark.parametrize("name", sorted(WARM_MUTANTS))
def test_warm_pins_reject_mutant(name, tmp_path):
    old, new = WARM_MUTANTS[name]
    assert _run_pins_on_mutant(tmp_path, "warm.c", old, new, "test_oracle_warm.py") != 0, \
        f"warm-start pins did not catch mutant '{name}'"
