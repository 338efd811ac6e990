"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a COPY of the C oracle (a dropped factor, a
wrong sign, a wrong normaliser, a transposed operand, ...), builds it into a
temporary library, and runs the pin suite against it in a subprocess: the
suite must fail.  Nothing here touches the committed oracle or any GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ptsne_oracle.c")

MUTANTS = {
    "gradient factor 2 instead of 4 (Eq. 6)":
        ("double c = 4.0 * (P[i * z + j] - q) * w;", "double c = 2.0 * (P[i * z + j] - q) * w;"),
    "p + q instead of p - q (Eq. 6)":
        ("double c = 4.0 * (P[i * z + j] - q) * w;", "double c = 4.0 * (P[i * z + j] + q) * w;"),
    "row-restricted gradient with p + q (Eq. 6)":
        ("double c = 4.0 * (Prows[r * z + j] - w / Z) * w;", "double c = 4.0 * (Prows[r * z + j] + w / Z) * w;"),
    "joint P divided by n instead of 2n (Eq. 3)":
        ("const double inv2n = 1.0 / (2.0 * (double)z);", "const double inv2n = 1.0 / ((double)z);"),
    "Z includes the diagonal (Eq. 4)":
        ("            if (l != k) s += cauchy(Y, od, k, l);", "            s += cauchy(Y, od, k, l);"),
    "Gaussian of the squared distance squared (Eq. 1)":
        ("        double e = exp(-beta * t);", "        double e = exp(-beta * t * t);"),
    "entropy drops beta (Eq. 2)":
        ("    return log(S) + beta * T / S;", "    return log(S) + T / S;"),
    "symmetrisation without the transpose (Eq. 3)":
        ("(C[i * z + j] + C[j * z + i])", "(C[i * z + j] + C[i * z + j])"),
    "ascent instead of descent (Eq. 12)":
        ("vel[i] = momentum * vel[i] - eta * gm * g;", "vel[i] = momentum * vel[i] + eta * gm * g;"),
    "gains rule inverted":
        ("gains[i] = differ ? gains[i] + 0.2 : gains[i] * 0.8;",
         "gains[i] = differ ? gains[i] * 0.8 : gains[i] + 0.2;"),
    "learning rate log n instead of log(n-1) (Eq. 13)":
        ("return log((double)(z - 1)) * (hi - lo) * 0.5;", "return log((double)(z)) * (hi - lo) * 0.5;"),
    "normalised cost denominator 2 log n (Eq. 9)":
        ("    return -H / (log((double)z) + log((double)(z - 1)));",
         "    return -H / (2.0 * log((double)z));"),
    "distance index mix-up":
        ("            double t = X[i * d + k] - X[j * d + k];",
         "            double t = X[i * d + k] - X[j * d + (k + 1) % d];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site vanished: {old}"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(mut),
                    "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, PTSNE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
