"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C sources (a dropped
term, a wrong sign, index or table, a transposed weight), builds the copy on
the CPU, and runs a pin file against it in a child process through
BSDE_ORACLE_LIB: at least one pin must fail.  A control build of the
unchanged sources passes the same way.
"""
import os
import shutil
import subprocess
import sys

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PINS = "tests/test_oracle_pins.py"
PINS_2D = "tests/test_oracle_2d.py"
PINS_GENERAL = "tests/test_oracle_general.py"
PINS_VARIANTS = "tests/test_oracle_variants.py"

# (name, source file, text, replacement, pin file)
MUTATIONS = [
    ("forward drift dropped from the node position (Eq. 21)", "oracle.c",
     "double X = xi + orc_fwd_a(p, xi) * j * dt + orc_fwd_b(p, xi) * dW;",
     "double X = xi + orc_fwd_b(p, xi) * dW;", PINS),
    ("Table 1 row read from Table 2", "oracle.c",
     "gy[j] = (double)ORC_GY_NUM[K - 1][j] / (double)ORC_GY_DEN[K - 1][j];",
     "gy[j] = (double)ORC_GZ_NUM[K - 1][j] / (double)ORC_GZ_DEN[K - 1][j];", PINS),
    ("E[f] in place of E[f DeltaW] in the z line (Eq. 20)", "oracle.c",
     "sfw += gz[j] * e[5 * (j - 1) + 2];", "sfw += gz[j] * e[5 * (j - 1) + 1];", PINS),
    ("sign of the explicit driver sum in A (Eq. 20)", "oracle.c",
     "double A = e[5 * (ky - 1) + 3] + h * sf;", "double A = e[5 * (ky - 1) + 3] - h * sf;",
     PINS),
    ("driver time t_{n+j-1} for t_{n+j}", "oracle.c",
     "double tj = (n + j) * dt;", "double tj = (n + j - 1) * dt;", PINS),
    ("DeltaW dropped from E[f DeltaW]", "oracle.c",
     "efw += w * F * dW;", "efw += w * F;", PINS),
    ("spline second derivative of the wrong node", "oracle.c",
     "(th * th * th - th) * M[c + 1]", "(th * th * th - th) * M[c]", PINS),
    ("E[y^] in place of E[z^] as the z line's first term", "oracle.c",
     "double first = p->zform ? e[4] / dt : e[0];",
     "double first = p->zform ? e[4] / dt : e[3];", PINS),
    ("Picard weight gamma_1 in place of gamma_0", "oracle.c",
     "double yn1 = A + h * gy[0] * orc_driver(p, tn, xi, y, z);",
     "double yn1 = A + h * gy[1] * orc_driver(p, tn, xi, y, z);", PINS),
    ("cell-averaged payoff: the -d term dropped in the strike's cell", "oracle.c",
     "*u = K * (expm1(d) - d) / dx;", "*u = K * expm1(d) / dx;", PINS),
    ("spline right-hand side 3 (second differences) in place of 6", "oracle.c",
     "double rhs = 6.0 * (v[q] - 2.0 * v[q + 1] + v[q + 2]) / (dx * dx);",
     "double rhs = 3.0 * (v[q] - 2.0 * v[q + 1] + v[q + 2]) / (dx * dx);", PINS),
    ("Gauss-Hermite Newton polish stepping the wrong way", "oracle.c",
     "a -= pL / d;", "a += pL / d;", PINS),
    ("one-step start-up with the main step dt instead of dt / S", "oracle.c",
     "q.N = p->N * S;", "q.N = p->N;", PINS_VARIANTS),
    ("2-D: the DeltaW components of the z line swapped", "oracle2d.c",
     "s += gz[j] * (E[j - 1][3 + d] - E[j - 1][d]);",
     "s += gz[j] * (E[j - 1][4 - d] - E[j - 1][d]);", PINS_2D),
    ("2-D: sign of a one-sided difference coefficient", "oracle2d.c",
     "48.0 * f[(i + 1) * s] - 36.0 * f[(i + 2) * s]",
     "48.0 * f[(i + 1) * s] + 36.0 * f[(i + 2) * s]", PINS_2D),
    ("2-D: sign of the outer central difference term", "oracle2d.c",
     "+ 8.0 * f[(i + 1) * s] - f[(i + 2) * s]) / 12.0;",
     "+ 8.0 * f[(i + 1) * s] + f[(i + 2) * s]) / 12.0;", PINS_2D),
    ("2-D: right slope weight of the Hermite basis negated", "oracle2d.c",
     "*h11 = t3 - t2;", "*h11 = t2 - t3;", PINS_2D),
    ("2-D: correlation term dropped from the second coordinate", "oracle2d.c",
     "const double X2 = x2 + p->a2 * j * dt + p->b21 * dW1 + p->b22 * dW2;",
     "const double X2 = x2 + p->a2 * j * dt + p->b22 * dW2;", PINS_2D),
    ("general forward: the slope of b(x) ignored", "oracle.c",
     "return p->forward == ORC_FWD_AFFINE ? p->b_x + p->b_1 * x : p->b_x;",
     "return p->forward == ORC_FWD_AFFINE ? p->b_x : p->b_x;", PINS_GENERAL),
]


def _build_copy(tmp_path, name=None, text=None, repl=None):
    for f in ("oracle.c", "oracle2d.c"):
        shutil.copy(os.path.join(ORACLE_DIR, f), tmp_path / f)
    if name is not None:
        path = tmp_path / name
        src = path.read_text()
        assert src.count(text) == 1, f"mutation target not unique in {name}: {text}"
        path.write_text(src.replace(text, repl))
    out = str(tmp_path / "liboracle_copy.so")
    O.compile_library(str(tmp_path / "oracle.c"), str(tmp_path / "oracle2d.c"), out)
    return out


def _run_pins(lib, pins):
    env = dict(os.environ, BSDE_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", pins, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    return r.returncode, r.stdout[-2000:]


def test_unchanged_copy_passes_the_pins(tmp_path):
    rc, out = _run_pins(_build_copy(tmp_path), PINS)
    assert rc == 0, out


@pytest.mark.parametrize("name,src,text,repl,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, src, text, repl, pins):
    rc, out = _run_pins(_build_copy(tmp_path, src, text, repl), pins)
    assert rc == 1, f"{name}: no pin failed (rc {rc})\n{out}"
