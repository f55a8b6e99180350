"""The oracle's pins catch plausible mistakes (CPU).

Each case plants one mistake in a copy of oracle/jefi_oracle.c -- a dropped
term, a wrong sign, a transposed operand, an off-by-one slot, a missing
factor, swapped interpolation weights -- builds it, and runs the pins of
test_oracle_pins.py (floor rule) or test_oracle_interp_pins.py (second-order
variant) against that library (JEFI_ORACLE_LIB).  Every mutant must fail at least one pin.  The
pins stop at the first failure, so a caught mutant costs little."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "jefi_oracle.c")

# (name, text in the floor-rule sum, planted replacement)
MUTANTS = [
    ("dJ/dt term of E dropped",
     "te[a] = D[a] * sc - dj[a] / (c * c * R);", "te[a] = D[a] * sc;"),
    ("dJ/dt term of E with the wrong sign",
     "te[a] = D[a] * sc - dj[a] / (c * c * R);", "te[a] = D[a] * sc + dj[a] / (c * c * R);"),
    ("dJ/dt term of E with 1/c instead of 1/c^2",
     "te[a] = D[a] * sc - dj[a] / (c * c * R);", "te[a] = D[a] * sc - dj[a] / (c * R);"),
    ("drho/dt term of E dropped",
     "const double sc = r_n / R3 + dr / (c * R2);", "const double sc = r_n / R3;"),
    ("drho/dt term of E without 1/c",
     "const double sc = r_n / R3 + dr / (c * R2);", "const double sc = r_n / R3 + dr / R2;"),
    ("backward difference without the previous slice",
     "dr = (r_n - r_prev) / dt;", "dr = r_n / dt;"),
    ("B as D x V instead of V x D",
     "nadd(&b[a], tb[a]);", "nadd(&b[a], -tb[a]);"),
    ("J components transposed in B",
     "V[a] = Jn[a] / R3 + dj[a] / (c * R2);", "V[a] = Jn[(a + 1) % 3] / R3 + dj[a] / (c * R2);"),
    ("dJ/dt term of B dropped",
     "V[a] = Jn[a] / R3 + dj[a] / (c * R2);", "V[a] = Jn[a] / R3;"),
    ("retarded slot one too late",
     "const int64_t n = (int64_t)floor((T - R / c) / dt);",
     "const int64_t n = (int64_t)floor((T - R / c) / dt) + 1;"),
    ("retarded time without 1/c",
     "const int64_t n = (int64_t)floor((T - R / c) / dt);",
     "const int64_t n = (int64_t)floor((T - R) / dt);"),
    ("cell centres at lo + i d",
     "double off = ((double)i + 0.5) * d;", "double off = ((double)i) * d;"),
    ("cell volume missing",
     "E[3 * o + a] = k_e * dV * nval(&e[a]);", "E[3 * o + a] = k_e * nval(&e[a]);"),
    ("screening box one axis only",
     "if (fabs(dx) <= screen[0] && fabs(dy) <= screen[1] && fabs(dz) <= screen[2])",
     "if (fabs(dx) <= screen[0])"),
]


def _run_pins(text, tmp, pins="test_oracle_pins.py"):
    src = os.path.join(tmp, "oracle_copy.c")
    lib = os.path.join(tmp, "liboracle_copy.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", lib, src, "-lm"], check=True)
    env = dict(os.environ, JEFI_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                           "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("pins", ["test_oracle_pins.py", "test_oracle_interp_pins.py"])
def test_unmutated_copy_passes(pins):
    """Control: the pins pass on a copy built the same way, so a failure
    below comes from the planted mistake."""
    with tempfile.TemporaryDirectory() as tmp:
        r = _run_pins(open(SRC).read(), tmp, pins)
    assert r.returncode == 0, r.stdout[-2000:]


# (name, text in the second-order sum, planted replacement): pinned by
# test_oracle_interp_pins.py
INTERP_MUTANTS = [
    ("interpolation weights swapped",
     "const double r_n = (1.0 - w) * r2[0] + w * r2[1];", "const double r_n = w * r2[0] + (1.0 - w) * r2[1];"),
    ("one-sided instead of central difference",
     "hist_at(rho, Ns, m + 1, cell, -1) - hist_at(rho, Ns, m - 1, cell, -1)",
     "hist_at(rho, Ns, m, cell, -1) - hist_at(rho, Ns, m - 1, cell, -1)"),
    ("drho/dt not interpolated",
     "const double dr = (1.0 - w) * dr2[0] + w * dr2[1];", "const double dr = dr2[0];"),
    ("dJ/dt not interpolated",
     "dj[a] = (1.0 - w) * dj2[0][a] + w * dj2[1][a];", "dj[a] = dj2[0][a];"),
    ("no interpolation weight (the floor rule)",
     "const double w = u - fl;", "const double w = 0.0;"),
    ("derivative before the first slice not zero",
     "if (m < 0) {", "if (m < -1) {"),
]


@pytest.mark.parametrize("name,old,new", INTERP_MUTANTS, ids=[m[0] for m in INTERP_MUTANTS])
def test_interp_pins_catch_planted_mistake(name, old, new):
    text = open(SRC).read()
    start = text.index("int oracle_fields_interp(")
    end = text.index("\n}\n", start)
    part = text[start:end]
    assert part.count(old) == 1, f"mutation site not unique: {old}"
    mutated = text[:start] + part.replace(old, new) + text[end:]
    with tempfile.TemporaryDirectory() as tmp:
        r = _run_pins(mutated, tmp, "test_oracle_interp_pins.py")
    assert r.returncode == 1, f"no pin caught: {name}\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new):
    text = open(SRC).read()
    # plant it in the floor-rule sum (cell centres: the shared helper before it)
    start = text.index("int oracle_fields(") if "off =" not in old else 0
    end = text.index("int oracle_fields_interp(")
    part = text[start:end]
    assert part.count(old) == 1, f"mutation site not unique: {old}"
    mutated = text[:start] + part.replace(old, new) + text[end:]
    with tempfile.TemporaryDirectory() as tmp:
        r = _run_pins(mutated, tmp)
    assert r.returncode == 1, f"no pin caught: {name}\n{r.stdout[-2000:]}"
