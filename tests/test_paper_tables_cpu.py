"""The paper's printed memory table against its own memory model (CPU).

Sec. 4 estimates the floats held on the GPU as
  N = (lts + 1) n_s^3 x 4  +  n_o^3 x 6
(rho, J for every resident slice; E, B once) and prints the occupied
memory in Table 3 (tests/golden/paper_table3_memory.txt).  With 4-byte
floats the model leaves a nearly constant remainder (the CUDA context and
libraries) across all fourteen entries, from 1.5 GB to 31 GB; with 8-byte
floats it exceeds the printed memory.  This is the evidence for reading the
paper's storage precision as FP32 (its precision is never stated)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
MIB = 1024.0 * 1024.0


def _table3():
    rows = np.loadtxt(os.path.join(HERE, "golden", "paper_table3_memory.txt"), comments="#")
    return rows[:, 0].astype(int), rows[:, 1].astype(int), rows[:, 2]


def _model_floats(n, lts):
    return (lts + 1) * n ** 3 * 4 + n ** 3 * 6


def test_table3_matches_the_memory_model_with_fp32_storage():
    n, lts, mib = _table3()
    assert len(n) == 14
    rest = mib - _model_floats(n, lts) * 4 / MIB
    # a constant overhead of ~300-360 MiB, independent of a 20x range of sizes
    assert np.all((rest > 250) & (rest < 400)), rest
    assert rest.max() - rest.min() < 100


def test_table3_rules_out_fp64_storage():
    n, lts, mib = _table3()
    over = _model_floats(n, lts) * 8 / MIB - mib
    assert np.all(over[mib > 5000] > 0.8 * mib[mib > 5000])
