"""Full-size parity of the dipole workload (point-list observers on four
shells, supplied and backward derivatives) and of the paper's own test
sources (Sec. 3.1 step-on constant, Sec. 3.2 sinusoidal) at the paper's
sizes.  FP64 within 1e-12 of the oracle; the FP32 errors are recorded per
shell and bounded."""
import json

import numpy as np
import pytest

import paper_2104_05426_gb300 as jefi
from jefi_cases import create, gpu_fields, history, oracle_fields, push_all, rel_l2
from workloads import c3_dipole, e1_constant, e2_sinusoidal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("supplied", [True, False])
def test_dipole_shells_full_size(gpu, supplied):
    p = c3_dipole()
    hist = history(p)
    times = p.times[:2]
    ref = oracle_fields(p, hist, times, supplied=supplied)
    radii = np.linalg.norm(p.obs_points, axis=1)
    report = {}
    for prec in ("fp64", "fp32c", "fp32"):
        h = create(p, prec, supplied=supplied)
        push_all(h, hist, supplied=supplied)
        E, B = gpu_fields(h, times)
        errs = {}
        for R in (5.0, 10.0, 20.0, 40.0):
            m = np.abs(radii - R) < 1e-6 * R
            errs[R] = max(max(rel_l2(E[i][m], ref[i][0][m]), rel_l2(B[i][m], ref[i][1][m]))
                          for i in range(len(times)))
        report[prec] = errs
        if prec == "fp64":
            assert max(errs.values()) <= 1e-12
        else:
            # measured on GB300: <= 2.0e-6 (compensated), <= 2.6e-6 (plain), worst
            # in the far zone where the dipole field cancels
            assert max(errs.values()) <= 1e-5
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)
    print("dipole rel-L2 vs oracle by shell", "supplied" if supplied else "backward",
          json.dumps({k: {str(r): f"{e:.2e}" for r, e in v.items()} for k, v in report.items()}))


@pytest.mark.parametrize("make", [e1_constant, e2_sinusoidal])
def test_paper_sources_at_paper_size(gpu, make):
    p = make()
    hist = history(p)
    ref = oracle_fields(p, hist, p.times)
    for prec, tol in (("fp64", 1e-12), ("fp32c", 1e-5)):
        h = create(p, prec)
        push_all(h, hist)
        E, B = gpu_fields(h, p.times)
        for i in range(len(p.times)):
            assert rel_l2(E[i], ref[i][0]) <= tol, (p.name, prec, i, rel_l2(E[i], ref[i][0]))
            assert rel_l2(B[i], ref[i][1]) <= tol, (p.name, prec, i, rel_l2(B[i], ref[i][1]))
        jefi.jefi_destroy(h)
