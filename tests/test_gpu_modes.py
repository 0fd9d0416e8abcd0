"""Mode-count error study (the synthetic analogue of the paper's error-versus-N
study, section 3.5): junction solves with N modes against a solve with more
modes, on an inflow rich in harmonics.  Every solve iterates to 1e-10 r_ref;
the space-time L2 error of the N-mode velocity (missing modes counted as
error) must fall as N grows, and it stays of the order of the inflow's own
truncation error."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_error_falls_with_the_number_of_modes():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    out = bench.run_mode_study(None, Ns=(2, 3, 5), N_ref=7, h=0.6, Re=50.0, Wo=8.0, amp=0.4)
    rows = {r["N"]: r for r in out["rows"]}
    assert all(r["converged"] for r in out["rows"]), out["rows"]
    errs = [rows[N]["field_rel_l2_vs_ref"] for N in (2, 3, 5)]
    assert errs[0] > errs[1] > errs[2] > 0.0, errs
    for N in (2, 3, 5):
        trunc = rows[N]["inflow_truncation_rel_l2"]
        assert 0.05 * trunc < rows[N]["field_rel_l2_vs_ref"] < 20.0 * trunc, rows[N]
