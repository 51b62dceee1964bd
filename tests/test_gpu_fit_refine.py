"""The fit's corrected semi-normal-equations step (Sec. 3 boundary fit) runs either always
(refine=1) or only when a probe of its correction on eight random right-hand-side combinations
exceeds 1e-11 of the solution (refine=0, the default).  Both fits give the same capacitance to
far below the FP64 parity bound, and both match the oracle's QR solution."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fits():
    import torch
    import paper_2605_13987_gb300 as P
    assert torch.cuda.is_available()
    w = W.workload("c1")
    out = {}
    for refine in (0, 1):
        sen = P.Sensor(w.grid, w.columns)
        sen.fit(refine=refine)
        out[refine] = (sen.capacitance(), sen.info())
        sen.close()
    return w, out


def test_always_refined_reports_the_full_correction(fits):
    _, out = fits
    info = out[1][1]
    assert info["fit_refined"] == 1
    assert 0.0 <= info["fit_correction"] < 1e-8


def test_probe_skips_a_negligible_correction(fits):
    _, out = fits
    info = out[0][1]
    # the single cell's scaled fit matrix is well conditioned: the correction the probe sees is
    # about cond(A_s)^2 eps (a few 1e-12), below the skip threshold, and the step is skipped
    assert info["fit_correction"] <= 1e-11
    assert info["fit_refined"] == 0
    # the probe estimates the full correction of the always-refined fit
    full = out[1][1]["fit_correction"]
    assert 0.2 * full <= info["fit_correction"] <= 5.0 * full


def test_both_fits_agree_and_match_the_oracle(fits):
    w, out = fits
    c0, c1 = out[0][0], out[1][0]
    assert rel_l2(c0, c1) < 5e-11
    sol = O.solve(w)
    assert rel_l2(c0, sol.fit["Cn"]) < 1e-10
    assert rel_l2(c1, sol.fit["Cn"]) < 1e-10


def test_refine_option_is_validated():
    import paper_2605_13987_gb300 as P
    w = W.workload("c1")
    sen = P.Sensor(w.grid, w.columns)
    with pytest.raises(P.WTError):
        sen.fit(refine=2)
    sen.close()
