"""The FP32 path's rank-r time basis (S5b) on both of its routes: the one-sided Jacobi on the
rows of R from a column-pivoted QR of the charge history (sources >= time samples) and the
Jacobi on the history's own rows (fewer sources than samples).  Against the oracle: the reported
per-sample truncation equals the exact SVD tail of the oracle's charge history, the rank is the
smallest that meets 1e-7 in every sample, and the FP32 field meets 1e-5 in every time sample."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu
UM = 1e-6


@pytest.fixture(scope="module")
def P():
    import torch
    import paper_2605_13987_gb300 as P
    assert torch.cuda.is_available()
    P.load_library()
    return P


# (nz, sources per column, time samples): 2 columns, so 2 m sources
CASES = {"pivoted_qr": (32, 32, 40), "direct": (24, 20, 96)}


@pytest.mark.parametrize("name", sorted(CASES))
def test_time_basis_against_the_oracle(P, name):
    nz, m, nt = CASES[name]
    w = W.tiny_cell(nx=16, nz=nz, n_t=nt, m_req=m, radius=8 * UM)
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    info = sen.info()
    ns = info["n_sources"]
    assert (ns >= nt) == (name == "pivoted_qr")
    Q = sol.q                                               # [ns][nt]
    U, sv, Vt = np.linalg.svd(Q, full_matrices=False)
    norms = np.linalg.norm(Q, axis=0)
    floor = 1e-6 * norms.max()

    def worst(r):
        tail = np.sqrt(((sv[r:, None] * Vt[r:]) ** 2).sum(0))
        return (tail / np.maximum(norms, floor)).max()

    r = info["rank"]
    assert 1 <= r <= 32
    assert abs(info["trunc_rel"] - worst(r)) <= 1e-3 * worst(r) + 1e-15
    assert info["trunc_rel"] <= 1e-7
    if r > 1:
        assert worst(r - 1) > 1e-7                           # the smallest rank that meets the target
    H32 = sen.extend("fp32").double().cpu().numpy()
    sen.close()
    ref = sol.H_full()
    for n in range(ref.shape[0]):
        assert rel_l2(H32[n], ref[n]) < 1e-5
