"""Relaxation modes from the divide-and-conquer eigensolver (tridiagonalisation,
Cuppen merges with deflation, blocked back-transformation) against the FP64
oracle and against the two-sided Jacobi solver, on a 3x3 pixel cell whose
columns all share one resistivity: the cell's fourfold symmetry gives exactly
degenerate modes, the case where the merges' deflation keeps the eigenvectors
orthogonal."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.configs import pixel_matrix, UM, OHM_CM
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def symmetric_cell():
    rng = np.random.default_rng(11)
    grid, cols = pixel_matrix(3, 55 * UM, 100 * UM, 24, 32, 5 * UM, 0.3 * OHM_CM, 0.3 * OHM_CM, 32, rng)
    return W.Workload("sym3x3", grid, cols, W.FitSpec(), W.log_times(48), seed=11)


@pytest.fixture(scope="module")
def case():
    import torch
    import paper_2605_13987_gb300 as P
    assert torch.cuda.is_available()
    w = symmetric_cell()
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    yield w, sol, sen
    sen.close()


def test_cell_has_degenerate_modes(case):
    w, sol, sen = case
    mu = np.sort(sol.rel["mu"])
    close = np.sum(np.diff(mu) <= 1e-9 * mu[1:])
    assert close >= 10, close


def test_modes_ascending_and_match_oracle(case):
    w, sol, sen = case
    mu = sen.modes()
    assert np.all(np.diff(mu) >= 0)
    assert rel_l2(mu, np.sort(sol.rel["mu"])) < TOL64
    assert np.max(np.abs(mu - np.sort(sol.rel["mu"])) / np.sort(sol.rel["mu"])) < 1e-6


def test_charge_history_matches_oracle(case):
    w, sol, sen = case
    q = sen.charges()
    assert rel_l2(q, sol.q.T) < TOL64
    for n in (0, 1, len(w.times) // 2, len(w.times) - 1):
        assert rel_l2(q[n], sol.q[:, n]) < 100 * TOL64


def test_same_history_as_jacobi(case, monkeypatch):
    import paper_2605_13987_gb300 as P
    w, sol, sen = case
    monkeypatch.setenv("WT_EIGEN", "jacobi")
    s2 = P.Sensor(w.grid, w.columns)
    s2.fit()
    s2.relax(w.times)
    try:
        assert rel_l2(np.sort(s2.modes()), sen.modes()) < 1e-12
        assert rel_l2(s2.charges(), sen.charges()) < TOL64
    finally:
        s2.close()


@pytest.mark.parametrize("nz,m", [(8, 8), (16, 16), (18, 17), (40, 40)])
def test_small_and_ragged_sizes(nz, m):
    """Problem sizes below, at and past one leaf (the reduced pencil has 2 m - 1 rows)."""
    import paper_2605_13987_gb300 as P
    w = W.tiny_cell(nx=8, nz=nz, n_t=12, m_req=m)
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    try:
        sen.fit()
        sen.relax(w.times)
        assert rel_l2(sen.modes(), np.sort(sol.rel["mu"])) < TOL64
        assert rel_l2(sen.charges(), sol.q.T) < TOL64
    finally:
        sen.close()
