"""Pins of the oracle's time relaxation (relax.py)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import relax, geometry
from workloads.configs import UM, OHM_CM


@pytest.fixture(scope="module")
def c1():
    return O.solve(W.workload("c1"))


@pytest.fixture(scope="module")
def tiny():
    return O.solve(W.tiny_cell(nx=8, nz=12, n_t=8))


def test_initial_final_and_neutral(c1):
    s = c1
    r = relax.relax(s.fit["Cn"], s.K, s.b, s.phi_dc, np.array([0.0, 1.0]))
    qinf = s.rel["q_inf"]
    sc = np.abs(qinf).max()
    assert np.abs(r["q"][:, 0]).max() < 1e-10 * sc                   # q(0) = 0
    assert np.abs(r["q"][:, 1] - qinf).max() < 1e-12 * sc              # q(inf) = C phi_DC
    assert np.abs(s.q.sum(axis=0)).max() < 1e-12 * sc                  # neutral at all t
    assert np.all(s.rel["mu"] > 0)
    # readout charge rises monotonically toward its DC value
    off = s.lay.col_off
    qr = s.q[off[0]:off[1]].sum(axis=0)
    assert np.all(np.diff(qr) >= -1e-14 * sc)


def test_modal_exponential_matches_expm(tiny):
    s = tiny
    qe = relax.relax_expm(s.fit["Cn"], s.K, s.b, s.phi_dc, s.times)
    assert np.linalg.norm(qe - s.q) < 1e-9 * np.linalg.norm(s.q)


def test_forward_euler_converges_to_exponential(tiny):
    """Sec. 3's forward-Euler iteration tends to the exact solution, first order in dt."""
    s = tiny
    t = s.times[[2, 5]]
    ref = relax.relax(s.fit["Cn"], s.K, s.b, s.phi_dc, t)["q"]
    mu_max = s.rel["mu"].max()
    errs = []
    for k in (1, 2, 4):
        dt = 1.0 / (mu_max * k)
        qe = relax.relax_euler(s.fit["Cn"], s.K, s.b, t, dt)
        errs.append(np.linalg.norm(qe - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[2] < 5e-2


def test_perfect_conductor_limit_is_static(c1):
    """rho -> 0: the charges sit at their DC values at every sample (static Ramo)."""
    w = W.configs.with_resistivity(W.workload("c1"), 1e-14)
    s = O.solve(w)
    qinf = s.rel["q_inf"]
    assert np.abs(s.q - qinf[:, None]).max() < 1e-12 * np.abs(qinf).max()
    # DC charges do not depend on the resistivity
    assert np.allclose(qinf, c1.rel["q_inf"], rtol=0, atol=1e-12 * np.abs(qinf).max())


def test_rc_line_slowest_mode():
    """Long readout line facing a perfectly conducting bias line: the slowest
    mode of an open-ended RC line driven at one end, mu_1 = pi^2/(4 L^2 R' C'),
    with C' = q_inf(readout) / (V_w L) and R' = rho / (pi r^2)."""
    L, pitch, r = 400 * UM, 20 * UM, 2.0 * UM
    grid = W.GridSpec(pitch, pitch, L, 16, 16, 128)
    rho = 1.0 * OHM_CM
    cols = [W.ColumnSpec(pitch / 2, pitch / 2, 0, L, r, rho, 1, 1, 128),
            W.ColumnSpec(0, 0, 0, L, r, 1e-12, 0, 0, 128)]
    s = O.solve(W.Workload("rc", grid, cols, W.FitSpec(), W.log_times(8)))
    qr = s.rel["q_inf"][:128].sum()
    Cp = qr / L
    Rp = rho / (math.pi * r * r)
    mu1 = math.pi ** 2 / (4 * L * L * Rp * Cp)
    assert abs(s.rel["mu"][0] / mu1 - 1.0) < 0.05
