"""Pins of the oracle's finite-difference gradient (the reference for the
library's hand-written derivative)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import adjoint as A
from workloads.configs import UM


def _case(rho=None):
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    if rho is not None:
        w = W.configs.with_resistivity(w, rho)
    tr = W.configs.mip_tracks(w.grid, 3, 12, np.random.default_rng(4))
    return w, tr


def test_fd_gradient_is_step_consistent():
    w, tr = _case()
    g1 = A.fd_grad(w, tr, rel_step=1e-4)
    g2 = A.fd_grad(w, tr, rel_step=4e-4)
    L = A.loss(w, tr)[0]
    assert np.all(np.isfinite(g1)) and L > 0
    assert np.allclose(g1, g2, rtol=2e-3, atol=1e-6 * L)


def test_perfect_conductor_has_no_resistivity_gradient():
    w, tr = _case(rho=1e-14)
    L = A.loss(w, tr)[0]
    g = A.fd_grad(w, tr, rel_step=1e-3, params=[0, 1])
    assert abs(g[0]) < 1e-8 * L and abs(g[1]) < 1e-8 * L


def test_readout_resistivity_dominates_bias():
    """Sec. 5: in a pixel matrix the bias electrodes barely affect the signal
    (their potential hardly changes), the readout's resistance does.  3x3
    matrix, tracks through the central (driven) pixel."""
    rng = np.random.default_rng(3)
    grid, cols = W.configs.pixel_matrix(3, 55 * UM, 60 * UM, 48, 16, 8 * UM, 0.75e-2, 0.75e-2, 16, rng)
    w = W.Workload("m3", grid, cols, W.FitSpec(), W.log_times(12))
    tr = W.configs.mip_tracks(grid, 4, 12, np.random.default_rng(5))
    tr.x = 55 * UM + np.mod(tr.x, 55 * UM)
    tr.y = 55 * UM + np.mod(tr.y, 55 * UM)
    g = A.fd_grad(w, tr, rel_step=1e-4, params=[0, 1])
    assert g[0] < 0 and abs(g[1]) < 0.2 * abs(g[0])


def test_current_tangents_give_the_loss_gradient():
    """Chain rule: dL/dtheta = 2 mean(i di/dtheta), with both sides taken by
    central differences of the oracle at the same step."""
    w, tr = _case()
    L, i = A.loss(w, tr)
    di = A.fd_currents(w, tr, rel_step=1e-4)
    g = A.fd_grad(w, tr, rel_step=1e-4)
    chain = 2.0 * np.mean(i[None] * di, axis=(1, 2))
    assert np.allclose(chain, g, rtol=1e-6, atol=1e-9 * L)
