"""Depth-dependent column resistivity (Sec. 5): the CUDA path against the
oracle with a resistivity profile, and the directional derivative of the
Eq. 1 loss along a profile change against the oracle's finite differences."""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import adjoint as A
from tests.gpu_common import rel_l2, device_tracks
from workloads.configs import UM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def P():
    import paper_2605_13987_gb300 as P
    return P


def _profiled():
    """Tiny cell whose readout column gets 4x the resistivity in the half
    away from its terminal, a linear ramp on the bias column."""
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    cols = list(w.columns)
    c0, c1 = cols
    m0 = c0.n_sources
    p0 = np.full(m0, c0.resistivity)
    p0[: m0 // 2] *= 4.0
    m1 = c1.n_sources
    p1 = c1.resistivity * np.linspace(0.5, 1.5, m1)
    cols = [replace(c0, rho_profile=tuple(p0)), replace(c1, rho_profile=tuple(p1))]
    return replace(w, columns=cols)


def test_profile_charges_and_field_match_oracle(P, torch):
    w = _profiled()
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    try:
        sen.fit()
        sen.relax(w.times)
        assert rel_l2(np.sort(sen.modes()), np.sort(sol.rel["mu"])) < 1e-10
        assert rel_l2(sen.charges(), sol.q.T) < 1e-10
        H = sen.extend("fp32")
        torch.cuda.synchronize()
        assert rel_l2(H.cpu().numpy(), sol.H_full()) < 1e-5
    finally:
        sen.close()


def test_uniform_profile_is_bitwise_uniform(P, torch):
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    a = P.Sensor(w.grid, w.columns)
    cols = [replace(c, rho_profile=tuple([c.resistivity] * c.n_sources)) for c in w.columns]
    b = P.Sensor(w.grid, cols)
    try:
        for s in (a, b):
            s.fit()
            s.relax(w.times)
        assert np.array_equal(a.charges(), b.charges())
    finally:
        a.close()
        b.close()


def test_profile_direction_matches_oracle_fd(P, torch):
    """dL/deps for rho_j -> rho_j (1 + eps delta_j), delta a ramp along the
    readout column and a constant on the bias column, against the oracle's
    FP64 central differences."""
    w = _profiled()
    tr = W.configs.mip_tracks(w.grid, 3, 12, np.random.default_rng(4))
    c0, c1 = w.columns
    d0 = np.linspace(-1.0, 1.0, c0.n_sources)
    d1 = np.full(c1.n_sources, 0.3)
    delta = np.concatenate([d0, d1])

    def at(eps):
        cols = [replace(c0, rho_profile=tuple(np.asarray(c0.rho_profile) * (1 + eps * d0))),
                replace(c1, rho_profile=tuple(np.asarray(c1.rho_profile) * (1 + eps * d1)))]
        return A.loss(replace(w, columns=cols), tr)[0]

    h = 1e-4
    fd = (at(h) - at(-h)) / (2 * h)
    sen = P.Sensor(w.grid, w.columns)
    try:
        sen.fit()
        sen.relax(w.times)
        L, g = sen.loss_grad_profile(device_tracks(tr, torch), delta)
        # the readout-scale component of the full gradient is the direction delta = 1 on that column
        L2, g4 = sen.loss_grad(device_tracks(tr, torch))
        _, g_r = sen.loss_grad_profile(device_tracks(tr, torch),
                                       np.concatenate([np.ones(c0.n_sources), np.zeros(c1.n_sources)]))
    finally:
        sen.close()
    print("profile dir", g, "fd", fd, "readout", g_r, g4[0])
    assert abs(g - fd) < 1e-4 * abs(fd)
    assert abs(g_r - g4[0]) < 1e-9 * abs(g4[0])


def test_profile_errors(P, torch):
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    s = P.Sensor(w.grid, w.columns)
    try:
        with pytest.raises(P.WTError, match="WT_ERR_ARG"):
            s.set_resistivity_profile(0, np.ones(3))
        with pytest.raises(P.WTError, match="WT_ERR_ARG"):
            s.set_resistivity_profile(5, np.ones(w.columns[0].n_sources))
        with pytest.raises(P.WTError, match="WT_ERR_ARG"):
            s.set_resistivity_profile(0, -np.ones(w.columns[0].n_sources))
        s.set_resistivity_profile(0, None)
    finally:
        s.close()
