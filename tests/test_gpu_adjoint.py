"""Derivative of the Eq. 1 loss (tangent-linear through fit, relaxation,
extension and Eq. 1) against central finite differences: the oracle's FP64
FD gradient on small cases, the library's own FP64 loss on the 3x3 cell of
grid 96x96x192, and the torch.autograd.Function built on it."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from tests.gpu_common import device_tracks
from workloads.configs import UM

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4     # relative, per component


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def P():
    import paper_2605_13987_gb300 as P
    return P


def _sensor(P, w):
    s = P.Sensor(w.grid, w.columns)
    s.fit(n_az=w.fit.n_az, n_h=w.fit.n_h, v_w=w.fit.v_w, az0=w.fit.az0)
    s.relax(w.times)
    return s


def _tiny():
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    tr = W.configs.mip_tracks(w.grid, 3, 12, np.random.default_rng(4))
    return w, tr


def _check_grad(g, fd, r, tol=GRAD_TOL):
    """Gradients in relative units (dL per relative change of each parameter;
    the radius one times r): the largest difference within tol of the largest
    component, and each component within 10 tol of itself or of that scale."""
    G = np.asarray(g, dtype=float) * np.array([1.0, 1.0, r, 1.0])[: len(g)]
    F = np.asarray(fd, dtype=float) * np.array([1.0, 1.0, r, 1.0])[: len(fd)]
    scale = np.max(np.abs(F))
    err = np.abs(G - F)
    assert np.max(err) <= tol * scale, (G, F, err / scale)
    assert np.all(err <= 10 * tol * np.maximum(np.abs(F), 0.1 * scale)), (G, F, err / np.abs(F))


def _rounded(tr):
    """The tracks as the library sees them (FP32 positions and velocities)."""
    from dataclasses import replace
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return replace(tr, x=f(tr.x), y=f(tr.y), z=f(tr.z), vx=f(tr.vx), vy=f(tr.vy), vz=f(tr.vz))


def test_loss_matches_oracle(P, torch):
    """FP64 field (FP64 interpolation, time weights and currents): within
    1e-9 for the tracks as the library sees them (FP32 positions and
    velocities); FP32 field: within the FP32 bound."""
    w, tr = _tiny()
    L_ref = A.loss(w, _rounded(tr))[0]
    sen = _sensor(P, w)
    try:
        t = device_tracks(tr, torch)
        assert abs(sen.loss(t, "fp64") - L_ref) < 1e-9 * L_ref
        assert abs(sen.loss(t, "fp32") - L_ref) < 1e-5 * L_ref
    finally:
        sen.close()


def test_gradient_matches_oracle_fd(P, torch):
    w, tr = _tiny()
    fd = A.fd_grad(w, tr, rel_step=1e-4)
    sen = _sensor(P, w)
    try:
        L, g = sen.loss_grad(device_tracks(tr, torch))
        trunc = sen.info()["grad_trunc_rel"]
    finally:
        sen.close()
    print("gpu", g, "fd", fd, "trunc", trunc)
    _check_grad(g, fd, w.columns[0].radius)


def test_host_tracks_give_the_same_gradient(P, torch):
    w, tr = _tiny()
    sen = _sensor(P, w)
    try:
        L1, g1 = sen.loss_grad(device_tracks(tr, torch))
        host = device_tracks(tr, torch, device="cpu")
        host = {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in host.items()}
        L2, g2 = sen.loss_grad(host)
    finally:
        sen.close()
    assert abs(L1 - L2) <= 1e-12 * L1 and np.allclose(g1, g2, rtol=1e-10, atol=0)


def test_readout_resistivity_dominates_bias(P, torch):
    """Sec. 5 ordering on a 3x3 matrix, and agreement with the oracle's FD
    gradient for the two resistivity scales."""
    rng = np.random.default_rng(3)
    grid, cols = W.configs.pixel_matrix(3, 55 * UM, 60 * UM, 48, 16, 8 * UM, 0.75e-2, 0.75e-2, 16, rng)
    w = W.Workload("m3", grid, cols, W.FitSpec(), W.log_times(12))
    tr = W.configs.mip_tracks(grid, 4, 12, np.random.default_rng(5))
    tr.x = 55 * UM + np.mod(tr.x, 55 * UM)
    tr.y = 55 * UM + np.mod(tr.y, 55 * UM)
    fd = A.fd_grad(w, tr, rel_step=1e-4, params=[0, 1])
    sen = _sensor(P, w)
    try:
        L, g = sen.loss_grad(device_tracks(tr, torch))
    finally:
        sen.close()
    assert g[0] < 0 and abs(g[1]) < 0.2 * abs(g[0])
    print("m3 gpu", g[:2], "fd", fd[:2])
    _check_grad(g[:2], fd[:2], 1.0)


def test_adjoint_workload_gradient_vs_fd_of_fp64_loss(P, torch):
    """3x3 cell at grid 96x96x192, 256 time samples, 1e4 tracks: the
    hand-written gradient against central differences of the library's FP64
    loss (plain FP64 field and Eq. 1) on re-fitted perturbed designs."""
    from paper_2605_13987_gb300.autograd import design_at
    w = W.workload("c4")                         # the configuration's 1e4 tracks of 100 steps
    tr = device_tracks(w.tracks, torch)
    base = np.array([1.0, 1.0, 0.0, 1.0])
    sen = _sensor(P, w)
    try:
        L, g = sen.loss_grad(tr)
        trunc = sen.info()["grad_trunc_rel"]
        L64 = sen.loss(tr, "fp64")
    finally:
        sen.close()
    assert abs(L - L64) < 1e-5 * L64
    def fd_at(k, h):
        vals = []
        for sgn in (+1, -1):
            th = base.copy()
            th[k] += sgn * h
            grid, cols, t = design_at(w.grid, w.columns, tr, th)
            s = P.Sensor(grid, cols)
            try:
                s.fit()
                s.relax(w.times)
                vals.append(s.loss(t, "fp64"))
            finally:
                s.close()
        return (vals[0] - vals[1]) / (2 * h)

    r = w.columns[0].radius
    fd = np.array([fd_at(0, 1e-4), fd_at(1, 1e-4), fd_at(2, 1e-4 * r), 0.0])
    # lambda rescales the FP32 track arrays, whose rounding moves the loss by ~1e-7 of itself:
    # larger steps with Richardson extrapolation keep that noise below the tolerance
    d1, d2 = fd_at(3, 5e-3), fd_at(3, 1e-2)
    fd[3] = (4 * d1 - d2) / 3
    print("c4 gpu", g, "fd", fd, "lambda steps", d1, d2, "trunc", trunc)
    _check_grad(g, fd, r)


def test_autograd_function(P, torch):
    from paper_2605_13987_gb300.autograd import eq1_loss, design_at
    w, tr = _tiny()
    t = device_tracks(tr, torch)
    theta0 = [1.2, 0.8, 0.5 * UM, 1.05]
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    L = eq1_loss(theta, w.grid, w.columns, w.times, t)
    L.backward()
    g = theta.grad.numpy()
    def fd_at(k, h):
        vals = []
        for sgn in (+1, -1):
            th = np.array(theta0)
            th[k] += sgn * h
            grid, cols, tk = design_at(w.grid, w.columns, t, th)
            s = P.Sensor(grid, cols)
            try:
                s.fit()
                s.relax(w.times)
                vals.append(s.loss(tk, "fp64"))
            finally:
                s.close()
        return (vals[0] - vals[1]) / (2 * h)

    r = w.columns[0].radius + theta0[2]
    fd = np.array([fd_at(0, 1e-4), fd_at(1, 1e-4), fd_at(2, 1e-4 * r),
                   (4 * fd_at(3, 5e-3) - fd_at(3, 1e-2)) / 3])
    print("autograd", g, "fd", fd)
    _check_grad(g, fd, r)


def test_loss_error_paths(P, torch):
    w, tr = _tiny()
    t = device_tracks(tr, torch)
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        with pytest.raises(P.WTError, match="WT_ERR_STATE"):
            s.loss_grad(t)
        s.relax(w.times)
        empty = dict(t, n_tracks=0)
        assert s.loss(empty) == 0.0
        L, g = s.loss_grad(empty)
        assert L == 0.0 and not np.any(g)
    finally:
        s.close()
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit(tikhonov=1e-12)
        s.relax(w.times)
        with pytest.raises(P.WTError, match="WT_ERR_UNSUPPORTED"):
            s.loss_grad(t)
    finally:
        s.close()


def test_gradient_stage_timing(P, torch):
    """The library's CUDA-event split of one loss derivative: every stage timed, none negative,
    zero again when timing is off."""
    w, tr = _tiny()
    s = _sensor(P, w)
    try:
        t = device_tracks(tr, torch)
        s.set_timing(True)
        L1, g1 = s.loss_grad(t)
        st = s.grad_timing()
        s.set_timing(False)
        L2, g2 = s.loss_grad(t)
        off = s.grad_timing()
    finally:
        s.close()
    assert set(st) == {"base", "shared", "fit_tangent", "modal_tangent", "tangent_basis", "tangent_fields"}
    assert all(v > 0.0 for v in st.values()), st
    assert all(v == 0.0 for v in off.values()), off
    # the loss reductions add block sums atomically: equal up to their order
    assert abs(L1 - L2) <= 1e-12 * abs(L1) and np.allclose(g1, g2, rtol=1e-9, atol=0)
