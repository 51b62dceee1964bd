"""Signal-shape features (wt_features), current tangents (wt_eq1_tangents)
and the geometry scan driver built on them, against the oracle: the
features kernel element by element on synthetic waveforms of ragged
lengths and degenerate shapes, the tangents against central differences of
the FP64 oracle's currents, and a bias-diameter scan's features and feature
sensitivities against the oracle's features of its own currents and
difference tangents."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from oracle import electronics as OE
from oracle import features as OF
from tests.gpu_common import device_tracks, rel_l2
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


@pytest.fixture(scope="module")
def sen(P):
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    s = P.Sensor(w.grid, w.columns)
    s.fit(n_az=w.fit.n_az, n_h=w.fit.n_h, v_w=w.fit.v_w, az0=w.fit.az0)
    s.relax(w.times)
    yield s, w
    s.close()


def _waveforms(n, rng):
    t = np.arange(n, dtype=np.float64)
    rows = []
    for k in range(9):
        a, b = rng.uniform(3, 40), rng.uniform(1, 8)
        x = (np.exp(-t / a) - np.exp(-t / b)) * rng.uniform(0.2, 3.0) + 1e-3 * rng.standard_normal(n)
        rows.append(-x if k % 2 else x)
    rows.append(np.zeros(n))                               # degenerate: zero waveform
    rows.append(np.full(n, 0.75))                          # all samples tie: first index
    z = np.zeros(n)
    z[0] = -2.0
    if n > 1:
        z[-1] = 2.0                                        # |x| ties with opposite signs: first index, A < 0
    rows.append(z)
    rows.append(np.linspace(1.0, 0.0, n))                  # maximum at index 0: no crossing
    rows.append(np.linspace(0.0, 1.0, n))                  # maximum at the last index
    return np.asarray(rows, dtype=np.float32)


def _check_features(f, ref, x, dt):
    f = np.asarray(f)
    assert np.array_equal(f[:, 0], ref[:, 0])              # the amplitude is a sample
    tscale = np.maximum(np.abs(ref[:, [1, 3, 4, 5]]), dt)
    assert np.all(np.abs(f[:, [1, 3, 4, 5]] - ref[:, [1, 3, 4, 5]]) <= 1e-12 * tscale)
    qscale = dt * np.abs(x.astype(np.float64)).sum(axis=1) + 1e-300
    assert np.all(np.abs(f[:, 2] - ref[:, 2]) <= 1e-12 * qscale)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 257, 1000])
def test_features_match_oracle(P, torch, sen, n):
    s, _ = sen
    rng = np.random.default_rng(n)
    x = _waveforms(n, rng)
    dx = rng.standard_normal((3,) + x.shape).astype(np.float32)
    dt, t0 = 2.5e-11, 1e-9
    xd = torch.tensor(x, device="cuda")
    dxd = torch.tensor(dx, device="cuda")
    f, df = s.features(xd, dt, t0, dx=dxd, lo=0.1, hi=0.9, cfd=0.3)
    torch.cuda.synchronize()
    ref = OF.features(x, t0, dt, 0.1, 0.9, 0.3)
    _check_features(f.cpu().numpy(), ref, x, dt)
    dref = OF.sensitivities(x, dx, t0, dt, 0.1, 0.9, 0.3)
    got = df.cpu().numpy()
    scale = np.maximum(np.abs(dref), np.array([1.0, dt, dt, dt, dt, dt]) * np.abs(dx).max())
    assert np.all(np.abs(got - dref) <= 1e-9 * scale)


def test_features_edge_arguments(P, torch, sen):
    s, _ = sen
    x = torch.zeros((0, 16), device="cuda")
    f, df = s.features(x, 1e-11)
    assert f.shape == (0, 6) and df is None
    y = torch.ones((2, 8), device="cuda")
    with pytest.raises(P.WTError):
        s.features(y, 1e-11, lo=0.0)
    with pytest.raises(P.WTError):
        s.features(y, -1.0)
    with pytest.raises(ValueError):
        s.features(y, 1e-11, dx=torch.ones((1, 2, 7), device="cuda"))
    with pytest.raises(ValueError):
        s.features(y.double(), 1e-11)


def test_current_tangents_match_oracle_fd(P, torch, sen):
    s, w = sen
    tr = W.configs.mip_tracks(w.grid, 3, 12, np.random.default_rng(4))
    t = device_tracks(tr, torch)
    i, di, L, g = s.tangents(t)
    L2, g2 = s.loss_grad(t)
    assert abs(L - L2) <= 1e-12 * L2 and np.allclose(g, g2, rtol=1e-12, atol=0)
    i_h, di_h = i.cpu().numpy().astype(np.float64), di.cpu().numpy().astype(np.float64)
    chain = 2.0 * np.mean(i_h[None] * di_h, axis=(1, 2))
    assert np.allclose(chain, g, rtol=1e-5, atol=1e-7 * np.abs(g).max())
    ref_i = A.loss(w, tr)[1]
    ref_di = A.fd_currents(w, tr, rel_step=1e-4)
    assert rel_l2(i_h, ref_i) < 1e-5
    for p in range(4):
        e = rel_l2(di_h[p], ref_di[p])
        print("param", p, "tangent rel L2", e)
        assert e < 2e-4, (p, e)


def _scan_points():
    pts = W.scan_bias_diameter(diameters_um=(6, 14), n_t=16, n_tracks=6, n_steps=24)
    return pts


def test_bias_diameter_scan_matches_oracle(P, torch):
    """Scan of two bias diameters with sensitivities: features against the
    oracle's features of its own FP64 currents; the library's current
    tangents against the oracle's difference tangents, both mapped through
    the features' linearisation at the library's currents (same decisions);
    the batched path (no sensitivities) gives the same features."""
    from paper_2605_13987_gb300.scan import run_scan
    pts = _scan_points()
    res = run_scan(pts, sensitivities=True, keep_waveforms=True)
    res_b = run_scan(pts, sensitivities=False)
    for (d, w), r, rb in zip(pts, res, res_b):
        tr = w.tracks
        dt = tr.dt
        ref_i = A.loss(w, tr)[1]
        assert rel_l2(r.waveforms, ref_i) < 1e-5
        ref_f = OF.features(ref_i, 0.0, dt)
        f = r.features
        amp = np.abs(ref_f[:, 0]).max()
        assert np.all(np.abs(f[:, 0] - ref_f[:, 0]) <= 1e-4 * amp)
        assert np.all(np.abs(f[:, [1, 3, 4, 5]] - ref_f[:, [1, 3, 4, 5]]) <= 2e-3 * dt)
        assert np.all(np.abs(f[:, 2] - ref_f[:, 2]) <= 1e-4 * dt * np.abs(ref_i).sum(axis=1))
        assert np.allclose(rb.features, f, rtol=1e-5, atol=1e-4 * dt)
        # the kernel's sensitivities are the oracle's linearisation of the library's own tangents
        own = OF.sensitivities(r.waveforms, r.tangents, 0.0, dt)
        assert np.allclose(r.dfeatures, own, rtol=1e-9, atol=1e-9 * np.abs(own).max())
        ref_di = A.fd_currents(w, tr, rel_step=1e-4)
        ref_df = OF.sensitivities(r.waveforms, ref_di, 0.0, dt)
        for p in range(4):
            assert rel_l2(r.tangents[p], ref_di[p]) < 2e-4
            for k in range(6):
                got, want = r.dfeatures[p, :, k], ref_df[p, :, k]
                e = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
                print("d", d, "param", p, "feature", k, "rel", e)
                assert e < 1e-3 or np.linalg.norm(want) < 1e-9 * np.abs(ref_df[p]).max() * len(want), (d, p, k, e)
        print("d", d, r.summary())


def test_shaped_scan_features_match_oracle(P, torch):
    from paper_2605_13987_gb300.scan import run_scan
    pts = _scan_points()[:1]
    tau, order = 0.3e-9, 2
    res = run_scan(pts, sensitivities=False, shaper=dict(tau=tau, order=order))
    d, w = pts[0]
    tr = w.tracks
    ref_v = OE.shape(A.loss(w, tr)[1], tr.dt, tau, order)
    ref_f = OF.features(ref_v, 0.0, tr.dt)
    f = res[0].features
    amp = np.abs(ref_f[:, 0]).max()
    assert np.all(np.abs(f[:, 0] - ref_f[:, 0]) <= 1e-4 * amp)
    assert np.all(np.abs(f[:, [1, 3, 4, 5]] - ref_f[:, [1, 3, 4, 5]]) <= 2e-3 * tr.dt)


def test_thickness_scan_through_the_batch_matches_oracle(P, torch):
    """Three thicknesses (Nz 40, 48, 64) in one captured batch of uneven
    grids: every variant's features against the oracle's features of its
    own FP64 currents."""
    from paper_2605_13987_gb300.scan import run_scan
    pts = W.scan_thickness(n_t=12, n_tracks=4, n_steps=20)
    res = run_scan(pts, sensitivities=False)
    for (th, w), r in zip(pts, res):
        tr = w.tracks
        ref_f = OF.features(A.loss(w, tr)[1], 0.0, tr.dt)
        amp = np.abs(ref_f[:, 0]).max()
        assert np.all(np.abs(r.features[:, 0] - ref_f[:, 0]) <= 1e-4 * amp), th
        assert np.all(np.abs(r.features[:, [1, 3, 4, 5]] - ref_f[:, [1, 3, 4, 5]]) <= 2e-3 * tr.dt), th
        print("thickness", th, r.summary())
