"""CUDA path vs FP64 oracle on the single-cell workload (55x55x100 um, grid
32x32x64, 2 columns x 64 sources, 64 time samples): every stage, full arrays."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import eq1 as OE, relax as OR
from tests.gpu_common import rel_l2, device_tracks

pytestmark = pytest.mark.gpu

TOL64 = 1e-10      # FP64 plain path and FP64 setup stages
TOL32 = 1e-5       # FP32 fast path: the accuracy target of the FP32 field against the FP64 oracle


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def case(torch):
    import paper_2605_13987_gb300 as P
    w = W.workload("c1")
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H64 = sen.extend("fp64")
    H32 = sen.extend("fp32")
    torch.cuda.synchronize()
    ref = sol.H_full()
    yield w, sol, sen, H64.cpu().numpy(), H32, ref
    sen.close()


def test_capacitance(case):
    w, sol, sen, *_ = case
    assert rel_l2(sen.capacitance(), sol.fit["Cn"]) < TOL64


def test_relaxation_rates(case):
    w, sol, sen, *_ = case
    assert rel_l2(np.sort(sen.modes()), np.sort(sol.rel["mu"])) < TOL64


def test_charge_history(case):
    w, sol, sen, *_ = case
    assert rel_l2(sen.charges(), sol.q.T) < TOL64


def test_H_fp64_full_grid(case):
    w, sol, sen, H64, H32, ref = case
    assert rel_l2(H64, ref) < TOL64
    # every time sample, not only the norm-dominant late ones
    for n in range(ref.shape[0]):
        assert rel_l2(H64[n], ref[n]) < 100 * TOL64


def test_H_fp32_full_grid(case):
    w, sol, sen, H64, H32, ref = case
    h = H32.double().cpu().numpy()
    assert rel_l2(h, ref) < TOL32
    assert rel_l2(h, H64) < TOL32
    # every time sample on its own, the early ones (t = 1 ps, the fast part of Eq. 1's signal)
    # included: one norm over all samples would be dominated by the late, relaxed ones
    per = [rel_l2(h[n], ref[n]) for n in range(ref.shape[0])]
    assert max(per) < TOL32, (int(np.argmax(per)), max(per))


def test_tensor_core_expansion_matches_fma_expansion(case, torch, monkeypatch):
    import paper_2605_13987_gb300 as P
    w, sol, sen, H64, H32, ref = case
    monkeypatch.setenv("WT_EXPAND", "simt")
    s2 = P.Sensor(w.grid, w.columns)
    s2.fit()
    s2.relax(w.times)
    Hs = s2.extend("fp32")
    torch.cuda.synchronize()
    s2.close()
    assert rel_l2(H32.double().cpu().numpy(), Hs.double().cpu().numpy()) < 2e-6


def test_point_samples(case):
    w, sol, sen, *_ = case
    rng = np.random.default_rng(0)
    g = w.grid
    pts = np.stack([rng.uniform(0, g.Lx, 8), rng.uniform(0, g.Ly, 8), rng.uniform(0, g.Lz, 8)], 1)
    ts = np.array([0.0, 3.3e-12, w.times[20], w.times[-1], 2e-8])
    got = sen.sample_H(pts, ts)
    q = OR.relax(sol.fit["Cn"], sol.K, sol.b, sol.phi_dc, ts)["q"]
    want = O.extend.field_points(sol.grid, sol.lay.src, q, pts)
    assert np.abs(got[0]).max() < 1e-9 * np.abs(want).max()       # H(t = 0) = 0
    assert rel_l2(got[1:], want[1:]) < TOL64


def test_eq1_currents(case, torch):
    w, sol, sen, H64, H32, ref = case
    tr = W.configs.mip_tracks(w.grid, 24, 40, np.random.default_rng(3))
    i = sen.eq1(H32, device_tracks(tr, torch))
    want = OE.currents(sol.grid, sol.times, ref, tr)
    assert rel_l2(i.cpu().numpy(), want) < TOL32


def test_eq1_direct_matches_oracle_and_eq1_on_H(case, torch):
    """Eq. 1 from the rank-r field form (no H): against the oracle, against
    Eq. 1 on the stored FP32 H, with host and device tracks, and with a
    ragged chunk of steps (37 steps: two full chunks of 16 and a tail)."""
    w, sol, sen, H64, H32, ref = case
    tr = W.configs.mip_tracks(w.grid, 24, 37, np.random.default_rng(8))
    t = device_tracks(tr, torch)
    i_h = sen.eq1(H32, t).cpu().numpy()
    i_d = sen.eq1_direct(t).cpu().numpy()
    want = OE.currents(sol.grid, sol.times, ref, tr)
    assert rel_l2(i_d, want) < TOL32
    assert rel_l2(i_d, i_h) < 2e-6
    host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in t.items()}
    out = np.zeros((tr.n_tracks, tr.n_out), dtype=np.float32)
    P = __import__("paper_2605_13987_gb300")
    P.wt_eq1_direct(sen.ctx, host, out)
    assert np.array_equal(out, i_d)


def test_diagnostics(case):
    w, sol, sen, *_ = case
    info = sen.info()
    assert info["n_sources"] == 128 and info["n_t"] == 64
    # the time basis: the smallest rank leaving <= 1e-7 in every time sample (exact SVD tail)
    assert 1 <= info["rank"] <= 32 and info["trunc_rel"] <= 1e-7
    Q = sol.q
    U, sv, Vt = np.linalg.svd(Q, full_matrices=False)
    r = info["rank"]
    tail = np.sqrt(((sv[r:, None] * Vt[r:]) ** 2).sum(0)) / np.linalg.norm(Q, axis=0)
    assert abs(tail.max() - info["trunc_rel"]) <= 1e-3 * info["trunc_rel"] + 1e-15
    tail1 = np.sqrt(((sv[r - 1:, None] * Vt[r - 1:]) ** 2).sum(0)) / np.linalg.norm(Q, axis=0)
    assert tail1.max() > 1e-7            # r is the smallest rank that meets the target
    assert info["boundary_residual"] < 1e-8
    assert info["asymmetry"] < 1e-8
    assert abs(info["mu_min"] / sol.rel["mu"].min() - 1) < 1e-9
