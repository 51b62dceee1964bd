"""Full-size parity in the launch configuration the bench times: the 3x3
cell at grid 128x128x256 with 512 time samples (FP32 fast path after the
autotuner, and the FP64 plain path), and four sensors of the 64-geometry
batch through wt_batch_run, each against the FP64 oracle on a random
subgrid of points and time samples that the oracle evaluates directly."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _sample(rng, w, n_t=4, n_side=8):
    """The first and last time samples (1 ps, 10 ns) and n_t - 2 random ones; a random subgrid."""
    g = w.grid
    nt = len(w.times)
    mid = rng.choice(np.arange(1, nt - 1), n_t - 2, replace=False)
    ti = np.sort(np.concatenate([[0, nt - 1], mid]))
    ix = np.sort(rng.choice(g.Nx, n_side, replace=False))
    iy = np.sort(rng.choice(g.Ny, n_side, replace=False))
    iz = np.sort(rng.choice(g.Nz, n_side, replace=False))
    return ti, ix, iy, iz


def _take(H, ti, ix, iy, iz, torch):
    ti_, ix_, iy_, iz_ = (torch.as_tensor(a, device=H.device) for a in (ti, ix, iy, iz))
    s = H.index_select(0, ti_).index_select(2, ix_).index_select(3, iy_).index_select(4, iz_)
    return s.double().cpu().numpy()


def test_c2_full_size(torch):
    import paper_2605_13987_gb300 as P
    w = W.workload("c2")
    sen = P.Sensor(w.grid, w.columns)
    try:
        sen.fit()
        sen.relax(w.times)
        H32 = sen.extend("fp32")                 # tuned launch shapes, as in the bench
        torch.cuda.synchronize()
        rng = np.random.default_rng(21)
        samp = _sample(rng, w)
        got32 = _take(H32, *samp, torch)
        del H32
        H64 = sen.extend("fp64")
        torch.cuda.synchronize()
        got64 = _take(H64, *samp, torch)
        del H64
    finally:
        sen.close()
    sol = O.solve(w)
    ref = sol.H_subgrid(t_idx=samp[0], ix=samp[1], iy=samp[2], iz=samp[3])
    e64, e32 = rel_l2(got64, ref), rel_l2(got32, ref)
    p32 = [rel_l2(got32[n], ref[n]) for n in range(len(ref))]
    p64 = [rel_l2(got64[n], ref[n]) for n in range(len(ref))]
    print("c2 full size: FP64", e64, "FP32", e32, "per time sample FP32", p32)
    assert e64 < TOL64 and e32 < TOL32
    assert max(p32) < TOL32 and max(p64) < 100 * TOL64


def _c3_pick():
    """One sensor of the 64-geometry batch per grid size (64, 80, 96, 112, 128), plus the two
    with the widest resistivity spreads (0.05 against 1.9 Ohm cm)."""
    ws = W.c3_batch(seed=3)
    pick = {}
    for i, w in enumerate(ws):
        pick.setdefault(w.grid.Nx, i)
    spread = sorted(range(len(ws)), key=lambda i: -max(c.resistivity for c in ws[i].columns)
                    / min(c.resistivity for c in ws[i].columns))[:2]
    idx = sorted(set(pick.values()) | set(spread))
    return [ws[i] for i in idx], idx


def test_c3_sensors_through_the_batch(torch):
    """Each picked sensor against the oracle, per time sample, from one batched launch."""
    import paper_2605_13987_gb300 as P
    ws, idx = _c3_pick()
    assert sorted({w.grid.Nx for w in ws}) == [64, 80, 96, 112, 128]
    sens, got, samps = [], [], []
    try:
        for w in ws:
            s = P.Sensor(w.grid, w.columns)
            s.fit()
            s.relax(w.times)
            sens.append(s)
        Hb = P.extend_batch(sens)
        torch.cuda.synchronize()
        rng = np.random.default_rng(22)
        for k, w in enumerate(ws):
            samp = _sample(rng, w)
            samps.append(samp)
            got.append(_take(Hb[k], *samp, torch))
        ranks = [s.info()["rank"] for s in sens]
    finally:
        for s in sens:
            s.close()
    for k, w in enumerate(ws):
        samp = samps[k]
        ref = O.solve(w).H_subgrid(t_idx=samp[0], ix=samp[1], iy=samp[2], iz=samp[3])
        per = [rel_l2(got[k][n], ref[n]) for n in range(len(ref))]
        print("c3 sensor", idx[k], w.grid.Nx, "rank", ranks[k], "FP32", rel_l2(got[k], ref), "per sample", per)
        assert rel_l2(got[k], ref) < TOL32 and max(per) < TOL32
