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
    g = w.grid
    ti = np.sort(rng.choice(len(w.times), n_t, replace=False))
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
    print("c2 full size: FP64", e64, "FP32", e32)
    assert e64 < TOL64 and e32 < TOL32


def test_c3_sensors_through_the_batch(torch):
    import paper_2605_13987_gb300 as P
    ws = W.c3_batch(seed=3)[:4]
    sens = []
    try:
        for w in ws:
            s = P.Sensor(w.grid, w.columns)
            s.fit()
            s.relax(w.times)
            sens.append(s)
        Hb = P.extend_batch(sens)
        torch.cuda.synchronize()
        k = int(np.argmax([w.grid.Nx for w in ws]))
        rng = np.random.default_rng(22)
        samp = _sample(rng, ws[k])
        got = _take(Hb[k], *samp, torch)
    finally:
        for s in sens:
            s.close()
    ref = O.solve(ws[k]).H_subgrid(t_idx=samp[0], ix=samp[1], iy=samp[2], iz=samp[3])
    err = rel_l2(got, ref)
    print("c3 sensor", k, ws[k].grid.Nx, "FP32", err)
    assert err < TOL32
