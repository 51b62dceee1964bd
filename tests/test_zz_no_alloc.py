"""The allocation-free Eq. 1 entry point (wt_eq1_noalloc) gives the same
currents as wt_eq1.

Some callers cannot call cudaMalloc (an arena manager that owns all device
memory, a real-time loop that must not hit the allocator, a plugin host that
only hands out its own buffers); wt_eq1_noalloc serves them with a fixed
device scratch array.  Two calls in a row with different output lengths
check that each call rewrites the shared scratch it uses.  This file is
collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

import workloads as W
from workloads.configs import UM
from tests.gpu_common import rel_l2, device_tracks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def test_noalloc_eq1_matches_eq1_on_two_calls(torch):
    import paper_2605_13987_gb300 as P
    w = W.tiny_cell(nx=16, nz=32, n_t=24, radius=8 * UM)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H = sen.extend("fp32")
    rng = np.random.default_rng(11)
    for n_tracks, n_steps, n_out in ((16, 30, 60), (9, 20, 130)):
        tr = W.configs.mip_tracks(w.grid, n_tracks, n_steps, rng)
        tr.n_out = n_out
        td = device_tracks(tr, torch)
        ref = sen.eq1(H, td)
        got = torch.full_like(ref, float("nan"))
        P.wt_eq1_noalloc(sen.ctx, H, td, got)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert rel_l2(g, r) < 1e-5
    sen.close()


def test_noalloc_eq1_rejects_what_it_cannot_do_without_allocating(torch):
    import paper_2605_13987_gb300 as P
    from paper_2605_13987_gb300 import _binding as B
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H = sen.extend("fp32")
    tr = W.configs.mip_tracks(w.grid, 2, 8, np.random.default_rng(1))
    td = device_tracks(tr, torch)
    out = torch.empty((2, 20000), device="cuda")
    big = dict(td, n_out=20000)
    with pytest.raises(P.WTError) as e:
        P.wt_eq1_noalloc(sen.ctx, H, big, out)
    assert e.value.code == B.WT_ERR_ARG
    host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in td.items()}
    with pytest.raises(P.WTError) as e:
        P.wt_eq1_noalloc(sen.ctx, H, host, torch.empty((2, tr.n_out), device="cuda"))
    assert e.value.code == B.WT_ERR_ARG
    sen.close()
