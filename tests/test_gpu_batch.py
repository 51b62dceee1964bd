"""Batched FP32 extension (wt_batch_run: one captured graph, one persistent
expansion launch over all contexts, autotuned launch shapes) on batches of
single cells with uneven grids: equal to wt_extend bit for bit, and to the
FP64 oracle within the FP32 bound."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def P():
    import paper_2605_13987_gb300 as P
    return P


def _sensors(P, ws):
    out = []
    for w in ws:
        s = P.Sensor(w.grid, w.columns)
        s.fit()
        s.relax(w.times)
        out.append(s)
    return out


def _close(sens):
    for s in sens:
        s.close()


@pytest.fixture(scope="module")
def small_batch(P, torch):
    ws = W.c3_batch(seed=11, n_sensors=6, nx_choices=(16, 20, 24, 28, 32), n_t=24)
    sens = _sensors(P, ws)
    yield ws, sens
    _close(sens)


def test_batch_equals_single_extend(P, torch, small_batch):
    ws, sens = small_batch
    assert len({w.grid.Nx for w in ws}) > 1          # uneven grids in one batch
    Hb = P.extend_batch(sens)
    torch.cuda.synchronize()
    for s, h in zip(sens, Hb):
        h1 = s.extend("fp32")
        torch.cuda.synchronize()
        assert torch.equal(h, h1)
    # graph replay: a second call gives the same arrays
    Hb2 = P.extend_batch(sens, outs=[torch.full_like(h, float("nan")) for h in Hb])
    torch.cuda.synchronize()
    for a, b in zip(Hb, Hb2):
        assert torch.equal(a, b)


def test_batch_matches_oracle(P, torch, small_batch):
    ws, sens = small_batch
    Hb = P.extend_batch(sens)
    torch.cuda.synchronize()
    k = int(np.argmax([w.grid.Nx for w in ws]))
    ref = O.solve(ws[k]).H_full()
    assert rel_l2(Hb[k].cpu().numpy(), ref) < TOL32


def test_tuned_shapes_are_candidates(P, torch, small_batch):
    ws, sens = small_batch
    P.extend_batch(sens)
    for s in sens:
        t = s.tuning()
        assert t["nb"] in (1, 2, 4) and t["lb"] in (16, 32, 64) and t["nch"] in (64, 128, 256)
        assert t["nepi"] in (8, 12, 16) and t["store_vec"] in (1, 2, 4)


def test_batch_fp64_equals_plain(P, torch, small_batch):
    ws, sens = small_batch
    Hb = P.extend_batch(sens[:2], precision="fp64")
    torch.cuda.synchronize()
    for s, h in zip(sens[:2], Hb):
        assert torch.equal(h, s.extend("fp64"))


def test_relax_again_recaptures(P, torch):
    ws = W.c3_batch(seed=12, n_sensors=3, nx_choices=(16, 24), n_t=16)
    sens = _sensors(P, ws)
    try:
        P.extend_batch(sens)
        sens[1].relax(W.log_times(20))            # new times: new charges, shapes and buffers
        Hb = P.extend_batch(sens)
        torch.cuda.synchronize()
        for s, h in zip(sens, Hb):
            assert h.shape[0] == len(s.times)
            assert torch.equal(h, s.extend("fp32"))
    finally:
        _close(sens)


def test_more_than_one_expansion_launch(P, torch):
    """65 contexts: the graph holds two persistent expansion launches."""
    ws = W.c3_batch(seed=13, n_sensors=65, nx_choices=(24, 28, 32), n_t=8)
    sens = _sensors(P, ws)
    try:
        Hb = P.extend_batch(sens)
        torch.cuda.synchronize()
        for i in (0, 31, 63, 64):
            assert torch.equal(Hb[i], sens[i].extend("fp32"))
    finally:
        _close(sens)


def test_batch_errors(P, torch, small_batch):
    ws, sens = small_batch
    B = P._binding
    with pytest.raises(P.WTError, match="WT_ERR_ARG"):
        B.wt_batch_run([sens[0].ctx, sens[0].ctx], B.WT_FP32,
                       [torch.empty(sens[0].h_shape(), device="cuda")] * 2)
    fresh = P.Sensor(ws[0].grid, ws[0].columns)
    try:
        fresh.fit()
        with pytest.raises(P.WTError, match="WT_ERR_STATE"):
            B.wt_batch_run([fresh.ctx], B.WT_FP32, [torch.empty(sens[0].h_shape(), device="cuda")])
    finally:
        fresh.close()
