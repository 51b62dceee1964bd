"""Basis fields from the per-column lateral tables (wt_tuning.table_rows > 0)
against the FP64 oracle and against the per-basis spectral passes, on grids
whose row count is not a multiple of the slab height (ragged last slab),
radix-5/7 lateral lengths, time-basis ranks in each accumulator width of the
combination kernel (<= 8, <= 16, <= 32), every time sample on its own."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.configs import UM
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _extend_with(P, w, shapes, monkeypatch, torch):
    if shapes is None:
        monkeypatch.delenv("WT_LAUNCH_SHAPES", raising=False)
    else:
        monkeypatch.setenv("WT_LAUNCH_SHAPES", ",".join(str(v) for v in shapes))
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        s.relax(w.times)
        H = s.extend("fp32")
        torch.cuda.synchronize()
        return H.double().cpu().numpy(), s.tuning(), s.info()
    finally:
        s.close()
        monkeypatch.delenv("WT_LAUNCH_SHAPES", raising=False)


@pytest.mark.parametrize("nx,nz,nt,ys", [(16, 32, 24, 4), (20, 36, 12, 8), (28, 40, 5, 16), (32, 64, 64, 4)])
def test_table_path_matches_oracle_and_per_basis_passes(torch, monkeypatch, nx, nz, nt, ys):
    import paper_2605_13987_gb300 as P
    if nx == 32:
        w = W.workload("c1")
    else:
        w = W.tiny_cell(nx=nx, nz=nz, n_t=nt, radius=6 * UM if nx >= 20 else 8 * UM)
    ref = O.solve(w).H_full()
    H0, tun, info = _extend_with(P, w, None, monkeypatch, torch)          # the tuner's own choice
    base = [tun[k] for k in ("nb", "lb", "nch", "nepi", "r_xy", "r_z", "x_direct", "two_pass", "store_vec")]
    Hb, tb, _ = _extend_with(P, w, base + [0], monkeypatch, torch)        # per-basis passes
    Ht, tt, _ = _extend_with(P, w, base + [ys], monkeypatch, torch)       # lateral tables
    assert tb["table_rows"] == 0 and tt["table_rows"] == ys
    for H in (H0, Hb, Ht):
        assert rel_l2(H, ref) < TOL32
        assert max(rel_l2(H[n], ref[n]) for n in range(len(ref))) < TOL32
    # the same sums in another order: FP32 rounding apart
    assert rel_l2(Ht, Hb) < 2e-6
    print(nx, nz, nt, "rank", info["rank"], "tables vs per-basis", rel_l2(Ht, Hb), "vs oracle", rel_l2(Ht, ref))


def test_tables_serve_the_batch_bit_for_bit(torch, monkeypatch):
    """wt_batch_run on contexts whose tuning uses the tables equals wt_extend on them."""
    import paper_2605_13987_gb300 as P
    ws = [W.tiny_cell(nx=16, nz=32, n_t=20, radius=8 * UM, seed=s) for s in (1, 2)]
    sens = []
    try:
        for w in ws:
            s = P.Sensor(w.grid, w.columns)
            s.fit()
            s.relax(w.times)
            sens.append(s)
        H1 = sens[0].extend("fp32")
        tun = sens[0].tuning()
        base = [tun[k] for k in ("nb", "lb", "nch", "nepi", "r_xy", "r_z", "x_direct", "two_pass", "store_vec")]
        monkeypatch.setenv("WT_LAUNCH_SHAPES", ",".join(str(v) for v in base + [4]))
        sens2 = []
        for w in ws:
            s = P.Sensor(w.grid, w.columns)
            s.fit()
            s.relax(w.times)
            sens2.append(s)
        Hb = P.extend_batch(sens2)
        He = [s.extend("fp32") for s in sens2]
        torch.cuda.synchronize()
        assert all(s.tuning()["table_rows"] == 4 for s in sens2)
        for a, b in zip(Hb, He):
            assert torch.equal(a, b)
        for s in sens2:
            s.close()
    finally:
        monkeypatch.delenv("WT_LAUNCH_SHAPES", raising=False)
        for s in sens:
            s.close()


@pytest.mark.parametrize("tf", [1, 2, 3, 4, 7])
def test_pipelined_and_discarding_slabs_are_bit_equal(torch, monkeypatch, tf):
    """Table flags (slabs pipelined on two streams, L2 lines of consumed slab rows dropped) change
    only the schedule and the caching: the fields are bit-equal to the one-stream path, through
    wt_extend and through a captured wt_batch_run."""
    import paper_2605_13987_gb300 as P
    w = W.workload("c1")                        # 32 x 32 x 64: two-pass z pass, 4-row slabs of 128 lines
    _, tun, _ = _extend_with(P, w, None, monkeypatch, torch)
    base = [tun["nb"], 64, tun["nch"], tun["nepi"], tun["r_xy"], tun["r_z"], tun["x_direct"],
            tun["two_pass"] | 1, tun["store_vec"]]
    Href, t0, _ = _extend_with(P, w, base + [4, 0], monkeypatch, torch)
    Ht, tt, _ = _extend_with(P, w, base + [4, tf], monkeypatch, torch)
    assert t0["table_flags"] == 0 and tt["table_flags"] == tf and tt["table_rows"] == 4
    assert np.array_equal(Ht, Href)
    monkeypatch.setenv("WT_LAUNCH_SHAPES", ",".join(str(v) for v in base + [4, tf]))
    sens = []
    try:
        for seed in (1, 2):
            s = P.Sensor(w.grid, w.columns)
            s.fit()
            s.relax(w.times)
            sens.append(s)
        Hb = P.extend_batch(sens)
        Hb2 = P.extend_batch(sens)                # the captured graph replayed
        torch.cuda.synchronize()
        for a, b in zip(Hb, Hb2):
            assert torch.equal(a, b)
        assert np.array_equal(Hb[0].double().cpu().numpy(), Href)
    finally:
        monkeypatch.delenv("WT_LAUNCH_SHAPES", raising=False)
        for s in sens:
            s.close()
