"""The allocation-free Eq. 1 entry point (wt_eq1_noalloc) gives the same
currents as wt_eq1.

Some callers cannot call cudaMalloc: an arena or pool manager that owns all
device memory, a real-time loop that must not take the allocator's locks, a
plugin host that hands out only its own buffers.  wt_eq1_noalloc serves them
with a fixed device scratch array.  Its lag table is built on the device by
the same double-precision rule as wt_eq1's host-built table and feeds the
same kernel, so the two agree bit for bit.  Two calls in a row with
different output lengths check that each call rewrites the shared scratch
it uses.  This file is collected last so that a failure here comes after
every other test.
"""
import numpy as np
import pytest

import workloads as W
from workloads.configs import UM
from tests.gpu_common import device_tracks

pytestmark = pytest.mark.gpu

MAX_OUT = 16384      # WT_EQ1_NOALLOC_MAX_OUT in include/wt.h


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def sensor(torch):
    import paper_2605_13987_gb300 as P
    w = W.tiny_cell(nx=16, nz=32, n_t=24, radius=8 * UM)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H = sen.extend("fp32")
    torch.cuda.synchronize()
    yield w, sen, H
    sen.close()


def test_noalloc_eq1_matches_eq1_on_two_calls(torch, sensor):
    import paper_2605_13987_gb300 as P
    w, sen, H = sensor
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
        assert np.array_equal(g, r)


def test_noalloc_eq1_at_the_largest_output_length(torch, sensor):
    """n_out exactly at the limit is served (every scratch entry in use); one more is refused."""
    import paper_2605_13987_gb300 as P
    from paper_2605_13987_gb300 import _binding as B
    w, sen, H = sensor
    tr = W.configs.mip_tracks(w.grid, 3, 40, np.random.default_rng(5))
    tr.n_out = MAX_OUT
    td = device_tracks(tr, torch)
    ref = sen.eq1(H, td)
    got = torch.full_like(ref, float("nan"))
    P.wt_eq1_noalloc(sen.ctx, H, td, got)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
    over = dict(td, n_out=MAX_OUT + 1)
    with pytest.raises(P.WTError) as e:
        P.wt_eq1_noalloc(sen.ctx, H, over, torch.empty((3, MAX_OUT + 1), device="cuda"))
    assert e.value.code == B.WT_ERR_ARG


def test_noalloc_eq1_leaves_device_memory_unchanged(torch, sensor):
    """After a first call (which looks up the scratch address), a call changes no free-memory count."""
    import paper_2605_13987_gb300 as P
    w, sen, H = sensor
    tr = W.configs.mip_tracks(w.grid, 8, 25, np.random.default_rng(9))
    td = device_tracks(tr, torch)
    out = torch.empty((tr.n_tracks, tr.n_out), device="cuda")
    P.wt_eq1_noalloc(sen.ctx, H, td, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    P.wt_eq1_noalloc(sen.ctx, H, td, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_eq1_rejects_what_it_cannot_do_without_allocating(torch, sensor):
    import paper_2605_13987_gb300 as P
    from paper_2605_13987_gb300 import _binding as B
    w, sen, H = sensor
    tr = W.configs.mip_tracks(w.grid, 2, 8, np.random.default_rng(1))
    td = device_tracks(tr, torch)
    out = torch.empty((2, tr.n_out), device="cuda")
    cases = [
        (H, {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in td.items()}, out),  # host tracks
        (H.double(), td, out),                                    # FP64 H read as FP32
        (H[:-1], td, out),                                        # H one value short
        (H, td, torch.empty((2, tr.n_out - 1), device="cuda")),  # currents buffer too small
        (H, td, out.double()),                                    # wrong output type
    ]
    for h, t, o in cases:
        with pytest.raises(P.WTError) as e:
            P.wt_eq1_noalloc(sen.ctx, h, t, o)
        assert e.value.code == B.WT_ERR_ARG
    # the C entry point itself refuses host memory (no staging without allocation)
    host_H = np.zeros(4, dtype=np.float32)
    tr_s = B._tracks_struct(td)
    import ctypes as C
    code = B.load_library().wt_eq1_noalloc(sen.ctx, B._ptr(host_H), C.byref(tr_s), B._ptr(out),
                                           B._stream_handle(None))
    assert code == B.WT_ERR_ARG


def test_noalloc_eq1_replays_from_a_captured_graph(torch, sensor):
    """After a first call (which looks up the scratch address), wt_eq1_noalloc can be captured
    into a CUDA graph: a replay gives wt_eq1's currents bit for bit, and a replay after the track
    arrays were rewritten in place follows the new tracks."""
    import paper_2605_13987_gb300 as P
    w, sen, H = sensor
    tr = W.configs.mip_tracks(w.grid, 12, 24, np.random.default_rng(21))
    tr.n_out = 50
    td = device_tracks(tr, torch)
    out = torch.zeros((tr.n_tracks, tr.n_out), dtype=torch.float32, device="cuda")
    P.wt_eq1_noalloc(sen.ctx, H, td, out)            # the first call resolves the scratch address
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        P.wt_eq1_noalloc(sen.ctx, H, td, out)
    torch.cuda.synchronize()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    ref = sen.eq1(H, td)
    assert torch.equal(out, ref)
    tr2 = W.configs.mip_tracks(w.grid, 12, 24, np.random.default_rng(22))
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        td[k].copy_(torch.tensor(np.ascontiguousarray(getattr(tr2, k)), dtype=torch.float32, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    ref2 = sen.eq1(H, td)
    assert torch.equal(out, ref2) and not torch.equal(ref, ref2)
