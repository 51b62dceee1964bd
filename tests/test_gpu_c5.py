"""The 5x5 pixel cell at full size (grid 192x192x384, 50 columns x 256
sources, 256 time samples, H 43.5 GB in FP32) in the bench's launch
configuration (autotuned FP32 fast path, and the FP64 plain path) against the
FP64 oracle's field on a seeded 8x8x8 subgrid at four time samples (1 ps,
10 ns and two drawn between them).  The oracle values are stored in
tests/golden/c5_oracle_subgrid.txt by tests/golden/make_c5_fixture.py, which
calls only the oracle: one oracle setup at this size takes about half an hour
on the host."""
import numpy as np
import pytest

import workloads as W
from tests.golden.make_c5_fixture import load
from tests.gpu_common import rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL64 = 1e-10
TOL32 = 1e-5


def _take(H, it, ix, iy, iz, torch):
    idx = [torch.as_tensor(a, device=H.device) for a in (it, ix, iy, iz)]
    s = H.index_select(0, idx[0]).index_select(2, idx[1]).index_select(3, idx[2]).index_select(4, idx[3])
    return s.double().cpu().numpy()


def test_c5_full_size_against_oracle_values():
    import torch
    import paper_2605_13987_gb300 as P
    assert torch.cuda.is_available()
    ix, iy, iz, it, ref = load()
    w = W.c5_large(n_tracks=1)
    assert ref.shape == (4, 3, 8, 8, 8) and it[0] == 0 and it[-1] == len(w.times) - 1
    sen = P.Sensor(w.grid, w.columns)
    try:
        sen.fit()
        sen.relax(w.times)
        H32 = sen.extend("fp32")
        torch.cuda.synchronize()
        got32 = _take(H32, it, ix, iy, iz, torch)
        del H32
        H64 = sen.extend("fp64")
        torch.cuda.synchronize()
        got64 = _take(H64, it, ix, iy, iz, torch)
        del H64
        info = sen.info()
    finally:
        sen.close()
    e64, e32 = rel_l2(got64, ref), rel_l2(got32, ref)
    p64 = [rel_l2(got64[n], ref[n]) for n in range(len(it))]
    p32 = [rel_l2(got32[n], ref[n]) for n in range(len(it))]
    print("c5 full size: rank", info["rank"], "FP64", e64, "per sample", p64, "FP32", e32, "per sample", p32)
    assert e64 < TOL64 and max(p64) < 100 * TOL64
    assert e32 < TOL32 and max(p32) < TOL32
