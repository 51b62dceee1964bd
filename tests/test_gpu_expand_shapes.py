"""The expansion's launch shapes (time samples per accumulator chunk, epilogue
warps, store width) only change how D = W E is moved out of tensor memory: every
combination gives H bit for bit equal, on a grid whose size is not a
multiple of the 128-point unit and a time count off the 32-sample tiling."""
import numpy as np
import pytest

import workloads as W
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
    P.load_library()
    return P


def test_every_epilogue_shape_gives_the_same_H(P, torch, monkeypatch):
    w = W.tiny_cell(nx=12, nz=20, n_t=300, radius=3 * UM)       # 2880 points, 300 time samples; r/h = 0.65
    ref = None
    for vec in (4, 2, 1):
        for nepi in (8, 12, 16):
            for nch in (64, 128, 256):
                monkeypatch.setenv("WT_LAUNCH_SHAPES", f"1,32,{nch},{nepi},3,5,0,0,{vec}")
                s = P.Sensor(w.grid, w.columns)
                try:
                    s.fit()
                    s.relax(w.times)
                    H = s.extend("fp32").cpu()
                    t = s.tuning()
                finally:
                    s.close()
                assert t["nepi"] == nepi and t["nch"] == nch and t["store_vec"] == vec
                if ref is None:
                    ref = H
                    assert torch.isfinite(ref).all() and ref.abs().max() > 0
                else:
                    assert torch.equal(H, ref), (vec, nepi, nch)
