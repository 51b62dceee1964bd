"""Every z-pass variant of the FP32 path (the register FFT at each lane
count, and the two-pass shared-memory FFT for Nz = 64, 128, 256), forced
through WT_LAUNCH_SHAPES, against the FP64 plain path of the same context
(itself checked against the oracle in test_gpu_c1 / test_gpu_edges) and,
for one case per length, against the oracle directly."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import rel_l2
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


def _variants(nz):
    out = []
    w = 32
    while w >= 4:
        if nz % w == 0 and nz // w in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 24):
            out.append((nz // w, 0))
        w //= 2
    if nz in (64, 128, 256):
        out.append((nz // 32, 1))
    return out


@pytest.mark.parametrize("nz", [64, 128, 256])
def test_every_z_variant_matches_fp64(P, torch, monkeypatch, nz):
    # a time count of its own per length keeps the process-wide tuning cache out of the way
    n_t = {64: 7, 128: 9, 256: 11}[nz]
    w = W.tiny_cell(nx=8, nz=nz, n_t=n_t, radius=5 * UM)
    ref = O.solve(w).H_full() if nz == 64 else None
    H64 = None
    for k, (rz, two_pass) in enumerate(_variants(nz)):
        monkeypatch.setenv("WT_LAUNCH_SHAPES", f"1,32,256,8,1,{rz},0,{two_pass}")
        s = P.Sensor(w.grid, w.columns)
        try:
            s.fit()
            s.relax(w.times)
            if H64 is None:
                H64 = s.extend("fp64").cpu().numpy()
                if ref is not None:
                    assert rel_l2(H64, ref) < 1e-10
            H32 = s.extend("fp32").double().cpu().numpy()
            t = s.tuning()
        finally:
            s.close()
        assert t["z_two_pass"] == two_pass and (two_pass or t["r_z"] == rz)
        e = rel_l2(H32, H64)
        print("nz", nz, "r_z", rz, "two-pass", two_pass, "rel L2", e)
        assert e < 1e-5, (nz, rz, two_pass, e)
