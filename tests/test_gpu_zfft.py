"""Every FFT variant of the FP32 path, forced through WT_LAUNCH_SHAPES:
the z pass by the register FFT at each lane count and by the two-pass
shared-memory FFT (Nz = 64, 96, 128, 160, 192, 224, 256, 384: radix-2, 3, 5
and 7 register DFTs), the y transforms of the plane pass
by the register FFT and by the two-pass FFT (Ny = 64, 128) at 16 and 32
lanes per x line, and two-pass x transforms on top, against the FP64 plain path of the same
context (itself checked against the oracle, here for Nz = 64 and in
test_gpu_c1 / test_gpu_edges)."""
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
    if nz in (64, 96, 128, 160, 192, 224, 256, 384):
        out.append((out[0][0], 1))
    return out


@pytest.mark.parametrize("nz", [64, 96, 128, 160, 192, 224, 256, 384])
def test_every_z_variant_matches_fp64(P, torch, monkeypatch, nz):
    # a time count of its own per length keeps the process-wide tuning cache out of the way
    n_t = {64: 7, 96: 8, 128: 9, 160: 10, 192: 13, 224: 14, 256: 11, 384: 15}[nz]
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
        assert t["two_pass"] == two_pass and (two_pass or t["r_z"] == rz)
        e = rel_l2(H32, H64)
        print("nz", nz, "r_z", rz, "two-pass", two_pass, "rel L2", e)
        assert e < 1e-5, (nz, rz, two_pass, e)


@pytest.mark.parametrize("n", [64, 128])
def test_two_pass_y_transforms_match_fp64(P, torch, monkeypatch, n):
    """Lateral grids of n x n (z: 16 cells), both x lane counts, staged and
    direct x stores."""
    n_t = {64: 5, 128: 6}[n]
    w = W.tiny_cell(nx=n, nz=16, n_t=n_t, pitch=55 * UM * n / 32, radius=5 * UM)
    H64 = None
    for rxy in (n // 32, n // 16):
        for xd in (0, 1):
            monkeypatch.setenv("WT_LAUNCH_SHAPES", f"2,32,256,8,{rxy},1,{xd},2")
            s = P.Sensor(w.grid, w.columns)
            try:
                s.fit()
                s.relax(w.times)
                if H64 is None:
                    H64 = s.extend("fp64").cpu().numpy()
                H32 = s.extend("fp32").double().cpu().numpy()
                t = s.tuning()
            finally:
                s.close()
            assert t["two_pass"] == 2 and t["r_xy"] == rxy and t["x_direct"] == xd
            e = rel_l2(H32, H64)
            print("n", n, "r_xy", rxy, "x_direct", xd, "rel L2", e)
            assert e < 1e-5, (n, rxy, xd, e)


@pytest.mark.parametrize("n", [64, 128])
def test_two_pass_x_transforms_match_fp64(P, torch, monkeypatch, n):
    """Two-pass y and x transforms (mask 6), with the register and the
    two-pass z pass (mask 7)."""
    n_t = {64: 3, 128: 2}[n]
    w = W.tiny_cell(nx=n, nz=64, n_t=n_t, pitch=55 * UM * n / 32, radius=5 * UM)
    H64 = None
    for mask in (6, 7):
        monkeypatch.setenv("WT_LAUNCH_SHAPES", f"1,32,256,8,{n // 32},2,1,{mask}")
        s = P.Sensor(w.grid, w.columns)
        try:
            s.fit()
            s.relax(w.times)
            if H64 is None:
                H64 = s.extend("fp64").cpu().numpy()
            H32 = s.extend("fp32").double().cpu().numpy()
            t = s.tuning()
        finally:
            s.close()
        assert t["two_pass"] == mask
        e = rel_l2(H32, H64)
        print("n", n, "mask", mask, "rel L2", e)
        assert e < 1e-5, (n, mask, e)
