"""Edge cases and error paths of the CUDA library (ragged FFT sizes, partial
tiles, host buffers, degenerate inputs, every host-side rejection)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.configs import UM
from tests.gpu_common import rel_l2, device_tracks

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


@pytest.mark.parametrize("nx,nz,nt", [(20, 36, 12), (28, 40, 5), (16, 30, 1)])
def test_ragged_grids(P, torch, nx, nz, nt):
    """Radix-5/7/3 FFT lengths, grid sizes that are not a multiple of the
    128-point tile, time counts below and off the 32-sample tiling."""
    w = W.tiny_cell(nx=nx, nz=nz, n_t=nt, radius=6 * UM if nx >= 20 else 8 * UM)
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H64 = sen.extend("fp64").cpu().numpy()
    H32 = sen.extend("fp32").double().cpu().numpy()
    ref = sol.H_full()
    sen.close()
    assert rel_l2(H64, ref) < 1e-10
    assert rel_l2(H32, ref) < 1e-5


def test_host_buffers_match_device(P, torch):
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    Hd = sen.extend("fp32")
    Hh = torch.empty(Hd.shape, dtype=torch.float32, pin_memory=True)
    sen.extend("fp32", out=Hh)
    Hp = np.empty(Hd.shape, dtype=np.float64)
    P.wt_extend(sen.ctx, P.WT_FP64, Hp)
    H64 = sen.extend("fp64")
    torch.cuda.synchronize()
    assert torch.equal(Hd.cpu(), Hh)
    assert np.array_equal(Hp, H64.cpu().numpy())
    # Eq. 1 with host track arrays and a host output
    tr = W.configs.mip_tracks(w.grid, 5, 12, np.random.default_rng(1))
    td = device_tracks(tr, torch)
    th = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in td.items()}
    i_dev = sen.eq1(Hd, td)
    i_host = np.zeros((5, tr.n_out), dtype=np.float32)
    P.wt_eq1(sen.ctx, Hd, th, i_host)
    sen.close()
    assert np.array_equal(i_dev.cpu().numpy(), i_host)


def test_zero_tracks_and_stationary(P, torch):
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H = sen.extend("fp32")
    tr = W.configs.mip_tracks(w.grid, 3, 10, np.random.default_rng(2))
    for a in ("vx", "vy", "vz"):
        setattr(tr, a, np.zeros_like(getattr(tr, a)))
    i = sen.eq1(H, device_tracks(tr, torch))
    assert float(i.abs().max()) == 0.0
    empty = dict(n_tracks=0, n_steps=4, n_out=8, dt=1e-11, x=H, y=H, z=H, vx=H, vy=H, vz=H)
    P.wt_eq1(sen.ctx, H, empty, torch.empty(0, device="cuda"))
    sen.close()


def _expect(P, code, fn, *a):
    with pytest.raises(P.WTError) as e:
        fn(*a)
    assert e.value.code == code, str(e.value)


def test_error_paths(P, torch):
    from paper_2605_13987_gb300 import _binding as B
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    # odd grid, unsupported FFT length (prime 11), bad device
    g_odd = W.GridSpec(w.grid.Lx, w.grid.Ly, w.grid.Lz, 15, 16, 32)
    _expect(P, B.WT_ERR_ARG, P.Sensor, g_odd, w.columns)
    g_11 = W.GridSpec(w.grid.Lx, w.grid.Ly, w.grid.Lz, 22, 16, 32)
    _expect(P, B.WT_ERR_UNSUPPORTED, P.Sensor, g_11, w.columns)
    _expect(P, B.WT_ERR_ARG, P.Sensor, w.grid, w.columns, 999)
    # overlap
    c0 = w.columns[0]
    bad = [c0, W.ColumnSpec(c0.x + 1e-6, c0.y, c0.z0, c0.z1, c0.radius, c0.resistivity, 0, 0, c0.n_sources)]
    s = P.Sensor(w.grid, bad)
    _expect(P, B.WT_ERR_GEOMETRY, s.fit)
    s.close()
    # order of calls, bad times, small buffer
    s = P.Sensor(w.grid, w.columns)
    _expect(P, B.WT_ERR_STATE, s.relax, w.times)
    s.fit()
    _expect(P, B.WT_ERR_STATE, s.fit)
    _expect(P, B.WT_ERR_ARG, s.relax, w.times[::-1])
    _expect(P, B.WT_ERR_ARG, s.relax, np.array([0.0, 1e-9]))
    s.relax(w.times)
    small = torch.empty(10, device="cuda")
    _expect(P, B.WT_ERR_ARG, P.wt_extend, s.ctx, P.WT_FP32, small)
    s.close()


def test_indefinite_capacitance_is_reported(P):
    """r/h ~ 1.45 on a 16x16x32 single cell: the band-limited kernel's axis
    ridge makes the fitted capacitance indefinite; the library says so."""
    from paper_2605_13987_gb300 import _binding as B
    w = W.tiny_cell(nx=16, nz=32, n_t=4, radius=5 * UM)
    s = P.Sensor(w.grid, w.columns)
    s.fit()
    _expect(P, B.WT_ERR_NOT_SPD, s.relax, w.times)
    s.close()
