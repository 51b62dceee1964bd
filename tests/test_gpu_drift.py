"""Static drift field and carrier drift on the GPU against the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import drift as D
from tests.gpu_common import rel_l2
from workloads.configs import UM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def case(torch):
    import paper_2605_13987_gb300 as P
    w = W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)
    sol = O.solve(w)
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    yield w, sol, sen
    sen.close()


def test_static_field_matches_oracle(torch, case):
    w, sol, sen = case
    phi = [0.0, 100.0]                       # readout at ground, bias at 100 V
    ref = D.static_field(sol, phi)
    E64 = sen.static_field(phi, "fp64")
    E32 = sen.static_field(phi, "fp32")
    torch.cuda.synchronize()
    assert rel_l2(E64.cpu().numpy(), ref) < 1e-10
    assert rel_l2(E32.double().cpu().numpy(), ref) < 1e-5
    Z = sen.static_field([5.0, 5.0], "fp64")
    assert float(Z.abs().max()) < 1e-9 * float(E64.abs().max())


def test_drift_matches_oracle(torch, case):
    w, sol, sen = case
    g = w.grid
    E32 = sen.static_field([0.0, 100.0], "fp32")
    rng = np.random.default_rng(9)
    n, n_steps, dt = 48, 60, 1e-12
    x0 = np.column_stack([rng.uniform(0, g.Lx, n), rng.uniform(0, g.Ly, n), rng.uniform(0.1, 0.9, n) * g.Lz])
    keep = [not D.inside_column(g, w.columns, p) for p in x0]
    x0 = x0[keep]
    n = len(x0)
    smu = np.where(np.arange(n) % 2 == 0, 0.2, -0.2)           # holes, electrons
    tr = sen.drift(E32, torch.tensor(x0, device="cuda"), torch.tensor(smu, device="cuda"), n_steps, dt)
    torch.cuda.synchronize()
    ref = D.drift(E32.double().cpu().numpy(), g, w.columns, x0, np.sign(smu), np.abs(smu), dt, n_steps)
    got = np.stack([tr[k].double().cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz")])
    # positions: FP32 output rounding; the same steps stop on both sides
    assert np.max(np.abs(got[:3] - ref[:3])) < 1e-6 * g.Lz
    assert np.array_equal(got[3:] == 0, ref[3:] == 0)
    assert rel_l2(got[3:], ref[3:]) < 1e-6
    assert np.any(ref[3:] == 0), "some carriers should reach a column or a face"
    # the tracks feed Eq. 1 directly
    H = sen.extend("fp32")
    i = sen.eq1(H, tr)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(i.cpu().numpy())) and float(i.abs().max()) > 0
