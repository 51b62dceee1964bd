"""CR-(RC)^n front-end shaping on the GPU against the oracle's FP64
convolution of the same currents (Eq. 1 currents of a small cell)."""
import numpy as np
import pytest

import workloads as W
from oracle import electronics as E
from tests.gpu_common import device_tracks, rel_l2
from workloads.configs import UM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def currents(torch):
    import paper_2605_13987_gb300 as P
    w = W.tiny_cell(nx=16, nz=32, n_t=12, radius=8 * UM)
    tr = W.configs.mip_tracks(w.grid, 5, 40, np.random.default_rng(6))
    sen = P.Sensor(w.grid, w.columns)
    sen.fit()
    sen.relax(w.times)
    H = sen.extend("fp32")
    i = sen.eq1(H, device_tracks(tr, torch))
    torch.cuda.synchronize()
    yield sen, i, tr.dt
    sen.close()


@pytest.mark.parametrize("order,tau_steps", [(0, 3.0), (1, 2.5), (4, 1.5)])
def test_shaping_matches_oracle(torch, currents, order, tau_steps):
    sen, i, dt = currents
    tau = tau_steps * dt
    rng = np.random.default_rng(order)
    noise = torch.tensor(rng.standard_normal(tuple(i.shape)), dtype=torch.float32, device="cuda")
    v = sen.shape(i, dt, tau, order, gain=2.5, noise=noise, noise_rms=0.05 * float(i.abs().max()))
    torch.cuda.synchronize()
    ref = E.shape(i.double().cpu().numpy(), dt, tau, order, gain=2.5, noise=noise.double().cpu().numpy(),
                  noise_rms=0.05 * float(i.abs().max()))
    assert rel_l2(v.double().cpu().numpy(), ref) < 1e-6


def test_shaping_errors(torch, currents):
    import paper_2605_13987_gb300 as P
    sen, i, dt = currents
    with pytest.raises(P.WTError, match="WT_ERR_ARG"):
        sen.shape(i, dt, -1.0, 2)
    with pytest.raises(P.WTError, match="WT_ERR_ARG"):
        sen.shape(i.cpu(), dt, 1e-9, 2)
