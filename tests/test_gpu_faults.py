"""Failure paths forced by host-side fault injection (WT_FAULT), none of
which faults, traps or hangs the GPU: a singular fit, failed allocations, a
non-finite charge, and a tensor-core expansion whose bounded waits run out
(the kernel unwinds, frees its tensor memory and reports WT_ERR_TIMEOUT);
after each the library keeps working."""
import os
import time
from contextlib import contextmanager

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


@contextmanager
def fault(name):
    os.environ["WT_FAULT"] = name
    try:
        yield
    finally:
        os.environ.pop("WT_FAULT", None)


def _w():
    return W.tiny_cell(nx=16, nz=32, n_t=8, radius=8 * UM)


def test_singular_fit_is_reported(P, torch):
    w = _w()
    s = P.Sensor(w.grid, w.columns)
    try:
        with fault("fit_singular"):
            with pytest.raises(P.WTError, match="WT_ERR_NOT_SPD"):
                s.fit()
    finally:
        s.close()
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        s.relax(w.times)
    finally:
        s.close()


def test_failed_allocations_are_reported(P, torch):
    w = _w()
    with fault("alloc"):
        with pytest.raises(P.WTError, match="WT_ERR_OOM"):
            P.Sensor(w.grid, w.columns)
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        s.relax(w.times)
        with fault("alloc"):
            with pytest.raises(P.WTError, match="WT_ERR_OOM"):
                s.extend("fp32")
        H = s.extend("fp32")
        torch.cuda.synchronize()
        assert torch.isfinite(H).all()
    finally:
        s.close()


def test_non_finite_charges_are_reported(P, torch):
    w = _w()
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        with fault("nan_q"):
            with pytest.raises(P.WTError, match="WT_ERR_NAN"):
                s.relax(w.times)
        s.relax(w.times)
        assert np.all(np.isfinite(s.charges()))
    finally:
        s.close()


def test_stalled_expansion_times_out_and_recovers(P, torch):
    w = _w()
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        s.relax(w.times)
        ref = s.extend("fp32")                  # tunes the launch shapes without the fault
        s.sync()
        with fault("queue_stall"):
            t0 = time.time()
            H = s.extend("fp32", out=torch.empty_like(ref))
            with pytest.raises(P.WTError, match="WT_ERR_TIMEOUT"):
                s.sync()
            host = torch.empty(tuple(ref.shape), dtype=torch.float32, pin_memory=True)
            with pytest.raises(P.WTError, match="WT_ERR_TIMEOUT"):
                s.extend("fp32", out=host)      # synchronous host path reports it directly
            assert time.time() - t0 < 60
        again = s.extend("fp32", out=torch.empty_like(ref))
        s.sync()
        assert torch.equal(again, ref)
    finally:
        s.close()


def test_truncated_time_basis_is_refused_by_the_fp32_paths(P, torch):
    """WT_FAULT=rank_cap caps the time basis at rank 4, far short of what the charge history
    needs: wt_relax still succeeds and reports the truncation, the FP32 field paths return
    WT_ERR_ACCURACY, and the FP64 path is unaffected."""
    from paper_2605_13987_gb300 import _binding as B
    w = W.tiny_cell(nx=16, nz=32, n_t=24, radius=8 * UM)
    s = P.Sensor(w.grid, w.columns)
    try:
        s.fit()
        with fault("rank_cap"):
            s.relax(w.times)
        info = s.info()
        assert info["rank"] == 4 and info["trunc_rel"] > 1e-6
        with pytest.raises(P.WTError) as e:
            s.extend("fp32")
        assert e.value.code == B.WT_ERR_ACCURACY
        H64 = s.extend("fp64")
        torch.cuda.synchronize()
        assert bool(torch.isfinite(H64).all())
        s.relax(w.times)                      # without the cap: a full basis, FP32 works again
        assert s.info()["trunc_rel"] <= 1e-7
        s.extend("fp32")
        torch.cuda.synchronize()
    finally:
        s.close()
