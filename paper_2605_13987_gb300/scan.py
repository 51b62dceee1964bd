"""Geometry what-if scans (Sec. 5: the bias-electrode diameter from 6 to
14 um in 2 um steps, and the diamond thickness), the sensor variants
compared by the shape of their signals.

For every variant: fit and relaxation (``Sensor.fit``, ``Sensor.relax``);
then either the fields of all variants in one captured batch
(``wt_batch_run``) followed by Eq. 1 per variant, or, with sensitivities,
``wt_eq1_tangents``, which gives each variant's currents together with
their derivatives along the four design parameters (readout and bias
resistivity scales, column radius, lateral scale).  An optional CR-(RC)^n
shaper (``wt_shape``) filters the currents, and, being linear, the tangents
with them.  ``wt_features`` reduces every waveform to amplitude, peak
time, collected charge, 10 %/90 % leading-edge times and a constant-fraction
time, and the tangents to those features' derivatives.  Every step runs in
the library; this module only sequences the calls and copies the small
results to the host.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _binding as B
from .sensor import Sensor, extend_batch

PARAMS = ("s_R", "s_B", "r", "lambda")


@dataclass
class ScanPoint:
    value: float                          # the scanned quantity (e.g. bias diameter in um)
    features: np.ndarray                  # [n_tracks, 6], see FEATURE_NAMES
    loss: Optional[float] = None          # mean i^2 (with sensitivities)
    grad: Optional[np.ndarray] = None     # [4] dL/d(s_R, s_B, r, lambda)
    dfeatures: Optional[np.ndarray] = None  # [4, n_tracks, 6] d feature / d parameter
    info: Dict = field(default_factory=dict)
    waveforms: Optional[np.ndarray] = None  # [n_tracks, n_out] (keep_waveforms)
    tangents: Optional[np.ndarray] = None   # [4, n_tracks, n_out] (keep_waveforms, sensitivities)

    def summary(self) -> Dict[str, float]:
        """Track medians of the features (times in s), plus the rise time."""
        f = self.features
        out = {name: float(np.median(f[:, k])) for k, name in enumerate(B.FEATURE_NAMES)}
        out["rise_time"] = float(np.median(f[:, 4] - f[:, 3]))
        return out


def _device_tracks(tr, torch, device):
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    return dict(n_tracks=tr.n_tracks, n_steps=tr.n_steps, n_out=tr.n_out, dt=tr.dt, charge=1.0,
                x=dev(tr.x), y=dev(tr.y), z=dev(tr.z), vx=dev(tr.vx), vy=dev(tr.vy), vz=dev(tr.vz),
                q=dev(tr.charge))


def run_scan(points: Sequence[Tuple[float, object]], sensitivities: bool = False, shaper: Optional[dict] = None,
             fractions: Tuple[float, float, float] = (0.1, 0.9, 0.5), device: int = 0,
             keep_waveforms: bool = False) -> List[ScanPoint]:
    """points: (value, workload) pairs (workloads with tracks, e.g. from
    ``workloads.scan_bias_diameter``).  shaper: dict(tau=..., order=...,
    gain=1.0) or None.  keep_waveforms: also return the (shaped) currents
    and their tangents.  Returns one ScanPoint per variant."""
    import torch
    dev = f"cuda:{device}"
    lo, hi, cfd = fractions
    sensors, tracks = [], []
    try:
        for value, w in points:
            s = Sensor(w.grid, w.columns, device=device)
            sensors.append(s)
            s.fit(n_az=w.fit.n_az, n_h=w.fit.n_h, tikhonov=w.fit.tikhonov, v_w=w.fit.v_w, az0=w.fit.az0)
            s.relax(w.times)
            tracks.append(_device_tracks(w.tracks, torch, dev))
        currents, tangents, losses, grads = [], [], [], []
        if sensitivities:
            for s, t in zip(sensors, tracks):
                i, di, L, g = s.tangents(t)
                currents.append(i)
                tangents.append(di)
                losses.append(L)
                grads.append(g)
        else:
            H = extend_batch(sensors, "fp32")
            for s, h, t in zip(sensors, H, tracks):
                currents.append(s.eq1(h, t))
            del H
        out = []
        for k, ((value, w), s, t) in enumerate(zip(points, sensors, tracks)):
            x, dx = currents[k], (tangents[k] if sensitivities else None)
            if shaper is not None:
                sh = {"gain": 1.0, **shaper}
                x = s.shape(x, t["dt"], sh["tau"], sh["order"], sh["gain"])
                if dx is not None:
                    n_tr, n_out = x.shape
                    dx = s.shape(dx.reshape(-1, n_out), t["dt"], sh["tau"], sh["order"], sh["gain"]).reshape(
                        4, n_tr, n_out)
            f, df = s.features(x, t["dt"], 0.0, dx=dx, lo=lo, hi=hi, cfd=cfd)
            s.sync()
            out.append(ScanPoint(value=value, features=f.cpu().numpy(),
                                 loss=losses[k] if sensitivities else None,
                                 grad=grads[k] if sensitivities else None,
                                 dfeatures=df.cpu().numpy() if df is not None else None,
                                 info=s.info(),
                                 waveforms=x.cpu().numpy() if keep_waveforms else None,
                                 tangents=dx.cpu().numpy() if (keep_waveforms and dx is not None) else None))
        return out
    finally:
        for s in sensors:
            s.close()
