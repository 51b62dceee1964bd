"""Front-end shaping of the induced currents (the readout electronics after
Eq. 1; the paper lists the electronics' response as a further step of the
signal chain without giving its transfer function, so it is parameterised
here as the common CR-(RC)^n shaper).

Impulse response of order n and time constant tau, unit area:
    h(t) = (t / tau)^n e^(-t / tau) / (n! tau),   t >= 0,
peaking at t = n tau.  The shaped signal on the output grid tau_m = (m + 1/2) dt
is the rectangle-rule convolution
    v_m = G sum_{k=0}^{m} h(k dt) dt i_{m-k}  +  sigma w_m,
with gain G, noise RMS sigma and the noise samples w_m passed in (drawn by the
caller).  TEST INFRASTRUCTURE ONLY: see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np


def impulse_response(n_taps, dt, tau, order):
    """h(k dt) for k = 0..n_taps-1 (FP64)."""
    t = np.arange(n_taps) * dt / tau
    return t ** order * np.exp(-t) / (math.factorial(order) * tau)


def shape(i, dt, tau, order, gain=1.0, noise=None, noise_rms=0.0):
    """v [n_tracks, n_out] from currents i [n_tracks, n_out] (FP64 direct
    convolution, np.convolve per track)."""
    i = np.atleast_2d(np.asarray(i, dtype=np.float64))
    n_out = i.shape[1]
    h = gain * impulse_response(n_out, dt, tau, order) * dt
    v = np.stack([np.convolve(row, h)[:n_out] for row in i])
    if noise is not None and noise_rms != 0.0:
        v = v + noise_rms * np.asarray(noise, dtype=np.float64).reshape(v.shape)
    return v
