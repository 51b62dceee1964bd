"""Signal-shape features of induced-current (or shaped) waveforms and their
first-order sensitivities, for the geometry scans of Sec. 5 (bias-electrode
diameter 6-14 um, diamond thickness), where the sensor variants are compared
by the shape of their signals.  The paper reports time resolution, which needs
the ionisation and noise model it takes from HEED/Garfield++; the features
here are the deterministic signal properties that time resolution is built
from (amplitude, peak time, collected charge, leading-edge threshold and
constant-fraction crossing times).

Definitions, for one waveform x_m on the grid tau_m = t0 + m dt, m = 0..n-1:

* amplitude  A = x_k, k the first index of the largest |x_m|; s = sign(A)
  (s = 1 when A = 0) and y_m = s x_m, so y_k = |A|.
* peak time  tau_k + dt delta, delta the vertex of the parabola through
  (k-1, k, k+1): delta = (y_{k-1} - y_{k+1}) / (2 (y_{k-1} - 2 y_k + y_{k+1}));
  delta = 0 at either end of the grid or for a zero denominator.
* charge     Q = dt sum_m x_m (rectangle rule on the output grid).
* crossing of fraction f on the leading edge: level l = f y_k; j the last
  index below k with y_j < l; the time is tau_j + dt (l - y_j) / (y_{j+1} - y_j)
  (linear interpolation).  Without such j (the waveform starts above the
  level, or A = 0) the crossing time is tau_0.
  Three crossings are reported: fractions lo, hi (rise time = t_hi - t_lo)
  and cfd (constant-fraction discrimination).

Feature vector: [A, t_peak, Q, t_lo, t_hi, t_cfd].

The integer decisions (k, j) are taken in float32 exactly as the library
takes them: |x| and s x are exact, l = f y_k is one rounded float32
product, comparisons are exact.  Everything after the decisions is float64.

Sensitivities: for a tangent waveform dx (d x / d theta for one parameter),
the derivative of each feature at fixed decisions (k, j):
  dA = dx_k;  d delta from the quotient rule;  dQ = dt sum dx;
  d t_f = dt [(f dy_k - dy_j)(y_{j+1} - y_j) - (l - y_j)(dy_{j+1} - dy_j)] / (y_{j+1} - y_j)^2.

TEST INFRASTRUCTURE ONLY: see the package docstring.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 6
NAMES = ("amplitude", "t_peak", "charge", "t_lo", "t_hi", "t_cfd")


def _decisions(x32, fracs32):
    """k, s, and the crossing indices j (or -1) from float32 samples."""
    a = np.abs(x32)
    k = int(np.argmax(a))                       # first index of the maximum
    s = np.float32(-1.0) if x32[k] < 0 else np.float32(1.0)
    y = s * x32
    js = []
    for f in fracs32:
        level = np.float32(f) * y[k]            # one float32 product
        below = np.nonzero(y[:k] < level)[0]
        js.append(int(below[-1]) if below.size else -1)
    return k, float(s), js


def features_one(x, t0, dt, lo=0.1, hi=0.9, cfd=0.5):
    """Feature vector (float64) of one waveform (values taken as float32)."""
    x32 = np.asarray(x, dtype=np.float32)
    fr = (np.float32(lo), np.float32(hi), np.float32(cfd))
    k, s, js = _decisions(x32, fr)
    y = s * x32.astype(np.float64)
    n = x32.size
    out = np.zeros(N_FEATURES)
    out[0] = float(x32[k])
    delta = 0.0
    if 0 < k < n - 1:
        den = y[k - 1] - 2.0 * y[k] + y[k + 1]
        if den != 0.0:
            delta = (y[k - 1] - y[k + 1]) / (2.0 * den)
    out[1] = t0 + dt * (k + delta)
    out[2] = dt * float(np.sum(x32.astype(np.float64)))
    for slot, (f, j) in enumerate(zip(fr, js)):
        if j < 0:
            out[3 + slot] = t0
        else:
            level = float(np.float32(f) * np.float32(y[k]))
            out[3 + slot] = t0 + dt * (j + (level - y[j]) / (y[j + 1] - y[j]))
    return out


def sensitivities_one(x, dx, t0, dt, lo=0.1, hi=0.9, cfd=0.5):
    """d(feature)/d(theta) for the tangent waveform dx, at fixed decisions."""
    x32 = np.asarray(x, dtype=np.float32)
    fr = (np.float32(lo), np.float32(hi), np.float32(cfd))
    k, s, js = _decisions(x32, fr)
    y = s * x32.astype(np.float64)
    dy = s * np.asarray(dx, dtype=np.float64)
    n = x32.size
    out = np.zeros(N_FEATURES)
    out[0] = s * dy[k]
    if 0 < k < n - 1:
        den = y[k - 1] - 2.0 * y[k] + y[k + 1]
        if den != 0.0:
            num = y[k - 1] - y[k + 1]
            dnum = dy[k - 1] - dy[k + 1]
            dden = dy[k - 1] - 2.0 * dy[k] + dy[k + 1]
            out[1] = dt * (dnum * den - num * dden) / (2.0 * den * den)
    out[2] = dt * float(np.sum(np.asarray(dx, dtype=np.float64)))
    for slot, (f, j) in enumerate(zip(fr, js)):
        if j >= 0:
            level = float(np.float32(f) * np.float32(y[k]))
            d = y[j + 1] - y[j]
            out[3 + slot] = dt * ((float(f) * dy[k] - dy[j]) * d - (level - y[j]) * (dy[j + 1] - dy[j])) / (d * d)
    return out


def features(x, t0, dt, lo=0.1, hi=0.9, cfd=0.5):
    """[n_tracks, 6] for waveforms x [n_tracks, n]."""
    x = np.atleast_2d(x)
    return np.stack([features_one(r, t0, dt, lo, hi, cfd) for r in x])


def sensitivities(x, dx, t0, dt, lo=0.1, hi=0.9, cfd=0.5):
    """[n_dir, n_tracks, 6] for waveforms x [n_tracks, n] and tangents dx [n_dir, n_tracks, n]."""
    x = np.atleast_2d(x)
    dx = np.asarray(dx).reshape((-1,) + x.shape)
    return np.stack([np.stack([sensitivities_one(r, d, t0, dt, lo, hi, cfd) for r, d in zip(x, dd)])
                     for dd in dx])
