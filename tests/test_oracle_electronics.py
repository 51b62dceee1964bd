"""Pins of the oracle's front-end shaping: closed forms of the CR-(RC)^n
impulse response (peak time, unit area, peak value) and of the shaped
response to a delta and to a step of current."""
import math

import numpy as np

from oracle import electronics as E


def test_impulse_response_closed_forms():
    tau, dt = 2e-9, 1e-12
    for n in (1, 2, 4):
        h = E.impulse_response(200_000, dt, tau, n)
        k = int(np.argmax(h))
        assert abs(k * dt - n * tau) <= dt                       # peak at t = n tau
        assert abs(h.sum() * dt - 1.0) < 1e-6                    # unit area
        peak = n ** n * math.exp(-n) / (math.factorial(n) * tau)
        assert abs(h.max() - peak) < 1e-6 * peak


def test_delta_current_gives_the_impulse_response():
    """A unit charge delivered in one output bin (i = 1/dt there) returns
    G h(k dt) shifted to that bin."""
    dt, tau, n, G = 25e-12, 1e-9, 2, 3.5
    i = np.zeros((1, 400))
    i[0, 7] = 1.0 / dt
    v = E.shape(i, dt, tau, n, gain=G)[0]
    k = np.arange(400 - 7)
    assert np.allclose(v[7:], G * E.impulse_response(400, dt, tau, n)[k], rtol=1e-13, atol=0)
    assert not np.any(v[:7])


def test_step_current_settles_at_gain_times_current():
    """A constant current I: v -> G I (the response integrates to one)."""
    dt, tau, n, G, I = 5e-12, 0.4e-9, 3, 2.0, 1e-6
    v = E.shape(np.full((1, 20_000), I), dt, tau, n, gain=G)[0]
    assert abs(v[-1] - G * I) < 1e-4 * G * I


def test_noise_is_added_scaled():
    rng = np.random.default_rng(0)
    i = rng.standard_normal((3, 50))
    w = rng.standard_normal((3, 50))
    a = E.shape(i, 1e-11, 1e-10, 1)
    b = E.shape(i, 1e-11, 1e-10, 1, noise=w, noise_rms=0.25)
    assert np.allclose(b - a, 0.25 * w, rtol=0, atol=1e-15)
