"""Pins of the oracle's signal-shape features and their sensitivities:
closed forms on pulses whose features are exact (linear edges, parabolic
peaks, a Gaussian's area), symmetry under sign and time shifts, and the
sensitivities against exact directional derivatives (scaling, translation)
and against central differences of the feature function itself."""
import math

import numpy as np

from oracle import features as F


def _triangle(n, m0, m1, slope, dt):
    """Zero until sample m0, rising with `slope` per second to sample m1, then
    falling at twice the rate to zero."""
    t = np.arange(n) * dt
    ta, tp = m0 * dt, m1 * dt
    A = slope * (tp - ta)
    x = np.where(t <= ta, 0.0, np.where(t <= tp, slope * (t - ta), np.maximum(A - 2 * slope * (t - tp), 0.0)))
    return x, A, ta


def test_triangle_pulse_closed_forms():
    dt, t0 = 25e-12, 0.0
    x, A, ta = _triangle(400, 40, 140, 1.0 / (100 * 25e-12), dt)      # peak value 1 at sample 140
    f = F.features_one(x, t0, dt, lo=0.1, hi=0.9, cfd=0.5)
    rise = A / (1.0 / (100 * 25e-12))
    assert abs(f[0] - A) < 1e-6
    assert abs(f[3] - (ta + 0.1 * rise)) < 1e-4 * dt                    # linear edge: exact crossing
    assert abs(f[4] - (ta + 0.9 * rise)) < 1e-4 * dt
    assert abs(f[5] - (ta + 0.5 * rise)) < 1e-4 * dt
    # area of the triangle (rise 100 dt, fall 50 dt, height 1): rectangle rule is exact on its samples' sum
    assert abs(f[2] - dt * x.astype(np.float32).astype(np.float64).sum()) < 1e-12 * dt
    assert abs(f[2] - 0.5 * 150 * dt) < 1e-3 * 75 * dt


def test_parabolic_peak_is_located_between_samples():
    dt, t0 = 1e-11, 3e-9
    n = 200
    tp = t0 + 87.3 * dt
    t = t0 + np.arange(n) * dt
    x = np.maximum(2.0 - ((t - tp) / (10 * dt)) ** 2, 0.0)             # exact parabola near the top
    f = F.features_one(x, t0, dt)
    assert abs(f[1] - tp) < 1e-4 * dt
    assert f[0] == float(np.float32(x[87]))                              # the float32 sample


def test_gaussian_area():
    dt, sig = 1e-11, 7.5e-11
    t = np.arange(600) * dt
    x = 3.0 * np.exp(-0.5 * ((t - 2e-9) / sig) ** 2)
    f = F.features_one(x, 0.0, dt)
    assert abs(f[2] - 3.0 * math.sqrt(2 * math.pi) * sig) < 1e-6 * 3.0 * math.sqrt(2 * math.pi) * sig


def test_sign_and_shift_symmetry():
    dt = 2e-11
    x, _, _ = _triangle(300, 30, 90, 1e9, dt)
    f = F.features_one(x, 0.0, dt)
    g = F.features_one(-x, 0.0, dt)
    assert g[0] == -f[0] and g[2] == -f[2]
    assert np.array_equal(g[[1, 3, 4, 5]], f[[1, 3, 4, 5]])
    xs = np.concatenate([np.zeros(17), x[:-17]])                      # 17 samples later
    h = F.features_one(xs, 0.0, dt)
    assert np.allclose(h[[1, 3, 4, 5]] - f[[1, 3, 4, 5]], 17 * dt, rtol=0, atol=1e-6 * dt)
    k = F.features_one(x, 5e-9, dt)                                   # t0 offsets every time feature
    assert np.allclose(k[[1, 3, 4, 5]] - f[[1, 3, 4, 5]], 5e-9, rtol=0, atol=1e-6 * dt)


def test_undefined_crossings_and_zero_waveform():
    dt = 1e-11
    z = F.features_one(np.zeros(50), 1e-9, dt)
    assert np.array_equal(z, [0.0, 1e-9, 0.0, 1e-9, 1e-9, 1e-9])
    x = np.linspace(1.0, 0.0, 50)                                      # starts at its maximum
    f = F.features_one(x, 0.0, dt)
    assert f[0] == 1.0 and f[1] == 0.0 and f[3] == 0.0 and f[4] == 0.0


def test_sensitivity_of_scaling_and_translation():
    """dx = x (scale): dA = A, dQ = Q, times fixed.  dx = -x' (translation by
    one unit of time) of a parabolic pulse: the interpolated peak moves by
    one, the peak sample with the pulse's slope there."""
    dt = 1e-11
    x, A, _ = _triangle(300, 30, 130, 1e9, dt)
    s = F.sensitivities_one(x, x, 0.0, dt)
    f = F.features_one(x, 0.0, dt)
    assert abs(s[0] - f[0]) < 1e-7 * abs(f[0]) and abs(s[2] - f[2]) < 1e-7 * abs(f[2])
    assert np.allclose(s[[1, 3, 4, 5]], 0.0, atol=1e-12)
    # translation: a parabola-topped pulse with linear flanks, differentiated analytically
    n = 400
    t = np.arange(n) * dt
    tp, w = 200.4 * dt, 30 * dt

    def pulse(tt):
        return np.maximum(1.0 - ((tt - tp) / w) ** 2, 0.0)

    def dpulse(tt):
        return np.where(np.abs(tt - tp) < w, -2.0 * (tt - tp) / w ** 2, 0.0)

    x = pulse(t)
    dx = -dpulse(t)                                                   # d/dshift of pulse(t - shift)
    s = F.sensitivities_one(x, dx, 0.0, dt)
    # the vertex of an exact parabola moves exactly; the samples are rounded to float32 first
    assert abs(s[1] - 1.0) < 1e-4
    # the amplitude is the peak sample, whose value moves with the pulse's slope there
    k = int(np.argmax(x))
    assert k == 200 and abs(s[0] - 2.0 * (t[k] - tp) / w ** 2) < 1e-9 * abs(s[0])
    # the flanks are curved here, so the crossing derivative is the interpolant's: check by differences
    eps = 1e-3 * dt
    fp = F.features_one(pulse(t - eps), 0.0, dt)
    fm = F.features_one(pulse(t + eps), 0.0, dt)
    fd = (fp - fm) / (2 * eps)
    assert np.allclose(s[3:], fd[3:], rtol=2e-3, atol=0)


def test_sensitivities_match_central_differences():
    """Smooth pulses and smooth tangent directions (so that the step stays far
    below the sample-to-sample differences at every crossing), fourth-order
    central differences."""
    rng = np.random.default_rng(11)
    dt = 1e-11
    t = np.arange(256) * dt
    fr = (np.float32(0.1), np.float32(0.9), np.float32(0.5))
    checked = 0
    for trial in range(8):
        t1, t2 = rng.uniform(25, 60) * dt, rng.uniform(5, 15) * dt
        x = (np.exp(-t / t1) - np.exp(-t / t2)) * rng.uniform(0.5, 2.0)
        if trial % 2:
            x = -x
        c = rng.standard_normal(3)
        dx = c[0] * x + c[1] * np.sin(t / (23 * dt)) * np.abs(x) + c[2] * np.exp(-t / (30 * dt))
        s = F.sensitivities_one(x, dx, 0.0, dt)
        eps = 4e-3                                                    # float32 inputs: not smaller
        dec = [F._decisions(np.asarray(x + e * eps * dx, np.float32), fr) for e in (-2, -1, 0, 1, 2)]
        if any(d != dec[2] for d in dec):
            continue                                                  # a decision flipped: no derivative
        f = [F.features_one(x + e * eps * dx, 0.0, dt) for e in (-2, -1, 1, 2)]
        fd = (8 * (f[2] - f[1]) - (f[3] - f[0])) / (12 * eps)
        scale = np.maximum(np.abs(fd), [np.abs(x).max(), dt, dt * np.abs(x).sum(), dt, dt, dt])
        assert np.all(np.abs(s - fd) <= 1e-3 * scale), (trial, s, fd)
        checked += 1
    assert checked >= 5


def test_batched_forms_stack_the_single_ones():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 64))
    dx = rng.standard_normal((3, 5, 64))
    f = F.features(x, 0.0, 1e-11)
    s = F.sensitivities(x, dx, 0.0, 1e-11)
    assert f.shape == (5, 6) and s.shape == (3, 5, 6)
    assert np.array_equal(f[2], F.features_one(x[2], 0.0, 1e-11))
    assert np.array_equal(s[1, 4], F.sensitivities_one(x[4], dx[1, 4], 0.0, 1e-11))
