"""Inputs of the geometry scans: the variants differ only in the scanned
quantity, every column radius stays below one lateral grid spacing (outside
the box-band kernel's indefinite windows), and the tracks enter through the
central pixel."""
import math

import numpy as np

import workloads as W
from workloads.configs import UM


def test_bias_diameter_scan_varies_only_the_bias_radius():
    pts = W.scan_bias_diameter(n_tracks=50, n_steps=20, n_t=8)
    assert [d for d, _ in pts] == [6.0, 8.0, 10.0, 12.0, 14.0]
    base = pts[0][1]
    for d, w in pts:
        assert w.grid == base.grid
        h = w.grid.Lx / w.grid.Nx
        for c0, c in zip(base.columns, w.columns):
            assert (c.x, c.y, c.z0, c.z1, c.terminal_top, c.driven, c.resistivity) == \
                   (c0.x, c0.y, c0.z0, c0.z1, c0.terminal_top, c0.driven, c0.resistivity)
            want = 5 * UM if c.terminal_top else 0.5 * d * UM
            assert abs(c.radius - want) < 1e-15
            assert c.radius < h and math.sin(math.pi * c.radius / h) > 0.4
        assert w.tracks is base.tracks
        assert sum(c.driven for c in w.columns) == 1


def test_scan_tracks_enter_the_central_pixel():
    for _, w in W.scan_bias_diameter(n_tracks=200, n_steps=30, n_t=8)[:1] + W.scan_thickness(n_tracks=200,
                                                                                                n_steps=30, n_t=8):
        tr = w.tracks
        p = 55 * UM
        assert np.all((tr.x[:, 0] >= p) & (tr.x[:, 0] < 2 * p) & (tr.y[:, 0] >= p) & (tr.y[:, 0] < 2 * p))
        assert np.all(tr.z[:, 0] == w.grid.Lz)
        assert tr.n_out == 60


def test_thickness_scan_keeps_the_vertical_spacing():
    pts = W.scan_thickness(n_tracks=10, n_steps=10, n_t=8)
    hz = [w.grid.Lz / w.grid.Nz for _, w in pts]
    assert [t for t, _ in pts] == [300.0, 400.0, 500.0]
    assert max(hz) / min(hz) < 1.12
    for _, w in pts:
        assert all(c.z1 == w.grid.Lz and c.z0 == 0.0 for c in w.columns)
