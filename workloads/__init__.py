"""Seeded synthetic inputs shared by the FP64 oracle and the GPU library.

This module holds no arithmetic of the solver: it only draws sensor
geometries, material values, time grids and carrier tracks from fixed seeds,
in SI units, with the shapes of the sensors and tracks the paper studies
(Sec. 5: 55 um pitch 3D pixels, ~6 um radius graphitised columns, 500 um
thick diamond, resistivity around 0.75 Ohm cm; Sec. 2: straight minimum-
ionising tracks crossing the sensor).  The paper's own inputs (Garfield++
carrier paths from 180 GeV/c pions, test-beam geometry files) are not
available; these generators stand in for them.
"""
from .configs import (  # noqa: F401
    GridSpec, ColumnSpec, FitSpec, TrackSet, Workload,
    workload, c1_single_cell, c2_pixel3x3, c3_batch, c4_adjoint, c5_large,
    tiny_cell, log_times, mip_tracks, drift_tracks, central_pixel_tracks, scan_bias_diameter, scan_thickness,
)
