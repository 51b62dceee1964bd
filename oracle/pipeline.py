"""Whole oracle pipeline for one sensor: geometry -> fit -> relaxation, with
field evaluation helpers.  See the sibling modules for the method readings."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import geometry, greens, fit as fitmod, relax as relaxmod, extend


@dataclass
class Solution:
    grid: object
    columns: list
    lay: object
    P: np.ndarray
    S: np.ndarray
    fit: dict
    K: np.ndarray
    b: np.ndarray
    phi_dc: np.ndarray
    times: np.ndarray
    rel: dict

    @property
    def q(self):
        return self.rel["q"]

    def H_subgrid(self, t_idx=None, ix=None, iy=None, iz=None):
        q = self.q if t_idx is None else self.q[:, t_idx]
        return extend.field_subgrid(self.grid, self.lay.src, q, ix, iy, iz)

    def H_full(self, t_idx=None):
        return self.H_subgrid(t_idx)

    def H_points(self, pts, q=None):
        return extend.field_points(self.grid, self.lay.src, self.q if q is None else q, pts)


def solve(w, times=None, want_cond=False):
    """Run the oracle on a workload (or anything with grid, columns, fit, times)."""
    grid, cols = w.grid, w.columns
    lay = geometry.layout(grid, cols, w.fit.n_az, w.fit.n_h, w.fit.az0)
    P = greens.potential_matrix(grid, lay.colloc, lay.src)
    S = geometry.interp_matrix(cols, lay)
    f = fitmod.fit(P, S, w.fit.tikhonov, want_cond=want_cond)
    K, b = geometry.resistive_line(cols, lay, w.fit.v_w)
    phi = geometry.phi_dc(cols, lay, w.fit.v_w)
    t = w.times if times is None else times
    rel = relaxmod.relax(f["Cn"], K, b, phi, t)
    return Solution(grid, cols, lay, P, S, f, K, b, phi, np.asarray(t), rel)
