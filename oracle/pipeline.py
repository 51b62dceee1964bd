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
    src: np.ndarray = None      # source positions when they differ from the nodes (a ring), else lay.src

    @property
    def sources(self):
        return self.lay.src if self.src is None else self.src

    @property
    def q(self):
        return self.rel["q"]

    def H_subgrid(self, t_idx=None, ix=None, iy=None, iz=None):
        q = self.q if t_idx is None else self.q[:, t_idx]
        return extend.field_subgrid(self.grid, self.sources, q, ix, iy, iz)

    def H_full(self, t_idx=None):
        return self.H_subgrid(t_idx)

    def H_points(self, pts, q=None):
        return extend.field_points(self.grid, self.sources, self.q if q is None else q, pts)


def solve(w, times=None, want_cond=False, n_ring=1, ring_frac=0.5, ring_az0=0.0):
    """Run the oracle on a workload (or anything with grid, columns, fit, times).

    n_ring > 1: the sources form a ring of lines inside each column (``geometry.ring_sources``);
    the nodes (one per column and source height) and the resistive lines stay as they are.  The
    fit then gives the source charges of node potentials, q = F phi (sources x nodes); the node
    capacitance is the charge each node's sources carry, C_n = N^T F symmetrised (N: source ->
    node), the relaxation runs on the nodes, and the sources take q(t) = F phi(t) with
    phi(t) = phi_DC + B zeta(t) the node potentials of the relaxation (``relax``)."""
    grid, cols = w.grid, w.columns
    lay = geometry.layout(grid, cols, w.fit.n_az, w.fit.n_h, w.fit.az0)
    S = geometry.interp_matrix(cols, lay)
    K, b = geometry.resistive_line(cols, lay, w.fit.v_w)
    phi = geometry.phi_dc(cols, lay, w.fit.v_w)
    t = w.times if times is None else times
    if n_ring == 1:
        P = greens.potential_matrix(grid, lay.colloc, lay.src)
        f = fitmod.fit(P, S, w.fit.tikhonov, want_cond=want_cond)
        rel = relaxmod.relax(f["Cn"], K, b, phi, t)
        return Solution(grid, cols, lay, P, S, f, K, b, phi, np.asarray(t), rel)
    src, node = geometry.ring_sources(cols, lay, n_ring, ring_frac, ring_az0, w.fit.n_az)
    P = greens.potential_matrix(grid, lay.colloc, src)
    f = fitmod.fit(P, S, w.fit.tikhonov, want_cond=want_cond)
    N = np.zeros((len(src), lay.n_src))
    N[np.arange(len(src)), node] = 1.0
    C = N.T @ f["F"]
    f["Cn"] = 0.5 * (C + C.T)
    f["asymmetry"] = np.linalg.norm(C - C.T) / np.linalg.norm(C)
    f["N"] = N
    rel = relaxmod.relax(f["Cn"], K, b, phi, t)
    zeta = rel["V"] @ (rel["amp"][:, None] * np.exp(-np.outer(rel["mu"], np.asarray(t, dtype=float))))
    phi_t = phi[:, None] + rel["B"] @ zeta
    rel["q_node"], rel["q_inf_node"] = rel["q"], rel["q_inf"]
    rel["phi"] = phi_t
    rel["q"] = f["F"] @ phi_t
    rel["q_inf"] = f["F"] @ phi
    return Solution(grid, cols, lay, P, S, f, K, b, phi, np.asarray(t), rel, src=src)
