"""Quasi-static relaxation of the electrode charges in time.

Reading of the Abstract (third-order PDE from the quasi-static limit of
Maxwell's equations): d/dt div(eps grad psi) + div(sigma grad psi) = 0 with
sigma = 1/rho inside the columns and 0 in the diamond.  The bulk stays
charge-free; each thin column is a resistive line (``geometry``), so with
node charges q = C_n phi (``fit``):

    C_n dphi/dt = K phi + b,   q(0) = 0,

V_w applied at t = 0 to the driven readout terminal (a step response; Eq. 1
uses V_w = 1 V).  Late-time state phi_DC: V_w on the driven column, 0 on the
others, so q_inf = C_n phi_DC.  With psi = phi - phi_DC = B zeta + beta 1
(B: basis of the complement of 1), neutrality 1^T K psi = 0 fixes beta and
turns K into Kt = K - K 1 1^T K / (1^T K 1).  The modes solve the symmetric-
definite generalised eigenproblem

    (-B^T Kt B) v = mu (B^T C_n B) v,   v^T (B^T C_n B) v = 1,

and q(t) = q_inf + C_n B sum_k v_k exp(-mu_k t) v_k^T B^T (-q_inf).

Sec. 3 describes an iterative forward-Euler procedure; ``relax_euler`` keeps
that scheme (charges -> potentials -> line currents -> charge update) as a
cross-check that converges to the exact exponential as dt -> 0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .fit import null_basis


def _reduced(Cn, K):
    n = Cn.shape[0]
    B = null_basis(n)
    one = np.ones(n)
    K1 = K @ one
    Kt = K - np.outer(K1, K1) / (one @ K1)
    Am = B.T @ Cn @ B
    Sm = -(B.T @ Kt @ B)
    return B, 0.5 * (Am + Am.T), 0.5 * (Sm + Sm.T)


def modes(Cn, K):
    B, Am, Sm = _reduced(Cn, K)
    mu, V = sla.eigh(Sm, Am)
    return mu, V, B


def relax(Cn, K, b, phi_dc, times):
    """q [Ns, Nt] at the given times (exact modal exponential)."""
    mu, V, B = modes(Cn, K)
    q_inf = Cn @ phi_dc
    c = V.T @ (B.T @ (-q_inf))                       # modal amplitudes
    E = np.exp(-np.outer(mu, times))                 # [modes, Nt]
    zeta = V @ (c[:, None] * E)
    q = q_inf[:, None] + Cn @ (B @ zeta)
    return {"q": q, "mu": mu, "q_inf": q_inf, "V": V, "amp": c, "B": B}


def relax_expm(Cn, K, b, phi_dc, times):
    """Same q(t) through scipy's matrix exponential of -Am^-1 Sm (cross-check)."""
    B, Am, Sm = _reduced(Cn, K)
    q_inf = Cn @ phi_dc
    zeta0 = np.linalg.solve(Am, B.T @ (-q_inf))
    M = -np.linalg.solve(Am, Sm)
    out = np.empty((Cn.shape[0], len(times)))
    for n, t in enumerate(times):
        out[:, n] = q_inf + Cn @ (B @ (sla.expm(M * t) @ zeta0))
    return out


def relax_euler(Cn, K, b, times, dt):
    """Forward Euler on the charges: potentials from charges through the
    capacitance (pseudo-inverse on the neutral subspace, the offset fixed by
    charge conservation), line currents K phi + b, explicit update."""
    n = Cn.shape[0]
    B = null_basis(n)
    Am = B.T @ Cn @ B
    one = np.ones(n)
    K1 = K @ one
    q = np.zeros(n)
    t = 0.0
    out = np.empty((n, len(times)))
    for i, tn in enumerate(times):
        while t < tn - 1e-30:
            h = min(dt, tn - t)
            zeta = np.linalg.solve(Am, B.T @ q)
            phi0 = B @ zeta
            beta = -(K1 @ phi0 + one @ b) / (one @ K1)
            phi = phi0 + beta * one
            q = q + h * (K @ phi + b)
            t += h
        out[:, i] = q
    return out
