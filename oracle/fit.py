"""Point-charge fit to the electrode boundary values (Abstract; Sec. 3).

For node potentials phi, the source charges q minimise

    || P q + c 1 - S phi ||^2   subject to   1^T q = 0,

with P[i, j] the potential at collocation point i from unit source j, c one
free potential offset (the periodic cell is neutral, so only potential
differences are defined) and S the boundary target of ``geometry``.  The
constraint is eliminated with an orthonormal basis B of the complement of the
all-ones vector (q = B z); the remaining unconstrained least-squares problem
in [z; c] is solved by a Householder QR factorisation (LAPACK), the textbook
stable route.  Linear in phi, so the fit is the matrix F (q = F phi).

Capacitance (Green reciprocity): C_n = (F + F^T) / 2.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def null_basis(n):
    """Orthonormal basis (n x n-1) of {v : sum(v) = 0}: the last n-1 columns of
    the Householder reflector that maps the all-ones vector to -sqrt(n) e_1."""
    v = np.ones(n)
    v[0] += np.sqrt(n)
    H = np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)
    return H[:, 1:]


def fit(P, S, tikhonov=0.0, want_cond=False):
    """Return dict with F (sources x nodes), offsets (nodes), Cn (when sources and nodes coincide),
    and diagnostics."""
    nc, ns = P.shape
    B = null_basis(ns)
    A = np.hstack([P @ B, np.ones((nc, 1))])
    rhs = S
    if tikhonov > 0.0:
        scale = np.max(np.sum(A[:, :-1] ** 2, axis=0))
        reg = np.zeros((ns - 1, ns))
        reg[:, :ns - 1] = np.sqrt(tikhonov * scale) * np.eye(ns - 1)
        A = np.vstack([A, reg])
        rhs = np.vstack([S, np.zeros((ns - 1, S.shape[1]))])
    # X = A^+ rhs via QR: rhs^T Q, R  (Q is never formed; A is a temporary and is factorised in place)
    QtR, R = sla.qr_multiply(A, rhs.T, mode="right", overwrite_a=True)
    X = sla.solve_triangular(R, QtR.T, lower=False)
    F = B @ X[:ns - 1]
    out = {"F": F, "offset": X[ns - 1], "B": B}
    if F.shape[0] == F.shape[1]:        # one source per node: F is the capacitance itself
        out["Cn"] = 0.5 * (F + F.T)
        out["asymmetry"] = np.linalg.norm(F - F.T) / np.linalg.norm(F)
    if want_cond:
        # condition number of A with unit-norm columns (the offset column and
        # the potential columns differ by ~1e15 in scale; QR is insensitive to
        # column scaling, so the equilibrated number is the meaningful one)
        Rs = R / np.linalg.norm(R, axis=0)[None, :]
        sv = np.linalg.svd(Rs, compute_uv=False)
        out["cond_A"] = sv[0] / sv[-1]
    return out


def boundary_residual(P, S, F, offset, phi):
    """|| P q + c - S phi || / || S phi || for node potentials phi."""
    q = F @ phi
    c = offset @ phi
    t = S @ phi
    return np.linalg.norm(P @ q + c - t) / np.linalg.norm(t)
