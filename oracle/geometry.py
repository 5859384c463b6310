"""Riemannian geometry of Stiefel and Grassmann manifolds, FP64, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Every operation is the paper's definition written out on dense matrices:
the projection of Eqs. (stiefel_gradient)/(grassmann_gradient), the
exponential retraction of Eq. (retraction) with the full n x n generator Q_X
and ``scipy.linalg.expm``, the transport of Eq. (transport) with the same
exponential, the metric g(X, Y) = Re Tr X^dag Y (Sec. 2.2) and the
preconditioner of Eqs. (preconditioner)/(preconditioner_solution).  None of
the low-rank shortcuts of the CUDA library are used here.

Pins (tests/test_oracle_geometry.py): R(0) = W, dR/dalpha(0) = X by central
differences, R^dag R = 1, transport preserves the metric and tangency,
projection is idempotent and orthogonal, the Grassmann closed form with
sines and cosines of singular values, and Eq. (preconditioner) at delta = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

STIEFEL = "stiefel"
GRASSMANN = "grassmann"


def dag(a):
    return a.conj().T


def inner(X, Y):
    """Euclidean metric on the product manifold: sum_v Re Tr(X_v^dag Y_v)."""
    return float(sum(np.real(np.vdot(x, y)) for x, y in zip(X, Y)))


def project(W, D, kind):
    """Orthogonal projection of D onto the tangent space at W (Sec. 2.2)."""
    if kind == STIEFEL:
        return D - 0.5 * W @ (dag(W) @ D + dag(D) @ W)
    return D - W @ (dag(W) @ D)


def generator(W, X):
    """Q_X = [W W_perp] [[A, -B^dag], [B, 0]] [W W_perp]^dag with X = W A + W_perp B,
    written without W_perp: Q_X = W A W^dag + Z W^dag - W Z^dag, Z = X - W A."""
    A = dag(W) @ X
    Z = X - W @ A
    return W @ A @ dag(W) + Z @ dag(W) - W @ dag(Z)


def retract(W, X, alpha):
    """R_W(X, alpha) = exp(alpha Q_X) W  (Eq. retraction), dense exponential."""
    return sla.expm(alpha * generator(W, X)) @ W


def transport(W, X, alpha, Y):
    """T_W(Y, X, alpha) = exp(alpha Q_X) Y  (Eq. transport)."""
    return sla.expm(alpha * generator(W, X)) @ Y


def polar(W):
    """Isometric polar factor U V^dag of W = U S V^dag (re-isometrisation)."""
    u, _, vh = np.linalg.svd(W, full_matrices=False)
    return u @ vh


def _regularised(rho, delta):
    lam, v = np.linalg.eigh(rho)
    return np.sqrt(lam**2 + delta**2), v


def precondition(W, X, rho, delta, kind):
    """Solve Re Tr[Y^dag Xt rho] = Re Tr[Y^dag X] for all tangent Y (Eq. preconditioner).

    With X = W A + W_perp B: Xt = W At + W_perp Bt, At rho + rho At = 2 A,
    Bt = B rho^{-1} (Eq. preconditioner_solution).  rho is replaced by its
    regularised version (rho^2 + delta^2)^{1/2}, i.e. eigenvalues
    lambda -> sqrt(lambda^2 + delta^2), in both the Sylvester and the inverse part.
    """
    lt, v = _regularised(rho, delta)
    A = dag(W) @ X if kind == STIEFEL else np.zeros((W.shape[1],) * 2, dtype=X.dtype)
    Z = X - W @ A
    Ah = dag(v) @ A @ v
    At = v @ (2.0 * Ah / (lt[:, None] + lt[None, :])) @ dag(v)
    Bt = Z @ (v @ np.diag(1.0 / lt) @ dag(v))
    return W @ At + Bt
