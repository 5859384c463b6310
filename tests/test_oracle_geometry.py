"""Pins of the oracle's Stiefel/Grassmann geometry (Sec. 2) and preconditioner
(Sec. 3) against closed forms, finite differences and invariants (CPU only)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import geometry as geo
from paper_2007_03638_gb300 import inputs as inp

CASES = [(16, 16, geo.STIEFEL), (16, 4, geo.GRASSMANN), (9, 3, geo.STIEFEL), (12, 5, geo.GRASSMANN)]


def _setup(n, p, kind, dt=np.float64, seed=0):
    rng = np.random.default_rng(seed)
    W = inp._haar_like(rng, n, p, dt)
    D = rng.standard_normal((n, p)) + (1j * rng.standard_normal((n, p)) if dt == np.complex128 else 0)
    X = geo.project(W, D, kind)
    Y = geo.project(W, rng.standard_normal((n, p)) + 0 * D, kind)
    return rng, W, D, X, Y


def _is_tangent(W, X, kind, tol=1e-12):
    A = W.conj().T @ X
    if kind == geo.STIEFEL:
        return np.abs(A + A.conj().T).max() < tol
    return np.abs(A).max() < tol


@pytest.mark.parametrize("n,p,kind", CASES)
@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_projection(n, p, kind, dt):
    rng, W, D, X, Y = _setup(n, p, kind, dt)
    assert _is_tangent(W, X, kind)
    assert np.abs(geo.project(W, X, kind) - X).max() < 1e-13           # idempotent
    assert abs(geo.inner([D - X], [Y])) < 1e-12                         # orthogonal
    assert abs(geo.inner([X], [Y]) - geo.inner([D], [Y])) < 1e-12       # g(G,Y) = Re Tr D^dag Y


@pytest.mark.parametrize("n,p,kind", CASES)
@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_retraction_and_transport(n, p, kind, dt):
    rng, W, D, X, Y = _setup(n, p, kind, dt, seed=1)
    a = 0.37
    R = geo.retract(W, X, a)
    assert np.abs(geo.retract(W, X, 0.0) - W).max() < 1e-14
    assert np.abs(R.conj().T @ R - np.eye(p)).max() < 1e-13
    h = 1e-5
    dR0 = (geo.retract(W, X, h) - geo.retract(W, X, -h)) / (2 * h)
    assert np.abs(dR0 - X).max() < 1e-8
    dRa = (geo.retract(W, X, a + h) - geo.retract(W, X, a - h)) / (2 * h)
    assert np.abs(dRa - geo.transport(W, X, a, X)).max() < 1e-8     # X' = T(X)
    TY, TX = geo.transport(W, X, a, Y), geo.transport(W, X, a, X)
    assert _is_tangent(R, TY, kind, 1e-12)
    assert abs(geo.inner([TY], [TX]) - geo.inner([Y], [X])) < 1e-12   # metric preserving
    assert abs(geo.inner([TY], [TY]) - geo.inner([Y], [Y])) < 1e-12


def test_unitary_closed_form():
    """Square case: exp(alpha Q_X) W = W exp(alpha W^dag X)."""
    _, W, _, X, _ = _setup(16, 16, geo.STIEFEL, seed=2)
    a = 0.8
    assert np.abs(geo.retract(W, X, a) - W @ sla.expm(a * W.T @ X)).max() < 1e-12


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_grassmann_closed_form(dt):
    """Grassmann case: with X = U S V^dag, exp(alpha Q_X) W = (W V cos(aS) + U sin(aS)) V^dag
    and T(Y) = Y - (W V sin(aS) + U (1 - cos(aS))) U^dag Y."""
    _, W, _, X, Y = _setup(16, 4, geo.GRASSMANN, dt, seed=3)
    a = 1.3
    U, s, Vh = np.linalg.svd(X, full_matrices=False)
    V = Vh.conj().T
    R = (W @ V @ np.diag(np.cos(a * s)) + U @ np.diag(np.sin(a * s))) @ Vh
    assert np.abs(geo.retract(W, X, a) - R).max() < 1e-12
    T = Y - (W @ V @ np.diag(np.sin(a * s)) + U @ np.diag(1 - np.cos(a * s))) @ (U.conj().T @ Y)
    assert np.abs(geo.transport(W, X, a, Y) - T).max() < 1e-12


@pytest.mark.parametrize("n,p,kind", CASES)
def test_preconditioner_identity(n, p, kind):
    """Eq. (preconditioner) at delta = 0: Re Tr[Y^dag Xt rho] = Re Tr[Y^dag X] for all
    tangent Y; Xt is tangent; with delta > 0 it is the same with rho -> (rho^2+delta^2)^1/2."""
    rng, W, D, X, _ = _setup(n, p, kind, seed=4)
    a = rng.standard_normal((p, p))
    rho = a @ a.T + 0.05 * np.eye(p)
    rho /= np.trace(rho)
    Xt = geo.precondition(W, X, rho, 0.0, kind)
    assert _is_tangent(W, Xt, kind, 1e-10)
    for _ in range(5):
        Y = geo.project(W, rng.standard_normal((n, p)), kind)
        assert abs(np.sum(Y * (Xt @ rho)) - np.sum(Y * X)) < 1e-10
    delta = 0.3
    lam, v = np.linalg.eigh(rho)
    rt = v @ np.diag(np.sqrt(lam**2 + delta**2)) @ v.T
    Xt = geo.precondition(W, X, rho, delta, kind)
    Y = geo.project(W, rng.standard_normal((n, p)), kind)
    assert abs(np.sum(Y * (Xt @ rt)) - np.sum(Y * X)) < 1e-10


def test_polar():
    rng = np.random.default_rng(5)
    W = inp._haar_like(rng, 16, 4, np.float64)
    P = geo.polar(W + 1e-9 * rng.standard_normal(W.shape))
    assert np.abs(P.T @ P - np.eye(4)).max() < 1e-14
    assert np.abs(P - W).max() < 1e-8
