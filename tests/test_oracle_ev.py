"""Pins of the Evenbly-Vidal oracle (oracle/ev.py) against facts that do not
come from its own code: the variational characterisation of the polar factor
(and its closed-form value, the sum of singular values), the equivalence of
its fixed points with a vanishing Stiefel gradient (App. ev_steplimit), and
the energy decrease of sweeps on a small critical-Ising MERA."""
import numpy as np
import pytest

from oracle import ev
from oracle import geometry as geo
from oracle import mera as om
from paper_2007_03638_gb300 import inputs as inp


def _iso(rng, n, p, dt):
    a = rng.standard_normal((n, p)) + (1j * rng.standard_normal((n, p)) if dt == np.complex128 else 0)
    q, _ = np.linalg.qr(a)
    return q


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_polar_factor_maximises_overlap(dt):
    rng = np.random.default_rng(11)
    n, p = 9, 4
    D = rng.standard_normal((n, p)) + (1j * rng.standard_normal((n, p)) if dt == np.complex128 else 0)
    Q = ev.polar_factor(D)
    assert np.abs(Q.conj().T @ Q - np.eye(p)).max() < 1e-13
    P = Q.conj().T @ D
    assert np.abs(P - P.conj().T).max() < 1e-12                       # Hermitian
    assert np.linalg.eigvalsh(0.5 * (P + P.conj().T)).min() > -1e-12  # positive semidefinite
    best = np.real(np.trace(D.conj().T @ Q))
    assert abs(best - np.linalg.svd(D, compute_uv=False).sum()) < 1e-12 * best
    for _ in range(200):
        W = _iso(rng, n, p, dt)
        assert np.real(np.trace(D.conj().T @ W)) <= best + 1e-12


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_fixed_points_have_zero_gradient(dt):
    """D = W M with M Hermitian negative definite: the update returns W and
    the Stiefel gradient of D at W vanishes; a tangent component moves it."""
    rng = np.random.default_rng(5)
    n, p = 16, 4
    W = _iso(rng, n, p, dt)
    a = rng.standard_normal((p, p)) + (1j * rng.standard_normal((p, p)) if dt == np.complex128 else 0)
    M = -(a @ a.conj().T + 0.5 * np.eye(p))
    D = W @ M
    assert np.abs(ev.ev_update(D) - W).max() < 1e-12
    assert np.abs(geo.project(W, D, geo.STIEFEL)).max() < 1e-12
    R = rng.standard_normal((n, p)) + (1j * rng.standard_normal((n, p)) if dt == np.complex128 else 0)
    X = geo.project(W, R, geo.STIEFEL)
    assert np.abs(ev.ev_update(D + 0.3 * X) - W).max() > 1e-3


def test_sweeps_lower_the_energy():
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    gamma = float(np.linalg.eigvalsh(h3).max()) + 0.5
    us, ws = inp.random_mera(4, 4, 2, seed=1)
    e = [om.energy(h3, us, ws)]
    for _ in range(3):
        us, ws, es = ev.ev_sweep(h3, us, ws, gamma)
        e.append(es[-1])
    assert all(b < a for a, b in zip(e, e[1:])), e
    # still a MERA: every tensor isometric
    for t in us + ws:
        assert np.abs(t.conj().T @ t - np.eye(t.shape[1])).max() < 1e-12


def test_sweeps_lower_the_ternary_energy():
    h = inp.ising_bond(1.0)
    gamma = float(np.linalg.eigvalsh(h).max()) + 0.5
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=5)
    from oracle import ternary as ot
    e = [ot.energy(h, us, ws)]
    for _ in range(3):
        us, ws, es = ev.ev_sweep(h, us, ws, gamma, network="ternary")
        e.append(es[-1])
    assert all(b < a for a, b in zip(e, e[1:])), e
