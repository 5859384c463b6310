"""Pins of the uniform-MPS oracle (oracle/mps.py, Sec. 5) against an exact
ground state (AKLT), closed forms, an independent power iteration, finite
differences and a long periodic chain computed with transfer matrices."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mps
from oracle import optim as oo
from paper_2007_03638_gb300 import inputs as inp


def test_aklt_is_an_exact_ground_state():
    A, h = inp.aklt_mps()
    M = mps.as_matrix(A)
    assert np.abs(M.T @ M - np.eye(2)).max() < 1e-14          # left-canonical
    e, D, rho = mps.energy_grad(A, h)
    assert abs(e + 2.0 / 3.0) < 1e-13
    assert abs(mps.energy(A, h) + 2.0 / 3.0) < 1e-13
    assert np.abs(mps.gradient(A, D)).max() < 1e-12            # stationary


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_product_state_closed_form(dt):
    rng = np.random.default_rng(1)
    c = rng.standard_normal(3) + (1j * rng.standard_normal(3) if dt == np.complex128 else 0)
    c /= np.linalg.norm(c)
    A = c.reshape(1, 3, 1)
    a = rng.standard_normal((9, 9)) + (1j * rng.standard_normal((9, 9)) if dt == np.complex128 else 0)
    h = 0.5 * (a + a.conj().T)
    cc = np.kron(c, c)
    assert abs(mps.energy(A, h) - np.real(cc.conj() @ h @ cc)) < 1e-13
    assert abs(mps.energy_grad(A, h)[0] - np.real(cc.conj() @ h @ cc)) < 1e-13


def test_right_fixed_point_by_power_iteration():
    A = inp.random_mps(5, 2, seed=3)
    rho = mps.right_fixed_point(A)
    y = np.eye(5) / 5
    for _ in range(2000):
        y = mps.transfer_right(A, y)
        y /= np.trace(y)
    assert np.abs(rho - y).max() < 1e-12
    assert np.linalg.eigvalsh(rho).min() > 0


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_gradient_finite_differences(dt):
    """de along a Grassmann tangent X equals Re sum conj(D) X (D = 2 de/d conj(A));
    the energy off the manifold uses both fixed points (no canonical form)."""
    A = inp.random_mps(4, 2, seed=7, dtype=dt)
    h = inp.ising_bond(1.0, 0.2).astype(dt)
    e, D, _ = mps.energy_grad(A, h)
    M = mps.as_matrix(A)
    rng = np.random.default_rng(2)
    for _ in range(3):
        Z = rng.standard_normal(M.shape) + (1j * rng.standard_normal(M.shape) if dt == np.complex128 else 0)
        X = mps.as_tensor(geo.project(M, Z, geo.GRASSMANN), 2)
        eps = 1e-5
        fd = (mps.energy(A + eps * X, h) - mps.energy(A - eps * X, h)) / (2 * eps)
        an = float(np.real(np.sum(D.conj() * X)))
        assert abs(fd - an) < 1e-8 * max(1.0, abs(an)), (fd, an)


def test_metric_is_the_hilbert_space_overlap():
    """Eq. mps_inner: for tangent tensors in the left gauge (M^dag X = 0) the
    overlap of the tangent states per site is Re Tr(X^dag Y rho).  Checked on
    a periodic chain of 200 sites with mixed transfer matrices (bra X at site
    0, ket Y at every site j), independently of the oracle's formula."""
    D, d, N = 3, 2, 200
    A = inp.random_mps(D, d, seed=4, dtype=np.complex128)
    M = mps.as_matrix(A)
    rng = np.random.default_rng(5)
    X, Y = (mps.as_tensor(geo.project(M, rng.standard_normal(M.shape) + 1j * rng.standard_normal(M.shape),
                                      geo.GRASSMANN), d) for _ in range(2))

    def E(P, Q):  # sum_s conj(P^s) (x) Q^s, acting on (bra, ket) virtual pairs
        return sum(np.kron(P[:, s, :].conj(), Q[:, s, :]) for s in range(d))

    EAA, EXA, EAY, EXY = E(A, A), E(X, A), E(A, Y), E(X, Y)
    powers = [np.eye(D * D)]
    for _ in range(N):
        powers.append(powers[-1] @ EAA)
    norm = np.trace(powers[N]).real
    tot = np.trace(EXY @ powers[N - 1])
    for j in range(1, N):
        tot += np.trace(EXA @ powers[j - 1] @ EAY @ powers[N - j - 1])
    rho = mps.right_fixed_point(A)
    want = np.trace(mps.as_matrix(X).conj().T @ mps.as_matrix(Y) @ rho)
    assert abs(tot / norm - want) < 1e-10 * abs(want)


def test_preconditioner_inverts_the_regularised_metric():
    A = inp.random_mps(4, 3, seed=8)
    rho = mps.right_fixed_point(A)
    rng = np.random.default_rng(9)
    M = mps.as_matrix(A)
    X = mps.as_tensor(geo.project(M, rng.standard_normal(M.shape), geo.GRASSMANN), 3)
    Y = mps.as_tensor(geo.project(M, rng.standard_normal(M.shape), geo.GRASSMANN), 3)
    delta = 0.05
    Xt = mps.precondition(X, rho, delta)
    lhs = np.trace(mps.as_matrix(Y).T @ mps.as_matrix(Xt) @ (rho + delta * np.eye(4)))
    assert abs(lhs - np.trace(mps.as_matrix(Y).T @ mps.as_matrix(X))) < 1e-12


def test_lbfgs_reaches_the_gapped_ising_energy():
    """Riemannian L-BFGS with the rho preconditioner on the transverse-field
    Ising chain at h = 1.5 (gapped): D = 6 within 1e-7 of the exact energy."""
    h = inp.ising_bond(1.5)
    A0 = inp.random_mps(6, 2, seed=11)
    prob = mps.MpsProblem(h, 2)
    pt, e, hist = oo.lbfgs(prob, [mps.as_matrix(A0)], m=8, maxiter=150, gtol=1e-9)
    exact = inp.exact_ising_energy_per_spin(1.5)
    assert abs(e - exact) < 1e-7, (e, exact, len(hist))
