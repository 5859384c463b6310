"""Pins of the ternary-MERA oracle (oracle/ternary.py) against dense periodic
state vectors built from the definition (tests/bruteforce.py), closed forms,
dense superoperators and finite differences (CPU only)."""
import numpy as np
import pytest

from oracle import ternary as ot
from paper_2007_03638_gb300 import inputs as inp
from tests import bruteforce as bf


def _swap2(r, c):
    """The same two-site operator with its two sites exchanged."""
    return r.reshape(c, c, c, c).transpose(1, 0, 3, 2).reshape(c * c, c * c)


def _top_rdm(top):
    """Position-averaged two-site density matrix of a 2-site periodic top state."""
    c = top.shape[0]
    p = top.reshape(c * c, 1)
    r = p @ p.conj().T
    return 0.5 * (r + _swap2(r, c))


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_bruteforce_6_sites(dt):
    """One layer: 2 top sites (dim 3) -> 6 spins.  The averaged 2-site density
    matrix of the dense state equals Dbar(rho_top); the energy density equals
    Tr(Abar(h) rho_top) (all three cone positions A_L, A_C, A_R)."""
    rng = np.random.default_rng(4)
    u = inp._haar_like(rng, 4, 4, dt)
    w = inp._haar_like(rng, 8, 3, dt)
    top = rng.standard_normal((3, 3)) + (1j * rng.standard_normal((3, 3)) if dt == np.complex128 else 0)
    top /= np.linalg.norm(top)
    psi = bf.finite_ternary_state(top, [(u, w)])
    assert psi.shape == (2,) * 6
    rho_top = _top_rdm(top)
    assert np.abs(bf.averaged_rdm2(psi) - ot.descend(rho_top, u, w)).max() < 1e-13
    bond = inp.xxz_bond(0.7) if dt == np.complex128 else inp.ising_bond(0.9)
    e_bf = bf.energy_density(psi, bond)
    assert abs(e_bf - np.real(np.trace(ot.ascend(bond, u, w) @ rho_top))) < 1e-13


def test_bruteforce_18_sites():
    """Two layers: 2 top sites (dim 2) -> 6 sites (dim 3) -> 18 spins."""
    rng = np.random.default_rng(9)
    u0 = inp._haar_like(rng, 4, 4, np.float64)
    w0 = inp._haar_like(rng, 8, 3, np.float64)
    u1 = inp._haar_like(rng, 9, 9, np.float64)
    w1 = inp._haar_like(rng, 27, 2, np.float64)
    top = rng.standard_normal((2, 2))
    top /= np.linalg.norm(top)
    psi = bf.finite_ternary_state(top, [(u1, w1), (u0, w0)])
    assert psi.shape == (2,) * 18
    rho_top = _top_rdm(top)
    rho_or = ot.descend(ot.descend(rho_top, u1, w1), u0, w0)
    assert np.abs(bf.averaged_rdm2(psi) - rho_or).max() < 1e-13
    bond = inp.ising_bond(1.0)
    e_or = np.trace(ot.ascend(ot.ascend(bond, u0, w0), u1, w1) @ rho_top)
    assert abs(bf.energy_density(psi, bond) - e_or) < 1e-13


@pytest.mark.parametrize("bond,exact", [(inp.ising_bond(0.7), -0.7), (inp.xxz_bond(0.4), 0.4)])
def test_product_state_closed_form(bond, exact):
    """u = 1, w|0> = |000>: the state |00...0>, energy per site <00|h|00>."""
    us, ws = inp.product_state_ternary_mera(2, 4, 1)
    assert abs(ot.energy(bond, us, ws) - exact) < 1e-12


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_unitality_trace_and_adjointness(dt):
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=2, dtype=dt)
    u, w = us[0], ws[0]
    rng = np.random.default_rng(1)
    for side in ot.SIDES:
        assert np.abs(ot.ascend_side(np.eye(4), u, w, side) - np.eye(16)).max() < 1e-13
        r = rng.standard_normal((16, 16)) + (1j * rng.standard_normal((16, 16)) if dt == np.complex128 else 0)
        o = rng.standard_normal((4, 4)) + (1j * rng.standard_normal((4, 4)) if dt == np.complex128 else 0)
        assert abs(np.trace(ot.descend_side(r, u, w, side)) - np.trace(r)) < 1e-12
        lhs = np.trace(ot.ascend_side(o, u, w, side) @ r)
        rhs = np.trace(o @ ot.descend_side(r, u, w, side))
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_fixed_point_and_series_vs_dense():
    """chi = 2 scale-invariant layer: the dense 16 x 16 superoperator's unit
    eigenvector and the dense solve of the series equation."""
    us, ws = inp.random_ternary_mera(2, 2, 0, seed=5)
    u, w = us[0], ws[0]
    n = 4
    Dm = np.zeros((n * n, n * n))
    Am = np.zeros((n * n, n * n))
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        Dm[:, k] = ot.descend(e.reshape(n, n), u, w).ravel()
        Am[:, k] = ot.ascend(e.reshape(n, n), u, w).ravel()
    vals, vecs = np.linalg.eig(Dm)
    k = int(np.argmin(np.abs(vals - 1.0)))
    assert abs(vals[k] - 1.0) < 1e-12
    rho = np.real(vecs[:, k]).reshape(n, n)
    rho /= np.trace(rho)
    assert np.abs(ot.si_fixed_point(u, w) - rho).max() < 1e-10
    h = inp.ising_bond(1.0)
    M = np.eye(n * n) - Am + np.outer(np.eye(n).ravel(), rho.T.ravel())
    x = np.linalg.solve(M, h.ravel()).reshape(n, n)
    assert np.abs(ot.si_env_series(h, rho, u, w) - 0.5 * (x + x.T)).max() < 1e-10


def _tangent(rng, W):
    Z = rng.standard_normal(W.shape)
    S = W.T @ Z
    return Z - W @ (0.5 * (S + S.T))


@pytest.mark.parametrize("which", ["u0", "w0", "uS", "wS", "all"])
def test_gradient_finite_differences(which):
    """Central differences of C(W + eps X) against sum D . X for tangent X
    (D_v = 2 dC/d conj(v); real tensors)."""
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=8)
    h = inp.ising_bond(1.0)
    pt = [t for pair in zip(us, ws) for t in pair]
    _, ds, _ = ot.energy_grad(h, us, ws)
    names = ["u0", "w0", "uS", "wS"]
    rng = np.random.default_rng(200 + (names + ["all"]).index(which))
    X = [np.zeros_like(t) for t in pt]
    for i, nm in enumerate(names):
        if which in ("all", nm):
            X[i] = _tangent(rng, pt[i])
    eps = 1e-5

    def C(t):
        p = [a + t * x for a, x in zip(pt, X)]
        return ot.energy(h, p[0::2], p[1::2])

    fd = (C(eps) - C(-eps)) / (2 * eps)
    an = sum(float(np.sum(d * x)) for d, x in zip(ds, X))
    assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (which, fd, an)


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_tensor_density_matrices_vs_dense(dt):
    """rho_u is the two-site density matrix of the isometry outputs that a u
    acts on: on a dense 6-site state before the disentanglers, the average
    over the two pairs (2, 3) and (5, 0) of their reduced density matrix;
    rho_w is the one-site marginal.  Both have unit trace."""
    rng = np.random.default_rng(12)
    w = inp._haar_like(rng, 8, 3, dt)
    top = rng.standard_normal((3, 3)) + (1j * rng.standard_normal((3, 3)) if dt == np.complex128 else 0)
    top /= np.linalg.norm(top)
    rho_top = _top_rdm(top)
    ru, rw = ot.tensor_density_matrices([rho_top], [w])
    psi = bf.apply_ternary_isometry_layer(top, w)   # W level: 6 sites, no u yet
    def rdm(i, j):
        p = np.moveaxis(psi, [i, j], [0, 1]).reshape(4, -1)
        return p @ p.conj().T
    dense = 0.5 * (rdm(2, 3) + rdm(5, 0))
    assert np.abs(ru - dense).max() < 1e-13
    t = top.reshape(9, 1) @ top.reshape(9, 1).conj().T
    t4 = t.reshape(3, 3, 3, 3)
    one = 0.5 * (np.einsum("abAb->aA", t4) + np.einsum("babA->aA", t4))
    assert np.abs(rw - one).max() < 1e-14
    assert abs(np.trace(ru) - 1) < 1e-13 and abs(np.trace(rw) - 1) < 1e-13


def test_lbfgs_on_the_ternary_network():
    """The oracle's Riemannian L-BFGS (Sec. 3) with the ternary preconditioner
    lowers the critical-Ising energy monotonically from a random chi = 4 start."""
    from oracle import optim as oo
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=6)
    prob = oo.TernaryProblem(inp.ising_bond(1.0))
    pt = [t for pair in zip(us, ws) for t in pair]
    e0 = ot.energy(inp.ising_bond(1.0), us, ws)
    _, e, hist = oo.lbfgs(prob, pt, m=8, maxiter=25)
    es = [h["energy"] for h in hist]
    assert e < e0 - 0.5
    assert all(b <= a + 1e-10 for a, b in zip(es, es[1:]))
