"""Pins of the oracle's optimizer (Sec. 3): L-BFGS two-loop against the dense
BFGS update on a Euclidean quadratic, Wolfe conditions of the Hager-Zhang line
search, convergence on a quadratic and a short MERA run (CPU only)."""
import math

import numpy as np
import pytest

from oracle import geometry as geo
from oracle import optim as oo
from paper_2007_03638_gb300 import inputs as inp


def test_two_loop_equals_dense_bfgs():
    """With P = identity and gamma from the newest pair, the two-loop recursion
    equals H_k g for the dense BFGS inverse-Hessian recursion
    H <- (1 - r s y^T) H (1 - r y s^T) + r s s^T started from gamma * 1."""
    rng = np.random.default_rng(0)
    n, m = 12, 5
    mem = []
    for _ in range(m):
        s = rng.standard_normal(n)
        y = s + 0.3 * rng.standard_normal(n)
        mem.append(([s], [y], 1.0 / float(s @ y)))
    g = rng.standard_normal(n)
    got = oo.two_loop([g], mem, lambda X: [x.copy() for x in X], geo.inner)[0]
    s, y, _ = mem[-1]
    gam = float(s[0] @ y[0]) / float(y[0] @ y[0])
    H = gam * np.eye(n)
    for s, y, r in mem:
        s, y = s[0], y[0]
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    assert np.abs(got - H @ g).max() < 1e-12


def test_hager_zhang_wolfe():
    """Accepted steps satisfy Wolfe or approximate Wolfe (Eqs. wolfe_1, wolfe_2)."""
    for k, (a0, scale) in enumerate([(1.0, 1.0), (1e-4, 1.0), (50.0, 1.0), (1.0, 30.0)]):
        def phi(a):
            f = scale * (a - 2.0) ** 2 + 0.3 * math.sin(3 * a)
            return f, 2 * scale * (a - 2.0) + 0.9 * math.cos(3 * a), None
        f0, df0, _ = phi(0.0)
        a, f, df, _, nev, ok = oo.hager_zhang(phi, f0, df0, a0)
        assert ok and nev <= 20
        wolfe = (f - f0 <= 0.1 * a * df0) and (df >= 0.9 * df0)
        approx = (-0.8 * df0 >= df >= 0.9 * df0) and (f <= f0 + 1e-6 * abs(f0))
        assert wolfe or approx


class _Quadratic:
    def __init__(self, n, seed):
        rng = np.random.default_rng(seed)
        q = np.linalg.qr(rng.standard_normal((n, n)))[0]
        self.A = q @ np.diag(np.logspace(0, 2, n)) @ q.T
        self.b = rng.standard_normal(n)

    def fg(self, p):
        x = p[0]
        return 0.5 * x @ self.A @ x - self.b @ x, [self.A @ x - self.b], None

    def precondition(self, p, aux, X):
        return [x.copy() for x in X]

    def retract(self, p, d, a):
        return [p[0] + a * d[0]]

    def transport(self, p, d, a, Y):
        return [y.copy() for y in Y]


def test_lbfgs_quadratic_converges():
    prob = _Quadratic(30, 1)
    p, e, hist = oo.lbfgs(prob, [np.zeros(30)], m=8, maxiter=200, gtol=1e-10)
    x = np.linalg.solve(prob.A, prob.b)
    assert np.abs(p[0] - x).max() < 1e-8
    assert hist[-1]["gnorm"] < 1e-10


def test_cg_quadratic_converges():
    prob = _Quadratic(30, 2)
    p, e, hist = oo.cg(prob, [np.zeros(30)], maxiter=400, gtol=1e-9)
    assert np.abs(p[0] - np.linalg.solve(prob.A, prob.b)).max() < 1e-7


def test_mera_lbfgs_short_run():
    """Config-1 shapes (chi=4, d_b=4, 2 transition layers): energy decreases every
    iteration, stays above the exact -4/pi per spin (variational bound), and the
    tensors stay isometric to 1e-13."""
    us, ws = inp.random_mera(4, 4, 2, seed=0)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    prob = oo.MeraProblem(h3)
    pt = [t for pair in zip(us, ws) for t in pair]
    p, e, hist = oo.lbfgs(prob, pt, m=8, maxiter=15)
    es = [h["energy"] for h in hist]
    assert all(b <= a + 1e-14 for a, b in zip(es, es[1:]))
    assert e / 2 > inp.EXACT_ISING_CRITICAL
    assert e / 2 < -1.1
    for t in p:
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-13


class _NewtonPreconditioned(_Quadratic):
    """The quadratic with the exact inverse Hessian as preconditioner."""

    def precondition(self, p, aux, X):
        return [np.linalg.solve(self.A, x) for x in X]


def test_gd_with_the_inverse_hessian_is_one_newton_step():
    """Preconditioned by A^-1, the descent direction is the Newton step and the
    line search's first trial (alpha = 1) is the exact minimiser."""
    prob = _NewtonPreconditioned(20, 3)
    p, e, hist = oo.gd(prob, [np.zeros(20)], maxiter=3, gtol=1e-10)
    x = np.linalg.solve(prob.A, prob.b)
    assert hist[0]["alpha"] == 1.0
    assert np.abs(p[0] - x).max() < 1e-10
    assert len(hist) <= 2


def test_gd_descends_and_converges_on_a_quadratic():
    """Identity preconditioner, condition number 10: the energy never rises by
    more than the approximate-Wolfe allowance (1e-6 |f|) and the iterates reach
    the minimiser."""
    prob = _Quadratic(20, 4)
    prob.A = np.diag(np.linspace(1.0, 10.0, 20))
    p, e, hist = oo.gd(prob, [np.zeros(20)], maxiter=500, gtol=1e-9)
    es = [h["energy"] for h in hist]
    assert all(b <= a + 1e-6 * abs(a) for a, b in zip(es, es[1:]))
    assert np.abs(p[0] - np.linalg.solve(prob.A, prob.b)).max() < 1e-8


def test_mera_gd_short_run():
    us, ws = inp.random_mera(4, 4, 2, seed=0)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    p, e, hist = oo.gd(oo.MeraProblem(h3), [t for pair in zip(us, ws) for t in pair], maxiter=10)
    es = [h["energy"] for h in hist]
    assert all(b <= a + 1e-14 for a, b in zip(es, es[1:]))
    assert e / 2 > inp.EXACT_ISING_CRITICAL


def test_hz_beta_with_exact_steps_gives_conjugate_directions():
    """On a strictly convex quadratic with exact line searches <d, g'> = 0, so
    the Hager-Zhang coefficient reduces to Hestenes-Stiefel's and nonlinear CG
    is linear CG: successive directions are A-conjugate and the minimiser is
    reached in n steps (textbook; Nocedal-Wright Thm. 5.2/5.3).  The bound
    does not act here (beta > 0)."""
    rng = np.random.default_rng(4)
    n = 7
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1.0, 9.0, n)) @ Q.T
    b = rng.standard_normal(n)
    inner = lambda u, v: float(np.dot(u, v))  # noqa: E731
    x = np.zeros(n)
    g = A @ x - b
    d = -g
    dirs = []
    for _ in range(n):
        alpha = -inner(g, d) / inner(d, A @ d)
        x = x + alpha * d
        g2 = A @ x - b
        dirs.append(d)
        if np.linalg.norm(g2) < 1e-13:
            break
        y = g2 - g
        beta = oo.hz_beta(inner, y, g2, y, d, g2, np.linalg.norm(g))
        assert beta > 0
        d = -g2 + beta * d
        g = g2
    assert np.linalg.norm(A @ x - b) < 1e-10
    for i in range(len(dirs)):
        for j in range(i):
            assert abs(dirs[i] @ A @ dirs[j]) < 1e-10 * np.linalg.norm(dirs[i]) * np.linalg.norm(dirs[j])


def test_hz_beta_bound_uses_the_previous_gradient():
    """The lower bound -1/(|d| min(eta, |g|)) acts when beta is very negative;
    it takes |g| of the point the direction started from."""
    inner = lambda u, v: float(np.dot(u, v))  # noqa: E731
    d = np.array([1.0, 0.0])
    y = np.array([1e-3, -1.0])   # <d, y> = 1e-3, <y, g'> = -5: beta = -5000
    g2 = np.array([0.0, 5.0])
    b = oo.hz_beta(inner, y, g2, y, d, g2, gnorm_old=0.004, eta=0.01)
    assert b == pytest.approx(-1.0 / (1.0 * 0.004))
    b = oo.hz_beta(inner, y, g2, y, d, g2, gnorm_old=2.0, eta=0.01)
    assert b == pytest.approx(-1.0 / (1.0 * 0.01))
