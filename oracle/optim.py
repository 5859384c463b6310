"""Riemannian L-BFGS / conjugate gradient with the Hager-Zhang line search, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3 of the paper: the search direction is built from the gradient, the
preconditioner and (transported) history; the step along the retraction is
chosen by the Hager-Zhang line search (Wolfe / approximate Wolfe conditions,
Eqs. wolfe_1, wolfe_2); vector transport brings the history to the new point.

Readings where the paper leaves details to the literature:
* line-search constants are the published Hager-Zhang defaults
  (delta=0.1, sigma=0.9, eps=1e-6, theta=0.5, gamma=0.66, expansion 5),
  with at most ``maxeval`` evaluations;
* L-BFGS is the Nocedal-Wright two-loop recursion with initial inverse
  Hessian gamma * P (P the preconditioner), gamma = <s,y>/<y,P y> of the
  newest pair; a pair is kept only if <s,y> > 1e-16 |s| |y|; if the
  direction is not a descent direction the memory is cleared and d = -P G;
* CG uses the preconditioned Hager-Zhang beta with the eta lower bound.

Pins (tests/test_oracle_optim.py): on a Euclidean quadratic the two-loop
equals the dense BFGS inverse-Hessian product; every accepted step satisfies
Wolfe or approximate Wolfe; L-BFGS on a strictly convex quadratic converges.
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry as geo
from . import mera as om


def lin(a, X, b=None, Y=None):
    """a X + b Y on tangent lists."""
    if Y is None:
        return [a * x for x in X]
    return [a * x + b * y for x, y in zip(X, Y)]


class _Found(Exception):
    def __init__(self, alpha):
        self.alpha = alpha


def hager_zhang(phi, f0, df0, alpha0, delta=0.1, sigma=0.9, eps=1e-6, theta=0.5,
                gamma=0.66, expand=5.0, maxeval=20):
    """Hager-Zhang line search.  ``phi(alpha) -> (f, df, payload)``.

    Returns (alpha, f, df, payload, n_evals, ok) for the first trial that meets
    the Wolfe conditions  f - f0 <= delta*alpha*df0  and  df >= sigma*df0,  or
    the approximate Wolfe conditions  (2 delta - 1) df0 >= df >= sigma df0  and
    f <= f0 + eps |f0|.  If ``maxeval`` is reached the trial with the lowest
    f is returned with ok=False.
    """
    assert df0 < 0
    epsk = eps * abs(f0)
    hist = {}

    def ev(a):
        if a in hist:
            return hist[a][0], hist[a][1]
        if len(hist) >= maxeval:
            raise StopIteration
        f, df, pay = phi(a)
        if not (np.isfinite(f) and np.isfinite(df)):
            f, df = math.inf, math.inf
        hist[a] = (f, df, pay)
        wolfe = (f - f0 <= delta * a * df0) and (df >= sigma * df0)
        approx = ((2 * delta - 1) * df0 >= df >= sigma * df0) and (f <= f0 + epsk)
        if wolfe or approx:
            raise _Found(a)
        return f, df

    def dfof(a):
        return df0 if a == 0 else hist[a][1]

    def fof(a):
        return f0 if a == 0 else hist[a][0]

    def u3(a, b):
        while True:
            d = (1 - theta) * a + theta * b
            fd, dfd = ev(d)
            if dfd >= 0:
                return a, d
            if fd <= f0 + epsk:
                a = d
            else:
                b = d

    def update(a, b, c):
        if not (a < c < b):
            return a, b
        fc, dfc = ev(c)
        if dfc >= 0:
            return a, c
        if fc <= f0 + epsk:
            return c, b
        return u3(a, c)

    def secant(a, b):
        da, db = dfof(a), dfof(b)
        if db == da:
            return 0.5 * (a + b)
        return (a * db - b * da) / (db - da)

    try:
        c = alpha0
        fc, dfc = ev(c)
        good = [0.0]
        while True:
            if dfc >= 0:
                a, b = good[-1], c
                break
            if fc > f0 + epsk:
                a, b = u3(0.0, c)
                break
            good.append(c)
            c = expand * c
            fc, dfc = ev(c)
        while True:
            c = secant(a, b)
            A, B = update(a, b, c)
            if c == B:
                A, B = update(A, B, secant(b, B))
            elif c == A:
                A, B = update(A, B, secant(a, A))
            if B - A > gamma * (b - a):
                A, B = update(A, B, 0.5 * (A + B))
            a, b = A, B
    except _Found as hit:
        f, df, pay = hist[hit.alpha]
        return hit.alpha, f, df, pay, len(hist), True
    except StopIteration:
        pass
    finite = [(v[0], a) for a, v in hist.items() if np.isfinite(v[0])]
    if not finite:
        return None, None, None, None, len(hist), False
    _, a = min(finite)
    f, df, pay = hist[a]
    return a, f, df, pay, len(hist), False


def two_loop(G, mem, precond, inner):
    """L-BFGS two-loop recursion: returns H(G) for the memory ``mem`` =
    [(s_i, y_i, rho_i)] (oldest first) with H0 = gamma * precond."""
    q = [g.copy() for g in G]
    alphas = []
    for s, y, r in reversed(mem):
        a = r * inner(s, q)
        alphas.append(a)
        q = lin(1.0, q, -a, y)
    if mem:
        s, y, _ = mem[-1]
        gam = inner(s, y) / inner(y, precond(y))
    else:
        gam = 1.0
    z = lin(gam, precond(q))
    for (s, y, r), a in zip(mem, reversed(alphas)):
        b = r * inner(y, z)
        z = lin(1.0, z, a - b, s)
    return z


class MeraProblem:
    """The MERA energy on the product manifold of its tensors (Sec. 4).

    The point is [u_0, w_0, ..., u_L, w_L]; u's are Stiefel (unitary), w's
    Grassmann unless ``w_stiefel``.  Retractions are followed by polar
    re-isometrisation.
    """

    def __init__(self, h0, w_stiefel=False, precond=True, tol=1e-14):
        self.h0 = h0
        self.w_kind = geo.STIEFEL if w_stiefel else geo.GRASSMANN
        self.use_precond = precond
        self.tol = tol

    def kinds(self, point):
        return [geo.STIEFEL if i % 2 == 0 else self.w_kind for i in range(len(point))]

    def fg(self, point):
        us, ws = point[0::2], point[1::2]
        e, ds, info = om.energy_grad(self.h0, us, ws, tol=self.tol)
        G = [geo.project(W, D, k) for W, D, k in zip(point, ds, self.kinds(point))]
        rv = om.tensor_density_matrices(info["rho"], ws)
        return e, G, {"rho_v": rv, "delta": [float(np.linalg.norm(g)) for g in G]}

    def precondition(self, point, aux, X):
        if not self.use_precond:
            return [x.copy() for x in X]
        return [geo.precondition(W, x, r, d, k) for W, x, r, d, k in
                zip(point, X, aux["rho_v"], aux["delta"], self.kinds(point))]

    def retract(self, point, d, alpha):
        return [geo.polar(geo.retract(W, x, alpha)) for W, x in zip(point, d)]

    def transport(self, point, d, alpha, Y):
        return [geo.transport(W, x, alpha, y) for W, x, y in zip(point, d, Y)]


def lbfgs(problem, point, m=8, maxiter=100, gtol=1e-6, callback=None, maxeval=20):
    """Riemannian L-BFGS (Sec. 3).  Returns (point, energy, history)."""
    inner = geo.inner
    e, G, aux = problem.fg(point)
    mem = []
    hist = []
    for it in range(maxiter):
        gnorm = math.sqrt(inner(G, G))
        hist.append({"iter": it, "energy": e, "gnorm": gnorm})
        if callback:
            callback(it, e, gnorm, point)
        if gnorm < gtol:
            break
        P = lambda X, _p=point, _a=aux: problem.precondition(_p, _a, X)
        d = lin(-1.0, two_loop(G, mem, P, inner))
        df0 = inner(G, d)
        if not df0 < 0:
            mem = []
            d = lin(-1.0, P(G))
            df0 = inner(G, d)

        def phi(a, _p=point, _d=d):
            p2 = problem.retract(_p, _d, a)
            e2, G2, aux2 = problem.fg(p2)
            d2 = problem.transport(_p, _d, a, _d)
            return e2, inner(G2, d2), (p2, G2, aux2, d2)

        alpha, e2, _, pay, nev, ok = hager_zhang(phi, e, df0, 1.0, maxeval=maxeval)
        hist[-1].update(alpha=alpha, nev=nev, ls_ok=ok)
        if alpha is None or (not ok and e2 >= e):
            mem = []
            continue
        p2, G2, aux2, d2 = pay
        mem = [(problem.transport(point, d, alpha, s), problem.transport(point, d, alpha, y), r)
               for s, y, r in mem]
        s = lin(alpha, d2)
        y = lin(1.0, G2, -1.0, problem.transport(point, d, alpha, G))
        sy = inner(s, y)
        if sy > 1e-16 * math.sqrt(inner(s, s) * inner(y, y)):
            mem.append((s, y, 1.0 / sy))
            if len(mem) > m:
                mem.pop(0)
        point, e, G, aux = p2, e2, G2, aux2
    return point, e, hist


def hz_beta(inner, y, Pg2, Py, d2, G2, gnorm_old, eta=0.01):
    """The preconditioned Hager-Zhang coefficient of the new direction
    d' = -P(g') + beta d (Sec. 3 uses the Hager-Zhang scheme):
    beta = (<y, P g'> - 2 <y, P y> <d, g'> / <d, y>) / <d, y>, y = g' - T(g),
    bounded below by -1 / (|d| min(eta, |g|)) with g the gradient where the
    searched direction d started.  All vectors at the new point (d and g
    transported)."""
    dy = inner(d2, y)
    beta = (inner(y, Pg2) - 2.0 * inner(y, Py) * inner(d2, G2) / dy) / dy
    dn = math.sqrt(inner(d2, d2))
    return max(beta, -1.0 / (dn * min(eta, gnorm_old)))


def cg(problem, point, maxiter=100, gtol=1e-6, eta=0.01, callback=None, maxeval=20):
    """Riemannian nonlinear CG with the preconditioned Hager-Zhang beta (Sec. 3)."""
    inner = geo.inner
    e, G, aux = problem.fg(point)
    Pg = problem.precondition(point, aux, G)
    d = lin(-1.0, Pg)
    alpha_prev = 1.0
    hist = []
    for it in range(maxiter):
        gnorm = math.sqrt(inner(G, G))
        hist.append({"iter": it, "energy": e, "gnorm": gnorm})
        if callback:
            callback(it, e, gnorm, point)
        if gnorm < gtol:
            break
        df0 = inner(G, d)
        if not df0 < 0:
            d = lin(-1.0, Pg)
            df0 = inner(G, d)

        def phi(a, _p=point, _d=d):
            p2 = problem.retract(_p, _d, a)
            e2, G2, aux2 = problem.fg(p2)
            d2 = problem.transport(_p, _d, a, _d)
            return e2, inner(G2, d2), (p2, G2, aux2, d2)

        alpha, e2, _, pay, nev, ok = hager_zhang(phi, e, df0, alpha_prev, maxeval=maxeval)
        hist[-1].update(alpha=alpha, nev=nev, ls_ok=ok)
        if alpha is None or (not ok and e2 >= e):
            d = lin(-1.0, Pg)
            continue
        p2, G2, aux2, d2 = pay
        y = lin(1.0, G2, -1.0, problem.transport(point, d, alpha, G))
        Pg2 = problem.precondition(p2, aux2, G2)
        # the lower bound takes the gradient where the searched direction
        # started (|T(d)| = |d|: the transport is isometric)
        beta = hz_beta(inner, y, Pg2, problem.precondition(p2, aux2, y), d2, G2, math.sqrt(inner(G, G)), eta)
        d = lin(-1.0, Pg2, beta, d2)
        point, e, G, aux, Pg, alpha_prev = p2, e2, G2, aux2, Pg2, alpha
    return point, e, hist


def gd(problem, point, maxiter=100, gtol=1e-6, callback=None, maxeval=20):
    """Riemannian gradient descent (Sec. 3): retract along the negative
    preconditioned gradient -P(G), the step from the Hager-Zhang line search
    started at the previous accepted step."""
    inner = geo.inner
    e, G, aux = problem.fg(point)
    alpha_prev = 1.0
    hist = []
    for it in range(maxiter):
        gnorm = math.sqrt(inner(G, G))
        hist.append({"iter": it, "energy": e, "gnorm": gnorm})
        if callback:
            callback(it, e, gnorm, point)
        if gnorm < gtol:
            break
        d = lin(-1.0, problem.precondition(point, aux, G))
        df0 = inner(G, d)

        def phi(a, _p=point, _d=d):
            p2 = problem.retract(_p, _d, a)
            e2, G2, aux2 = problem.fg(p2)
            d2 = problem.transport(_p, _d, a, _d)
            return e2, inner(G2, d2), (p2, G2, aux2)

        alpha, e2, _, pay, nev, ok = hager_zhang(phi, e, df0, alpha_prev, maxeval=maxeval)
        hist[-1].update(alpha=alpha, nev=nev, ls_ok=ok)
        if alpha is None or (not ok and e2 >= e):
            break
        point, G, aux = pay
        e, alpha_prev = e2, alpha
    return point, e, hist


class TernaryProblem(MeraProblem):
    """The ternary-MERA energy (oracle/ternary.py) on the same product manifold:
    u's Stiefel (unitary), w's Grassmann, the ternary density matrices in the
    preconditioner."""

    def fg(self, point):
        from . import ternary as ot
        us, ws = point[0::2], point[1::2]
        e, ds, info = ot.energy_grad(self.h0, us, ws, tol=self.tol)
        G = [geo.project(W, D, k) for W, D, k in zip(point, ds, self.kinds(point))]
        rv = ot.tensor_density_matrices(info["rho"], ws)
        return e, G, {"rho_v": rv, "delta": [float(np.linalg.norm(g)) for g in G]}
