"""Binary MERA energy and partial derivatives, FP64, written from the definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Network (Sec. 4; the paper defers the binary network to Evenbly-Vidal and
its diagrams are not in the text, so the standard binary MERA is written out
here).  One layer maps a coarse lattice to a fine one as |fine> = U W |coarse>:

* ``w`` sends coarse site j to the fine pair (2j, 2j+1):  w[x_2j x_2j+1, c_j];
* ``u`` acts on the fine pair (2j+1, 2j+2):               u[f f', x x'].

A 3-site operator on fine sites (0,1,2) lies in the causal cone of coarse
sites (-1,0,1) ("left" map A_L); one on fine sites (1,2,3) lies in the cone of
coarse sites (0,1,2) ("right" map A_R).  The averaged ascending superoperator
is Abar = (A_L + A_R)/2 and the descending one Dbar is its Hilbert-Schmidt
adjoint, so that Tr(h rho) is the same at every level and equals the energy
per (bottom) site.

Leg names below: ``f``/``g`` are fine legs of the operator (ket/bra side),
``x`` legs sit between the conjugated u and w copies, ``y`` legs between the
plain copies; ``a b c`` (``A B C``) are the coarse legs of the conjugated
(plain) isometries.  Each network is evaluated with ``numpy.einsum`` as a
single library call; the pairwise order is numpy's own choice.

Parity pins (tests/test_oracle_mera.py): brute-force state vectors of finite
periodic MERAs, the closed-form product state, dense superoperator
eigen/linear solves on small bonds, central finite differences of the energy,
unitality and trace preservation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def _contract(pairs, out):
    """einsum over named legs: ``pairs`` is a list of (array, "leg leg ...")."""
    table = {}

    def sub(legs):
        s = ""
        for name in legs.split():
            if name not in table:
                table[name] = _LETTERS[len(table)]
            s += table[name]
        return s

    subs = [sub(legs) for _, legs in pairs]
    expr = ",".join(subs) + "->" + sub(out)
    return np.einsum(expr, *[a for a, _ in pairs], optimize=("greedy", 2**62))


def _dims(u, w):
    c = int(round(np.sqrt(u.shape[0])))
    return c, w.shape[1]


def _network(side, u, w):
    """Leaves of the ascending network A_side without the operator.

    Returns (leaves, op_legs, out_legs, rho_legs); each leaf is
    (array, legs, role) with role in {"u", "ub", "w", "wb"} ("b" = complex
    conjugated copy, i.e. on the bra side of <MERA| ... |MERA>).
    """
    c, cp = _dims(u, w)
    u4 = u.reshape(c, c, c, c)
    w3 = w.reshape(c, c, cp)
    ub, wb = u4.conj(), w3.conj()
    if side == "L":
        # operator on fine sites (0,1,2); u on (-1,0) and (1,2); w_-1, w_0, w_1
        leaves = [
            (ub, "fm f0 xm x0", "ub"), (ub, "f1 f2 x1 x2", "ub"),
            (wb, "xl xm a", "wb"), (wb, "x0 x1 b", "wb"), (wb, "x2 x3 c", "wb"),
            (u4, "fm g0 ym y0", "u"), (u4, "g1 g2 y1 y2", "u"),
            (w3, "xl ym A", "w"), (w3, "y0 y1 B", "w"), (w3, "y2 x3 C", "w"),
        ]
        return leaves, "f0 f1 f2 g0 g1 g2", "a b c A B C", "A B C a b c"
    if side == "R":
        # operator on fine sites (1,2,3); u on (1,2) and (3,4); w_0, w_1, w_2
        leaves = [
            (ub, "f1 f2 x1 x2", "ub"), (ub, "f3 f4 x3 x4", "ub"),
            (wb, "x0 x1 a", "wb"), (wb, "x2 x3 b", "wb"), (wb, "x4 x5 c", "wb"),
            (u4, "g1 g2 y1 y2", "u"), (u4, "g3 f4 y3 y4", "u"),
            (w3, "x0 y1 A", "w"), (w3, "y2 y3 B", "w"), (w3, "y4 x5 C", "w"),
        ]
        return leaves, "f1 f2 f3 g1 g2 g3", "a b c A B C", "A B C a b c"
    raise ValueError(side)


def ascend_side(o, u, w, side):
    """A_side(o): 3-site fine operator -> 3-site coarse operator (W^dag U^dag o U W)."""
    c, cp = _dims(u, w)
    leaves, op_legs, out_legs, _ = _network(side, u, w)
    pairs = [(o.reshape((c,) * 6), op_legs)] + [(a, l) for a, l, _ in leaves]
    return _contract(pairs, out_legs).reshape(cp**3, cp**3)


def descend_side(r, u, w, side):
    """D_side(r), the adjoint of A_side: Tr(A_side(o) r) = Tr(o D_side(r))."""
    c, cp = _dims(u, w)
    leaves, op_legs, _, rho_legs = _network(side, u, w)
    pairs = [(a, l) for a, l, _ in leaves] + [(r.reshape((cp,) * 6), rho_legs)]
    f = op_legs.split()
    return _contract(pairs, " ".join(f[3:] + f[:3])).reshape(c**3, c**3)


def ascend(o, u, w):
    """Averaged ascending superoperator Abar(o) = (A_L(o) + A_R(o)) / 2."""
    return 0.5 * (ascend_side(o, u, w, "L") + ascend_side(o, u, w, "R"))


def descend(r, u, w):
    """Averaged descending superoperator Dbar(r) = (D_L(r) + D_R(r)) / 2."""
    return 0.5 * (descend_side(r, u, w, "L") + descend_side(r, u, w, "R"))


def layer_derivatives(h, r, u, w):
    """Partial derivatives D_u, D_w of C = Tr(Abar(h) r) for one layer.

    D_v = 2 dC/d(conj v) (Sec. 2.3, Sec. 4): the sum, over every conjugated
    occurrence of v in the two networks, of the network with that copy
    removed.  The 1/2 of Abar cancels the 2 of the convention.
    """
    c, cp = _dims(u, w)
    du = np.zeros((c, c, c, c), dtype=np.result_type(h, r, u, w))
    dw = np.zeros((c, c, cp), dtype=du.dtype)
    for side in ("L", "R"):
        leaves, op_legs, _, rho_legs = _network(side, u, w)
        base = [(h.reshape((c,) * 6), op_legs), (r.reshape((cp,) * 6), rho_legs)]
        for k, (_, legs, role) in enumerate(leaves):
            if role not in ("ub", "wb"):
                continue
            rest = base + [(a, l) for j, (a, l, _) in enumerate(leaves) if j != k]
            env = _contract(rest, legs)
            if role == "ub":
                du += env
            else:
                dw += env
    return du.reshape(c * c, c * c), dw.reshape(c * c, cp)


def si_fixed_point(u, w, tol=1e-14, v0=None):
    """Scale-invariant density matrix: the eigenvector of Dbar_S with the
    eigenvalue of largest modulus (= 1), by a Krylov (Arnoldi) eigensolver
    (App. B), normalised to unit trace and hermitised.  Returns (rho, lambda)."""
    c, cp = _dims(u, w)
    assert c == cp
    n = c**6
    dt = np.result_type(u, w)

    def mv(v):
        return descend(v.reshape(c**3, c**3).astype(dt, copy=False), u, w).ravel()

    op = spla.LinearOperator((n, n), matvec=mv, dtype=dt)
    if v0 is None:
        v0 = (np.eye(c**3) / c**3).ravel().astype(dt)
    vals, vecs = spla.eigs(op, k=1, which="LM", v0=v0, tol=tol, ncv=min(n - 1, 24))
    rho = vecs[:, 0].reshape(c**3, c**3)
    rho = rho / np.trace(rho)
    rho = 0.5 * (rho + rho.conj().T)
    if np.dtype(dt).kind != "c":
        rho = rho.real.copy()
    return rho, complex(vals[0])


def si_env_series(h, rho, u, w, tol=1e-14, x0=None):
    """x = sum_i <h| A'^i with A' = A - |rho><1| (App. B, Eq. scale_invariant_partial),
    obtained from the linear problem x (1 - A') = <h|, i.e.
    x - Abar_S(x) + Tr(x rho) 1 = h, by restarted GMRES."""
    c, _ = _dims(u, w)
    n = c**6
    dt = np.result_type(h, rho, u, w)
    one = np.eye(c**3, dtype=dt)

    def mv(v):
        X = v.reshape(c**3, c**3)
        return (X - ascend(X, u, w) + np.trace(X @ rho) * one).ravel()

    op = spla.LinearOperator((n, n), matvec=mv, dtype=dt)
    b = h.astype(dt).ravel()
    x, info = spla.gmres(op, b, x0=None if x0 is None else x0.ravel(), rtol=tol,
                         atol=0.0, restart=min(n, 60), maxiter=400)
    x = x.reshape(c**3, c**3)
    x = 0.5 * (x + x.conj().T)
    return x


def energy_grad(h0, us, ws, tol=1e-14):
    """Energy per bottom site and partial derivatives of the infinite MERA.

    ``us``/``ws``: transition layers 0..L-1 followed by the scale-invariant
    layer L.  Steps: ascend h through the transition layers; fixed point rho_S
    of the scale-invariant descending map; environment series x of App. B;
    descend rho through the transition layers; e = Tr(h_0 rho_0); D_v of each
    transition layer from (h_l, rho_{l+1}) and of the scale-invariant layer
    from (x, rho_S).

    Returns (e, [D_u0, D_w0, ..., D_uL, D_wL], info) with info holding the
    ascended operators ``h``, density matrices ``rho`` and the series ``x``.
    """
    L = len(us) - 1
    hs = [np.asarray(h0)]
    for l in range(L):
        hs.append(ascend(hs[l], us[l], ws[l]))
    rho_s, lam = si_fixed_point(us[L], ws[L], tol=tol)
    x = si_env_series(hs[L], rho_s, us[L], ws[L], tol=tol)
    rhos = [None] * (L + 1)
    rhos[L] = rho_s
    for l in reversed(range(L)):
        rhos[l] = descend(rhos[l + 1], us[l], ws[l])
    e = float(np.real(np.trace(hs[0] @ rhos[0])))
    ds = []
    for l in range(L + 1):
        hl = hs[l] if l < L else x
        du, dw = layer_derivatives(hl, rhos[l + 1] if l < L else rho_s, us[l], ws[l])
        ds += [du, dw]
    return e, ds, {"h": hs, "rho": rhos, "x": x, "lambda": lam}


def energy(h0, us, ws, tol=1e-14):
    """Energy per bottom site only (ascend, fixed point, one trace)."""
    L = len(us) - 1
    h = np.asarray(h0)
    for l in range(L):
        h = ascend(h, us[l], ws[l])
    rho_s, _ = si_fixed_point(us[L], ws[L], tol=tol)
    return float(np.real(np.trace(h @ rho_s)))


def tensor_density_matrices(rhos, ws):
    """Reduced density matrices on the top legs of every tensor (Sec. 4):
    rho_w of layer l is the one-site (middle site) marginal of rho_{l+1};
    rho_u of layer l is the two-site state W rho2 W^dag on the pair of fine
    legs that u's columns connect to, with rho2 the marginal of rho_{l+1}
    on its first two sites.  ``rhos[l]`` is the 3-site density matrix at
    level l (rhos[L] = rho_S)."""
    L = len(ws) - 1
    out = []
    for l in range(L + 1):
        r = rhos[l + 1] if l < L else rhos[L]
        w = ws[l]
        c = int(round(np.sqrt(w.shape[0])))
        cp = w.shape[1]
        r6 = r.reshape((cp,) * 6)
        r1 = _contract([(r6, "a b c a B c")], "b B")
        r2 = _contract([(r6, "a b c A B c")], "a b A B")
        w3 = w.reshape(c, c, cp)
        ru = _contract([(w3, "x0 x1 a"), (w3, "x2 x3 b"), (r2, "a b A B"),
                        (w3.conj(), "x0 X1 A"), (w3.conj(), "X2 x3 B")],
                       "x1 x2 X1 X2").reshape(c * c, c * c)
        out += [ru, r1]
    return out
