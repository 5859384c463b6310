"""Ternary MERA: ascending/descending superoperators, scale-invariant layer,
energy and partial derivatives, FP64 (the network of the paper's benchmark).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading (the paper uses the ternary MERA of Evenbly and Vidal and draws no
diagram): |fine> = U W |coarse>; w (c^3 x c') maps coarse site j to the fine
triple (3j, 3j+1, 3j+2), row-major w[f_a f_b f_c, k]; u (c^2 x c^2) is
unitary on the fine pairs (3j+2, 3j+3), u[f_a f_b, x_a x_b].  Local operators
are two-site (c^2 x c^2, rows = bra legs).  A two-site operator on fine sites
(s, s+1) ascends to coarse sites
  A_L: s = 3j      -> (j-1, j)   (u on (3j-1, 3j); site 3j+1 under no u),
  A_R: s = 3j+1    -> (j, j+1)   (site 3j+1 free; u on (3j+2, 3j+3)),
  A_C: s = 3j+2    -> (j, j+1)   (both sites under one u),
and Abar = (A_L + A_C + A_R) / 3 (translation average).  Descending maps are
their adjoints, Tr(A(o) r) = Tr(o D(r)).  Energy per site e = Tr(h_0 rho_0);
D_v = 2 dC / d conj(v) for C = Tr(Abar(h) rho): (2/3) times the sum, over the
three networks and every conjugated copy of v, of the network with that copy
removed.  Scale-invariant layer, series and the level sweep as in
``oracle/mera.py`` (App. B).

Index names: ``f``/``g`` bra/ket fine legs of the operator, ``x`` legs between
the conjugated copies, ``y`` between the plain copies, ``p``/``q`` legs traced
between a conjugated and a plain isometry, ``a b`` (``A B``) coarse legs of
the conjugated (plain) isometries.

Pins (tests/test_oracle_ternary.py): dense periodic ternary MERA states of 6
and 18 sites; the product-state closed form; unitality, trace preservation
and adjointness; dense superoperator fixed point and series at chi = 2;
central finite differences of the energy in every tensor; the tensors'
density matrices against reduced density matrices of a dense state.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .mera import _contract

SIDES = ("L", "C", "R")


def _dims(u, w):
    c = int(round(np.sqrt(u.shape[0])))
    return c, w.shape[1]


def _network(side, u, w):
    """Leaves (array, legs, role) of the ascending network A_side without the
    operator; role in {"u", "ub", "w", "wb"} ("b": conjugated copy)."""
    c, cp = _dims(u, w)
    u4 = u.reshape(c, c, c, c)
    w4 = w.reshape(c, c, c, cp)
    ub, wb = u4.conj(), w4.conj()
    if side == "L":
        return [
            (ub, "fm f0 xm x0", "ub"), (wb, "p1 p2 xm a", "wb"), (wb, "x0 f1 q2 b", "wb"),
            (u4, "fm g0 ym y0", "u"), (w4, "p1 p2 ym A", "w"), (w4, "y0 g1 q2 B", "w"),
        ]
    if side == "R":
        return [
            (wb, "p0 f0 x2 a", "wb"), (ub, "f1 fp x2 x3", "ub"), (wb, "x3 p4 p5 b", "wb"),
            (w4, "p0 g0 y2 A", "w"), (u4, "g1 fp y2 y3", "u"), (w4, "y3 p4 p5 B", "w"),
        ]
    if side == "C":
        return [
            (ub, "f0 f1 x2 x3", "ub"), (wb, "p0 p1 x2 a", "wb"), (wb, "x3 p4 p5 b", "wb"),
            (u4, "g0 g1 y2 y3", "u"), (w4, "p0 p1 y2 A", "w"), (w4, "y3 p4 p5 B", "w"),
        ]
    raise ValueError(side)


OP_LEGS, OUT_LEGS, RHO_LEGS = "f0 f1 g0 g1", "a b A B", "A B a b"


def ascend_side(o, u, w, side):
    """A_side(o): two-site fine operator -> two-site coarse operator (Sec. 4)."""
    c, cp = _dims(u, w)
    pairs = [(o.reshape((c,) * 4), OP_LEGS)] + [(a, l) for a, l, _ in _network(side, u, w)]
    return _contract(pairs, OUT_LEGS).reshape(cp**2, cp**2)


def descend_side(r, u, w, side):
    """D_side(r), the adjoint of A_side (Sec. 4)."""
    c, cp = _dims(u, w)
    pairs = [(a, l) for a, l, _ in _network(side, u, w)] + [(r.reshape((cp,) * 4), RHO_LEGS)]
    return _contract(pairs, "g0 g1 f0 f1").reshape(c**2, c**2)


def ascend(o, u, w):
    """Abar(o) = (A_L + A_C + A_R)(o) / 3 (Sec. 4)."""
    return sum(ascend_side(o, u, w, s) for s in SIDES) / 3.0


def descend(r, u, w):
    """Dbar(r) = (D_L + D_C + D_R)(r) / 3 (Sec. 4)."""
    return sum(descend_side(r, u, w, s) for s in SIDES) / 3.0


def layer_derivatives(h, r, u, w):
    """D_u, D_w of C = Tr(Abar(h) r) for one layer (D_v = 2 dC/d conj(v),
    Sec. 2.3 and Sec. 4)."""
    c, cp = _dims(u, w)
    dt = np.result_type(h, r, u, w)
    du = np.zeros((c,) * 4, dtype=dt)
    dw = np.zeros((c, c, c, cp), dtype=dt)
    for side in SIDES:
        leaves = _network(side, u, w)
        base = [(h.reshape((c,) * 4), OP_LEGS), (r.reshape((cp,) * 4), RHO_LEGS)]
        for k, (_, legs, role) in enumerate(leaves):
            if role not in ("ub", "wb"):
                continue
            rest = base + [(a, l) for j, (a, l, _) in enumerate(leaves) if j != k]
            env = _contract(rest, legs)
            if role == "ub":
                du += env
            else:
                dw += env
    return (2.0 / 3.0) * du.reshape(c * c, c * c), (2.0 / 3.0) * dw.reshape(c**3, cp)


def si_fixed_point(u, w, tol=1e-14):
    """rho_S = Dbar_S(rho_S), unit trace, hermitised (Krylov eigensolver, App. B)."""
    c, cp = _dims(u, w)
    n = c**4
    dt = np.result_type(u, w)

    def mv(v):
        return descend(v.reshape(c**2, c**2).astype(dt, copy=False), u, w).ravel()

    op = spla.LinearOperator((n, n), matvec=mv, dtype=dt)
    v0 = (np.eye(c**2) / c**2).ravel().astype(dt)
    _, vecs = spla.eigs(op, k=1, which="LM", v0=v0, tol=tol, ncv=min(n - 1, 20))
    rho = vecs[:, 0].reshape(c**2, c**2)
    rho = rho / np.trace(rho)
    rho = 0.5 * (rho + rho.conj().T)
    if np.dtype(dt).kind != "c":
        rho = rho.real.copy()
    return rho


def si_env_series(h, rho, u, w, tol=1e-14):
    """x with x - Abar_S(x) + Tr(x rho) 1 = h (the series of App. B,
    Eq. scale_invariant_partial)."""
    c, _ = _dims(u, w)
    n = c**4
    dt = np.result_type(h, rho, u, w)
    one = np.eye(c**2, dtype=dt)

    def mv(v):
        X = v.reshape(c**2, c**2)
        return (X - ascend(X, u, w) + np.trace(X @ rho) * one).ravel()

    op = spla.LinearOperator((n, n), matvec=mv, dtype=dt)
    x, _ = spla.gmres(op, h.astype(dt).ravel(), rtol=tol, atol=0.0, restart=min(n, 60), maxiter=400)
    x = x.reshape(c**2, c**2)
    return 0.5 * (x + x.conj().T)


def energy_grad(h0, us, ws, tol=1e-14):
    """Energy per site and partial derivatives of the infinite ternary MERA
    (transition layers 0..L-1, scale-invariant layer L).  Returns
    (e, [D_u0, D_w0, ..., D_uL, D_wL], info)."""
    L = len(us) - 1
    hs = [np.asarray(h0)]
    for l in range(L):
        hs.append(ascend(hs[l], us[l], ws[l]))
    rho_s = si_fixed_point(us[L], ws[L], tol=tol)
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
    return e, ds, {"h": hs, "rho": rhos, "x": x}


def energy(h0, us, ws, tol=1e-14):
    """Energy per site only: ascending sweep and scale-invariant fixed point (Sec. 4, App. B)."""
    L = len(us) - 1
    h = np.asarray(h0)
    for l in range(L):
        h = ascend(h, us[l], ws[l])
    rho_s = si_fixed_point(us[L], ws[L], tol=tol)
    return float(np.real(np.trace(h @ rho_s)))


def tensor_density_matrices(rhos, ws):
    """Reduced density matrices on the top legs of every tensor (Sec. 4) for
    the ternary network: rho_w of layer l is the one-site marginal of the
    two-site rho_{l+1} (average of its left and right sites, equal for a
    translation-averaged state); rho_u is the two-site state on the isometry
    outputs that u acts on, the third leg of w_j and the first of w_{j+1}:
    W rho_{l+1} W^dag with the other four isometry legs traced.  ``rhos[l]``
    is the two-site density matrix at level l (rhos[L] = rho_S)."""
    L = len(ws) - 1
    out = []
    for l in range(L + 1):
        r = rhos[l + 1] if l < L else rhos[L]
        w = ws[l]
        cp = w.shape[1]
        c = int(round(w.shape[0] ** (1.0 / 3.0)))
        r4 = r.reshape(cp, cp, cp, cp)
        rw = 0.5 * (_contract([(r4, "a b A b")], "a A") + _contract([(r4, "b a b A")], "a A"))
        w4 = w.reshape(c, c, c, cp)
        ru = _contract([(w4, "p0 p1 x2 a"), (w4, "x3 p4 p5 b"), (r4, "a b A B"),
                        (w4.conj(), "p0 p1 X2 A"), (w4.conj(), "X3 p4 p5 B")],
                       "x2 x3 X2 X3").reshape(c * c, c * c)
        out += [ru, rw]
    return out
