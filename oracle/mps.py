"""Uniform (translation-invariant, one-site) MPS on the Grassmann manifold,
FP64: energy per site, partial derivative, preconditioner (Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The state is |psi> = sum_{...s_n...} (... A^{s_1} A^{s_2} ...) |... s_1 s_2 ...>
with A of shape (D, d, D), A^s = A[:, s, :], kept left-canonical: the matrix
M = A.reshape(D d, D) is an isometry (sum_s A^s^dag A^s = 1), a point of the
Grassmann manifold (right unitary rotations are gauge).  Transfer maps on
D x D matrices:
  E_L(x) = sum_s A^s^dag x A^s   (E_L(1) = 1 for left-canonical A),
  E_R(y) = sum_s A^s y A^s^dag,  rho = its unit-trace fixed point.
Readings (the section's diagrams are absent):
* the Hamiltonian is a nearest-neighbour two-site term h (d^2 x d^2, rows =
  bra legs), the simplest MPO; the cost is the energy per site
  e = Tr[(A^s A^t)^dag A^s' A^t' rho] h[(s t), (s' t')] (summed);
* the partial derivative D = 2 de / d conj(A) is the sum over the bra copies
  of A: the two local terms (the bra copy under h) and the left and right
  energy environments H_l, H_r, geometric sums of the transfer maps applied
  to the left- and right-contracted shifted term h - e 1 (the shift makes the
  sums converge and removes the normalisation terms), obtained from the
  nonsingular systems (1 - E_L + |1)(rho|) H_l = h_l and
  (1 - E_R + |rho)(1|) H_r = h_r;
* preconditioner: X -> X (rho + delta 1)^{-1} on the Grassmann tangent, with
  delta = |G|^2 (the regularisation the section states);
* the energy off the manifold (for the finite-difference pins) is
  Tr(l T_h(r)) / (lambda^2 Tr(l r)) with l, r the left and right dominant
  eigenvectors of the transfer maps and lambda their eigenvalue.

Pins (tests/test_oracle_mps.py): the AKLT state is an exact ground state
(energy -2/3 per bond, zero gradient); product-state closed form; the
transfer fixed point against a dense eigensolve; central finite differences
of the off-manifold energy along tangent directions; the preconditioner
inverts the metric Re Tr(X^dag Y (rho + delta 1)).
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo


def as_matrix(A):
    D, d, _ = A.shape
    return A.reshape(D * d, D)


def as_tensor(M, d):
    D = M.shape[1]
    return M.reshape(D, d, D)


def transfer_right(A, y):
    """E_R(y) = sum_s A^s y A^s^dag, the map of Eq. mps_right_transfermatrix."""
    return np.einsum("asb,bc,dsc->ad", A, y, A.conj())


def transfer_left(A, x):
    """E_L(x) = sum_s A^s^dag x A^s (E_L(1) = 1: Eq. mps_isometricity)."""
    return np.einsum("asb,ac,csd->bd", A.conj(), x, A)


def _dense(fn, A):
    D = A.shape[0]
    E = np.zeros((D * D, D * D), dtype=np.result_type(A, 1.0))
    for k in range(D * D):
        e = np.zeros(D * D, dtype=E.dtype)
        e[k] = 1.0
        E[:, k] = fn(A, e.reshape(D, D)).ravel()
    return E


def fixed_points(A):
    """Left and right dominant eigenvectors (l, r) of the transfer maps and
    their eigenvalue, normalised Tr(l r) = 1 and Tr r = 1, hermitised."""
    D = A.shape[0]
    vals, vecs = np.linalg.eig(_dense(transfer_right, A))
    k = int(np.argmax(np.abs(vals)))
    r = vecs[:, k].reshape(D, D)
    r = r / np.trace(r)
    r = 0.5 * (r + r.conj().T)
    vl, vecl = np.linalg.eig(_dense(transfer_left, A))
    kl = int(np.argmax(np.abs(vl)))
    l = vecl[:, kl].reshape(D, D)
    l = l / np.trace(l @ r)
    l = 0.5 * (l + l.conj().T)
    return l, r, vals[k].real


def _two_site(A):
    """B[a, s, t, c] = (A^s A^t)[a, c]."""
    return np.einsum("asb,btc->astc", A, A)


def _t_h(A, h, y):
    """T_h(y) = sum h[(s t), (s' t')] A^s' A^t' y (A^s A^t)^dag."""
    d = A.shape[1]
    B = _two_site(A)
    h4 = h.reshape(d, d, d, d)
    return np.einsum("stuv,auvb,bc,dstc->ad", h4, B, y, B.conj())


def energy(A, h):
    """Energy per site of the normalised infinite MPS of Eq. mps (valid off the
    manifold), Sec. 5."""
    l, r, lam = fixed_points(A)
    return float(np.real(np.trace(l @ _t_h(A, h, r)) / (lam**2 * np.trace(l @ r))))


def right_fixed_point(A):
    """rho = E_R(rho), Tr rho = 1 (left-canonical A): Eq. mps_right_transfermatrix."""
    return fixed_points(A)[1]


def energy_grad(A, h):
    """(e, D, rho) at a left-canonical A: D = 2 de/d conj(A), shape (D, d, D),
    with the energy environments of Eq. mps_derivative (Sec. 5)."""
    Dd, d, _ = A.shape
    rho = right_fixed_point(A)
    one = np.eye(Dd)
    e = float(np.real(np.trace(_t_h(A, h, rho))))
    ht = h - e * np.eye(d * d)
    h4 = ht.reshape(d, d, d, d)
    B = _two_site(A)
    # left- and right-contracted shifted term
    h_l = np.einsum("stuv,astc,auvd->cd", h4, B.conj(), B)
    h_r = _t_h(A, ht, rho)
    # geometric sums: (1 - E_L + |1)(rho|) H_l = h_l, (1 - E_R + |rho)(1|) H_r = h_r
    EL = _dense(transfer_left, A)
    ER = _dense(transfer_right, A)
    n = Dd * Dd
    ML = np.eye(n) - EL + np.outer(one.ravel(), rho.T.ravel())
    MR = np.eye(n) - ER + np.outer(rho.ravel(), one.ravel())
    H_l = np.linalg.solve(ML, h_l.ravel()).reshape(Dd, Dd)
    H_r = np.linalg.solve(MR, h_r.ravel()).reshape(Dd, Dd)
    # bra copy at site 0: local (h on (0,1) and (-1,0)) and environment terms
    loc1 = np.einsum("stuv,auvb,bc,dtc->asd", h4, B, rho, A.conj())
    loc2 = np.einsum("tsuv,etc,euvb,bd->csd", h4, A.conj(), B, rho)
    env = np.einsum("ab,bsc,cd->asd", H_l, A, rho) + np.einsum("asb,bc->asc", A, H_r)
    D = 2.0 * (loc1 + loc2 + env)
    return e, D, rho


def gradient(A, D):
    """Grassmann projection of D at A (matrix form), Eq. grassmann_gradient."""
    d = A.shape[1]
    return as_tensor(geo.project(as_matrix(A), as_matrix(D), geo.GRASSMANN), d)


def precondition(X, rho, delta):
    """X -> X (rho + delta 1)^{-1} (matrix form, right virtual index):
    Eq. mps_preconditioning with the regularisation of Sec. 5; it inverts the
    metric of Eq. mps_inner."""
    d = X.shape[1]
    M = as_matrix(X)
    return as_tensor(M @ np.linalg.inv(rho + delta * np.eye(rho.shape[0])), d)


class MpsProblem:
    """The uniform-MPS energy on the Grassmann manifold, for oracle/optim.py."""

    def __init__(self, h, d, precond=True):
        self.h = h
        self.d = d
        self.use_precond = precond

    def fg(self, point):
        A = as_tensor(point[0], self.d)
        e, D, rho = energy_grad(A, self.h)
        G = geo.project(point[0], as_matrix(D), geo.GRASSMANN)
        return e, [G], {"rho": rho, "delta": float(np.linalg.norm(G)) ** 2}

    def precondition(self, point, aux, X):
        if not self.use_precond:
            return [x.copy() for x in X]
        return [X[0] @ np.linalg.inv(aux["rho"] + aux["delta"] * np.eye(aux["rho"].shape[0]))]

    def retract(self, point, d, alpha):
        return [geo.polar(geo.retract(point[0], d[0], alpha))]

    def transport(self, point, d, alpha, Y):
        return [geo.transport(point[0], d[0], alpha, Y[0])]
