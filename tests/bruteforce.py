"""Brute-force constructions used to pin the oracle: dense state vectors of
finite periodic binary MERAs and dense causal-cone isometries.  Written from
the definition |fine> = U W |coarse> with w on pairs (2j, 2j+1) and u on pairs
(2j+1, 2j+2); shares nothing with ``oracle/``."""
import numpy as np


def apply_two_site(psi, op, i, j):
    """Apply a (d*d, d*d) operator to legs i, j of the state tensor psi."""
    d = psi.shape[i]
    op4 = op.reshape(d, d, d, d)
    out = np.tensordot(op4, psi, axes=([2, 3], [i, j]))
    return np.moveaxis(out, [0, 1], [i, j])


def apply_isometry_layer(psi, w):
    """Each site k of psi (dim c') becomes the pair (2k, 2k+1) via w (c*c, c')."""
    n = psi.ndim
    c = int(round(np.sqrt(w.shape[0])))
    w3 = w.reshape(c, c, w.shape[1])
    for k in reversed(range(n)):
        psi = np.tensordot(psi, w3, axes=([k], [2]))  # new legs appended at end
        psi = np.moveaxis(psi, [psi.ndim - 2, psi.ndim - 1], [k, k + 1])
    return psi


def apply_disentangler_layer(psi, u):
    """u on every pair (2k+1, 2k+2), periodic."""
    n = psi.ndim
    for k in range(n // 2):
        psi = apply_two_site(psi, u, (2 * k + 1) % n, (2 * k + 2) % n)
    return psi


def finite_mera_state(top, layers):
    """top: state tensor on the top sites; layers: [(u, w), ...] from the top down."""
    psi = top
    for u, w in layers:
        psi = apply_isometry_layer(psi, w)
        psi = apply_disentangler_layer(psi, u)
    return psi


def energy_density(psi, bond):
    """<psi| sum_i bond(i, i+1) |psi> / N for a periodic chain."""
    n = psi.ndim
    tot = 0.0
    for i in range(n):
        tot += np.vdot(psi, apply_two_site(psi, bond, i, (i + 1) % n)).real
    return tot / n / np.vdot(psi, psi).real


def averaged_rdm3(psi):
    """Average over positions of the 3-site reduced density matrix (periodic)."""
    n = psi.ndim
    d = psi.shape[0]
    acc = np.zeros((d**3, d**3), dtype=np.result_type(psi, 1.0))
    for i in range(n):
        keep = [i % n, (i + 1) % n, (i + 2) % n]
        p = np.moveaxis(psi, keep, [0, 1, 2]).reshape(d**3, -1)
        acc += p @ p.conj().T
    return acc / n


def cone_isometry(u, w, side):
    """Dense map from 3 coarse sites to the 6 fine sites of one causal cone.

    side 'L': coarse (-1,0,1) -> fine (-2..3), u on fine pairs (-1,0), (1,2);
    side 'R': coarse (0,1,2) -> fine (0..5), u on (1,2), (3,4).
    Returns (V, keep) with V of shape (c**6, cp**3) and ``keep`` the positions
    (within the 6 fine sites) of the 3 sites the local operator lives on.
    """
    c = int(round(np.sqrt(u.shape[0])))
    w3 = np.kron(np.kron(w, w), w)  # (c**6, cp**3), fine order = site order
    one = np.eye(c)
    U = np.kron(np.kron(one, u), np.kron(u, one))
    keep = [2, 3, 4] if side == "L" else [1, 2, 3]
    return U @ w3, keep


def dense_descend(rho, u, w, side):
    V, keep = cone_isometry(u, w, side)
    c = int(round(np.sqrt(u.shape[0])))
    big = (V @ rho @ V.conj().T).reshape((c,) * 12)
    rest = [k for k in range(6) if k not in keep]
    perm = keep + rest + [6 + k for k in keep] + [6 + k for k in rest]
    big = np.transpose(big, perm).reshape(c**3, c**3, c**3, c**3)
    return np.einsum("aibi->ab", big)


# ------------------------------------------------------------- ternary ----
# |fine> = U W |coarse> with w mapping coarse site k to the fine triple
# (3k, 3k+1, 3k+2) and u acting on the fine pairs (3k+2, 3k+3), periodic.

def apply_ternary_isometry_layer(psi, w):
    """Each site k of psi (dim c') becomes the triple (3k, 3k+1, 3k+2) via w (c**3, c')."""
    n = psi.ndim
    c = int(round(w.shape[0] ** (1.0 / 3.0)))
    w4 = w.reshape(c, c, c, w.shape[1])
    for k in reversed(range(n)):
        psi = np.tensordot(psi, w4, axes=([k], [3]))  # three new legs appended at the end
        psi = np.moveaxis(psi, [psi.ndim - 3, psi.ndim - 2, psi.ndim - 1], [k, k + 1, k + 2])
    return psi


def apply_ternary_disentangler_layer(psi, u):
    """u on every pair (3k+2, 3k+3), periodic."""
    n = psi.ndim
    for k in range(n // 3):
        psi = apply_two_site(psi, u, (3 * k + 2) % n, (3 * k + 3) % n)
    return psi


def finite_ternary_state(top, layers):
    """top: state tensor on the top sites; layers: [(u, w), ...] from the top down."""
    psi = top
    for u, w in layers:
        psi = apply_ternary_isometry_layer(psi, w)
        psi = apply_ternary_disentangler_layer(psi, u)
    return psi


def averaged_rdm2(psi):
    """Average over positions of the 2-site reduced density matrix (periodic)."""
    n = psi.ndim
    d = psi.shape[0]
    acc = np.zeros((d**2, d**2), dtype=np.result_type(psi, 1.0))
    for i in range(n):
        p = np.moveaxis(psi, [i % n, (i + 1) % n], [0, 1]).reshape(d**2, -1)
        acc += p @ p.conj().T
    return acc / n / np.vdot(psi, psi).real
