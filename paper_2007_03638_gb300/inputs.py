"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the optimisation method itself: it only
builds the problem data (local Hamiltonian terms on Pauli matrices, blocked
into three-site terms) and seeded random starting tensors (QR of Gaussian
matrices).  Both implementations receive the same bytes from here.

Conventions
-----------
* A 3-site operator ``o`` on sites of dimension ``d`` is a ``(d**3, d**3)``
  matrix ``o[f0 f1 f2, g0 g1 g2] = <f0 f1 f2| o |g0 g1 g2>`` (row-major, left
  site most significant).
* A disentangler ``u`` of a layer with fine dimension ``c`` is a ``(c*c, c*c)``
  unitary ``u[f_a f_b, x_a x_b]`` (rows: fine/output legs, columns: legs that
  connect to the isometries above).
* An isometry ``w`` maps one coarse site (dimension ``c'``) to a pair of fine
  sites: a ``(c*c, c')`` matrix ``w[x_a x_b, k]`` with ``w^dag w = 1``.
"""
from __future__ import annotations

import numpy as np

PAULI_X = np.array([[0.0, 1.0], [1.0, 0.0]])
PAULI_Y = np.array([[0.0, -1.0j], [1.0j, 0.0]])
PAULI_Z = np.array([[1.0, 0.0], [0.0, -1.0]])
ID2 = np.eye(2)


def ising_bond(h: float = 1.0, hx: float = 0.0) -> np.ndarray:
    """Two-spin term of H = -sum(X X + h Z + hx X) with the one-site fields
    split evenly over the two bonds that touch a spin (4x4, real)."""
    t = -np.kron(PAULI_X, PAULI_X)
    t = t - 0.5 * h * (np.kron(PAULI_Z, ID2) + np.kron(ID2, PAULI_Z))
    t = t - 0.5 * hx * (np.kron(PAULI_X, ID2) + np.kron(ID2, PAULI_X))
    return t


def xxz_bond(delta: float = 1.0) -> np.ndarray:
    """Two-spin term X X + Y Y + delta Z Z on Pauli matrices (4x4, real)."""
    t = np.kron(PAULI_X, PAULI_X) + np.kron(PAULI_Y, PAULI_Y) + delta * np.kron(PAULI_Z, PAULI_Z)
    return np.real_if_close(t).astype(np.float64)


def three_site_unblocked(bond: np.ndarray) -> np.ndarray:
    """3-site term on spin sites (d=2) whose translates sum to sum_i bond(i,i+1)."""
    return 0.5 * (np.kron(bond, ID2) + np.kron(ID2, bond))


def three_site_blocked(bond: np.ndarray) -> np.ndarray:
    """3-site term on blocked sites of dimension 4 (spins 2i, 2i+1 form site i).

    The blocked two-site term keeps half of each block's internal bond plus the
    bond between the blocks; the 3-site term is the average of the two-site
    term on its left and right pairs.  Translates of the result sum to the spin
    Hamiltonian, so the energy per blocked site is twice the energy per spin.
    """
    id4 = np.eye(4)
    intra = 0.5 * (np.kron(bond, id4) + np.kron(id4, bond))
    inter = np.kron(np.kron(ID2, bond), ID2)
    hb = intra + inter
    return 0.5 * (np.kron(hb, id4) + np.kron(id4, hb))


def layer_dims(d_b: int, chi: int, n_trans: int) -> list[int]:
    """Bond dimensions chi_0 = d_b, chi_{l+1} = min(chi, chi_l**2); the last
    entry (index n_trans) is the scale-invariant layer's dimension, forced to chi."""
    dims = [d_b]
    for _ in range(n_trans):
        dims.append(min(chi, dims[-1] ** 2))
    if dims[-1] != chi:
        raise ValueError(f"transition layers cannot reach chi={chi} from d_b={d_b}")
    return dims


def _haar_like(rng: np.random.Generator, n: int, p: int, dtype) -> np.ndarray:
    g = rng.standard_normal((n, p))
    if np.dtype(dtype).kind == "c":
        g = g + 1j * rng.standard_normal((n, p))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r).real)
    s[s == 0] = 1.0
    return (q * s[None, :]).astype(dtype)


def random_mera(d_b: int, chi: int, n_trans: int, seed: int, dtype=np.float64):
    """Seeded starting point: per layer (transition layers, then the
    scale-invariant one) a unitary u (QR of a square Gaussian) and an isometry w
    (thin QR of a Gaussian), columns sign-fixed by diag(R)."""
    rng = np.random.default_rng(seed)
    dims = layer_dims(d_b, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        us.append(_haar_like(rng, c * c, c * c, dtype))
        ws.append(_haar_like(rng, c * c, cp, dtype))
    return us, ws


def product_state_mera(d_b: int, n_trans: int, chi: int | None = None):
    """u = 1 and w|k> = |k>|0>: a MERA for the product state |0 0 ...>."""
    chi = d_b if chi is None else chi
    dims = layer_dims(d_b, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        us.append(np.eye(c * c))
        w = np.zeros((c * c, cp))
        for k in range(min(cp, c)):
            w[k * c + 0, k] = 1.0
        ws.append(w)
    return us, ws


def random_tangent_like(rng: np.random.Generator, tensors, dtype=np.float64):
    out = []
    for t in tensors:
        g = rng.standard_normal(t.shape)
        if np.dtype(dtype).kind == "c":
            g = g + 1j * rng.standard_normal(t.shape)
        out.append(g.astype(dtype))
    return out


def exact_ising_energy_per_spin(h: float = 1.0, n: int = 200000) -> float:
    """Ground-state energy per spin of -sum(X X + h Z) (free fermions):
    -(1/pi) int_0^pi sqrt(1 + h^2 + 2 h cos k) dk, by the midpoint rule."""
    k = (np.arange(n) + 0.5) * np.pi / n
    return float(-np.mean(np.sqrt(1.0 + h * h + 2.0 * h * np.cos(k))))


EXACT_ISING_CRITICAL = -4.0 / np.pi
EXACT_XXZ_DELTA1 = 1.0 - 4.0 * np.log(2.0)


def ternary_layer_dims(d: int, chi: int, n_trans: int) -> list[int]:
    """Ternary MERA bond dimensions chi_0 = d, chi_{l+1} = min(chi, chi_l**3);
    the last entry (index n_trans) is the scale-invariant layer's, forced to chi."""
    dims = [d]
    for _ in range(n_trans):
        dims.append(min(chi, dims[-1] ** 3))
    if dims[-1] != chi:
        raise ValueError(f"transition layers cannot reach chi={chi} from d={d}")
    return dims


def random_ternary_mera(d: int, chi: int, n_trans: int, seed: int, dtype=np.float64):
    """Seeded ternary starting point: per layer a unitary u (c^2 x c^2) and an
    isometry w (c^3 x c'), QR of Gaussians with columns sign-fixed by diag(R)."""
    rng = np.random.default_rng(seed)
    dims = ternary_layer_dims(d, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        us.append(_haar_like(rng, c * c, c * c, dtype))
        ws.append(_haar_like(rng, c**3, cp, dtype))
    return us, ws


def product_state_ternary_mera(d: int, chi: int, n_trans: int):
    """u = 1 and w|k> = the k-th basis vector of the fine triple (so
    w|0> = |000>): the scale-invariant product state |00...0>."""
    dims = ternary_layer_dims(d, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        us.append(np.eye(c * c))
        ws.append(np.eye(c**3, cp))
    return us, ws


def random_mps(D: int, d: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded left-canonical uniform-MPS tensor A (D, d, D): thin QR of a
    Gaussian (D d) x D matrix, columns sign-fixed by diag(R)."""
    rng = np.random.default_rng(seed)
    return _haar_like(rng, D * d, D, dtype).reshape(D, d, D)


def aklt_mps():
    """The AKLT state (spin 1, D = 2) as a left-canonical uniform-MPS tensor
    A (2, 3, 2) (physical basis m = +1, 0, -1) and its bond term
    S.S + (S.S)^2 / 3, whose exact ground state it is (energy -2/3 per bond)."""
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    A = np.zeros((2, 3, 2))
    A[:, 0, :] = np.sqrt(2.0 / 3.0) * sp
    A[:, 1, :] = -np.sqrt(1.0 / 3.0) * np.diag([1.0, -1.0])
    A[:, 2, :] = -np.sqrt(2.0 / 3.0) * sp.T
    s = 1.0 / np.sqrt(2.0)
    Sx = s * np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=complex)
    Sy = s * np.array([[0, -1j, 0], [1j, 0, -1j], [0, 1j, 0]])
    Sz = np.diag([1.0, 0.0, -1.0]).astype(complex)
    SS = np.real(np.kron(Sx, Sx) + np.kron(Sy, Sy) + np.kron(Sz, Sz))
    return A, SS + SS @ SS / 3.0


def z2_parities(dim: int) -> np.ndarray:
    """Z2 charges of the basis of a leg of dimension dim: the first ceil(dim/2)
    states even (0), the rest odd (1).  For a spin-1/2 leg (dim 2) this is the
    eigenbasis of Z: |0> even, |1> odd, the parity of the Ising chain."""
    return np.array([0] * ((dim + 1) // 2) + [1] * (dim // 2), dtype=np.int64)


def fused_parities(*dims: int) -> np.ndarray:
    """Charges of the product basis of several legs (last leg fastest)."""
    p = np.zeros(1, dtype=np.int64)
    for d in dims:
        p = (p[:, None] + z2_parities(d)[None, :]).ravel() % 2
    return p


def _z2_block_isometry(rng, row_par, col_par, dtype):
    """Isometry (rows x cols) mapping each column charge into the rows of the
    same charge only (block diagonal in the charge basis)."""
    W = np.zeros((row_par.size, col_par.size), dtype=dtype)
    for q in (0, 1):
        r, c = np.flatnonzero(row_par == q), np.flatnonzero(col_par == q)
        if c.size:
            W[np.ix_(r, c)] = _haar_like(rng, r.size, c.size, dtype)
    return W


def random_z2_ternary_mera(chi: int, n_trans: int, seed: int, dtype=np.float64):
    """Seeded Z2-symmetric ternary MERA on spins (d = 2): every u and w maps
    each charge sector into the same sector (parities of fine legs fused, coarse
    legs charged by z2_parities)."""
    rng = np.random.default_rng(seed)
    dims = ternary_layer_dims(2, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        pair = fused_parities(c, c)
        us.append(_z2_block_isometry(rng, pair, pair, dtype))
        ws.append(_z2_block_isometry(rng, fused_parities(c, c, c), z2_parities(cp), dtype))
    return us, ws


# Basis of a blocked spin pair (s1 s2) ordered by parity: the even states
# |00>, |11> first, then the odd |01>, |10>, so that the first half of the
# site's basis is even (the grading of the library's Z2 mode).
PAIR_PARITY_ORDER = np.array([0, 3, 1, 2])


def parity_ordered_three_site(h3: np.ndarray) -> np.ndarray:
    """A three-site term on blocked spin pairs (three_site_blocked) in the
    parity-ordered site basis: P h3 P^T with P the permutation
    PAIR_PARITY_ORDER on each of the three sites."""
    perm = np.array([(a * 16 + b * 4 + c) for a in PAIR_PARITY_ORDER for b in PAIR_PARITY_ORDER
                     for c in PAIR_PARITY_ORDER])
    return h3[np.ix_(perm, perm)]


def random_z2_mera(d_b: int, chi: int, n_trans: int, seed: int, dtype=np.float64):
    """Seeded Z2-symmetric binary MERA: every u and w maps each charge sector
    into the same sector (parities of fine legs fused, every leg graded with
    the first half of its basis even)."""
    rng = np.random.default_rng(seed)
    dims = layer_dims(d_b, chi, n_trans)
    us, ws = [], []
    for l in range(n_trans + 1):
        c = dims[l]
        cp = dims[l + 1] if l < n_trans else dims[n_trans]
        pair = fused_parities(c, c)
        us.append(_z2_block_isometry(rng, pair, pair, dtype))
        ws.append(_z2_block_isometry(rng, pair, z2_parities(cp), dtype))
    return us, ws
