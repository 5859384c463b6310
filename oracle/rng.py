"""Seeded random isometries, FP64: the counter-based generator and the
sign-fixed QR-of-Gaussian initialisation, restated from their definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The library's ``mera_init_random`` draws the starting point itself, so the
random numbers cannot be passed in as inputs; this module implements the same
generator from its published definition (SplitMix64: Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; normals by the
Box-Muller transform, 1958) and the same factorisation (the thin QR factor of
the Gaussian matrix with R's diagonal real and positive, the unique one), with
NumPy's QR as the library primitive.

Definition (shared with ``include/mera.h``): x_k(s) = mix(s + k gamma) for
k >= 1 with gamma = 0x9E3779B97F4A7C15 and mix the SplitMix64 output function;
stream i under seed uses base = x_{i+1}(seed) and u_k = ((x_k(base) >> 11) +
0.5) 2^-53; the pair j, j+1 (j even) of normals is r cos t, r sin t with
r = sqrt(-2 ln u_{j+1}), t = 2 pi u_{j+2}.  The Gaussian matrix of a tensor
is row-major (interleaved real and imaginary parts for complex tensors).

Pins (tests/test_oracle_rng.py): the published first outputs of SplitMix64
for seed 0; the normals' mean, variance and distribution (Kolmogorov-Smirnov);
the isometry is the QR factor (Q^dag G upper triangular with a positive real
diagonal, Q R = G); charge blocks are factored on their own.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def mix(z: int) -> int:
    """SplitMix64's output function of a 64-bit state."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def output(state: int, k: int) -> int:
    """The k-th output (k >= 1) of SplitMix64 started at `state`."""
    return mix((state + k * GAMMA) & MASK)


def gaussians(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` standard normals of stream `stream` (Box-Muller on SplitMix64 uniforms)."""
    base = output(seed & MASK, stream + 1)
    out = np.empty(count)
    for j in range(0, count, 2):
        u1 = ((output(base, j + 1) >> 11) + 0.5) * 2.0**-53
        u2 = ((output(base, j + 2) >> 11) + 0.5) * 2.0**-53
        r, t = np.sqrt(-2.0 * np.log(u1)), 2.0 * np.pi * u2
        out[j] = r * np.cos(t)
        if j + 1 < count:
            out[j + 1] = r * np.sin(t)
    return out


def qr_positive(G: np.ndarray) -> np.ndarray:
    """The thin QR factor of G (n >= p) whose R has a real positive diagonal."""
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :]


def random_isometry(seed: int, stream: int, n: int, p: int, cplx: bool = False, row_charge=None,
                    col_charge=None) -> np.ndarray:
    """The isometry mera_init_random puts in tensor `stream` (n x p): the
    sign-fixed QR factor of the stream's Gaussian matrix, or, with charges,
    of each charge block (rows and columns of charge q in ascending order),
    zero between charges."""
    g = gaussians(seed, stream, n * p * (2 if cplx else 1))
    G = (g[0::2] + 1j * g[1::2]).reshape(n, p) if cplx else g.reshape(n, p)
    if row_charge is None:
        return qr_positive(G)
    out = np.zeros_like(G)
    for q in (0, 1):
        rows = np.flatnonzero(np.asarray(row_charge) == q)
        cols = np.flatnonzero(np.asarray(col_charge) == q)
        if cols.size:
            out[np.ix_(rows, cols)] = qr_positive(G[np.ix_(rows, cols)])
    return out
