"""Z2 symmetry of isometric tensors, FP64 (Sec. 6: symmetric tensors are block
diagonal in the charge basis, and the isometry condition, the projection, the
retraction and the transport act on the individual blocks; the benchmark of
Sec. 4, Fig. 2, enforces Z2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A tensor W (rows = its output legs fused, columns = its input legs fused, as
stored by the MERA code) carries Z2 charges on both sides
(``inputs.fused_parities`` of the leg dimensions); it is symmetric when it maps
each charge sector into the same sector, i.e. W[i, j] = 0 unless the row charge
of i equals the column charge of j.  Readings: charges of a leg follow
``inputs.z2_parities`` (the first half of a leg's basis even); the blockwise
geometry is the dense geometry of ``oracle/geometry.py`` applied to each
(row sector, column sector) block.

Pins (tests/test_oracle_z2.py): the Ising term is symmetric; a symmetric MERA
under a symmetric Hamiltonian has symmetric derivatives, level operators and
density matrices; projection, retraction and transport of symmetric inputs
are symmetric and equal their blockwise forms.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo


def violation(W, row_par, col_par):
    """Largest entry of W that connects different charges (zero for a
    symmetric tensor, Sec. 6)."""
    bad = row_par[:, None] != col_par[None, :]
    return float(np.abs(W[bad]).max()) if bad.any() else 0.0


def symmetrize(W, row_par, col_par):
    """Orthogonal projection onto the symmetric subspace (zero the entries
    that connect different charges)."""
    out = W.copy()
    out[row_par[:, None] != col_par[None, :]] = 0
    return out


def blocks(W, row_par, col_par):
    """The charge blocks {q: W[rows of q, cols of q]}."""
    return {q: W[np.ix_(np.flatnonzero(row_par == q), np.flatnonzero(col_par == q))] for q in (0, 1)}


def assemble(bl, row_par, col_par, dtype):
    out = np.zeros((row_par.size, col_par.size), dtype=dtype)
    for q, b in bl.items():
        out[np.ix_(np.flatnonzero(row_par == q), np.flatnonzero(col_par == q))] = b
    return out


def _blockwise(fn, row_par, col_par, *mats):
    bs = [blocks(M, row_par, col_par) for M in mats]
    out = {q: (fn(*[b[q] for b in bs]) if bs[0][q].size else bs[0][q]) for q in (0, 1)}
    return assemble(out, row_par, col_par, np.result_type(*mats))


def project_blockwise(W, D, kind, row_par, col_par):
    """Eqs. stiefel_gradient / grassmann_gradient on each charge block (Sec. 6)."""
    return _blockwise(lambda w, d: geo.project(w, d, kind), row_par, col_par, W, D)


def retract_blockwise(W, X, alpha, row_par, col_par):
    """The retraction of Sec. 2.3 on each charge block (Sec. 6)."""
    return _blockwise(lambda w, x: geo.retract(w, x, alpha), row_par, col_par, W, X)


def transport_blockwise(W, X, alpha, Y, row_par, col_par):
    """The vector transport of Sec. 2.3 on each charge block (Sec. 6)."""
    return _blockwise(lambda w, x, y: geo.transport(w, x, alpha, y), row_par, col_par, W, X, Y)
