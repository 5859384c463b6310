"""Pins of the Z2 utilities (oracle/z2.py): the Ising chain's parity, symmetry
of a symmetric MERA's derivatives and level operators, and the blockwise
geometry of Sec. 6 (projection, retraction and transport per charge block)
against the dense geometry."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import ternary as ot
from oracle import z2
from paper_2007_03638_gb300 import inputs as inp


def _charges(us, ws):
    """(row, column) charges of every tensor of a ternary MERA on spins."""
    out = []
    for u, w in zip(us, ws):
        c = int(round(np.sqrt(u.shape[0])))
        pair = inp.fused_parities(c, c)
        out += [(pair, pair), (inp.fused_parities(c, c, c), inp.z2_parities(w.shape[1]))]
    return out


def test_ising_term_is_symmetric_and_a_field_breaks_it():
    p = inp.fused_parities(2, 2)
    assert z2.violation(inp.ising_bond(1.0), p, p) == 0.0
    assert z2.violation(inp.xxz_bond(0.7), p, p) == 0.0
    assert z2.violation(inp.ising_bond(1.0, 0.3), p, p) > 0.1


def test_symmetric_initial_point():
    us, ws = inp.random_z2_ternary_mera(8, 2, seed=0)
    for t, (r, c) in zip([t for p in zip(us, ws) for t in p], _charges(us, ws)):
        assert z2.violation(t, r, c) == 0.0
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-13


def test_derivatives_and_level_operators_stay_symmetric():
    us, ws = inp.random_z2_ternary_mera(4, 1, seed=2)
    pt = [t for p in zip(us, ws) for t in p]
    e, ds, info = ot.energy_grad(inp.ising_bond(1.0), us, ws)
    for d, (r, c) in zip(ds, _charges(us, ws)):
        assert z2.violation(d, r, c) < 1e-13 * np.abs(d).max()
    for l, (h, rho) in enumerate(zip(info["h"], info["rho"])):
        cl = int(round(np.sqrt(h.shape[0])))
        p = inp.fused_parities(cl, cl)
        assert z2.violation(h, p, p) < 1e-13 and z2.violation(rho, p, p) < 1e-13
    # a symmetry-breaking field shows up in the derivatives
    _, ds2, _ = ot.energy_grad(inp.ising_bond(1.0, 0.3), us, ws)
    assert max(z2.violation(d, r, c) for d, (r, c) in zip(ds2, _charges(us, ws))) > 1e-3


def test_blockwise_geometry_equals_dense_geometry():
    us, ws = inp.random_z2_ternary_mera(4, 1, seed=4)
    pt = [t for p in zip(us, ws) for t in p]
    _, ds, _ = ot.energy_grad(inp.ising_bond(1.0), us, ws)
    rng = np.random.default_rng(1)
    for i, (W, D, (r, c)) in enumerate(zip(pt, ds, _charges(us, ws))):
        kind = geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN
        G = geo.project(W, D, kind)
        assert z2.violation(G, r, c) < 1e-13 * max(1.0, np.abs(G).max())
        assert np.abs(G - z2.project_blockwise(W, D, kind, r, c)).max() < 1e-13
        Y = geo.project(W, z2.symmetrize(rng.standard_normal(W.shape), r, c), kind)
        R = geo.retract(W, G, 0.3)
        assert z2.violation(R, r, c) < 1e-12
        assert np.abs(R - z2.retract_blockwise(W, G, 0.3, r, c)).max() < 1e-12
        T = geo.transport(W, G, 0.3, Y)
        assert np.abs(T - z2.transport_blockwise(W, G, 0.3, Y, r, c)).max() < 1e-12
