"""Host-side set-up of the optimisation program solve.py (no GPU): the binary network on
blocked sites with a three-site term, the ternary network and the uniform MPS
on spins with a two-site term, Z2-symmetric ternary starting points."""
import numpy as np
import pytest

from oracle import z2
from paper_2007_03638_gb300 import inputs as inp
from paper_2007_03638_gb300 import solve


def test_binary_problem():
    h, d_b, tensors, spins = solve.problem("ising", 1.0, 8, 3)
    assert (h.shape, d_b, spins, len(tensors)) == ((64, 64), 4, 2, 8)


def test_ternary_z2_problem_is_the_figure_2_setting():
    h, d_b, tensors, spins = solve.problem("ising", 1.0, 8, 2, network="ternary", z2=True)
    assert (h.shape, d_b, spins, len(tensors)) == ((4, 4), 2, 1, 6)
    assert [t.shape for t in tensors] == [(4, 4), (8, 8), (64, 64), (512, 8), (64, 64), (512, 8)]
    p = inp.fused_parities(2, 2)
    assert z2.violation(h, p, p) == 0.0
    w0 = tensors[1]
    assert z2.violation(w0, inp.fused_parities(2, 2, 2), inp.z2_parities(8)) == 0.0


def test_binary_z2_problem_is_parity_ordered():
    h, d_b, tensors, spins = solve.problem("ising", 1.0, 8, 3, z2=True)
    p3 = inp.fused_parities(4, 4, 4)
    assert (h.shape, d_b, spins, len(tensors)) == ((64, 64), 4, 2, 8)
    assert z2.violation(h, p3, p3) == 0.0
    pair = inp.fused_parities(4, 4)
    assert z2.violation(tensors[0], pair, pair) == 0.0


def test_mps_problem():
    h, d_b, tensors, spins = solve.problem("xxz", 1.0, 12, 0, network="mps")
    assert (h.shape, d_b, spins, len(tensors)) == ((4, 4), 2, 1, 1)
    A = tensors[0]
    assert A.shape == (24, 12)
    assert np.abs(A.T @ A - np.eye(12)).max() < 1e-13
    with pytest.raises(ValueError):
        solve.problem("ising", 1.0, 8, 0, network="mps", z2=True)


@pytest.mark.parametrize("network,z2", [("binary", False), ("binary", True), ("ternary", True)])
def test_figure_2_start_has_identity_disentanglers(network, z2):
    """--start fig2: the random start's isometries, identity disentanglers."""
    _, _, rand, _ = solve.problem("ising", 1.0, 8, 2 if network == "ternary" else 3, network=network, z2=z2)
    _, _, fig2, _ = solve.problem("ising", 1.0, 8, 2 if network == "ternary" else 3, network=network, z2=z2,
                                  start="fig2")
    assert len(fig2) == len(rand)
    for i, (a, b) in enumerate(zip(fig2, rand)):
        if i % 2 == 0:
            assert a.shape == b.shape and np.array_equal(a, np.eye(a.shape[0]))
        else:
            assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        solve.problem("ising", 1.0, 8, 0, network="mps", start="fig2")
    with pytest.raises(ValueError):
        solve.problem("ising", 1.0, 8, 3, start="zeros")
