"""Writes ternary_ising_chi4_L1_z2_lbfgs.npz: a Z2-symmetric ternary MERA for
the critical Ising chain (spins at the bottom, the Z eigenbasis ordered by
parity; chi = 4 with two even and two odd states; one transition layer plus
the scale-invariant layer), optimised by the oracle's preconditioned L-BFGS
(Sec. 3, m = 8) until |G| < 1e-9 or 1500 iterations.  The starting point is
the one of the paper's Fig. 2: the seeded symmetric random isometries
(seed 0) with identity disentanglers (from random disentanglers the
optimisation at this small chi stalls in a poor local minimum).  Every
retraction is followed by the projection of each tensor onto its charge
blocks (Sec. 6), so rounding cannot lead the optimisation out of the
symmetric tensors.

Only the oracle and the seeded input generators run here; the file holds the
tensors u_0, w_0, u_S, w_S, the final energy per spin and the iteration
count.  tests/test_oracle_scaling.py reads it.

    python tests/golden/make_ternary_ising_chi4_optimized.py    (about 2 minutes on 8 cores)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import geometry as geo  # noqa: E402
from oracle import optim as oo  # noqa: E402
from oracle import z2  # noqa: E402
from paper_2007_03638_gb300 import inputs as inp  # noqa: E402

CHI, N_TRANS, ITERS = 4, 1, 1500


def charges():
    """(row, column) charges of every tensor of the ternary MERA point."""
    dims = inp.ternary_layer_dims(2, CHI, N_TRANS)
    out = []
    for l in range(N_TRANS + 1):
        c, cp = dims[l], dims[min(l + 1, N_TRANS)]
        pair = inp.fused_parities(c, c)
        out += [(pair, pair), (inp.fused_parities(c, c, c), inp.z2_parities(cp))]
    return out


class SymmetricTernaryProblem(oo.TernaryProblem):
    """The oracle's ternary MERA problem with every retracted tensor projected
    onto its charge blocks before the polar re-isometrisation."""

    def __init__(self, h, ch):
        super().__init__(h)
        self.ch = ch

    def retract(self, point, d, alpha):
        return [geo.polar(z2.symmetrize(geo.retract(W, x, alpha), r, c))
                for W, x, (r, c) in zip(point, d, self.ch)]


def main():
    h = inp.ising_bond(1.0)
    _, ws = inp.random_z2_ternary_mera(CHI, N_TRANS, seed=0)
    dims = inp.ternary_layer_dims(2, CHI, N_TRANS)
    us = [np.eye(dims[l] ** 2) for l in range(N_TRANS + 1)]
    point = [t for pair in zip(us, ws) for t in pair]
    p, e, hist = oo.lbfgs(SymmetricTernaryProblem(h, charges()), point, m=8, maxiter=ITERS, gtol=1e-9)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ternary_ising_chi4_L1_z2_lbfgs.npz")
    np.savez(out, *p, energy_per_spin=e, iterations=len(hist))
    print(f"wrote {out}: {len(hist)} iterations, energy per spin {e:.10f} "
          f"({e - inp.EXACT_ISING_CRITICAL:.3e} above -4/pi), |G| {hist[-1]['gnorm']:.2e}")


if __name__ == "__main__":
    main()
