"""Writes ising_chi4_L2_z2_lbfgs.npz: a Z2-symmetric binary MERA for the
critical Ising chain (two spins per bottom site, the site basis ordered by
parity; chi = 4 with two even and two odd states; 2 transition layers plus
the scale-invariant layer), optimised by the oracle's preconditioned L-BFGS
(Sec. 3, m = 8) from the seeded symmetric random point (seed 0) for 1000
iterations.  Every retraction is followed by the projection of each tensor
onto its charge blocks (Sec. 6), so rounding cannot lead the optimisation
out of the symmetric tensors.  (Without the symmetry the optimum at this
small chi breaks the chain's Z2 symmetry, and the scale-invariant layer then
has no Ising spectrum to compare with.)

Only the oracle and the seeded input generators run here; the file holds the
tensors u_0, w_0, u_1, w_1, u_S, w_S, the final energy per spin and the
iteration count.  tests/test_oracle_scaling.py reads it.

    python tests/golden/make_ising_chi4_optimized.py    (about 6 minutes on 8 cores;
                                                         reruns reproduce the file bit for bit)
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

ITERS = 1000


def charges(point):
    """(row, column) charges of every tensor of a binary MERA point."""
    out = []
    for i, t in enumerate(point):
        c = int(round(np.sqrt(t.shape[0])))
        pair = inp.fused_parities(c, c)
        out.append((pair, pair) if i % 2 == 0 else (pair, inp.z2_parities(t.shape[1])))
    return out


class SymmetricProblem(oo.MeraProblem):
    """The oracle's MERA problem with every retracted tensor projected onto its
    charge blocks before the polar re-isometrisation."""

    def __init__(self, h0, ch):
        super().__init__(h0)
        self.ch = ch

    def retract(self, point, d, alpha):
        return [geo.polar(z2.symmetrize(geo.retract(W, x, alpha), r, c))
                for W, x, (r, c) in zip(point, d, self.ch)]


def main():
    h3 = inp.parity_ordered_three_site(inp.three_site_blocked(inp.ising_bond(1.0)))
    us, ws = inp.random_z2_mera(4, 4, 2, seed=0)
    point = [t for pair in zip(us, ws) for t in pair]
    p, e, hist = oo.lbfgs(SymmetricProblem(h3, charges(point)), point, m=8, maxiter=ITERS, gtol=1e-9)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ising_chi4_L2_z2_lbfgs.npz")
    np.savez(out, *p, energy_per_spin=e / 2, iterations=len(hist))
    print(f"wrote {out}: {len(hist)} iterations, energy per spin {e / 2:.10f} "
          f"({e / 2 - inp.EXACT_ISING_CRITICAL:.3e} above -4/pi)")


if __name__ == "__main__":
    main()
