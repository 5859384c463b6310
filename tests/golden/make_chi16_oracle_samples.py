"""Writes chi16_ising_L1_oracle_samples.json: the oracle's energy and sampled
partial derivatives of one chi = 16 binary MERA, for GPU parity at a size
whose oracle evaluation takes too long to repeat inside a test.

The point is the seeded QR-of-Gaussian start inputs.random_mera(4, 16, 1,
seed=7) (one transition layer 4 -> 16, then the scale-invariant layer at
chi = 16, whose chi^9 products are the largest of the evaluation), the
Hamiltonian the critical Ising chain on blocked spin pairs.  One transition
layer keeps the derivatives of the scale-invariant layer at the size they
have in the parity cases at chi <= 12 (Frobenius norms 0.03 to 0.1; after
three random layers at chi = 16 they are 1e-3) and the oracle's run to about
12 minutes.  Stored: the energy per bottom site e = Tr(h rho) (Sec. 4), and for every tensor v the
Frobenius norm and the largest magnitude of D_v = 2 dC/d conj(v) (Sec. 2.3)
with SAMPLES entries at seeded positions (row, column, value).  Only the
oracle and the seeded input generators run here.

    python tests/golden/make_chi16_oracle_samples.py    (about 12 minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import mera as om  # noqa: E402
from paper_2007_03638_gb300 import inputs as inp  # noqa: E402

CHI, N_TRANS, SEED, SAMPLES = 16, 1, 7, 64


def main():
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    us, ws = inp.random_mera(4, CHI, N_TRANS, seed=SEED)
    e, ds, _ = om.energy_grad(h3, us, ws)
    rng = np.random.default_rng(12345)
    tensors = []
    for d in ds:
        rows = rng.integers(0, d.shape[0], SAMPLES)
        cols = rng.integers(0, d.shape[1], SAMPLES)
        tensors.append({"shape": list(d.shape), "fro": float(np.linalg.norm(d)), "max_abs": float(np.abs(d).max()),
                        "rows": rows.tolist(), "cols": cols.tolist(), "values": d[rows, cols].tolist()})
    out = {"model": "critical Ising, blocked spin pairs (d_b = 4)", "chi": CHI, "n_trans": N_TRANS, "seed": SEED,
           "energy": e, "tensors": tensors}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chi16_ising_L1_oracle_samples.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"wrote {path}: e = {e!r}")


if __name__ == "__main__":
    main()
