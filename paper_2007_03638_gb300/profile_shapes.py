"""Per-shape contraction profile of one L-BFGS iteration.

Builds the XXZ (Delta = 1) problem on blocked sites (d_b = 4) with three
transition layers, starts from the seeded random point, runs one
energy/gradient evaluation (which fills the Krylov warm starts), then times
one L-BFGS iteration with profiling on and writes the library's per-shape
table (mera_profile_dump: every contraction shape with its path, call count
and device time, plus the operand-packing and eigensolver phases) as CSV.

    python -m paper_2007_03638_gb300.profile_shapes --chi 32 --prec 2 --out shapes.csv
"""
import argparse
import json
import time

from . import inputs as inp
from . import mera as gm


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--chi", type=int, default=32)
    ap.add_argument("--prec", type=int, default=2, help="0 FP64, 1 3xTF32, 2 split-BF16")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", required=True, help="CSV file for the per-shape table")
    a = ap.parse_args(argv)
    cfg = gm.default_config(4, a.chi, 3, prec=a.prec, lbfgs_m=16, krylov_dim=4)
    m = gm.Mera(cfg, inp.three_site_blocked(inp.xxz_bond(1.0)))
    us, ws = inp.random_mera(4, a.chi, 3, seed=a.seed)
    m.set_tensors([t for p in zip(us, ws) for t in p])
    m.energy_grad()
    m.stats(reset=True)
    m.profile(True)
    t = time.perf_counter()
    info = m.lbfgs_step()
    wall = time.perf_counter() - t
    m.profile_dump(a.out)
    st = m.stats()
    print(json.dumps({"chi": a.chi, "prec": a.prec, "step_s": wall, "iter": info, "stats": st}))


if __name__ == "__main__":
    main()
