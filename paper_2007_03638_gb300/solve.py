"""Run a MERA (or uniform-MPS) ground-state optimisation and log every iteration.

    python -m paper_2007_03638_gb300.solve --model ising --chi 4 --n-trans 2 --iters 300
    python -m paper_2007_03638_gb300.solve --model xxz --delta 1 --chi 8 --prec 1 --method cg
    python -m paper_2007_03638_gb300.solve --network ternary --z2 --chi 8 --n-trans 2 --method ev
    python -m paper_2007_03638_gb300.solve --network ternary --z2 --chi 4 --n-trans 1 --start fig2
    python -m paper_2007_03638_gb300.solve --network mps --model ising --field 1.5 --chi 16

Each iteration prints one JSON record: energy per spin, its distance to the
exact value (critical Ising -4/pi or Ising at field h by quadrature, XXZ at
Delta = 0 or 1 in closed form), |G|, the accepted step, the number of
energy/gradient evaluations and superoperator applications, and the
wall time.  The last record carries the summary.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as inp
from . import mera as gm


def exact_energy(model, par):
    if model == "ising":
        return inp.exact_ising_energy_per_spin(par)
    if abs(par - 1.0) < 1e-15:
        return inp.EXACT_XXZ_DELTA1
    if abs(par) < 1e-15:
        return -4.0 / math.pi
    return None


def problem(model, par, chi, n_trans, network="binary", z2=False, seed=0, start="random"):
    """(h, d_b, tensors, spins per bottom site) of a run: the binary network on
    blocked sites (two spins, three-site term), the ternary one and the uniform
    MPS (bond dimension chi, n_trans unused) on spins (two-site term); z2:
    Z2-symmetric starting point (binary: blocked pairs in the parity-ordered
    basis), and run() sets the library's Z2 mode, which contracts by charge
    sector.  start: "random" (seeded random isometries and disentanglers) or
    "fig2" (the start of the paper's Fig. 2: the same random isometries with
    identity disentanglers; MERA networks only)."""
    if start not in ("random", "fig2"):
        raise ValueError(f"unknown start {start!r}")
    if start == "fig2" and network == "mps":
        raise ValueError("the Fig. 2 start sets disentanglers, which the MPS has none of")
    h, d_b, tensors, spins = _problem(model, par, chi, n_trans, network, z2, seed)
    if start == "fig2":
        tensors = [np.eye(t.shape[0], dtype=t.dtype) if i % 2 == 0 else t for i, t in enumerate(tensors)]
    return h, d_b, tensors, spins


def _problem(model, par, chi, n_trans, network, z2, seed):
    bond = inp.ising_bond(par) if model == "ising" else inp.xxz_bond(par)
    if network == "mps":
        if z2:
            raise ValueError("Z2-symmetric starting points are built for the ternary network")
        A = inp.random_mps(chi, 2, seed=seed)
        return bond, 2, [A.reshape(chi * 2, chi)], 1
    if network == "ternary":
        us, ws = (inp.random_z2_ternary_mera(chi, n_trans, seed=seed) if z2
                  else inp.random_ternary_mera(2, chi, n_trans, seed=seed))
        return bond, 2, [t for p in zip(us, ws) for t in p], 1
    if z2:  # blocked spin pairs in the parity-ordered basis, symmetric tensors
        us, ws = inp.random_z2_mera(4, chi, n_trans, seed=seed)
        return (inp.parity_ordered_three_site(inp.three_site_blocked(bond)), 4,
                [t for p in zip(us, ws) for t in p], 2)
    us, ws = inp.random_mera(4, chi, n_trans, seed=seed)
    return inp.three_site_blocked(bond), 4, [t for p in zip(us, ws) for t in p], 2


def run(model="ising", par=1.0, chi=4, n_trans=2, prec=0, method=0, iters=300, gtol=1e-6, seed=0,
        lbfgs_m=8, krylov_dim=20, out=print, ev_gamma=None, network="binary", z2=False, start="random"):
    """method: 0 L-BFGS, 1 CG, 2 Evenbly-Vidal sweeps (one record per sweep;
    ev_gamma = the Hamiltonian shift, default the largest eigenvalue of the
    Hamiltonian term plus 0.5), 3 gradient descent.  network: "binary", "ternary" or "mps".
    start: as in problem()."""
    h3, d_b, tensors, spins = problem(model, par, chi, n_trans, network, z2, seed, start)
    net = {"binary": gm.MERA_BINARY, "ternary": gm.MERA_TERNARY, "mps": gm.MERA_MPS}[network]
    cfg = gm.default_config(d_b, chi, 0 if network == "mps" else n_trans, prec=prec, lbfgs_m=lbfgs_m,
                            krylov_dim=krylov_dim, network=net, z2=int(z2))
    m = gm.Mera(cfg, h3)
    m.set_tensors(tensors)
    ex = exact_energy(model, par)
    if method == 2 and ev_gamma is None:
        ev_gamma = float(np.linalg.eigvalsh(h3).max()) + 0.5
    t0 = time.perf_counter()
    rec = None
    evals = 0
    for it in range(iters):
        info = (m.cg_step() if method == 1 else m.ev_sweep(ev_gamma) if method == 2 else m.gd_step() if method == 3
                else m.lbfgs_step())
        evals += info["n_evals"]
        e_spin = info["energy"] / spins
        rec = {"iter": it + 1, "energy_per_spin": e_spin,
               "error": (e_spin - ex) if ex is not None else None, "gnorm": info["gnorm"],
               "alpha": info["alpha"], "n_evals": info["n_evals"], "krylov_matvecs": info["krylov_matvecs"],
               "time_s": time.perf_counter() - t0}
        out(json.dumps(rec))
        if info["gnorm"] < gtol:
            break
    summary = {"summary": True, "model": model, "param": par, "network": network, "z2": z2, "chi": chi,
               "n_trans": n_trans, "start": start,
               "prec": ["fp64", "3xtf32", "split_bf16", "split_fp16"][prec],
               "method": ["lbfgs", "cg", "ev", "gd"][method],
               "iters": rec["iter"], "energy_per_spin": rec["energy_per_spin"], "exact": ex,
               "error": rec["error"], "gnorm": rec["gnorm"], "evals": evals, "time_s": rec["time_s"]}
    if prec != 0:
        # the point the mixed-precision run reached, evaluated in FP64
        final = m.get_tensors()
        cfg64 = gm.default_config(d_b, chi, 0 if network == "mps" else n_trans, prec=0, lbfgs_m=lbfgs_m,
                                  krylov_dim=krylov_dim, network=net, z2=int(z2))
        m64 = gm.Mera(cfg64, h3)
        m64.set_tensors(final)
        e64, g64 = m64.energy_grad()
        summary["energy_per_spin_fp64"] = e64 / spins
        summary["gnorm_fp64"] = float(np.sqrt(sum(float(np.vdot(g, g).real) for g in g64)))
        m64.close()
    out(json.dumps(summary))
    m.close()
    return summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="ising", choices=["ising", "xxz"])
    ap.add_argument("--field", type=float, default=1.0, help="Ising transverse field h")
    ap.add_argument("--delta", type=float, default=1.0, help="XXZ anisotropy")
    ap.add_argument("--chi", type=int, default=4)
    ap.add_argument("--n-trans", type=int, default=2)
    ap.add_argument("--prec", type=int, default=0, help="0 FP64, 1 3xTF32, 2 split-BF16, 3 scaled split-FP16")
    ap.add_argument("--method", default="lbfgs", choices=["lbfgs", "cg", "ev", "gd"])
    ap.add_argument("--network", default="binary", choices=["binary", "ternary", "mps"])
    ap.add_argument("--z2", action="store_true",
                    help="Z2-symmetric problem (ternary, or binary up to chi = 16): contractions by charge sector")
    ap.add_argument("--ev-gamma", type=float, default=None,
                    help="Evenbly-Vidal Hamiltonian shift (default: largest eigenvalue of the 3-site term + 0.5)")
    ap.add_argument("--start", default="random", choices=["random", "fig2"],
                    help="starting point: seeded random tensors, or the paper's Fig. 2 start (identity disentanglers)")
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--gtol", type=float, default=1e-6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--m", type=int, default=8)
    ap.add_argument("--krylov-dim", type=int, default=20)
    a = ap.parse_args()
    par = a.field if a.model == "ising" else a.delta
    method = {"lbfgs": 0, "cg": 1, "ev": 2, "gd": 3}[a.method]
    run(a.model, par, a.chi, a.n_trans, a.prec, method, a.iters, a.gtol, a.seed, a.m, a.krylov_dim,
        ev_gamma=a.ev_gamma, network=a.network, z2=a.z2, start=a.start)


if __name__ == "__main__":
    main()
