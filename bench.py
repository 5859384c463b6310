#!/usr/bin/env python
"""Benchmark: MERA gradient evaluations per second (one GB300 per rank).

A step is one full Riemannian L-BFGS iteration of the scale-invariant binary
MERA (two-loop direction with the preconditioner, Hager-Zhang line search
with as many energy/gradient evaluations as it needs, retraction, transport
of the history); other workloads take the same step for the ternary MERA
(with or without Z2 charge sectors), the uniform MPS or complex tensors.  The reported value is energy/gradient evaluations per
second over the timed steps, summed over ranks (independent replicas: the
optimisation does not shard across GPUs, so N GPUs run N problems).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU FP64 oracle, same metric
    python bench.py --shapes-out shapes.csv  # per-shape device time of one L-BFGS iteration

Inputs are synthetic and seeded (QR-of-Gaussian tensors, Z2-symmetric blocks
for the z2 workloads; critical Ising, Ising with a longitudinal field or the
Heisenberg chain, on blocked spin pairs for the binary MERA and on spins
otherwise).  L2 is flushed (256 MiB write) between timed steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_03638_gb300 import inputs as inp  # noqa: E402

WORKLOADS = {
    # name: (hamiltonian, d_b, chi, n_trans, prec, extra config)
    # prec: 0 FP64, 1 3xTF32, 2 split-BF16, 3 scaled split-FP16
    "ising_chi4_L2_fp64": ("ising", 4, 4, 2, 0, {}),
    "ising_chi8_L3_fp64": ("ising", 4, 8, 3, 0, {}),
    "ising_chi12_L3_fp64": ("ising", 4, 12, 3, 0, {}),
    "ising_chi12_L3_3xtf32": ("ising", 4, 12, 3, 1, {}),
    "ising_chi12_L3_bf16": ("ising", 4, 12, 3, 2, {}),
    "xxz_chi16_L3_3xtf32": ("xxz", 4, 16, 3, 1, {"lbfgs_m": 16}),
    "xxz_chi16_L3_bf16": ("xxz", 4, 16, 3, 2, {"lbfgs_m": 16}),
    "xxz_chi24_L3_3xtf32": ("xxz", 4, 24, 3, 1, {"lbfgs_m": 16}),
    "xxz_chi24_L3_bf16": ("xxz", 4, 24, 3, 2, {"lbfgs_m": 16}),
    "xxz_chi32_L3_3xtf32": ("xxz", 4, 32, 3, 1, {"lbfgs_m": 16, "krylov_dim": 4}),
    "xxz_chi32_L3_bf16": ("xxz", 4, 32, 3, 2, {"lbfgs_m": 16, "krylov_dim": 4}),
    "xxz_chi32_L3_fp16": ("xxz", 4, 32, 3, 3, {"lbfgs_m": 16, "krylov_dim": 4}),
    "xxz_chi24_L3_fp16": ("xxz", 4, 24, 3, 3, {"lbfgs_m": 16}),
    "xxz_chi16_L3_fp16": ("xxz", 4, 16, 3, 3, {"lbfgs_m": 16}),
    "ising_chi12_L3_fp16": ("ising", 4, 12, 3, 3, {}),
    # the same with environment recomputation (one set of intermediates for all layers)
    "xxz_chi32_L3_bf16_recompute": ("xxz", 4, 32, 3, 2, {"lbfgs_m": 16, "krylov_dim": 4, "recompute_env": 1}),
    "xxz_chi32_L3_fp16_recompute": ("xxz", 4, 32, 3, 3, {"lbfgs_m": 16, "krylov_dim": 4, "recompute_env": 1}),
    # extra config fields: network 1 = ternary, 2 = uniform MPS (chi = bond
    # dimension D); z2 = 1: Z2 charge sectors; dtype 1 = complex128
    "ternary_ising_chi8_L2_fp64": ("ising", 2, 8, 2, 0, {"network": 1}),
    "ternary_ising_chi8_L2_fp64_z2": ("ising", 2, 8, 2, 0, {"network": 1, "z2": 1}),
    "ternary_xxz_chi16_L2_3xtf32": ("xxz", 2, 16, 2, 1, {"network": 1}),
    "ternary_xxz_chi16_L2_3xtf32_z2": ("xxz", 2, 16, 2, 1, {"network": 1, "z2": 1}),
    "mps_xxz_D32_fp64": ("xxz", 2, 32, 0, 0, {"network": 2}),
    "ising_chi16_L3_3xtf32_z2": ("ising", 4, 16, 3, 1, {"z2": 1, "lbfgs_m": 16}),
    "ising_hz_chi8_L3_c128_fp64": ("ising_hz", 4, 8, 3, 0, {"dtype": 1}),
    "ising_hz_chi16_L3_c128_3xtf32": ("ising_hz", 4, 16, 3, 1, {"dtype": 1, "lbfgs_m": 16}),
}
# Workloads whose CPU baseline times whole oracle energy/gradient evaluations
# (seconds each): the ternary and MPS ones and every binary one up to chi = 12;
# the others time one layer's ascending map and extrapolate by flop count.
def whole_eval(name):
    kind, d_b, chi, L, prec, extra = WORKLOADS[name]
    return extra.get("network", 0) in (1, 2) or chi <= 12
DEFAULT_WORKLOAD = "xxz_chi32_L3_fp16"
# Algorithmic flops of one energy/gradient evaluation as the GPU path counts
# them inside L-BFGS steps (measured by this script's own GPU runs); used only
# to express the reference arm's bounded sample in gradient evaluations.
FLOPS_PER_GRAD = {
    "xxz_chi32_L3_bf16": 4.1e15, "xxz_chi32_L3_3xtf32": 4.1e15, "xxz_chi32_L3_bf16_recompute": 4.1e15,
    # split-FP16 at chi = 32: 7.75 superoperator applications per gradient
    # (3.0e14 flops each); the recompute figure was measured at 9.75
    "xxz_chi32_L3_fp16_recompute": 4.72e15,
    "xxz_chi32_L3_fp16": 3.82e15,
    "xxz_chi24_L3_3xtf32": 4.7e14, "xxz_chi24_L3_bf16": 4.7e14, "xxz_chi24_L3_fp16": 4.7e14,
    "xxz_chi16_L3_3xtf32": 1.45e13, "xxz_chi16_L3_bf16": 1.2e13, "xxz_chi16_L3_fp16": 1.2e13,
    "ising_chi12_L3_fp64": 1.6e12, "ising_chi12_L3_3xtf32": 1.13e12, "ising_chi12_L3_bf16": 1.13e12,
    "ising_chi12_L3_fp16": 1.13e12,
    "ising_chi8_L3_fp64": 5e10, "ising_chi4_L2_fp64": 1.2e8,
    # complex workloads: 4 x the real workload's (8 real flops per complex
    # multiply-add), an estimate until measured
    "ising_hz_chi8_L3_c128_fp64": 2e11, "ising_hz_chi16_L3_c128_3xtf32": 5.8e13,
    # Z2 workloads: the dense evaluation's count (the oracle contracts densely)
    "ising_chi16_L3_3xtf32_z2": 1.45e13,
}
METRIC = "MERA grad evals/s"
UNIT = "grad_evals/s"

# FP64 FMA throughput of GB300: the nominal 1.25 TFLOP/s at the 2070 MHz
# boost clock is 2 FP64 FMA per clock per SM over 152 SMs.
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2070e6

# Tensor-core peaks: the measured dense BF16 GEMM rate (MEASURED_PEAKS.json)
# sustained over seconds under the power cap (the contractions are timed
# inside steps of tens of seconds), and TF32 from it by the nominal TF32/BF16
# ratio (1.1 / 2.25 PFLOP/s).
def tensor_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        j = json.load(open(path))
        bf16 = float(j["bf16_tflops_sustained"]) * 1e12
        src = "measured bf16, sustained (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        bf16 = 1.7e15
        src = "fallback bf16 sustained 1.7 PFLOP/s"
    # FP16 products (kind::f16) run at the BF16 rate
    return {2: (bf16, src), 3: (bf16, src + " (fp16 = bf16 rate)"),
            1: (bf16 * 1.1 / 2.25, src + " x nominal tf32/bf16 ratio 1.1/2.25")}


# DRAM traffic per launch of the dominant kernel from an ncu capture of the
# same workload, kept only while the kernel is unchanged since the capture
# (none is: the roofline's traffic is reported as null).
GETT_TRAFFIC_BYTES = {}


def hamiltonian(kind, d_b, network=0, z2=False):
    """The workload's Hamiltonian term: critical Ising, Ising with a
    longitudinal field h_z = 0.13 (-h_z X per spin) or the Heisenberg chain;
    three-site (blocked spin pairs when d_b = 4) for the binary MERA, the
    two-site bond for the ternary MERA and the MPS; blocked pairs in the
    parity-ordered basis for Z2-symmetric binary problems."""
    bond = (inp.ising_bond(1.0) if kind == "ising" else inp.ising_bond(1.0, 0.13) if kind == "ising_hz"
            else inp.xxz_bond(1.0))
    if network in (1, 2):
        return bond
    h3 = inp.three_site_blocked(bond) if d_b == 4 else inp.three_site_unblocked(bond)
    return inp.parity_ordered_three_site(h3) if (z2 and d_b == 4) else h3


def initial_point(d_b, chi, L, extra, seed):
    """Seeded starting tensors of a workload (QR of Gaussian matrices; Z2-symmetric
    blocks when z2 is set; complex when dtype = 1)."""
    net = extra.get("network", 0)
    dt = np.complex128 if extra.get("dtype", 0) == 1 else np.float64
    if net == 2:
        return [inp.random_mps(chi, d_b, seed=seed, dtype=dt).reshape(chi * d_b, chi)]
    if net == 1:
        us, ws = (inp.random_z2_ternary_mera(chi, L, seed=seed, dtype=dt) if extra.get("z2")
                  else inp.random_ternary_mera(d_b, chi, L, seed=seed, dtype=dt))
    elif extra.get("z2"):
        us, ws = inp.random_z2_mera(d_b, chi, L, seed=seed, dtype=dt)
    else:
        us, ws = inp.random_mera(d_b, chi, L, seed=seed, dtype=dt)
    return [t for p in zip(us, ws) for t in p]


def ascend_flops(cf, cc=None):
    """Algorithmic flops of one averaged ascending map of a layer with fine
    bond cf and coarse bond cc (both sides; the library's contraction tree,
    whose ten steps cost cf^3cc^2, cf^8, cf^8, cf^5cc, cf^8cc, cf^5cc, cf^7cc^2,
    cf^4cc^4, cf^3cc^2, cf^2cc^6 multiply-adds; 2 chi^9 + 4 chi^8 + ... at cf = cc)."""
    cc = cf if cc is None else cc
    f, c = float(cf), float(cc)
    macs = (f**3 * c**2 + 2 * f**8 + f**5 * c + f**8 * c + f**5 * c + f**7 * c**2 + f**4 * c**4
            + f**3 * c**2 + f**2 * c**6)
    return 2 * 2.0 * macs


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path, gpu):
        self.path, self.gpu, self.p = path, gpu, None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.close()

    def summary(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def sample_layer(d_b, chi, L):
    """The largest layer of the workload whose oracle ascending map stays a
    bounded (seconds-scale) sample: the scale-invariant layer up to chi=16,
    otherwise transition layer 1."""
    dims = inp.layer_dims(d_b, chi, L)
    if chi <= 16:
        return L, dims[L], dims[L]
    return 1, dims[1], dims[2]


def oracle_sample(d_b, chi, L, seconds=10.0, seed=0, cplx=False):
    """Time the oracle's ascending map of one layer of the workload (seeded
    tensors of that layer, random Hermitian operator) on the host cores: both
    sides up to chi=16, the left side A_L alone above (half the flops)."""
    from oracle import mera as om
    layer, cf, cc = sample_layer(d_b, chi, L)
    one_side = chi > 16
    us, ws = inp.random_mera(d_b, chi, L, seed=seed, dtype=np.complex128 if cplx else np.float64)
    u, w = us[layer], ws[layer]
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((cf**3, cf**3)) + (1j * rng.standard_normal((cf**3, cf**3)) if cplx else 0)
    h = 0.5 * (h + h.conj().T)
    n, t0 = 0, time.perf_counter()
    while True:
        if one_side:
            om.ascend_side(h, u, w, "L")
        else:
            om.ascend(h, u, w)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return dt / n, n, layer, cf, cc, (0.5 if one_side else 1.0)


def oracle_eval_sample(wl, seconds=10.0, seed=0):
    """Time whole oracle energy/gradient evaluations of the workload (the
    binary, ternary or MPS oracle) at its seeded point on the host cores,
    at least one and until `seconds` have passed.  Returns (seconds per
    evaluation, evaluations)."""
    kind, d_b, chi, L, prec, extra = wl
    net = extra.get("network", 0)
    h = hamiltonian(kind, d_b, net, bool(extra.get("z2", 0)))
    point = initial_point(d_b, chi, L, extra, seed)
    if net == 2:
        from oracle import mps
        A = point[0].reshape(chi, d_b, chi)
        run = lambda: mps.energy_grad(A, h)  # noqa: E731
    elif net == 1:
        from oracle import ternary as ot
        run = lambda: ot.energy_grad(h, point[0::2], point[1::2])  # noqa: E731
    else:
        from oracle import mera as om
        run = lambda: om.energy_grad(h, point[0::2], point[1::2])  # noqa: E731
    n, t0 = 0, time.perf_counter()
    while True:
        run()
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return dt / n, n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(t_ms, units, dist=None, device="cpu"):
    """Whole-job numbers over ranks: the slowest rank's time and the summed
    units (replicas: every rank solves its own problem)."""
    if dist is None:
        return t_ms, units
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


def run_reference(args, wl):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    kind, d_b, chi, L, prec, extra = wl
    cplx = extra.get("dtype", 0) == 1
    per = []
    # samples of tens of seconds (chi = 32: one side of a layer's ascending
    # map) run at most 1 + 3 times, so that the arm ends within minutes
    steps, warmup = args.steps, args.warmup
    if not whole_eval(args.workload) and chi > 16:
        steps, warmup = min(steps, 3), min(warmup, 1)
    if whole_eval(args.workload):
        for i in range(warmup + steps):
            t, n = oracle_eval_sample(wl, seconds=args.ref_seconds)
            if i >= warmup:
                per.append(t)
        t = sum(per) / len(per)
        value = 1.0 / t
        sample = f"oracle (NumPy FP64) energy/gradient evaluations of the workload at its seeded point, {t:.2f} s each"
    else:
        flops_grad = args.ref_flops_per_grad or FLOPS_PER_GRAD[args.workload]
        for i in range(warmup + steps):
            t, n, layer, cf, cc, part = oracle_sample(d_b, chi, L, seconds=args.ref_seconds, seed=i, cplx=cplx)
            if i >= warmup:
                per.append(t)
        frac = part * ascend_flops(cf, cc) * (4 if cplx else 1) / flops_grad
        t = sum(per) / len(per)
        value = frac / t
        sample = (f"extrapolated: oracle (NumPy FP64) {'one side of the ' if part < 1 else ''}ascending map of "
                  f"layer {layer} (chi {cf}->{cc}), {t:.2f} s each = {frac:.3g} of one gradient evaluation's "
                  f"algorithmic flops ({flops_grad:.3g}), scaled by that fraction")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128" if cplx else "f64",
            "data": "synthetic", "config": {"workload": args.workload, "chi": chi, "n_trans": L},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": sample, "extrapolated": not whole_eval(args.workload)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def accuracy_probe(gm, prec, seed=0):
    """The workload's arithmetic against the FP64 oracle at a size the oracle
    evaluates in seconds: critical Ising, chi = 8, three transition layers, the
    seeded point; energy error (absolute and relative to max(1, |e|)) and the
    largest per-tensor relative error of the derivatives."""
    from oracle import mera as om
    us, ws = inp.random_mera(4, 8, 3, seed=seed)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    m = gm.Mera(gm.default_config(4, 8, 3, prec=prec), h3)
    m.set_tensors([t for p in zip(us, ws) for t in p])
    e, G, D = m.energy_grad(deriv=True)
    m.close()
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    return {"case": "critical Ising, chi=8, 3 transition layers, seeded point", "energy": e_ref,
            "energy_abs_error": abs(e - e_ref), "energy_rel_error": abs(e - e_ref) / max(1.0, abs(e_ref)),
            "deriv_rel_error_max": max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(D, ds))}


def serve_measure(n, chis, maxiter, workers, prec, seed):
    """Reduced serving stream through the native server (Poisson arrivals at
    50/s, Ising h ~ U[0.5,1.5] or XXZ Delta ~ U[0,2], chi drawn from `chis`,
    stop at |G| < 1e-6 or `maxiter` iterations), against the same stream
    solved one request at a time on the same GPU."""
    import torch
    from paper_2007_03638_gb300 import serve
    reqs = serve.poisson_stream(n, rate=50.0, chis=chis, seed=seed, prec=prec)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.8)
    warm = serve.poisson_stream(2, rate=1000.0, chis=chis[:1], seed=seed + 99, prec=prec)
    serve.run_stream(warm, budget, workers=2, maxiter=2)
    mixed = serve.run_stream(reqs, budget, workers=workers, maxiter=maxiter)
    seq = serve.run_sequential(reqs, maxiter=maxiter)
    same = all(a["iters"] == b_["iters"] and a["energy"] == b_["energy"]
               for a, b_ in zip(mixed["results"], seq["results"]))
    return {"metric": "serve solves/s", "value": mixed["solves_per_s"], "unit": "solves/s",
            "p50_latency_s": mixed["p50_latency_s"], "p99_latency_s": mixed["p99_latency_s"],
            "sequential": {"solves_per_s": seq["solves_per_s"], "p50_latency_s": seq["p50_latency_s"],
                           "p99_latency_s": seq["p99_latency_s"]},
            "same_results_alone_and_mixed": same,
            "batched_evaluations": sum(r["batched_evals"] for r in mixed["results"]),
            "evaluations": sum(r["n_evals"] for r in mixed["results"]),
            "iterations_total": sum(r["iters"] for r in mixed["results"]),
            "config": {"workload": "poisson_stream", "requests": n, "rate_per_s": 50.0, "chis": list(chis),
                       "maxiter": maxiter, "gtol": 1e-6, "prec": ["fp64", "3xtf32", "split_bf16", "split_fp16"][prec],
                       "workers": workers, "budget_bytes": budget},
            "deviation": (f"reduced stream: {n} requests, chi in {list(chis)}, at most {maxiter} iterations "
                          "(the full 512-request stream with chi up to 32 and 1000 iterations takes far more "
                          "than a bench run)")}


def run_serve(args):
    """The serving workload alone, as its own JSON line."""
    from paper_2007_03638_gb300 import build as b
    b.build()
    chis = tuple(int(x) for x in args.serve_chis.split(","))
    res = serve_measure(args.serve_n, chis, args.serve_maxiter, args.serve_workers, args.serve_prec, args.seed)
    line = {"metric": res.pop("metric"), "value": res.pop("value"), "unit": res.pop("unit"), "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic"}
    line.update(res)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--ref-flops-per-grad", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving workload: a seeded Poisson request stream through the native server, "
                         "against the same stream solved one request at a time")
    ap.add_argument("--serve-n", type=int, default=24)
    ap.add_argument("--serve-chis", default="4,8,12")
    ap.add_argument("--serve-maxiter", type=int, default=40)
    ap.add_argument("--serve-workers", type=int, default=12)
    ap.add_argument("--serve-prec", type=int, default=3, help="mixed mode of the served requests (see WORKLOADS)")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the reduced serving stream out of the default line")
    ap.add_argument("--energy-once", action="store_true",
                    help="set the seeded point, run one energy/gradient evaluation and exit (profiling case)")
    ap.add_argument("--shapes-out", default=None,
                    help="per-shape profile: from the seeded point, one evaluation (filling the Krylov warm "
                         "starts), then one L-BFGS iteration with the library's per-shape timing on; writes "
                         "that table (mera_profile_dump) as CSV to this path and exits")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args, wl)
        return
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera as gm

    kind, d_b, chi, L, prec, extra = wl
    net, cplx = extra.get("network", 0), extra.get("dtype", 0) == 1
    h3 = hamiltonian(kind, d_b, net, bool(extra.get("z2", 0)))
    stream = torch.cuda.current_stream()
    cfg = gm.default_config(d_b, chi, L, prec=prec, **extra)
    free0, _ = torch.cuda.mem_get_info()
    m = gm.Mera(cfg, h3, stream=stream.cuda_stream)
    point = initial_point(d_b, chi, L, extra, args.seed + rank)
    m.set_tensors(point)
    free1, _ = torch.cuda.mem_get_info()
    memory = {"device_bytes": int(free0 - free1), "footprint_bytes": gm.footprint_bytes(cfg)}
    if args.energy_once:
        print(json.dumps({"workload": args.workload, "energy": m.energy(), "launches": m.launch_count()}))
        return
    if args.shapes_out:
        m.energy_grad()
        m.stats(reset=True)
        m.profile(True)
        t0 = time.perf_counter()
        info = m.lbfgs_step()
        wall = time.perf_counter() - t0
        m.profile_dump(args.shapes_out)
        print(json.dumps({"workload": args.workload, "step_s": wall, "iter": info, "stats": m.stats()}))
        return
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        m.lbfgs_step()
    m.stats(reset=True)
    m.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    # nvidia-smi samples of the timed region: $MERA_BENCH_CLOCKS_DIR (kept) or a temporary directory
    clk_dir = os.environ.get("MERA_BENCH_CLOCKS_DIR") or tempfile.mkdtemp(prefix="mera_bench_clocks_")
    clk_path = os.path.join(clk_dir, f"clocks_rank{rank}.csv")
    os.makedirs(clk_dir, exist_ok=True)
    infos = []
    with Clocks(clk_path, local) as clocks:
        # named range: a profiler can select exactly the timed launches
        torch.cuda.nvtx.range_push("timed_steps")
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            infos.append(m.lbfgs_step())
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    m.profile(False)
    st = m.stats(reset=True)
    t_ms = sum(a.elapsed_time(b_) for a, b_ in ev)
    grads = st["energy_grad_calls"]
    t_ms, grads_all = aggregate(t_ms, grads, pg, "cuda")
    value = grads_all / (t_ms / 1e3)
    gett_flops_per_grad = st["gett_flops"] / max(1, grads)

    # end to end: the call a user makes per evaluation, host (pinned) tensors
    # in and the host gradient out.  The points are ones the optimisation
    # visits (recorded one L-BFGS iteration apart after the timed steps) and
    # are evaluated in reverse order, so each evaluation starts its Krylov
    # solves from the previous point's solutions, one iteration away, as the
    # evaluations inside the timed steps do.
    gout = [torch.empty(s, dtype=torch.complex128 if cplx else torch.float64).pin_memory() for s in m.shapes]
    big = chi >= 24
    n_e2e = 1 if big else max(2, args.steps)
    visited = []
    for _ in range(n_e2e + 1):
        visited.append([torch.from_numpy(np.ascontiguousarray(t)).pin_memory() for t in m.get_tensors()])
        m.lbfgs_step()
    visited.reverse()
    h2d = sum(t.numel() * t.element_size() for t in visited[0])
    d2h = sum(t.numel() * t.element_size() for t in gout) + 8
    m.set_tensors(visited[0])  # untimed warm-up call
    m.energy_grad_into(gout)
    m.stats(reset=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        m.set_tensors(visited[1 + k])
        m.energy_grad_into(gout)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    st_e2e = m.stats(reset=True)
    t_e2e, _ = aggregate(t_e2e, 0, pg, "cuda")
    e2e_value = world * n_e2e / t_e2e

    achieved = st["gett_flops"] / (st["gett_ms"] / 1e3) if st["gett_ms"] > 0 else None
    if prec == 0:
        peak, psrc, kname, bound = FP64_PEAK_FLOPS, "derived FP64 FMA rate (152 SMs x 2 FMA/clk x 2070 MHz)", \
            "gett_c128_kernel" if cplx else "gett_f64_kernel", "alu"
    else:
        peak, psrc = tensor_peaks()[prec]
        kname, bound = "tc_gemm_kernel (%s)" % {1: "3xTF32", 2: "split-BF16", 3: "split-FP16"}[prec], "tensor"
    roof = {"bound": bound, "kernel": kname, "achieved": achieved / 1e12 if achieved else None,
            "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "traffic": GETT_TRAFFIC_BYTES.get(args.workload),
            "peak_source": psrc,
            "flops_counted": "algorithmic 2*M*N*K per contraction (each split mode issues 3 tensor-core products per MAC)",
            "launches_timed": st["gett_timed"],
            "share_of_step": (st["gett_ms"] / t_ms) if t_ms > 0 else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("complex " if cplx else "") + ["f64", "tf32x3+f32acc (f64 Krylov/geometry)",
                                                     "bf16x3+f32acc (f64 Krylov/geometry)",
                                                     "fp16x3 scaled+f32acc (f64 Krylov/geometry)"][prec],
            "data": "synthetic",
            "config": {"workload": args.workload, "hamiltonian": kind, "d_b": d_b, "chi": chi,
                       "n_trans": L, "prec": ["fp64", "3xtf32", "split_bf16", "split_fp16"][prec],
                       "network": ["binary", "ternary", "mps"][net], "z2": bool(extra.get("z2", 0)),
                       "element": "complex128" if cplx else "float64",
                       "step": "one L-BFGS iteration (m=%d)" % extra.get("lbfgs_m", 8), "l2": "flushed (256 MiB write) between steps",
                       "parallelism": f"replicas x{world}"},
            "lbfgs_iters_per_s": world * args.steps / (t_ms / 1e3),
            "grad_evals_per_step": grads / args.steps,
            "krylov_matvecs_per_grad": st["krylov_matvecs"] / max(1, grads),
            "gett_gflop_per_grad": gett_flops_per_grad / 1e9,
            "energy_last": infos[-1]["energy"],
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": "mera_set_tensors(host) + mera_energy_grad(grad -> host)",
                    "evaluations": n_e2e,
                    "points": "visited by the optimisation, one L-BFGS iteration apart, in reverse order",
                    "krylov_matvecs_per_grad": st_e2e["krylov_matvecs"] / max(1, n_e2e)},
            "gpu_launches": st["launches"],
            "memory": memory,
            "clocks": clocks.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if whole_eval(args.workload):
            t, n = oracle_eval_sample(wl, seconds=args.cpu_seconds)
            line["cpu_baseline"] = {"value": 1.0 / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                                    "sample": f"{n} x oracle (NumPy FP64) energy/gradient evaluation of the "
                                              f"workload at its seeded point, {t:.2f} s each",
                                    "extrapolated": False}
        else:
            t, n, layer, cf, cc, part = oracle_sample(d_b, chi, L, seconds=args.cpu_seconds, cplx=cplx)
            # the oracle contracts densely: a Z2 workload's fraction is of the dense count
            per_grad = FLOPS_PER_GRAD[args.workload] if extra.get("z2") else gett_flops_per_grad
            frac = part * ascend_flops(cf, cc) * (4 if cplx else 1) / per_grad
            line["cpu_baseline"] = {"value": frac / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                                    "sample": f"extrapolated: {n} x oracle (NumPy FP64) "
                                              f"{'one side of the ' if part < 1 else ''}ascending map of layer "
                                              f"{layer} (chi {cf}->{cc}), {t:.2f} s each = {frac:.3g} of one "
                                              f"gradient evaluation's algorithmic flops, scaled by that fraction",
                                    "extrapolated": True}
    if rank == 0 and world == 1 and prec != 0:
        line["accuracy_vs_oracle"] = accuracy_probe(gm, prec, args.seed)
    if rank == 0 and world == 1 and not args.no_serve:
        # the serving workload (config 5) on the same GPU, bounded: the
        # problem above is released first
        m.close()
        del flush
        torch.cuda.empty_cache()
        chis = tuple(int(x) for x in args.serve_chis.split(","))
        line["serve"] = serve_measure(args.serve_n, chis, args.serve_maxiter, args.serve_workers, args.serve_prec,
                                      args.seed)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
