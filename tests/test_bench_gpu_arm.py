"""bench.py's own arm without a GPU: the device layer (torch.cuda streams,
events, pinned memory) and the library object are replaced by host stand-ins
that return fixed counters, so that the arm's control flow and the JSON line it
assembles (the keys of the benchmark contract, the roofline and CPU-baseline
objects, the end-to-end and clock records) are checked on the CPU for every
workload family.  The numbers are meaningless here; the GPU runs measure."""
import json
import sys
import time

import numpy as np
import pytest

import bench
from paper_2007_03638_gb300 import mera as gm


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return 1e3 * (other.t - self.t) + 1.0


class _Stream:
    cuda_stream = 0


class _Mera:
    """Stands in for paper_2007_03638_gb300.mera.Mera: shapes from the config,
    fixed counters per L-BFGS step."""

    def __init__(self, cfg, h3, stream=None):
        self.cfg = cfg
        self.grads = 0
        if cfg.network == gm.MERA_MPS:
            self.shapes = [(cfg.chi * cfg.d_b, cfg.chi)]
        else:
            from paper_2007_03638_gb300 import inputs as inp
            tern = cfg.network == gm.MERA_TERNARY
            dims = (inp.ternary_layer_dims if tern else inp.layer_dims)(cfg.d_b, cfg.chi, cfg.n_trans)
            self.shapes = []
            for l in range(cfg.n_trans + 1):
                cf, cc = dims[l], dims[min(l + 1, cfg.n_trans)]
                self.shapes += [(cf * cf, cf * cf), (cf ** (3 if tern else 2), cc)]
        self.dtype = np.complex128 if cfg.dtype == gm.MERA_C128 else np.float64

    def set_tensors(self, tensors):
        assert [tuple(np.shape(t)) for t in tensors] == self.shapes

    def energy(self):
        self.grads += 1
        return -0.5

    def lbfgs_step(self):
        self.grads += 3
        return {"iter": 1, "energy": -0.6, "gnorm": 0.1, "alpha": 1.0, "n_evals": 3, "ls_ok": 1, "krylov_matvecs": 9}

    def stats(self, reset=False):
        st = {"launches": 1000, "gett_launches": 400, "gett_flops": 1e9 * max(1, self.grads), "gett_timed": 400,
              "gett_ms": 0.5, "energy_grad_calls": max(1, self.grads), "krylov_matvecs": 9}
        if reset:
            self.grads = 0
        return st

    def profile(self, enable=True):
        pass

    def get_tensors(self, device=False):
        return [np.zeros(s, dtype=self.dtype) for s in self.shapes]

    def energy_grad_into(self, G):
        return -0.5

    def launch_count(self):
        return 0

    def close(self):
        pass


@pytest.fixture
def fake_device(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: _Stream())
    free = iter([10 * 2**30, 7 * 2**30] * 4)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (next(free), 16 * 2**30))
    monkeypatch.setattr(torch.cuda.nvtx, "range_push", lambda *a: None)
    monkeypatch.setattr(torch.cuda.nvtx, "range_pop", lambda *a: None)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: empty(*a, **k))
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(gm, "Mera", _Mera)
    # the oracle comparison evaluates on the GPU: a stand-in here
    monkeypatch.setattr(bench, "accuracy_probe", lambda gm_, prec, seed=0: {
        "energy_abs_error": 1e-7, "energy_rel_error": 1e-7, "deriv_rel_error_max": 1e-5})
    # the serving stream needs the native server: its summary is a stand-in here
    monkeypatch.setattr(bench, "serve_measure", lambda n, chis, maxiter, workers, prec, seed: {
        "metric": "serve solves/s", "value": 1.0, "unit": "solves/s", "p50_latency_s": 0.5, "p99_latency_s": 0.9,
        "sequential": {"solves_per_s": 0.5}, "same_results_alone_and_mixed": True, "batched_evaluations": 3,
        "deviation": "stand-in", "config": {"requests": n, "chis": list(chis)}})


CONTRACT = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks")


@pytest.mark.parametrize("workload", ["ising_chi4_L2_fp64", "ising_chi12_L3_bf16", "ising_chi12_L3_fp16",
                                      "ternary_ising_chi8_L2_fp64_z2",
                                      "mps_xxz_D32_fp64", "ising_hz_chi8_L3_c128_fp64",
                                      "ising_chi16_L3_3xtf32_z2"])
def test_gpu_arm_line(fake_device, monkeypatch, capsys, workload):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", workload, "--steps", "2", "--warmup", "3",
                                      "--cpu-seconds", "0.1"])
    kind, d_b, chi, L, prec, extra = bench.WORKLOADS[workload]
    if extra.get("network", 0) == 0 and chi > 8:
        # a whole binary oracle evaluation at chi = 12 takes tens of seconds on
        # the CPU: its timing is replaced (the control flow is what is checked)
        monkeypatch.setattr(bench, "oracle_eval_sample", lambda wl, seconds=10.0, seed=0: (30.0, 1))
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in CONTRACT:
        assert k in line, k
    assert line["config"]["workload"] == workload and line["steps"] == 2 and line["warmup"] == 3
    extra = bench.WORKLOADS[workload][5]
    assert line["config"]["network"] == ["binary", "ternary", "mps"][extra.get("network", 0)]
    assert line["config"]["z2"] == bool(extra.get("z2", 0))
    assert line["config"]["element"] == ("complex128" if extra.get("dtype", 0) else "float64")
    assert line["n_gpus"] == 1 and line["scaling"] == "weak" and line["higher_is_better"] is True
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert line["roofline"]["frac"] == pytest.approx(line["roofline"]["achieved"] / line["roofline"]["peak"])
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"], k
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["extrapolated"] == (not bench.whole_eval(workload))
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    assert line["e2e"]["h2d_bytes_per_step"] > 0
    assert line["e2e"]["evaluations"] >= 1 and line["e2e"]["krylov_matvecs_per_grad"] >= 0
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in line["clocks"], k
    assert line["memory"]["device_bytes"] == 3 * 2**30 and line["memory"]["footprint_bytes"] > 0
    for k in ("value", "p50_latency_s", "p99_latency_s", "sequential", "same_results_alone_and_mixed", "deviation"):
        assert k in line["serve"], k
    assert ("accuracy_vs_oracle" in line) == (bench.WORKLOADS[workload][4] != 0)
