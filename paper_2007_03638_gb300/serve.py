"""Serving many MERA optimisations on one GPU (binding of mera_server_*).

``Server`` wraps the library's native scheduler: requests are admitted by
device footprint, each keeps its state on the device on its own stream,
worker threads interleave their iterations, and the energy/gradient
evaluations of same-configuration requests run together as batched launches.  ``poisson_stream`` builds the
seeded request stream of the serving workload (Ising with transverse field
h ~ U[0.5, 1.5] or XXZ with Delta ~ U[0, 2], bond dimension drawn from a set,
exponential inter-arrival gaps); ``run_stream`` replays it in real time and
reports solves/s and latency percentiles; ``run_sequential`` is the same
stream solved one request at a time on the same GPU.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import inputs as inp
from . import mera as gm


def request_sizes(cfg):
    """Elements of the Hamiltonian term and of each tensor that
    mera_server_submit copies for this config: the level dimensions
    chi_{l+1} = min(chi, chi_l^2) (binary) or min(chi, chi_l^3) (ternary) from
    chi_0 = d_b, the scale-invariant layer keeping the last one."""
    tern = cfg.network == gm.MERA_TERNARY
    n_op = int(cfg.d_b) ** (2 if tern else 3)
    dims = [int(cfg.d_b)]
    for _ in range(int(cfg.n_trans)):
        dims.append(min(int(cfg.chi), dims[-1] ** (3 if tern else 2)))
    sizes = []
    for l in range(int(cfg.n_trans) + 1):
        cf = dims[l]
        cc = dims[l + 1] if l < cfg.n_trans else dims[l]
        sizes += [cf ** 4, (cf ** 3 if tern else cf ** 2) * cc]
    return n_op * n_op, sizes


def check_request(cfg, h3, tensors):
    """Refuses a request whose arrays are shorter or longer than what the
    library copies from them (it reads that many elements behind each
    pointer).  MPS requests are left to the library, which refuses them."""
    if cfg.network == gm.MERA_MPS:
        return
    n_h, sizes = request_sizes(cfg)
    if int(np.size(h3)) != n_h:
        raise ValueError(f"the Hamiltonian term has {np.size(h3)} elements, expected {n_h}")
    if len(tensors) != len(sizes):
        raise ValueError(f"expected {len(sizes)} tensors, got {len(tensors)}")
    for i, (t, n) in enumerate(zip(tensors, sizes)):
        if gm._numel(t) != n:
            raise ValueError(f"tensor {i} has {gm._numel(t)} elements, expected {n}")


class Server:
    def __init__(self, budget_bytes: int, workers: int = 4):
        self.L = gm.load()
        h = C.c_void_p()
        rc = self.L.mera_server_create(int(budget_bytes), int(workers), C.byref(h))
        if rc != 0:
            raise gm.MeraError(rc, self.L.mera_strerror(rc).decode())
        self.h = h

    def submit(self, cfg, h3, tensors, method=0, gtol=1e-6, maxiter=100) -> int:
        keep = []
        rid = C.c_int64()
        dt = np.complex128 if cfg.dtype == gm.MERA_C128 else np.float64
        h3 = np.ascontiguousarray(h3, dtype=dt)
        check_request(cfg, h3, tensors)
        rc = self.L.mera_server_submit(self.h, C.byref(cfg), C.c_void_p(h3.ctypes.data),
                                       gm._ptrs(tensors, keep, dt), int(method), float(gtol), int(maxiter),
                                       C.byref(rid))
        if rc != 0:
            raise gm.MeraError(rc, self.L.mera_strerror(rc).decode())
        return rid.value

    def poll(self, rid):
        st = gm.RequestStatus()
        rc = self.L.mera_server_poll(self.h, int(rid), C.byref(st))
        if rc != 0:
            raise gm.MeraError(rc, self.L.mera_strerror(rc).decode())
        return {f: getattr(st, f) for f, _ in gm.RequestStatus._fields_}

    def wait(self, timeout=3600.0):
        rc = self.L.mera_server_wait(self.h, float(timeout))
        if rc != 0:
            raise gm.MeraError(rc, "requests still running after the timeout")

    def close(self):
        if getattr(self, "h", None):
            self.L.mera_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_stream(n, rate=50.0, chis=(4, 8, 12, 16, 24, 32), n_trans=2, prec=1, seed=0):
    """Seeded request stream: list of dicts with arrival time, model, config,
    Hamiltonian term and starting tensors."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        chi = int(rng.choice(chis))
        if rng.random() < 0.5:
            model, par = "ising", float(rng.uniform(0.5, 1.5))
            h3 = inp.three_site_blocked(inp.ising_bond(par))
        else:
            model, par = "xxz", float(rng.uniform(0.0, 2.0))
            h3 = inp.three_site_blocked(inp.xxz_bond(par))
        us, ws = inp.random_mera(4, chi, n_trans, seed=int(rng.integers(1 << 31)))
        extra = {"krylov_dim": 4} if chi >= 32 else {}
        out.append({"i": i, "t": t, "model": model, "param": par, "chi": chi, "h3": h3,
                    "tensors": [x for p in zip(us, ws) for x in p],
                    "cfg": (4, chi, n_trans, prec, extra)})
    return out


def _cfg(spec):
    d_b, chi, n_trans, prec, extra = spec
    return gm.default_config(d_b, chi, n_trans, prec=prec, **extra)


def _summary(lat, wall, results):
    lat = np.array(lat)
    return {"solves": len(lat), "wall_s": wall, "solves_per_s": len(lat) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "results": results}


def run_stream(reqs, budget_bytes, workers=4, gtol=1e-6, maxiter=100, timeout=3600.0):
    """Replay the stream in real time through the native server."""
    sv = Server(budget_bytes, workers)
    ids = []
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        ids.append(sv.submit(_cfg(r["cfg"]), r["h3"], r["tensors"], gtol=gtol, maxiter=maxiter))
    sv.wait(timeout)
    wall = time.perf_counter() - t0
    res = [sv.poll(i) for i in ids]
    sv.close()
    lat = [x["t_done"] - x["t_submit"] for x in res]
    return _summary(lat, wall, [{k: x[k] for k in ("state", "iters", "energy", "gnorm", "error", "message",
                                                    "batched_evals", "n_evals")}
                                for x in res])


def run_sequential(reqs, gtol=1e-6, maxiter=100):
    """The same stream, one request at a time on the same GPU (arrival order)."""
    t0 = time.perf_counter()
    lat, results = [], []
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        m = gm.Mera(_cfg(r["cfg"]), r["h3"])
        m.set_tensors(r["tensors"])
        out = m.solve(maxiter=maxiter, gtol=gtol)
        m.close()
        done = time.perf_counter() - t0
        lat.append(done - r["t"])
        results.append({"state": 2, "iters": out["iters"], "energy": out["energy"], "gnorm": out["gnorm"]})
    return _summary(lat, time.perf_counter() - t0, results)
