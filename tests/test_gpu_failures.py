"""Failure paths through the C ABI, each made on the host or by a bounded
device wait that is told to expire; no test faults, traps or hangs the GPU.

* a NaN in a host-side input (tensor, Hamiltonian term, retraction step)
  gives MERA_ERR_NONFINITE and leaves the point unchanged;
* a Krylov iteration cap too small to converge gives MERA_ERR_NOCONV;
* a device allocator that refuses memory gives MERA_ERR_OOM with nothing
  leaked, and the server defers a request whose creation ran out of memory
  while another ran, then solves it with the result it has alone;
* a tensor-core pipeline wait limit far below the kernel's latencies makes
  the kernel stop early: MERA_ERR_DEVICE_TIMEOUT, and with the limit restored
  the same object evaluates to the bit-identical result of a fresh one."""
import threading

import numpy as np
import pytest

from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu

NONFINITE, NOCONV, OOM, TIMEOUT = -3, -4, -2, -5


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera
    yield mera
    mera.set_allocator()


def _h3():
    return inp.three_site_blocked(inp.ising_bond(1.0))


def _point(chi, L, seed):
    us, ws = inp.random_mera(4, chi, L, seed=seed)
    return [t for p in zip(us, ws) for t in p]


def test_nonfinite_inputs(gm):
    pt = _point(4, 2, 0)
    m = gm.Mera(gm.default_config(4, 4, 2), _h3())
    m.set_tensors(pt)
    e0 = m.energy()
    bad = [t.copy() for t in pt]
    bad[2][1, 3] = np.nan
    with pytest.raises(gm.MeraError) as ei:
        m.set_tensors(bad)
    assert ei.value.code == NONFINITE
    bad[2][1, 3] = np.inf
    with pytest.raises(gm.MeraError) as ei:
        m.set_tensors(bad)
    assert ei.value.code == NONFINITE
    for a, b in zip(m.get_tensors(), pt):
        assert np.array_equal(a, b)
    # a NaN step is refused before the point moves
    e, G = m.energy_grad()
    step = [-g for g in G]
    step[1][0, 0] = np.nan
    with pytest.raises(gm.MeraError) as ei:
        m.retract(step, 0.1)
    assert ei.value.code == NONFINITE
    for a, b in zip(m.get_tensors(), pt):
        assert np.array_equal(a, b)
    assert m.energy() == e0
    h = _h3()
    h[5, 5] = np.nan
    with pytest.raises(gm.MeraError) as ei:
        gm.Mera(gm.default_config(4, 4, 2), h)
    assert ei.value.code == NONFINITE


def test_krylov_cap_gives_noconv(gm):
    pt = _point(4, 2, 1)
    m = gm.Mera(gm.default_config(4, 4, 2, krylov_dim=2, krylov_maxiter=2), _h3())
    m.set_tensors(pt)
    with pytest.raises(gm.MeraError) as ei:
        m.energy_grad()
    assert ei.value.code == NOCONV
    assert "GMRES" in str(ei.value)
    for a, b in zip(m.get_tensors(), pt):
        assert np.array_equal(a, b)
    with pytest.raises(gm.MeraError) as ei:
        m.lbfgs_step()
    assert ei.value.code == NOCONV


class _Bounded:
    """A device allocator with a byte limit (through the CUDA runtime of torch's
    caching allocator); counts live bytes."""

    def __init__(self, limit):
        import torch
        self.torch = torch
        self.limit, self.live, self.sizes, self.refused = limit, 0, {}, 0
        self.mu = threading.Lock()

    def alloc(self, n):
        with self.mu:
            if self.live + n > self.limit:
                self.refused += 1
                return 0
            p = self.torch.cuda.caching_allocator_alloc(n)
            self.live += n
            self.sizes[p] = n
            return p

    def free(self, p):
        with self.mu:
            self.live -= self.sizes.pop(p)
        self.torch.cuda.caching_allocator_delete(p)


def test_allocator_refusal_gives_oom(gm):
    cfg = gm.default_config(4, 8, 3)
    a = _Bounded(gm.footprint_bytes(cfg) // 4)
    gm.set_allocator(a.alloc, a.free)
    try:
        with pytest.raises(gm.MeraError) as ei:
            gm.Mera(cfg, _h3())
        assert ei.value.code == OOM
        assert a.refused >= 1 and a.live == 0  # what the failed creation had allocated is back
    finally:
        gm.set_allocator()
    pt = _point(8, 3, 2)
    ref = gm.Mera(cfg, _h3())
    ref.set_tensors(pt)
    e_ref, G_ref = ref.energy_grad()
    ref.close()
    # the same problem with all of its memory from torch's caching allocator
    gm.use_torch_allocator()
    try:
        m = gm.Mera(cfg, _h3())
        m.set_tensors(pt)
        e, G = m.energy_grad()
        m.close()
    finally:
        gm.set_allocator()
    assert e == e_ref
    for x, y in zip(G, G_ref):
        assert np.array_equal(x, y)


def test_server_defers_on_oom(gm):
    from paper_2007_03638_gb300 import serve
    cfg = gm.default_config(4, 8, 3, prec=gm.PREC_3XTF32)
    pts = [_point(8, 3, 10 + k) for k in range(2)]
    iters = 6
    # alone, through a counting allocator: the results and one problem's peak memory
    count = _Bounded(1 << 62)
    gm.set_allocator(count.alloc, count.free)
    alone, peak = [], 0
    try:
        for pt in pts:
            m = gm.Mera(cfg, _h3())
            m.set_tensors(pt)
            for _ in range(iters):
                info = m.lbfgs_step()
            peak = max(peak, count.live)
            alone.append(info["energy"])
            m.close()
    finally:
        gm.set_allocator()
    assert count.live == 0 and peak > 0
    # one problem's memory fits under the limit, two do not: the request whose
    # creation comes second runs out of memory and waits for the first
    a = _Bounded(int(1.5 * peak))
    gm.set_allocator(a.alloc, a.free)
    try:
        sv = serve.Server(4 * gm.footprint_bytes(cfg), workers=2)
        ids = [sv.submit(cfg, _h3(), pt, maxiter=iters, gtol=0.0) for pt in pts]
        sv.wait(600)
        st = [sv.poll(i) for i in ids]
        sv.close()
    finally:
        gm.set_allocator()
    assert all(s["state"] == 2 for s in st), st
    assert sum(s["deferred"] for s in st) >= 1 and a.refused >= 1
    for s, e in zip(st, alone):
        assert s["iters"] == iters and s["energy"] == e
    assert a.live == 0


@pytest.mark.parametrize("prec", [1, 2])
def test_device_wait_expiry(gm, prec):
    cfg = gm.default_config(4, 8, 3, prec=prec)
    pt = _point(8, 3, 4)
    ref = gm.Mera(cfg, _h3())
    ref.set_tensors(pt)
    e_ref, G_ref = ref.energy_grad()
    ref.close()
    m = gm.Mera(cfg, _h3())
    m.set_tensors(pt)
    m.set_device_wait(1e-9)
    with pytest.raises(gm.MeraError) as ei:
        m.energy_grad()
    assert ei.value.code == TIMEOUT
    for a, b in zip(m.get_tensors(), pt):
        assert np.array_equal(a, b)
    m.set_device_wait(1.0)
    e, G = m.energy_grad()
    assert e == e_ref
    for x, y in zip(G, G_ref):
        assert np.array_equal(x, y)
    with pytest.raises(gm.MeraError):
        m.set_device_wait(0.0)
