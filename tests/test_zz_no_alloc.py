"""The allocation-free dot-product entry point (mera_dots_noalloc) against the
library's regular inner product (mera_inner), through the C ABI, on two calls
in a row.

mera_dots_noalloc exists for callers that cannot allocate device memory (a
host application that owns all GPU memory and offers no allocator, or code
that must not trigger cudaMalloc's device synchronisation): it needs no
mera_t and keeps its partial sums in a fixed device array inside the library.
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera as gm
    return torch, gm


def test_dots_noalloc_matches_inner(env):
    torch, gm = env
    us, ws = inp.random_mera(4, 4, 2, seed=3)
    m = gm.Mera(gm.default_config(4, 4, 2), inp.three_site_blocked(inp.ising_bond()))
    m.set_tensors([t for p in zip(us, ws) for t in p])
    rng = np.random.default_rng(0)
    k = 5
    Xs = [[rng.standard_normal(s) for s in m.shapes] for _ in range(k)]
    Y = [rng.standard_normal(s) for s in m.shapes]
    ref = np.array([m.inner(X, Y) for X in Xs])
    n = sum(a.size for a in Y)
    Xdev = torch.from_numpy(np.stack([np.concatenate([a.ravel() for a in X]) for X in Xs])).cuda()
    ydev = torch.from_numpy(np.concatenate([a.ravel() for a in Y])).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = np.full(k, np.nan)
        gm.dots_noalloc(Xdev, ydev, k, n, n, out, stream)
        assert np.all(np.abs(out - ref) <= TOL * np.maximum(1.0, np.abs(ref))), (call, out, ref)
    # device output and a single vector
    out_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    gm.dots_noalloc(Xdev[2], ydev, 1, n, n, out_dev, stream)
    assert abs(out_dev.item() - ref[2]) <= TOL * max(1.0, abs(ref[2]))


def test_dots_noalloc_rejects_too_many_vectors(env):
    torch, gm = env
    x = torch.zeros(33 * 8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = np.zeros(33)
    with pytest.raises(gm.MeraError) as ex:
        gm.dots_noalloc(x, y, 33, 8, 8, out, 0)
    assert ex.value.code == -1
