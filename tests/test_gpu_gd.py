"""Riemannian gradient descent (mera_gd_step, Sec. 3) on the GPU against the
oracle's (oracle.optim.gd): the same iterates' energies on the config-1
shapes, descent, isometry kept; mera_solve with method 2."""
import numpy as np
import pytest

from oracle import optim as oo
from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera
    return mera


def test_gd_follows_the_oracle(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=0)
    pt = [t for p in zip(us, ws) for t in p]
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    m = gm.Mera(gm.default_config(4, 4, 2), h3)
    m.set_tensors(pt)
    got = [m.gd_step()["energy"] for _ in range(6)]
    _, _, hist = oo.gd(oo.MeraProblem(h3), pt, maxiter=7)
    ref = [h["energy"] for h in hist[1:7]]
    for g, r in zip(got, ref):
        assert abs(g - r) < 1e-9 * abs(r), (g, r)
    for t in m.get_tensors():
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-13


def test_solve_with_gradient_descent(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=1)
    m = gm.Mera(gm.default_config(4, 4, 2), inp.three_site_blocked(inp.ising_bond(1.0)))
    m.set_tensors([t for p in zip(us, ws) for t in p])
    e0 = m.energy()
    r = m.solve(maxiter=5, gtol=1e-12, method=2)
    assert r["iters"] == 5 and r["energy"] < e0
