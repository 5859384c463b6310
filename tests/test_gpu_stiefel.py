"""Isometries on the Stiefel manifold (mera_config.w_stiefel = 1) on the GPU
against the oracle's geometry (Sec. 2.3): the Stiefel projection, the
retraction e^{alpha Q_X} W and the transport e^{alpha Q_X} Y of non-square
isometries (computed on the span of W and an orthonormal basis of
(1 - W W^dag) X, the construction the paper describes), the preconditioner's
Stiefel form, and L-BFGS following the oracle's trajectory; real and
complex."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
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


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


@pytest.mark.parametrize("cplx", [False, True])
def test_stiefel_geometry_parity(gm, cplx):
    dt = np.complex128 if cplx else np.float64
    us, ws = inp.random_mera(4, 4, 2, seed=12, dtype=dt)
    pt = _flat(us, ws)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0, 0.2)).astype(dt)
    m = gm.Mera(gm.default_config(4, 4, 2, w_stiefel=1, dtype=gm.MERA_C128 if cplx else gm.MERA_F64), h3)
    m.set_tensors(pt)
    rng = np.random.default_rng(3)

    def rnd(shape):
        return rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0)

    X = [geo.project(W, rnd(W.shape), geo.STIEFEL) for W in pt]
    Y = [geo.project(W, rnd(W.shape), geo.STIEFEL) for W in pt]
    assert all(np.abs(a - geo.project(W, x, geo.STIEFEL)).max() < 1e-13
               for a, W, x in zip(m.project(X), pt, X))
    alpha = 0.4
    for W, x, y, ty in zip(pt, X, Y, m.transport(X, alpha, Y)):
        assert np.abs(ty - geo.transport(W, x, alpha, y)).max() < 1e-12
    e, G = m.energy_grad()
    e_ref, ds, info = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) < 1e-12 * max(1.0, abs(e_ref))
    for W, d, g in zip(pt, ds, G):
        assert np.abs(g - geo.project(W, d, geo.STIEFEL)).max() < 1e-12 * max(1.0, np.abs(d).max())
    rv = om.tensor_density_matrices(info["rho"], ws)
    deltas = [float(np.linalg.norm(geo.project(W, d, geo.STIEFEL))) for W, d in zip(pt, ds)]
    for W, x, r, dl, xt in zip(pt, X, rv, deltas, m.precondition(X)):
        ref = geo.precondition(W, x, r, dl, geo.STIEFEL)
        assert np.abs(xt - ref).max() < 1e-11 * max(1, np.abs(ref).max())
    Xp = m.retract(X, alpha, want_xprime=True)
    for W, x, wn, xp in zip(pt, X, m.get_tensors(), Xp):
        assert np.abs(wn - geo.polar(geo.retract(W, x, alpha))).max() < 1e-12
        assert np.abs(xp - geo.transport(W, x, alpha, x)).max() < 1e-12
        assert np.abs(wn.conj().T @ wn - np.eye(wn.shape[1])).max() < 1e-14


def test_stiefel_lbfgs_follows_oracle(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=13)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    m = gm.Mera(gm.default_config(4, 4, 2, w_stiefel=1), h3)
    m.set_tensors(_flat(us, ws))
    got = [m.lbfgs_step()["energy"] for _ in range(6)]
    _, _, hist = oo.lbfgs(oo.MeraProblem(h3, w_stiefel=True), _flat(us, ws), m=8, maxiter=7)
    ref = [h["energy"] for h in hist[1:7]]
    for g, r in zip(got, ref):
        assert abs(g - r) < 1e-9 * abs(r), (g, r)
