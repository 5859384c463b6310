"""Ternary MERA (mera_config.network = MERA_TERNARY) on the GPU against the
ternary oracle (oracle/ternary.py), through the C ABI: energy per site and
every partial derivative D_v = 2 dC/d conj(v) at 1e-12 (FP64, real and
complex), within the mixed-precision bound for 3xTF32; the preconditioner
with the ternary density matrices; L-BFGS and Evenbly-Vidal sweeps descend."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import ternary as ot
from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cfg(gm, chi, L, **kw):
    return gm.default_config(2, chi, L, network=gm.MERA_TERNARY, **kw)


@pytest.mark.parametrize("chi,L,seed", [(4, 1, 0), (8, 1, 1)])
def test_ternary_energy_grad_parity(gm, chi, L, seed):
    h = inp.ising_bond(1.0)
    us, ws = inp.random_ternary_mera(2, chi, L, seed=seed)
    m = gm.Mera(_cfg(gm, chi, L), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref)), (e, e_ref)
    pt = _flat(us, ws)
    for i, (W, d_ref) in enumerate(zip(pt, ds)):
        assert D[i].shape == d_ref.shape
        assert _rel(D[i], d_ref) < TOL, (i, _rel(D[i], d_ref))
        k = geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN
        assert np.abs(G[i] - geo.project(W, d_ref, k)).max() < TOL * np.abs(d_ref).max(), i


def test_ternary_complex_parity(gm):
    X, Y = inp.PAULI_X, inp.PAULI_Y
    h = inp.xxz_bond(0.5).astype(np.complex128) + 0.7 * (np.kron(X, Y) - np.kron(Y, X))
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=2, dtype=np.complex128)
    m = gm.Mera(_cfg(gm, 4, 1, dtype=gm.MERA_C128), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref))
    for i, d_ref in enumerate(ds):
        assert _rel(D[i], d_ref) < TOL, (i, _rel(D[i], d_ref))


def test_ternary_mixed_precision(gm):
    """3xTF32 tensor-core contractions, FP64 Krylov and reductions."""
    h = inp.ising_bond(1.0)
    us, ws = inp.random_ternary_mera(2, 8, 1, seed=4)
    m = gm.Mera(_cfg(gm, 8, 1, prec=1), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) / max(1.0, abs(e_ref)) < 2e-6
    assert max(_rel(D[i], ds[i]) for i in range(len(ds))) < 2e-5


def test_ternary_lbfgs_and_ev_descend(gm):
    h = inp.ising_bond(1.0)
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=5)
    m = gm.Mera(_cfg(gm, 4, 1), h)
    m.set_tensors(_flat(us, ws))
    e0 = m.energy()
    es = [m.lbfgs_step()["energy"] for _ in range(8)]
    assert es[-1] < e0 - 1e-2
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))
    gamma = float(np.linalg.eigvalsh(h).max()) + 0.5
    m.set_tensors(_flat(us, ws))
    ev = [m.ev_sweep(gamma)["energy"] for _ in range(3)]
    assert ev[0] < e0 and all(b < a for a, b in zip(ev, ev[1:]))
    for t in m.get_tensors():
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-12


@pytest.mark.parametrize("dt", [np.float64, np.complex128])
def test_ternary_preconditioner_parity(gm, dt):
    """Eq. preconditioner with the ternary density matrices (rho_w the
    one-site marginal, rho_u the state on a u's isometry outputs) against the
    oracle's, delta_v = |G_v|."""
    if dt == np.complex128:
        X, Y = inp.PAULI_X, inp.PAULI_Y
        h = inp.xxz_bond(0.5).astype(np.complex128) + 0.7 * (np.kron(X, Y) - np.kron(Y, X))
        m = gm.Mera(_cfg(gm, 4, 1, dtype=gm.MERA_C128), h)
    else:
        h = inp.ising_bond(1.0)
        m = gm.Mera(_cfg(gm, 4, 1), h)
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=7, dtype=dt)
    pt = _flat(us, ws)
    m.set_tensors(pt)
    m.energy_grad()
    e_ref, ds, info = ot.energy_grad(h, us, ws)
    rv = ot.tensor_density_matrices(info["rho"], ws)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    Gr = [geo.project(W, d, k) for W, d, k in zip(pt, ds, kinds)]
    deltas = [float(np.linalg.norm(g)) for g in Gr]
    rng = np.random.default_rng(3)
    Xs = []
    for W, k in zip(pt, kinds):
        Z = rng.standard_normal(W.shape) + (1j * rng.standard_normal(W.shape) if dt == np.complex128 else 0)
        Xs.append(geo.project(W, Z, k))
    Xt = m.precondition(Xs)
    for W, x, r, dl, k, xt in zip(pt, Xs, rv, deltas, kinds, Xt):
        ref = geo.precondition(W, x, r, dl, k)
        assert np.abs(xt - ref).max() < 1e-11 * max(1, np.abs(ref).max())
