"""Uniform MPS (mera_config.network = MERA_MPS, Sec. 5) on the GPU against the
MPS oracle (oracle/mps.py), through the C ABI: energy per site, the partial
derivative D = 2 de/d conj(A) of Eq. mps_derivative and its Grassmann
projection at 1e-12 (real and complex, bond dimensions from 1 to 16, a ragged
physical dimension 3); the preconditioner X (rho + |G|^2 1)^(-1); the AKLT
state as an exact stationary point; L-BFGS on the gapped Ising chain to the
exact energy; the configurations the MPS path refuses."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mps as om
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


def _problem(gm, A, h, **kw):
    D, d, _ = A.shape
    dt = gm.MERA_C128 if np.iscomplexobj(A) else gm.MERA_F64
    m = gm.Mera(gm.default_config(d, D, 0, network=gm.MERA_MPS, dtype=dt, **kw), h)
    m.set_tensors([om.as_matrix(A)])
    return m


def _hermitian(n, seed, cplx):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    return 0.5 * (a + a.conj().T)


@pytest.mark.parametrize("D,d,cplx,seed", [(1, 2, False, 0), (5, 2, False, 1), (16, 2, False, 2),
                                           (7, 3, False, 3), (6, 2, True, 4), (9, 3, True, 5)])
def test_mps_energy_grad_parity(gm, D, d, cplx, seed):
    dt = np.complex128 if cplx else np.float64
    A = inp.random_mps(D, d, seed=seed, dtype=dt)
    h = _hermitian(d * d, seed + 100, cplx)
    m = _problem(gm, A, h)
    e, G, Dv = m.energy_grad(deriv=True)
    e_ref, D_ref, _ = om.energy_grad(A, h)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref)), (e, e_ref)
    Dm = om.as_matrix(D_ref)
    scale = max(np.abs(Dm).max(), 1.0)
    assert Dv[0].shape == Dm.shape
    assert np.abs(Dv[0] - Dm).max() < TOL * scale
    G_ref = geo.project(om.as_matrix(A), Dm, geo.GRASSMANN)
    assert np.abs(G[0] - G_ref).max() < TOL * scale
    assert abs(m.energy_only() - e_ref) <= TOL * max(1.0, abs(e_ref))


@pytest.mark.parametrize("cplx", [False, True])
def test_mps_preconditioner_parity(gm, cplx):
    dt = np.complex128 if cplx else np.float64
    D, d = 8, 2
    A = inp.random_mps(D, d, seed=21, dtype=dt)
    h = inp.ising_bond(1.0, 0.3).astype(dt)
    m = _problem(gm, A, h)
    _, G = m.energy_grad()
    _, _, rho = om.energy_grad(A, h)
    M = om.as_matrix(A)
    rng = np.random.default_rng(22)
    Z = rng.standard_normal(M.shape) + (1j * rng.standard_normal(M.shape) if cplx else 0)
    X = geo.project(M, Z, geo.GRASSMANN)
    delta = float(np.linalg.norm(G[0])) ** 2
    want = X @ np.linalg.inv(rho + delta * np.eye(D))
    got = m.precondition([X])[0]
    assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()


def test_mps_aklt_is_stationary(gm):
    A, h = inp.aklt_mps()
    m = _problem(gm, A, h)
    e, G = m.energy_grad()
    assert abs(e + 2.0 / 3.0) < 1e-13
    assert np.abs(G[0]).max() < 1e-12


def test_mps_geometry_keeps_the_point_isometric(gm):
    A = inp.random_mps(6, 2, seed=31)
    m = _problem(gm, A, inp.ising_bond(1.0))
    _, G = m.energy_grad()
    m.retract([-G[0]], 0.3)
    W = m.get_tensors()[0]
    assert np.abs(W.T @ W - np.eye(6)).max() < 1e-13


def test_mps_lbfgs_reaches_the_gapped_ising_energy(gm):
    """Same problem as the oracle's L-BFGS pin: h = 1.5, D = 6."""
    A = inp.random_mps(6, 2, seed=11)
    m = _problem(gm, A, inp.ising_bond(1.5))
    e = None
    for _ in range(150):
        info = m.lbfgs_step()
        e = info["energy"]
        if info["gnorm"] < 1e-9:
            break
    exact = inp.exact_ising_energy_per_spin(1.5)
    assert abs(e - exact) < 1e-7, (e, exact)


def test_mps_refusals(gm):
    A = inp.random_mps(4, 2, seed=41)
    h = inp.ising_bond(1.0)
    with pytest.raises(gm.MeraError) as ei:
        _problem(gm, A, h, prec=gm.PREC_3XTF32)
    assert ei.value.code == -8
    with pytest.raises(gm.MeraError) as ei:
        _problem(gm, A, h, w_stiefel=1)
    assert ei.value.code == -8
    m = _problem(gm, A, h)
    with pytest.raises(gm.MeraError) as ei:
        m.ev_sweep(2.0)
    assert ei.value.code == -8
