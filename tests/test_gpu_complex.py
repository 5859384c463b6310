"""Complex tensors (MERA_C128, FP64 path) against the CPU FP64 oracle,
element by element, through the C ABI.  A complex Hermitian Hamiltonian
(an XXZ chain with a Dzyaloshinskii-Moriya term, whose matrix elements are
imaginary, or a random Hermitian 3-site term) and complex Haar-like
isometries, so that every conjugation on the bra side of the network
(Sec. 2.3), every conjugate transpose in the geometry (Sec. 3) and the
Hermitian eigenproblems of the preconditioner are exercised.  Tolerance:
1e-12 relative, as for the real FP64 path."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
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


def _dm_bond(dm=0.7):
    """XXZ bond plus dm (X Y - Y X): Hermitian with imaginary off-diagonal elements."""
    X, Y = inp.PAULI_X, inp.PAULI_Y
    return inp.xxz_bond(0.5).astype(np.complex128) + dm * (np.kron(X, Y) - np.kron(Y, X))


def _ham(d_b, kind, seed):
    if kind == "dm":
        b = _dm_bond()
        return inp.three_site_blocked(b) if d_b == 4 else inp.three_site_unblocked(b)
    rng = np.random.default_rng(seed)
    n = d_b**3
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (a + a.conj().T)


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _kinds(n):
    return [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(n)]


CASES = [
    (4, 4, 2, "dm", 0),      # blocked spin-1/2 chain, dims 4,4,4
    (2, 3, 2, "dm", 1),      # unblocked, ragged tiles: dims 2,3,3
    (3, 5, 2, "random", 2),  # odd dims 3,5,5, random Hermitian term
]


@pytest.mark.parametrize("d_b,chi,L,kind,seed", CASES)
def test_energy_grad_parity_complex(gm, d_b, chi, L, kind, seed):
    us, ws = inp.random_mera(d_b, chi, L, seed=seed, dtype=np.complex128)
    h3 = _ham(d_b, kind, seed)
    m = gm.Mera(gm.default_config(d_b, chi, L, dtype=gm.MERA_C128), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    assert G[0].dtype == np.complex128
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref)), (e, e_ref)
    pt = _flat(us, ws)
    for i, (W, d_ref, k) in enumerate(zip(pt, ds, _kinds(len(pt)))):
        assert _rel(D[i], d_ref) < TOL, (i, _rel(D[i], d_ref))
        g_ref = geo.project(W, d_ref, k)
        assert np.abs(G[i] - g_ref).max() < TOL * np.abs(d_ref).max(), i
    # the imaginary parts carry weight: dropping them changes the energy
    m_re = gm.Mera(gm.default_config(d_b, chi, L, dtype=gm.MERA_C128), h3.real.astype(np.complex128))
    m_re.set_tensors(_flat(us, ws))
    assert abs(m_re.energy() - e) > 1e-6


def test_real_data_through_complex_path(gm):
    """A real problem run as complex gives the real path's numbers."""
    us, ws = inp.random_mera(4, 4, 2, seed=3)
    h3 = inp.three_site_blocked(inp.ising_bond(1.0, 0.3))
    mr = gm.Mera(gm.default_config(4, 4, 2), h3)
    mr.set_tensors(_flat(us, ws))
    er, Gr = mr.energy_grad()
    mc = gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128), h3.astype(np.complex128))
    mc.set_tensors([t.astype(np.complex128) for t in _flat(us, ws)])
    ec, Gc = mc.energy_grad()
    assert abs(ec - er) < 1e-13 * abs(er)
    for a, b in zip(Gc, Gr):
        assert np.abs(a.imag).max() < 1e-14
        assert np.abs(a.real - b).max() < 1e-12 * max(1.0, np.abs(b).max())


def test_geometry_parity_complex(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=7, dtype=np.complex128)
    pt = _flat(us, ws)
    h3 = _ham(4, "dm", 0)
    m = gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128), h3)
    m.set_tensors(pt)
    rng = np.random.default_rng(1)
    kinds = _kinds(len(pt))

    def crandn(shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    Draw = [crandn(t.shape) for t in pt]
    X = m.project(Draw)
    X_ref = [geo.project(W, d, k) for W, d, k in zip(pt, Draw, kinds)]
    for a, b in zip(X, X_ref):
        assert np.abs(a - b).max() < 1e-13
    Y = [geo.project(W, crandn(W.shape), k) for W, k in zip(pt, kinds)]
    ip = geo.inner(X_ref, Y)
    assert abs(m.inner(X, Y) - ip) < 1e-12 * abs(ip)
    alpha = 0.3
    TY = m.transport(X_ref, alpha, Y)
    for W, x, y, ty in zip(pt, X_ref, Y, TY):
        assert np.abs(ty - geo.transport(W, x, alpha, y)).max() < 1e-12
    e, G = m.energy_grad()
    e_ref, ds, info = om.energy_grad(h3, us, ws)
    rv = om.tensor_density_matrices(info["rho"], ws)
    Gr = [geo.project(W, d, k) for W, d, k in zip(pt, ds, kinds)]
    deltas = [float(np.linalg.norm(g)) for g in Gr]
    Xt = m.precondition(X_ref)
    for W, x, r, dl, k, xt in zip(pt, X_ref, rv, deltas, kinds, Xt):
        ref = geo.precondition(W, x, r, dl, k)
        assert np.abs(xt - ref).max() < 1e-11 * max(1, np.abs(ref).max())
    Xp = m.retract(X_ref, alpha, want_xprime=True)
    Wn = m.get_tensors()
    for W, x, wn, xp in zip(pt, X_ref, Wn, Xp):
        assert np.abs(wn - geo.polar(geo.retract(W, x, alpha))).max() < 1e-12
        assert np.abs(xp - geo.transport(W, x, alpha, x)).max() < 1e-12
        assert np.abs(wn.conj().T @ wn - np.eye(wn.shape[1])).max() < 1e-14


def test_lbfgs_complex_descends(gm):
    us, ws = inp.random_mera(4, 4, 2, seed=4, dtype=np.complex128)
    m = gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128), _ham(4, "dm", 0))
    m.set_tensors(_flat(us, ws))
    e0 = m.energy()
    es = [m.lbfgs_step()["energy"] for _ in range(6)]
    assert es[-1] < e0 - 1e-3
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))
    for t in m.get_tensors():
        assert np.abs(t.conj().T @ t - np.eye(t.shape[1])).max() < 1e-13
