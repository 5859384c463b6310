"""Complex tensors in the mixed-precision modes (MERA_C128 with 3xTF32 or
split-BF16 contractions): each complex product runs as four real tensor-core
products of the real views (Re C = Re A Re B - Im A Im B, Im C = Re A Im B +
Im A Re B, conjugated bra leaves by sign), FP64 Krylov solves and geometry.
Against the complex FP64 oracle within the bounds of the real mixed-precision
tests (energy 2e-6 / 2e-4 relative, derivatives 10x that), for the binary
network (also with the sliced chain) and the ternary one; a central difference
of the energy along the retraction matches Re <G, X>."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
from oracle import ternary as ot
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


def _dm_bond(dm=0.7):
    X, Y = inp.PAULI_X, inp.PAULI_Y
    return inp.xxz_bond(0.5).astype(np.complex128) + dm * (np.kron(X, Y) - np.kron(Y, X))


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [  # prec, tol, chi, n_trans, b_chunk, seed
    (1, 2e-6, 4, 2, 0, 0),
    (2, 2e-4, 4, 2, 0, 1),
    (1, 2e-6, 8, 3, 4, 2),  # the chi^9 chain sliced over b (4 values per slice)
    (3, 2e-6, 4, 2, 0, 3),  # scaled split-FP16
    (3, 2e-6, 8, 3, 4, 4),
]


@pytest.mark.parametrize("prec,tol,chi,L,chunk,seed", CASES)
def test_complex_mixed_binary(gm, prec, tol, chi, L, chunk, seed):
    h3 = inp.three_site_blocked(_dm_bond())
    us, ws = inp.random_mera(4, chi, L, seed=seed, dtype=np.complex128)
    m = gm.Mera(gm.default_config(4, chi, L, dtype=gm.MERA_C128, prec=prec, b_chunk=chunk), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) / max(1.0, abs(e_ref)) < tol
    assert max(_rel(D[i], ds[i]) for i in range(len(ds))) < 10 * tol


def test_complex_mixed_ternary(gm):
    h = _dm_bond()
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=3, dtype=np.complex128)
    m = gm.Mera(gm.default_config(2, 4, 1, network=gm.MERA_TERNARY, dtype=gm.MERA_C128, prec=1), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) / max(1.0, abs(e_ref)) < 2e-6
    assert max(_rel(D[i], ds[i]) for i in range(len(ds))) < 2e-5


def test_complex_mixed_directional_derivative(gm):
    """Ising chain with a longitudinal field (-h_z X, h_z = 0.13) on complex
    tensors, 3xTF32: (e(R(eps X)) - e(R(-eps X))) / (2 eps) against
    Re <G, X> for random tangents X."""
    h3 = inp.three_site_blocked(inp.ising_bond(1.0, 0.13).astype(np.complex128))
    us, ws = inp.random_mera(4, 4, 2, seed=5, dtype=np.complex128)
    pt = _flat(us, ws)
    m = gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128, prec=1), h3)
    m.set_tensors(pt)
    _, G = m.energy_grad()
    rng = np.random.default_rng(6)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    eps = 1e-3
    for _ in range(4):
        X = [geo.project(W, rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape), k)
             for W, k in zip(pt, kinds)]
        nx = np.sqrt(sum(float(np.vdot(x, x).real) for x in X))
        X = [x / nx for x in X]
        e = {}
        for a in (eps, -eps):
            m.set_tensors(pt)
            m.retract(X, a)
            e[a] = m.energy_only()
        fd = (e[eps] - e[-eps]) / (2 * eps)
        an = sum(float(np.vdot(g, x).real) for g, x in zip(G, X))
        assert abs(fd - an) < 1e-3 * max(1.0, abs(an)), (fd, an)


def test_complex_mixed_chi16_64_directions(gm):
    """The field-Ising workload at its full size (chi = 16, 3 transition
    layers: dims 4, 16, 16, 16, 16) on complex tensors in scaled split-FP16:
    along 64 seeded unit tangents X the central difference of the energy
    along the retraction (step 1e-3) matches Re <G, X> to 1% of |G|, which a
    missing or wrong derivative term would exceed by orders of magnitude."""
    h3 = inp.three_site_blocked(inp.ising_bond(1.0, 0.13).astype(np.complex128))
    us, ws = inp.random_mera(4, 16, 3, seed=7, dtype=np.complex128)
    pt = _flat(us, ws)
    m = gm.Mera(gm.default_config(4, 16, 3, dtype=gm.MERA_C128, prec=3), h3)
    m.set_tensors(pt)
    _, G = m.energy_grad()
    gn = np.sqrt(sum(float(np.vdot(g, g).real) for g in G))
    rng = np.random.default_rng(16)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    eps = 1e-3
    worst = 0.0
    for _ in range(64):
        X = [geo.project(W, rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape), k)
             for W, k in zip(pt, kinds)]
        nx = np.sqrt(sum(float(np.vdot(x, x).real) for x in X))
        X = [x / nx for x in X]
        e = {}
        for a in (eps, -eps):
            m.set_tensors(pt)
            m.retract(X, a)
            e[a] = m.energy_only()
        fd = (e[eps] - e[-eps]) / (2 * eps)
        an = sum(float(np.vdot(g, x).real) for g, x in zip(G, X))
        worst = max(worst, abs(fd - an) / gn)
    assert worst < 1e-2, worst
