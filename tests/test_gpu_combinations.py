"""Combinations of the library's options on the GPU: Z2 charge sectors with
complex data (FP64 and 3xTF32: sector plans on the real views), the uniform
MPS with complex tensors under L-BFGS, and environment recomputation in a mixed
mode (shared intermediates, 256-byte aligned, give bit-identical results)."""
import numpy as np
import pytest

from oracle import mps as om_mps
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


def _flat(us, ws):
    return [t for p in zip(us, ws) for t in p]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_z2_complex(gm, prec, tol):
    X, Y = inp.PAULI_X, inp.PAULI_Y
    # XXZ plus an X Y - Y X term: complex, and even under the Z parity
    h = inp.xxz_bond(0.5).astype(np.complex128) + 0.7 * (np.kron(X, Y) - np.kron(Y, X))
    us, ws = inp.random_z2_ternary_mera(4, 1, seed=6, dtype=np.complex128)
    m = gm.Mera(gm.default_config(2, 4, 1, network=gm.MERA_TERNARY, dtype=gm.MERA_C128, z2=1, prec=prec), h)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = ot.energy_grad(h, us, ws)
    assert abs(e - e_ref) <= tol * max(1.0, abs(e_ref))
    assert max(_rel(D[i], ds[i]) for i in range(len(ds))) < 10 * tol


def test_mps_complex_lbfgs(gm):
    D, d = 6, 2
    A = inp.random_mps(D, d, seed=9, dtype=np.complex128)
    h = inp.ising_bond(1.5, 0.1).astype(np.complex128)
    m = gm.Mera(gm.default_config(d, D, 0, network=gm.MERA_MPS, dtype=gm.MERA_C128), h)
    m.set_tensors([om_mps.as_matrix(A)])
    e0 = m.energy()
    es = [m.lbfgs_step()["energy"] for _ in range(20)]
    assert es[-1] < e0
    assert all(b <= a + 1e-6 * abs(a) for a, b in zip(es, es[1:]))
    W = m.get_tensors()[0]
    assert np.abs(W.conj().T @ W - np.eye(D)).max() < 1e-13


def test_recompute_env_mixed_is_bit_identical(gm):
    us, ws = inp.random_mera(4, 8, 3, seed=10)
    h3 = inp.three_site_blocked(inp.xxz_bond(1.0))
    out = []
    for rec in (0, 1):
        m = gm.Mera(gm.default_config(4, 8, 3, prec=gm.PREC_SPLIT_BF16, recompute_env=rec), h3)
        m.set_tensors(_flat(us, ws))
        out.append(m.energy_grad(deriv=True))
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][2], out[1][2]):
        assert np.array_equal(a, b)
