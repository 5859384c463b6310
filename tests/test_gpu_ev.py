"""Evenbly-Vidal sweeps (mera_ev_sweep) against the oracle's sweep
(oracle/ev.py), through the C ABI: same tensors after one sweep (every
tensor replaced by minus the polar factor of its environment for the
shifted Hamiltonian, App. ev_steplimit), same energy at the new point."""
import numpy as np
import pytest

from oracle import ev
from oracle import mera as om
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


def _case(kind):
    if kind == "real":
        h3 = inp.three_site_blocked(inp.ising_bond(1.0))
        us, ws = inp.random_mera(4, 4, 2, seed=1)
    else:
        X, Y = inp.PAULI_X, inp.PAULI_Y
        bond = inp.xxz_bond(0.5).astype(np.complex128) + 0.7 * (np.kron(X, Y) - np.kron(Y, X))
        h3 = inp.three_site_blocked(bond)
        us, ws = inp.random_mera(4, 4, 2, seed=2, dtype=np.complex128)
    gamma = float(np.linalg.eigvalsh(h3).max()) + 0.5
    return h3, us, ws, gamma


@pytest.mark.parametrize("kind", ["real", "complex"])
def test_ev_sweep_matches_oracle(gm, kind):
    h3, us, ws, gamma = _case(kind)
    dt = gm.MERA_C128 if kind == "complex" else gm.MERA_F64
    m = gm.Mera(gm.default_config(4, 4, 2, dtype=dt), h3)
    m.set_tensors(_flat(us, ws))
    info = m.ev_sweep(gamma)
    assert info["n_evals"] == 2 * len(us) + 1
    us_r, ws_r, es = ev.ev_sweep(h3, us, ws, gamma)
    got = m.get_tensors()
    for a, b in zip(got, _flat(us_r, ws_r)):
        assert np.abs(a - b).max() < 1e-9, np.abs(a - b).max()
        assert np.abs(a.conj().T @ a - np.eye(a.shape[1])).max() < 1e-13
    assert abs(info["energy"] - es[-1]) < 1e-10 * abs(es[-1])
    # the reported energy is the unshifted one at the new point
    assert abs(info["energy"] - om.energy(h3, us_r, ws_r)) < 1e-10 * abs(es[-1])


def test_ev_sweeps_descend_mixed_precision(gm):
    """3xTF32 contractions, chi = 8, 3 transition layers: sweeps lower the
    energy from a random start, tensors stay isometric, and L-BFGS can take
    over from the point a sweep leaves."""
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    gamma = float(np.linalg.eigvalsh(h3).max()) + 0.5
    us, ws = inp.random_mera(4, 8, 3, seed=3)
    m = gm.Mera(gm.default_config(4, 8, 3, prec=1), h3)
    m.set_tensors(_flat(us, ws))
    e = [m.energy()]
    for _ in range(3):
        e.append(m.ev_sweep(gamma)["energy"])
    assert all(b < a for a, b in zip(e, e[1:])), e
    for t in m.get_tensors():
        assert np.abs(t.T @ t - np.eye(t.shape[1])).max() < 1e-12
    assert m.lbfgs_step()["energy"] < e[-1]
