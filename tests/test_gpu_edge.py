"""Degenerate shapes on the GPU against the oracle: a square isometry
(chi_{l+1} = chi_l^2, a point of the trivial Grassmann manifold Gr(n, n),
whose Riemannian gradient vanishes while its partial derivative does not) in a
transition layer, and the smallest network (one transition layer), through
the FP64 and 3xTF32 paths; an L-BFGS step leaves the square isometry's
subspace unchanged.  Hamiltonian terms that are not Hermitian or not finite are
refused at creation."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_square_isometry(gm, prec, tol):
    # d_b = 2, chi = 4, one transition layer: dims 2, 4; w_0 is 4 x 4
    h3 = inp.three_site_unblocked(inp.ising_bond(1.0))
    us, ws = inp.random_mera(2, 4, 1, seed=8)
    assert ws[0].shape == (4, 4)
    m = gm.Mera(gm.default_config(2, 4, 1, prec=prec), h3)
    m.set_tensors(_flat(us, ws))
    e, G, D = m.energy_grad(deriv=True)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e - e_ref) <= tol * max(1.0, abs(e_ref))
    assert np.abs(D[1] - ds[1]).max() <= 10 * tol * np.abs(ds[1]).max()
    assert np.abs(ds[1]).max() > 1e-3  # the derivative is not zero ...
    assert np.abs(G[1]).max() < 1e-12 * np.abs(ds[1]).max() + (0 if prec == 0 else 1e-9)  # ... the gradient is
    w0 = ws[0]
    m.lbfgs_step()
    w1 = m.get_tensors()[1]
    # the span of a square isometry is the whole space: W^T W = 1 and W W^T = 1 before and after
    assert np.abs(w1 @ w1.T - np.eye(4)).max() < 1e-12 and np.abs(w0 @ w0.T - np.eye(4)).max() < 1e-12


def test_hamiltonian_checks(gm):
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    bad = h3.copy()
    bad[0, 1] += 1e-3
    with pytest.raises(gm.MeraError) as ei:
        gm.Mera(gm.default_config(4, 4, 2), bad)
    assert ei.value.code == -1
    bad = h3.copy()
    bad[3, 3] = np.nan
    with pytest.raises(gm.MeraError) as ei:
        gm.Mera(gm.default_config(4, 4, 2), bad)
    assert ei.value.code == -3  # MERA_ERR_NONFINITE
    hc = h3.astype(np.complex128)
    hc[0, 1] += 1e-3j
    hc[1, 0] -= 1e-3j  # still Hermitian
    gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128), hc).close()
