"""The GPU path at a converged point rather than a random one.

The point is the fixture of tests/test_oracle_scaling.py: a Z2-symmetric
chi = 4 MERA of the critical Ising chain (two transition layers) that the
oracle's L-BFGS optimised to 1.4e-6 per spin above -4/pi.  Its
scale-invariant maps are near-critical (subleading eigenvalue 0.917 =
2^(-1/8), the spin field), the regime in which the Krylov solves of App. B
converge slowest, and the gradient is small (|G| = 1.6e-5 against entries of
the partial derivatives near 10), so the projection cancels almost all of D.

FP64, dense and by charge sector: energy and every partial derivative
against the oracle at 1e-12, the projected gradient to 1e-12 of the
derivatives' scale.  Mixed modes: the energy against the oracle within ten
times the random-point bound of the 22-bit modes, since slow modes amplify
the fixed-point solve's residual floor near an optimum."""
import os

import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu
TOL = 1e-12
FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ising_chi4_L2_z2_lbfgs.npz")


@pytest.fixture(scope="module")
def gm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera
    return mera


@pytest.fixture(scope="module")
def problem():
    z = np.load(FIXTURE)
    point = [z[f"arr_{i}"] for i in range(6)]
    h3 = inp.parity_ordered_three_site(inp.three_site_blocked(inp.ising_bond(1.0)))
    e, ds, _ = om.energy_grad(h3, point[0::2], point[1::2])
    gs = [geo.project(W, D, geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN) for i, (W, D) in enumerate(zip(point, ds))]
    return h3, point, e, ds, gs


@pytest.mark.parametrize("z2", [0, 1])
def test_fp64_at_the_optimised_point(gm, problem, z2):
    h3, point, e_ref, ds, gs = problem
    m = gm.Mera(gm.default_config(4, 4, 2, z2=z2), h3)
    m.set_tensors(point)
    e, G, D = m.energy_grad(deriv=True)
    assert abs(e - e_ref) <= TOL * max(1.0, abs(e_ref)), (e, e_ref)
    scale = max(np.abs(d).max() for d in ds)
    for i in range(len(ds)):
        assert np.abs(D[i] - ds[i]).max() < TOL * np.abs(ds[i]).max(), i
        assert np.abs(G[i] - gs[i]).max() < TOL * scale, i
    gnorm = np.sqrt(sum(np.sum(g * g) for g in G))
    assert abs(gnorm - np.sqrt(geo.inner(gs, gs))) < 1e-10


@pytest.mark.parametrize("prec,z2", [(1, 1), (3, 0)])
def test_mixed_energy_at_the_optimised_point(gm, problem, prec, z2):
    h3, point, e_ref, ds, _ = problem
    m = gm.Mera(gm.default_config(4, 4, 2, z2=z2, prec=prec), h3)
    m.set_tensors(point)
    e, G, D = m.energy_grad(deriv=True)
    err_e = abs(e - e_ref) / max(1.0, abs(e_ref))
    err_d = max(np.abs(D[i] - ds[i]).max() / np.abs(ds[i]).max() for i in range(len(ds)))
    print(f"prec {prec}: energy error {err_e:.2e}, derivative error {err_d:.2e}")
    assert err_e < 2e-5, err_e
    assert err_d < 2e-4, err_d
