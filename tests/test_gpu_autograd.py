"""Differentiation: the torch.autograd.Function's gradient against the oracle
and against central finite differences along the retraction on 64 seeded
tangent directions (step 1e-6)."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import mera as om
from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import autograd as ag
    from paper_2007_03638_gb300 import mera as gm
    return torch, gm, ag


def _setup(gm, hz=0.13, seed=4, chi=4, L=2, prec=0):
    bond = inp.ising_bond(1.0, hx=hz)   # critical Ising with a longitudinal (X) field
    h3 = inp.three_site_blocked(bond)
    us, ws = inp.random_mera(4, chi, L, seed=seed)
    pt = [t for p in zip(us, ws) for t in p]
    return gm.Mera(gm.default_config(4, chi, L, prec=prec), h3), h3, us, ws, pt


def test_autograd_matches_oracle(env):
    torch, gm, ag = env
    m, h3, us, ws, pt = _setup(gm)
    ts = [torch.from_numpy(t).cuda().requires_grad_(True) for t in pt]
    e = ag.mera_energy(m, ts)
    grads = torch.autograd.grad(e, ts)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e.item() - e_ref) < 1e-12 * abs(e_ref)
    for g, d in zip(grads, ds):
        assert np.abs(g.cpu().numpy() - d).max() < 1e-12 * np.abs(d).max()
    # grad_output scales the result
    e2 = ag.mera_energy(m, ts)
    g2 = torch.autograd.grad(3.0 * e2, ts)
    assert torch.allclose(g2[0], 3.0 * grads[0], rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec,tol", [(0, 2e-7), (1, 2e-4)])
def test_finite_differences_64_directions(env, prec, tol):
    """d/de C(R_W(X, e)) at e = 0 equals g(G, X) = <grad, X> (R'(0) = X)."""
    torch, gm, ag = env
    m, h3, us, ws, pt = _setup(gm, prec=prec)
    ts = [torch.from_numpy(t).cuda().requires_grad_(True) for t in pt]
    grads = [g.cpu().numpy() for g in torch.autograd.grad(ag.mera_energy(m, ts), ts)]
    rng = np.random.default_rng(64)
    kinds = [geo.STIEFEL if i % 2 == 0 else geo.GRASSMANN for i in range(len(pt))]
    eps = 1e-6 if prec == 0 else 1e-3
    errs = []
    for _ in range(64):
        X = [geo.project(W, rng.standard_normal(W.shape), k) for W, k in zip(pt, kinds)]
        vals = []
        for sgn in (1.0, -1.0):
            m.set_tensors(pt)
            m.retract(X, sgn * eps)
            vals.append(m.energy_only())
        fd = (vals[0] - vals[1]) / (2 * eps)
        an = sum(float(np.sum(g * x)) for g, x in zip(grads, X))
        scale = np.sqrt(sum(float(np.sum(g * g)) for g in grads) * sum(float(np.sum(x * x)) for x in X))
        errs.append(abs(fd - an) / scale)
    assert max(errs) < tol, max(errs)


def test_autograd_complex_matches_oracle(env):
    """Complex tensors (MERA_C128) and a complex Hermitian Hamiltonian: the
    gradient torch receives is the library's D_v = 2 dC/d conj(v), which is
    also torch's own convention for a real function of complex inputs."""
    torch, gm, ag = env
    X, Y = inp.PAULI_X, inp.PAULI_Y
    bond = inp.ising_bond(1.0, hx=0.13).astype(np.complex128) + 0.4 * (np.kron(X, Y) - np.kron(Y, X))
    h3 = inp.three_site_blocked(bond)
    us, ws = inp.random_mera(4, 4, 2, seed=6, dtype=np.complex128)
    pt = [t for p in zip(us, ws) for t in p]
    m = gm.Mera(gm.default_config(4, 4, 2, dtype=gm.MERA_C128), h3)
    ts = [torch.from_numpy(t).cuda().requires_grad_(True) for t in pt]
    e = ag.mera_energy(m, ts)
    grads = torch.autograd.grad(e, ts)
    e_ref, ds, _ = om.energy_grad(h3, us, ws)
    assert abs(e.item() - e_ref) < 1e-12 * abs(e_ref)
    for g, d in zip(grads, ds):
        assert g.dtype == torch.complex128
        assert np.abs(g.cpu().numpy() - d).max() < 1e-12 * np.abs(d).max()
