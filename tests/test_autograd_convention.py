"""CPU pin of the gradient convention the autograd wrapper relies on: for a
real function of complex tensors torch returns 2 dC/d conj(z), the same
normalisation as the paper's partial derivative D_v (Sec. 2.3), so the
wrapper passes D_v through without a factor."""
import numpy as np
import pytest


def test_torch_complex_gradient_is_twice_conjugate_wirtinger():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    H = torch.from_numpy(0.5 * (A + A.conj().T))            # Hermitian
    z0 = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    z = torch.from_numpy(z0).requires_grad_(True)
    C = (z.conj() @ H @ z).real                              # C = z^dag H z, real
    (g,) = torch.autograd.grad(C, z)
    # dC/d conj(z) = H z, so 2 dC/d conj(z) = 2 H z
    assert np.abs(g.numpy() - 2 * (H.numpy() @ z0)).max() < 1e-12
    # first-order change: dC = Re sum conj(g) dz
    dz = 1e-7 * (rng.standard_normal(5) + 1j * rng.standard_normal(5))
    zp = z0 + dz
    dC = float(np.real(zp.conj() @ H.numpy() @ zp) - np.real(z0.conj() @ H.numpy() @ z0))
    assert abs(dC - float(np.real(np.sum(g.numpy().conj() * dz)))) < 1e-12
