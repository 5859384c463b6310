"""mera_init_random through the C ABI: the point it leaves on the device is,
tensor by tensor, oracle/rng.py's sign-fixed QR-of-Gaussian isometry of the
same seed and stream (binary real and complex, ternary with Z2 charge blocks,
the MPS), and an evaluation there matches the oracle's energy."""
import numpy as np
import pytest

from oracle import mera as om
from oracle import rng
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


def _charges(gm, m, i, chi, L):
    if not m.cfg.z2:
        return None, None
    dims = inp.ternary_layer_dims(2, chi, L)
    l = i // 2
    cf, cc = dims[l], dims[min(l + 1, L)]
    if i % 2 == 0:
        return inp.fused_parities(cf, cf), inp.fused_parities(cf, cf)
    return inp.fused_parities(cf, cf, cf), inp.z2_parities(cc)


@pytest.mark.parametrize("case", ["binary", "binary_c128", "ternary_z2", "mps"])
def test_init_random_matches_oracle(gm, case):
    seed = 31
    if case.startswith("binary"):
        dt = gm.MERA_C128 if case.endswith("c128") else gm.MERA_F64
        chi, L = 4, 2
        h = inp.three_site_blocked(inp.ising_bond(1.0))
        cfg = gm.default_config(4, chi, L, dtype=dt)
    elif case == "ternary_z2":
        chi, L = 8, 2
        h = inp.ising_bond(1.0)
        cfg = gm.default_config(2, chi, L, network=gm.MERA_TERNARY, z2=1)
    else:
        chi, L = 6, 0
        h = inp.xxz_bond(1.0)
        cfg = gm.default_config(2, chi, 0, network=gm.MERA_MPS)
    m = gm.Mera(cfg, h)
    m.init_random(seed)
    got = m.get_tensors()
    for i, (W, (n, p)) in enumerate(zip(got, m.shapes)):
        rq, cq = _charges(gm, m, i, chi, L)
        want = rng.random_isometry(seed, i, n, p, cfg.dtype == gm.MERA_C128, rq, cq)
        assert np.abs(W - want).max() < 1e-12, (case, i)
    e = m.energy()
    if case.startswith("binary"):
        e_ref, _, _ = om.energy_grad(h.astype(got[0].dtype), got[0::2], got[1::2])
        assert abs(e - e_ref) < 1e-12 * max(1.0, abs(e_ref))
    assert np.isfinite(e)
