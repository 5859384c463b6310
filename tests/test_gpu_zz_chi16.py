"""Parity at chi = 16 (binary MERA, one transition layer 4 -> 16 and the
scale-invariant layer at chi = 16), a size whose oracle evaluation takes
about 12 minutes.  The oracle's energy and sampled partial derivatives at the
seeded point are stored in tests/golden/chi16_ising_L1_oracle_samples.json,
written by the committed script beside it, which runs only the oracle.

FP64: the energy within 1e-12 of max(1, |e|), every sampled entry of every D_v at
1e-12 of that D_v's largest entry, and the Frobenius norms at 1e-12.  Mixed
modes (3xTF32, scaled split-FP16): the energy within 2e-6 of max(1, |e|),
the bound the 22-bit modes meet at chi <= 12, and the sampled entries within
1e-4 of each D_v's largest entry (at chi <= 12 they stay near 1e-5; the
tensor cores' FP32 accumulation grows with the summed extents)."""
import json
import os

import numpy as np
import pytest

from paper_2007_03638_gb300 import inputs as inp

pytestmark = pytest.mark.gpu
SAMPLES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "chi16_ising_L1_oracle_samples.json")


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
def reference():
    with open(SAMPLES) as f:
        ref = json.load(f)
    us, ws = inp.random_mera(4, ref["chi"], ref["n_trans"], seed=ref["seed"])
    return ref, [t for p in zip(us, ws) for t in p]


def _evaluate(gm, ref, point, prec):
    h3 = inp.three_site_blocked(inp.ising_bond(1.0))
    m = gm.Mera(gm.default_config(4, ref["chi"], ref["n_trans"], prec=prec), h3)
    m.set_tensors(point)
    e, _, D = m.energy_grad(deriv=True)
    m.close()
    return e, D


def _sample_errors(ref, D):
    errs = []
    for t, d in zip(ref["tensors"], D):
        assert list(d.shape) == t["shape"]
        got = d[np.array(t["rows"]), np.array(t["cols"])]
        errs.append(np.abs(got - np.array(t["values"])).max() / t["max_abs"])
    return errs


def test_fp64_chi16_matches_the_oracle(gm, reference):
    ref, point = reference
    e, D = _evaluate(gm, ref, point, 0)
    assert abs(e - ref["energy"]) <= 1e-12 * max(1.0, abs(ref["energy"])), (e, ref["energy"])
    errs = _sample_errors(ref, D)
    assert max(errs) < 1e-12, errs
    for i, (t, d) in enumerate(zip(ref["tensors"], D)):
        assert abs(np.linalg.norm(d) - t["fro"]) < 1e-12 * t["fro"], (i, np.linalg.norm(d), t["fro"])


@pytest.mark.parametrize("prec", [1, 3])
def test_mixed_chi16_matches_the_oracle(gm, reference, prec):
    ref, point = reference
    e, D = _evaluate(gm, ref, point, prec)
    assert abs(e - ref["energy"]) / max(1.0, abs(ref["energy"])) < 2e-6, (e, ref["energy"])
    errs = _sample_errors(ref, D)
    assert max(errs) < 1e-4, errs
