"""Serving: requests run concurrently on one GPU give the same results as
each request alone, and admission respects the memory budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import serve
    return serve


def test_same_alone_and_in_the_mix(sv):
    reqs = sv.poisson_stream(6, rate=200.0, chis=(4, 8), seed=3)
    mixed = sv.run_stream(reqs, budget_bytes=8 << 30, workers=4, maxiter=12)
    alone = sv.run_sequential(reqs, maxiter=12)
    for a, b in zip(mixed["results"], alone["results"]):
        assert a["state"] == 2
        assert a["iters"] == b["iters"]
        assert abs(a["energy"] - b["energy"]) <= 1e-12 * max(1.0, abs(b["energy"]))
        assert abs(a["gnorm"] - b["gnorm"]) <= 1e-10 * max(1.0, abs(b["gnorm"]))
    assert mixed["p99_latency_s"] >= mixed["p50_latency_s"] > 0


def test_admission_budget(sv):
    from paper_2007_03638_gb300 import mera as gm
    reqs = sv.poisson_stream(3, rate=1000.0, chis=(8,), seed=5)
    need = gm.footprint_bytes(sv._cfg(reqs[0]["cfg"]))
    # a budget for one request at a time still completes the stream
    out = sv.run_stream(reqs, budget_bytes=int(need * 1.5), workers=2, maxiter=3)
    assert all(r["state"] == 2 for r in out["results"])
    server = sv.Server(need // 2, 1)
    with pytest.raises(gm.MeraError):
        server.submit(sv._cfg(reqs[0]["cfg"]), reqs[0]["h3"], reqs[0]["tensors"])
    server.close()
