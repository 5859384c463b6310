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
    """Requests of the same bond dimension evaluate together (batched launches
    over a cohort), the others overlap on their streams; every result equals
    the request's result alone, bit for bit."""
    reqs = sv.poisson_stream(8, rate=400.0, chis=(4, 8), seed=3)
    mixed = sv.run_stream(reqs, budget_bytes=8 << 30, workers=8, maxiter=12)
    alone = sv.run_sequential(reqs, maxiter=12)
    for a, b in zip(mixed["results"], alone["results"]):
        assert a["state"] == 2
        assert a["iters"] == b["iters"]
        assert a["energy"] == b["energy"]
        assert a["gnorm"] == b["gnorm"]
    assert sum(r["batched_evals"] for r in mixed["results"]) > 0
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
