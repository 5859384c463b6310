"""Host-side checks of the serving client (no GPU): the sizes a request's
arrays must have are the ones mera_server_submit copies (the binding refuses
anything else before the call), for every bond dimension of the request
stream and for the ternary network."""
import numpy as np
import pytest

from paper_2007_03638_gb300 import inputs as inp
from paper_2007_03638_gb300 import mera as gm
from paper_2007_03638_gb300 import serve


def test_stream_requests_have_the_sizes_the_library_copies():
    for r in serve.poisson_stream(24, chis=(4, 8, 12, 16, 24, 32), seed=3):
        cfg = serve._cfg(r["cfg"])
        n_h, sizes = serve.request_sizes(cfg)
        assert n_h == r["h3"].size
        assert sizes == [t.size for t in r["tensors"]]
        serve.check_request(cfg, r["h3"], r["tensors"])


def test_ternary_request_sizes():
    us, ws = inp.random_ternary_mera(2, 8, 2, seed=0)
    cfg = gm.default_config(2, 8, 2, network=gm.MERA_TERNARY)
    n_h, sizes = serve.request_sizes(cfg)
    assert n_h == 16 and sizes == [t.size for p in zip(us, ws) for t in p]


def test_mis_sized_requests_are_refused():
    r = serve.poisson_stream(1, chis=(8,), seed=4)[0]
    cfg = serve._cfg(r["cfg"])
    with pytest.raises(ValueError):
        serve.check_request(cfg, r["h3"], r["tensors"][:-1])          # a tensor short
    short = list(r["tensors"])
    short[1] = short[1][:, :-1]
    with pytest.raises(ValueError):
        serve.check_request(cfg, r["h3"], short)                      # a short tensor
    with pytest.raises(ValueError):
        serve.check_request(cfg, np.zeros((16, 16)), r["tensors"])    # a two-site term for the binary network
