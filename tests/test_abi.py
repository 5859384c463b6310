"""The C-ABI library loads and exports every symbol that include/mera.h
declares; host-only calls work without a GPU (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera as gm
    return gm.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "mera.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mera_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2007_03638_gb300 import mera as gm
    assert sorted(gm.EXPORTS) == _declared()


def test_host_only_calls(lib):
    from paper_2007_03638_gb300 import mera as gm
    cfg = gm.default_config(4, 8, 3)
    assert (cfg.d_b, cfg.chi, cfg.n_trans, cfg.krylov_dim) == (4, 8, 3, 20)
    assert gm.footprint_bytes(cfg) > 0
    big = gm.footprint_bytes(gm.default_config(4, 16, 3))
    assert big > gm.footprint_bytes(cfg)
    assert lib.mera_strerror(-4) == b"iteration did not converge"
    assert lib.mera_launch_count(None) == 0
