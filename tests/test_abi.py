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


def test_footprint_accounts_for_element_type_and_precision(lib):
    """mera_footprint_bytes (a dry run of every allocation, no GPU) against
    what the layout implies: complex data doubles every array; at chi = 16 the
    mixed modes' float intermediates and packed planes undercut FP64; the
    slice length of the chi^9 chain bounds the 7-leg intermediate; invalid
    configurations give 0."""
    from paper_2007_03638_gb300 import mera as gm
    real = gm.footprint_bytes(gm.default_config(4, 8, 3))
    cplx = gm.footprint_bytes(gm.default_config(4, 8, 3, dtype=gm.MERA_C128))
    assert 1.8 * real < cplx < 4.2 * real
    f64 = gm.footprint_bytes(gm.default_config(4, 16, 3))
    bf16 = gm.footprint_bytes(gm.default_config(4, 16, 3, prec=2))
    assert 0 < bf16 < f64
    # chi = 16, N5 = 16^7 entries: slicing the coarse leg b into 2 or 4 slices
    # shrinks the transient buffers
    whole = gm.footprint_bytes(gm.default_config(4, 16, 3, prec=2))
    halves = gm.footprint_bytes(gm.default_config(4, 16, 3, prec=2, b_chunk=8))
    quarters = gm.footprint_bytes(gm.default_config(4, 16, 3, prec=2, b_chunk=4))
    assert quarters < halves < whole
    # chi = 32 split-BF16 (the bench workload) fits one GB300's 288 GB
    big = gm.footprint_bytes(gm.default_config(4, 32, 3, prec=2, lbfgs_m=16, krylov_dim=4))
    assert 50e9 < big < 280e9
    # invalid: no transition layer; chi = 64 unreachable from d_b = 4 in one layer (4 -> 16)
    assert gm.footprint_bytes(gm.default_config(4, 3, 0)) == 0
    assert gm.footprint_bytes(gm.default_config(4, 64, 1)) == 0
