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


def test_enums_match_header():
    """The binding's enum values are the header's."""
    from paper_2007_03638_gb300 import mera as gm
    src = open(os.path.join(ROOT, "include", "mera.h")).read()
    for name in ("MERA_F64", "MERA_C128", "MERA_BINARY", "MERA_TERNARY", "MERA_MPS",
                 "MERA_PREC_FP64", "MERA_PREC_3XTF32", "MERA_PREC_SPLIT_BF16"):
        val = int(re.search(rf"\b{name}\s*=\s*(\d+)", src).group(1))
        py = {"MERA_PREC_FP64": "PREC_FP64", "MERA_PREC_3XTF32": "PREC_3XTF32",
              "MERA_PREC_SPLIT_BF16": "PREC_SPLIT_BF16"}.get(name, name)
        assert getattr(gm, py) == val, name


def test_mps_footprint(lib):
    """mera_footprint_bytes for a uniform MPS (network = MERA_MPS): positive,
    growing like the D^2 d^2 two-site buffers and the tangent lists, doubled by
    complex data, and 0 for what the MPS path does not serve (transition
    layers, mixed precision, Stiefel, a one-dimensional site)."""
    from paper_2007_03638_gb300 import mera as gm

    def fp(d, D, n_trans=0, **kw):
        return gm.footprint_bytes(gm.default_config(d, D, n_trans, network=gm.MERA_MPS, **kw))

    small, big = fp(2, 8), fp(2, 64)
    assert 0 < small < big
    # at D = 64, d = 2 the (D d d D) buffers, the Krylov vectors and 2m + 10
    # tensors of D d D reals dominate: within a factor 2 of that count
    D, d, k, m = 64, 2, 20, 8
    est = 8 * (3 * D * d * d * D + (k + 4) * D * D + (2 * m + 10) * D * d * D)
    assert est < big < 2 * est
    assert 1.8 * big < fp(2, 64, dtype=gm.MERA_C128) < 4.2 * big
    assert fp(3, 1) > 0
    assert fp(2, 8, n_trans=1) == 0
    assert fp(2, 8, prec=gm.PREC_SPLIT_BF16) == 0
    assert fp(2, 8, w_stiefel=1) == 0
    assert fp(1, 8) == 0


def test_z2_flag_footprint(lib):
    """mera_config.z2: served for the ternary network, and for the binary one
    where its chi^9 chain runs unsliced (the footprint, a dry run of the
    allocations, is 0 for what mera_create refuses)."""
    from paper_2007_03638_gb300 import mera as gm
    tern = gm.footprint_bytes(gm.default_config(2, 8, 2, network=gm.MERA_TERNARY, z2=1))
    assert tern > 0
    assert gm.footprint_bytes(gm.default_config(2, 8, 2, network=gm.MERA_TERNARY, z2=2)) == 0
    assert gm.footprint_bytes(gm.default_config(4, 8, 3, z2=1)) > 0
    assert gm.footprint_bytes(gm.default_config(4, 32, 3, z2=1)) == 0  # sliced chain
    assert gm.footprint_bytes(gm.default_config(2, 8, 0, network=gm.MERA_MPS, z2=1)) == 0
    assert gm.default_config(4, 8, 3).z2 == 0


def test_recompute_env_shares_the_operator_nodes(lib):
    """With recompute_env = 1 the binary network keeps one set of its
    operator-dependent intermediates (N3, N7, N8) for all layers and sides:
    at chi = 32 split-BF16 about 41 GB less (two transition layers' worth and
    one side's, 4 x 4.3 GB per layer and side, float)."""
    from paper_2007_03638_gb300 import mera as gm
    kw = dict(prec=gm.PREC_SPLIT_BF16, lbfgs_m=16, krylov_dim=4)
    keep = gm.footprint_bytes(gm.default_config(4, 32, 3, **kw))
    share = gm.footprint_bytes(gm.default_config(4, 32, 3, recompute_env=1, **kw))
    assert 40e9 < keep - share < 43e9
    assert gm.footprint_bytes(gm.default_config(4, 8, 3, recompute_env=1)) < gm.footprint_bytes(
        gm.default_config(4, 8, 3))



def test_create_refuses_configs_out_of_range(lib):
    """mera_create checks the config before any device work, so invalid ones
    are refused with MERA_ERR_ARG on a machine without a GPU too."""
    import ctypes as C

    import numpy as np

    from paper_2007_03638_gb300 import mera as gm
    h = np.zeros((64, 64))
    bad = [dict(precond=2), dict(krylov_tol=0.0), dict(krylov_tol=float("nan")), dict(krylov_tol=1.5),
           dict(krylov_maxiter=0), dict(krylov_dim=0), dict(lbfgs_m=0), dict(b_chunk=-1), dict(w_stiefel=3),
           dict(recompute_env=-1), dict(network=7), dict(dtype=5), dict(prec=9), dict(z2=3),
           dict(device_wait_s=0.0), dict(device_wait_s=61.0), dict(device_wait_s=float("nan"))]
    for kw in bad:
        cfg = gm.default_config(4, 8, 3, **kw)
        handle = C.c_void_p()
        rc = lib.mera_create(C.byref(cfg), C.c_void_p(h.ctypes.data), None, C.byref(handle))
        assert rc == -1 and not handle.value, kw
        if "network" not in kw:
            assert gm.footprint_bytes(cfg) == 0, kw


def test_allocator_hook_arguments(lib):
    """mera_set_allocator needs a deallocator with an allocator; NULL
    restores the CUDA allocator (host-side bookkeeping only)."""
    from paper_2007_03638_gb300 import mera as gm
    a = gm.ALLOC_FN(lambda n, user: None)
    assert lib.mera_set_allocator(a, gm.C.cast(None, gm.FREE_FN), None) == -1
    assert lib.mera_set_allocator(gm.C.cast(None, gm.ALLOC_FN), gm.C.cast(None, gm.FREE_FN), None) == 0
    gm.set_allocator(lambda n: 0, lambda p: None)
    gm.set_allocator()


def test_dots_noalloc_wrapper_checks_sizes(lib):
    """The binding refuses arrays shorter than the sizes it passes on, before
    any call into the library."""
    import numpy as np
    import pytest

    from paper_2007_03638_gb300 import mera as gm
    x, y = np.zeros(20), np.zeros(8)
    with pytest.raises(ValueError):
        gm.dots_noalloc(x, y, 3, 8, 8, np.zeros(3))      # X needs 2 * 8 + 8 = 24
    with pytest.raises(ValueError):
        gm.dots_noalloc(np.zeros(24), y, 3, 8, 8, np.zeros(2))  # out needs 3
    with pytest.raises(ValueError):
        gm.dots_noalloc(np.zeros(24), np.zeros(7), 3, 8, 8, np.zeros(3))
    with pytest.raises(TypeError):
        gm.dots_noalloc(np.zeros(24, dtype=np.complex128), y, 3, 8, 8, np.zeros(3))


def test_binding_checks_tensor_counts_and_sizes(lib):
    """Per-tensor lists must hold one array per tensor with the tensor's
    element count, and the Hamiltonian term its operator's: the library reads
    and writes that many elements behind every pointer, so the binding refuses
    anything else before a call."""
    import numpy as np
    import pytest

    from paper_2007_03638_gb300 import mera as gm
    sizes = [256, 64]
    keep = []
    assert len(gm._ptrs([np.zeros((16, 16)), np.zeros((16, 4))], keep, np.float64, sizes)) == 2
    with pytest.raises(ValueError):
        gm._ptrs([np.zeros((16, 16))], keep, np.float64, sizes)  # one tensor short
    with pytest.raises(ValueError):
        gm._ptrs([np.zeros((16, 16)), np.zeros((16, 3))], keep, np.float64, sizes)  # a short tensor
    with pytest.raises(ValueError):  # a real view of complex data has twice the elements
        gm._ptrs([np.zeros((16, 32)), np.zeros((16, 8))], keep, np.complex128, sizes)
    with pytest.raises(ValueError):  # binary network: a three-site term, 4^3 x 4^3 at d_b = 4
        gm.Mera(gm.default_config(4, 8, 3), np.zeros((16, 16)))
    with pytest.raises(ValueError):  # ternary network: a two-site term, 2^2 x 2^2 at d = 2
        gm.Mera(gm.default_config(2, 8, 2, network=gm.MERA_TERNARY), np.zeros((8, 8)))


def test_gemm_wrapper_checks_shapes(lib):
    """mera_gemm reads M K and K N elements and writes M N: the binding
    refuses mismatched extents and non-double arrays before the call."""
    import numpy as np
    import pytest

    from paper_2007_03638_gb300 import mera as gm
    with pytest.raises(ValueError):
        gm.gemm(1, np.zeros((4, 3)), np.zeros((2, 5)), np.zeros((4, 5)))   # inner extents differ
    with pytest.raises(ValueError):
        gm.gemm(1, np.zeros((4, 3)), np.zeros((3, 5)), np.zeros((4, 4)))   # out too small
    with pytest.raises(ValueError):
        gm.gemm(1, np.zeros(12), np.zeros((3, 5)), np.zeros((4, 5)))       # A not a matrix
    with pytest.raises(TypeError):
        gm.gemm(1, np.zeros((4, 3), dtype=np.complex128), np.zeros((3, 5)), np.zeros((4, 5)))
