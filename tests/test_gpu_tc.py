"""Tensor-core contraction kernel (tcgen05, 3xTF32 / split-BF16 with FP32
accumulation) against an FP64 product, through the C ABI (mera_gemm)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128, 32), (200, 130, 70), (1, 1, 1), (1024, 512, 1000), (4100, 257, 2049),
          (256, 200, 40000), (100, 130, 9000)]  # the last two split K


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03638_gb300 import build as b
    b.build()
    from paper_2007_03638_gb300 import mera as gm
    return torch, gm


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 4e-6), (2, 2e-4), (3, 4e-6)])
def test_gemm_modes(env, shape, prec, tol):
    torch, gm = env
    M, N, K = shape
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    ref = A @ B
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    Cd = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    gm.gemm(prec, Ad, Bd, Cd)
    C = Cd.cpu().numpy()
    assert np.all(np.isfinite(C))
    # error relative to the natural scale of the entries (sqrt(K) for N(0,1) data)
    err = np.abs(C - ref).max() / np.sqrt(K)
    assert err < tol, (prec, shape, err)


# products whose output tiles do not fill the GPU split K over several CTAs
# (partials summed in a fixed order by a second kernel); odd tile counts and
# single-row outputs exercise the padding of the last tiles
SPLIT_SHAPES = [(384, 384, 8192), (4100, 257, 2049), (256, 200, 40000), (1, 300, 6400), (130, 1, 70000)]


@pytest.mark.parametrize("shape", SPLIT_SHAPES)
@pytest.mark.parametrize("prec,tol", [(1, 4e-6), (2, 2e-4), (3, 4e-6)])
def test_gemm_split_k_shapes(env, shape, prec, tol):
    torch, gm = env
    M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 5 * K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    ref = A @ B
    Cd = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    gm.gemm(prec, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd)
    C = Cd.cpu().numpy()
    assert np.all(np.isfinite(C))
    err = np.abs(C - ref).max() / np.sqrt(K)
    assert err < tol, (prec, shape, err)


@pytest.mark.parametrize("sa,sb", [(1e-20, 1e15), (1e12, 1e-30), (3e-5, 3e-5), (1.0, 65504.0 * 4)])
def test_fp16_planes_scale_any_magnitude(env, sa, sb):
    """Scaled split-FP16: each operand is scaled by a power of two from its
    largest entry before it is split, so operands far outside FP16's range
    (or entries at the size of a unit-trace chi^6 density matrix, 3e-5) keep
    the 22-bit accuracy of the unscaled case; a row a thousand times larger
    than the rest does not cost the others their accuracy beyond that."""
    torch, gm = env
    M, N, K = 200, 130, 3000
    rng = np.random.default_rng(5)
    A = rng.standard_normal((M, K)) * sa
    B = rng.standard_normal((K, N)) * sb
    A[7] *= 1e3
    ref = A @ B
    Cd = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    gm.gemm(3, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd)
    C = Cd.cpu().numpy()
    assert np.all(np.isfinite(C))
    rows = np.arange(M) != 7
    scale = np.sqrt(K) * sa * sb
    assert np.abs(C[rows] - ref[rows]).max() / scale < 8e-6
    assert np.abs(C[7] - ref[7]).max() / (1e3 * scale) < 4e-6
    # zero operand: zero product, no NaN from the scale of an all-zero maximum
    Z = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    gm.gemm(3, Z, torch.from_numpy(B).cuda(), Cd)
    assert torch.count_nonzero(Cd).item() == 0
