"""The library's own dense product (iga_gemm_batched) against a plain
torch product in FP64 on the same inputs: every FP64 tile shape (64 x 64,
64 x 16, 16 x 64, 16 x 16, picked by the output's padding), both transposes,
reductions split over K (few output tiles, long K) and batched products, with
beta both zero and nonzero.  FP32 against the FP64 product of the FP32
inputs, within a bound from the reduction length."""
import pytest

from gpu_util import ctx_and_torch

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return ctx_and_torch()[0]


# (count, M, N, K): shapes that pick each FP64 tile and the split reduction
SHAPES = [
    (1, 256, 1, 71),       # matrix-vector, split over K (16 x 16 tiles)
    (3, 4225, 17, 65),     # tall, 17 columns (64 x 16 tiles)
    (1, 17, 1105, 65),     # wide, 17 rows (16 x 64 tiles)
    (2, 130, 150, 300),    # full 64 x 64 tiles with ragged edges
    (5, 17, 17, 17),       # Gram-sized
    (1, 33, 40, 5000),     # long reduction, few tiles
    (64, 9, 13, 7),        # long batch of tiny products
]


def _ref(A, B, C0, alpha, beta, tA, tB):
    a = A.transpose(1, 2) if tA else A
    b = B.transpose(1, 2) if tB else B
    return alpha * torch.bmm(a.double(), b.double()) + beta * C0.double()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("tA,tB", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_fp64_matches_torch(ctx, shape, tA, tB):
    from paper_1811_06797_gb300 import iga
    count, M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M * 7919 + N * 31 + K + 2 * tA + tB)
    A = torch.randn((count, K, M) if tA else (count, M, K), device="cuda", dtype=torch.float64,
                    generator=g)
    B = torch.randn((count, N, K) if tB else (count, K, N), device="cuda", dtype=torch.float64,
                    generator=g)
    C0 = torch.randn((count, M, N), device="cuda", dtype=torch.float64, generator=g)
    for alpha, beta in ((1.0, 0.0), (-0.5, 2.0)):
        C = C0.clone()
        iga.iga_gemm_batched(ctx, A, B, C, alpha=alpha, beta=beta, tA=tA, tB=tB)
        ref = _ref(A, B, C0, alpha, beta, tA, tB)
        # FP64 round-off of a K-term sum of products of unit normals
        tol = 4 * K * 2.0 ** -52 * (abs(alpha) * K ** 0.5 + abs(beta)) * 8
        err = (C - ref).abs().max().item()
        assert err <= tol, (shape, tA, tB, alpha, beta, err, tol)


@pytest.mark.parametrize("shape", [(1, 256, 1, 71), (2, 130, 150, 300), (1, 33, 40, 5000)])
def test_gemm_fp32_matches_fp64_product(ctx, shape):
    from paper_1811_06797_gb300 import iga
    count, M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(K)
    A = torch.randn((count, M, K), device="cuda", dtype=torch.float32, generator=g)
    B = torch.randn((count, K, N), device="cuda", dtype=torch.float32, generator=g)
    C = torch.zeros((count, M, N), device="cuda", dtype=torch.float32)
    iga.iga_gemm_batched(ctx, A, B, C)
    ref = torch.bmm(A.double(), B.double())
    # FP32 accumulation: about K eps |a||b| in the worst case, sqrt(K) typical
    tol = 8 * K ** 0.5 * 2.0 ** -23 * K ** 0.5 * 4
    assert (C.double() - ref).abs().max().item() <= tol


def test_gemm_is_deterministic(ctx):
    from paper_1811_06797_gb300 import iga
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn((1, 33, 5000), device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn((1, 5000, 40), device="cuda", dtype=torch.float64, generator=g)
    C1 = torch.zeros((1, 33, 40), device="cuda", dtype=torch.float64)
    C2 = torch.zeros_like(C1)
    iga.iga_gemm_batched(ctx, A, B, C1)
    iga.iga_gemm_batched(ctx, A, B, C2)
    assert torch.equal(C1, C2)


def test_gemm_rejects_mismatched_shapes(ctx):
    from paper_1811_06797_gb300 import iga
    A = torch.zeros((1, 4, 5), device="cuda", dtype=torch.float64)
    B = torch.zeros((1, 6, 3), device="cuda", dtype=torch.float64)
    C = torch.zeros((1, 4, 3), device="cuda", dtype=torch.float64)
    with pytest.raises(iga.IgaError):
        iga.iga_gemm_batched(ctx, A, B, C)
    with pytest.raises(iga.IgaError):
        iga.iga_gemm_batched(ctx, A, B.float(), C)


# shapes whose leading dimensions are multiples of 4 (16-byte operand loads,
# with ragged tiles) and shapes whose are not (scalar loads)
@pytest.mark.parametrize("shape", [(4, 128, 256, 96), (2, 260, 44, 36), (1, 300, 40, 70),
                                   (3, 775, 38, 190), (2, 33, 17, 5), (1, 1000, 130, 33)])
@pytest.mark.parametrize("tA,tB", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_tf32_tensor_cores_match_torch(ctx, shape, tA, tB):
    """The tcgen05 TF32 product against the FP64 product of the same FP32
    inputs, within the TF32 rounding of the operands (10-bit mantissa)."""
    from paper_1811_06797_gb300 import iga
    count, M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K)
    A = torch.randn((count, K, M) if tA else (count, M, K), device="cuda", dtype=torch.float32,
                    generator=g)
    B = torch.randn((count, N, K) if tB else (count, K, N), device="cuda", dtype=torch.float32,
                    generator=g)
    C0 = torch.randn((count, M, N), device="cuda", dtype=torch.float32, generator=g)
    C = C0.clone()
    iga.iga_gemm_batched(ctx, A, B, C, alpha=0.5, beta=-1.0, tA=tA, tB=tB, tf32=True)
    a = A.transpose(1, 2) if tA else A
    b = B.transpose(1, 2) if tB else B
    ref = 0.5 * torch.bmm(a.double(), b.double()) - C0.double()
    tol = 4 * 2.0 ** -10 * K ** 0.5 + 1e-5
    assert (C.double() - ref).abs().max().item() <= tol
