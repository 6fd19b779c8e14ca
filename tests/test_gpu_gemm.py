"""GPU parity: the tcgen05 BF16 and TF32 GEMMs against a float64 product of
the same bf16- or tf32-rounded operands.  FP32 accumulation:
|C - ref| <= 2e-5 sum_k |a_ik b_jk|.  Shapes cover both output tile widths
(128 and 256 columns), ragged M, N and K (zero-filled tiles, masked
stores), split-K, and more work items than SMs (the persistent loop with
its two alternating accumulators)."""
import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (128, 128, 256, 1),
                                          (256, 384, 640, 1), (256, 384, 640, 3),
                                          (128, 256, 2560, 8), (384, 128, 1024, 5),
                                          (64, 200, 520, 1), (130, 300, 136, 2),
                                          (96, 4000, 1336, 3), (2560, 4096, 128, 1)])
def test_gemm_bf16_parity(env, M, N, K, splits):
    torch, sp, ctx = env
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).bfloat16()
    B = torch.randn(N, K, generator=g).bfloat16()
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    work = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
    sp.specula_gemm_bf16(ctx, Ad, Bd, C, splits=splits, work=work)
    torch.cuda.synchronize()
    assert sp.specula_ctx_status(ctx) == 0
    a = A.float().numpy().astype(np.float64)
    b = B.float().numpy().astype(np.float64)
    ref = a @ b.T
    mag = np.abs(a) @ np.abs(b).T
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 2e-5 * mag + 1e-30), np.max(np.abs(got - ref) / mag)


def test_gemm_deterministic_and_rejects_shapes(env):
    torch, sp, ctx = env
    A = torch.randn(256, 512, device="cuda").bfloat16()
    B = torch.randn(256, 512, device="cuda").bfloat16()
    C1 = torch.empty(256, 256, device="cuda")
    C2 = torch.empty(256, 256, device="cuda")
    w = torch.empty(4 * 256 * 256, device="cuda")
    sp.specula_gemm_bf16(ctx, A, B, C1, splits=4, work=w)
    sp.specula_gemm_bf16(ctx, A, B, C2, splits=4, work=w)
    torch.cuda.synchronize()
    assert torch.equal(C1, C2)
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_gemm_bf16(ctx, A[:, :100].contiguous(), B[:, :100].contiguous(),
                             torch.empty(256, 256, device="cuda"))
    assert e.value.status == sp.EUNSUPPORTED


def tf32_round(x):
    """Round float32 values to tf32 (10-bit mantissa), to nearest, ties away
    from zero: the values the tensor cores then read exactly."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 32, 1), (128, 128, 256, 1),
                                          (256, 384, 640, 1), (256, 384, 640, 3),
                                          (384, 128, 960, 5), (72, 200, 100, 1)])
def test_gemm_tf32_parity(env, M, N, K, splits):
    torch, sp, ctx = env
    rng = np.random.default_rng(M * 5 + N + K)
    a = tf32_round(rng.standard_normal((M, K)).astype(np.float32))
    b = tf32_round(rng.standard_normal((N, K)).astype(np.float32))
    C = torch.full((M, N), float("nan"), device="cuda")
    work = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
    sp.specula_gemm_tf32(ctx, torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"), C,
                         splits=splits, work=work)
    torch.cuda.synchronize()
    assert sp.specula_ctx_status(ctx) == 0
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    ref = a64 @ b64.T
    mag = np.abs(a64) @ np.abs(b64).T
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 2e-5 * mag + 1e-30), np.max(np.abs(got - ref) / mag)


def test_gemm_tf32_reads_only_the_tf32_bits(env):
    """Operands that differ only below the tf32 mantissa give the same product."""
    torch, sp, ctx = env
    rng = np.random.default_rng(3)
    a = tf32_round(rng.standard_normal((128, 64)).astype(np.float32))
    b = tf32_round(rng.standard_normal((128, 64)).astype(np.float32))
    noisy = (a.view(np.uint32) | np.uint32(0x0FFF)).view(np.float32)   # low bits set
    C1 = torch.empty(128, 128, device="cuda")
    C2 = torch.empty(128, 128, device="cuda")
    bd = torch.tensor(b, device="cuda")
    sp.specula_gemm_tf32(ctx, torch.tensor(a, device="cuda"), bd, C1)
    sp.specula_gemm_tf32(ctx, torch.tensor(noisy, device="cuda"), bd, C2)
    torch.cuda.synchronize()
    assert torch.equal(C1, C2)
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_gemm_tf32(ctx, torch.zeros(128, 50, device="cuda"),
                             torch.zeros(128, 50, device="cuda"), C1)
    assert e.value.status == sp.EUNSUPPORTED
