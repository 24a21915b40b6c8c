"""Tensor-core complex GEMM (split BF16 operands, FP32 accumulation) against
a numpy complex128 product (run with -m gpu).

Bound: with x = hi + lo + e, |e| <= 2^-16 |x| (two BF16 roundings) and the
lo*lo term dropped, every product carries at most ~3 * 2^-16 of |a||b|;
the test allows 8e-5 * (|A| @ |B|) per entry plus FP32 accumulation.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    import paper_2505_00715_gb300 as td
    return td


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


def _rand(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (1, 1, 1), (130, 129, 65), (257, 300, 200), (64, 513, 7),
                                   (300, 40, 128)])
def test_zgemm_matches_numpy(td, ctx, M, N, K):
    import torch
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A, B = _rand(rng, (M, K)), _rand(rng, (K, N))
    D = td.zgemm(ctx, torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")).cpu().numpy()
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    err = np.abs(D - ref)
    assert np.all(err <= 8e-5 * bound + 1e-6), float(np.max(err / (bound + 1e-30)))
    print("M %d N %d K %d: max error / (|A||B|) = %.2e" % (M, N, K, float(np.max(err / bound))))


def test_zgemm_scales_and_zero_k(td, ctx):
    import torch
    rng = np.random.default_rng(5)
    # widely different magnitudes per row / column stay relative
    A = _rand(rng, (200, 96)) * (10.0 ** rng.uniform(-6, 3, (200, 1))).astype(np.float32)
    B = _rand(rng, (96, 150)) * (10.0 ** rng.uniform(-4, 4, (1, 150))).astype(np.float32)
    D = td.zgemm(ctx, torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")).cpu().numpy()
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.all(np.abs(D - ref) <= 8e-5 * bound + 1e-30)
    Z = td.zgemm(ctx, torch.zeros((3, 0), dtype=torch.complex64, device="cuda"),
                 torch.zeros((0, 5), dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert np.all(Z == 0)
    ctx.sync()


def test_tensor_core_wait_gives_up_and_context_stays_usable(td, ctx):
    """Failure detection of the bounded tensor-core waits: with a poll limit
    of 1 every wait on the MMA completion barrier gives up before the MMAs
    finish; the kernel records the failure, lets its own MMAs finish, frees
    its tensor memory and returns, and the call reports TDBEM_ERR_CUDA.  With
    the default limit restored the same context computes correctly again."""
    import torch
    rng = np.random.default_rng(4)
    A, B = _rand(rng, (256, 192)), _rand(rng, (192, 256))
    At, Bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(td.TdbemError) as ei:
            td.zgemm(ctx, At, Bt)
        assert "gave up" in str(ei.value)
    finally:
        ctx.set_wait_limit(0)
    ctx.sync()  # the status word was cleared by the failing call
    D = td.zgemm(ctx, At, Bt).cpu().numpy()
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    bound = 8e-5 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(D - ref) <= bound)
    with pytest.raises(td.TdbemError):
        ctx.set_wait_limit(-1)
