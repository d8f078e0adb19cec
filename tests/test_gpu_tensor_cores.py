"""The tensor-core contraction (peps_tc_gemm: tcgen05, error-free BF16 slices)
through the C ABI.  First exactly: with one slice the result is the exact
product of the first slices, which the test forms on the CPU from the
splitting's definition (integer products, exact in FP64) -- any error in the
operand layout or the MMA descriptors shows here.  Then at full accuracy
against the FP64 product on the shapes of the strip column steps, with
CUDA-core contract() in float-float and FP64 beside it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def first_slices(X, axis):
    """The one-slice image of X along `axis` (the reduction index): scale by
    2^-e (e: exponent of the largest |entry| of each row or column) and round
    to 7 bits (to nearest, halves away from zero); returns the slice values
    times their scale."""
    mx = np.max(np.abs(X), axis=axis, keepdims=True)
    e = np.where(mx > 0, np.frexp(mx)[1], 0)
    r = np.ldexp(X, -e)
    q = np.sign(r) * np.floor(np.abs(r) * 128.0 + 0.5)
    return np.ldexp(q / 128.0, e)


def test_one_slice_is_the_exact_product_of_the_first_slices():
    from paper_1806_03761_gb300 import Contraction
    rng = np.random.default_rng(0)
    M, N, K, B = 128, 16, 16, 1
    A = rng.standard_normal((B, M, K))
    Bm = rng.standard_normal((B, K, N))
    c = Contraction(M, N, K, B, slices=1)
    C = c.tensor_cores(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda())
    torch.cuda.synchronize()
    assert int(c.status.item()) == 0
    want = np.einsum("bmk,bkn->bmn", first_slices(A, 2), first_slices(Bm, 1))
    got = C.cpu().numpy()
    assert np.array_equal(got, want), np.max(np.abs(got - want))


@pytest.mark.parametrize("M,N,K,B,shared", [(128, 16, 16, 2, False), (300, 36, 36, 3, True),
                                             (3456, 36, 36, 4, False), (864, 144, 36, 2, False)])
def test_seven_slices_match_the_fp64_product(M, N, K, B, shared):
    from paper_1806_03761_gb300 import Contraction
    rng = np.random.default_rng(M + N)
    A = rng.standard_normal((B, M, K)) * np.exp(rng.uniform(-8, 8, (B, M, 1)))  # rows of mixed scale
    Bm = rng.standard_normal((1 if shared else B, K, N))
    c = Contraction(M, N, K, B, b_shared=shared, slices=7)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()
    C = c.tensor_cores(Ad, Bd).cpu().numpy()
    assert int(c.status.item()) == 0
    Bx = np.broadcast_to(Bm, (B, K, N))
    exact = np.einsum("bmk,bkn->bmn", A, Bx)
    scale = np.einsum("bmk,bkn->bmn", np.abs(A), np.abs(Bx))
    err = np.max(np.abs(C - exact) / scale)
    # the omitted remainders: 2^-49 of each row / column scale, times K
    assert err < 2.0 ** -45, err
    # float-float output (hi, lo): the same sum rounded to about 48 bits
    Cf = c.tensor_cores(Ad, Bd, out="mixed").cpu().numpy().astype(np.float64)
    err_ff = np.max(np.abs(Cf[..., 0] + Cf[..., 1] - exact) / scale)
    assert err_ff < 2.0 ** -44, err_ff
    for prec, tol in (("mixed", 2.0 ** -40), ("fp64", 2.0 ** -46)):
        Cc = c.cuda_cores(Ad, Bd, precision=prec).cpu().numpy()
        e2 = np.max(np.abs(Cc - exact) / scale)
        print(M, N, K, prec, "%.2e" % e2, "tensor cores %.2e" % err)
        assert e2 < tol
