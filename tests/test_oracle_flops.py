"""The oracle's operation counter (oracle/flops.py): its counts are pinned by
hand counts of single operations, counting leaves the oracle's results
bit-identical, and the library's own flop model (peps_flops_per_sample, the
kernels' work) lies within a stated band of the oracle's count.

The band: the kernels never form the absorbed tensor N_j = M_j T_j nor the
thin Q of the QR sweep (they carry R_j into the next column's contraction),
so they do less work than the oracle for the same result; the model must
come out between 0.5 and 1.0 of the oracle's count of the fused step
(evaluation + one sweep, without the sweep's own rebuild of the lower
environments and without the strip rebuilds after an accepted exchange)."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from oracle import flops as F
from synth import make_peps, random_sz0_configs


def test_counts_of_single_operations():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((3, 4, 5)), rng.standard_normal((5, 4, 6))
    with F.counting() as c:
        r = F.tensordot(a, b, axes=([1, 2], [1, 0]))   # (3,6) from K = 20
    assert np.array_equal(r, np.tensordot(a, b, axes=([1, 2], [1, 0])))
    assert c.by_class() == {"contraction": 2.0 * 3 * 6 * 20}
    with F.counting() as c:
        F.einsum("ab,bc->ac", rng.standard_normal((2, 3)), rng.standard_normal((3, 7)))
        F.einsum("a,b->ab", rng.standard_normal(4), rng.standard_normal(5))   # outer product
        F.einsum("xyz,xyz->", a, a)                                           # dot product
    assert c.by_class() == {"contraction": 2.0 * 2 * 3 * 7 + 4 * 5 + 2.0 * 60}
    # the leading-order Householder count 2 m n^2 - 2 n^3 / 3 (m >= n), per factor
    with F.counting() as c:
        F.qr(rng.standard_normal((9, 3)))
        F.qr(rng.standard_normal((3, 9)))               # wide: the roles swap
    want = 2 * (2.0 * 9 * 9 - (2.0 / 3.0) * 27)
    assert c.by_class()["qr"] == pytest.approx(want) and c.by_class()["qr_q"] == pytest.approx(want)
    # SVD of 6 x 4 keeping 2: bidiagonalisation 4*6*16 - 4/3*64, vectors 2*(4*6*4-2*16) + 2*(4*4*4-2*16)
    with F.counting() as c:
        F.svd(rng.standard_normal((6, 4)), keep=2)
    assert c.by_class()["svd"] == pytest.approx(4 * 6 * 16 - 64 * 4 / 3 + 2 * (96 - 32) + 2 * (64 - 32))


def test_tags_and_nesting():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 4))
    with F.counting() as c:
        F.einsum("ab,bc->ac", x, x)
        with F.tagged("rebuild"):
            F.einsum("ab,bc->ac", x, x)
    assert c.total() == 2 * 128.0
    assert c.total(exclude_tags=("rebuild",)) == 128.0
    # outside a counting block nothing is recorded and nothing fails
    F.einsum("ab,bc->ac", x, x)


def test_counting_leaves_the_results_unchanged():
    L, D, Dc = 4, 2, 3
    A = make_peps(L, D, seed=3)
    s = random_sz0_configs(L, 1, seed=4)[0]
    r0 = oracle.evaluate(A, s, L, Dc, want_delta=True)
    with F.counting() as c:
        r1 = oracle.evaluate(A, s, L, Dc, want_delta=True)
    assert c.total() > 0
    for k in r0:
        assert np.array_equal(np.asarray(r0[k]), np.asarray(r1[k])), k


def test_product_state_counts_follow_the_network():
    """D = 1: every bond has extent 1, so a strip column step is three
    pairwise contractions of scalars; the count grows with the number of
    sites and never with D."""
    def count(L):
        A = make_peps(L, 1, seed=5)
        s = random_sz0_configs(L, 1, seed=6)[0]
        with F.counting() as c:
            oracle.evaluate(A, s, L, 2, want_delta=False)
        return c.total()
    n3, n4 = count(3), count(4)
    assert 0 < n3 < n4 < 10 * n3


@pytest.fixture(scope="module")
def lib():
    from paper_1806_03761_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1806_03761_gb300 import build
        build.build()
    return _lib.load()


@pytest.mark.parametrize("L,D,Dc,kind", [(6, 3, 4, "gauss"), (8, 4, 16, "neel"), (10, 4, 16, "gauss")])
def test_kernel_model_within_band_of_oracle_count(lib, L, D, Dc, kind):
    from paper_1806_03761_gb300 import _lib
    A = make_peps(L, D, seed=4, kind=kind)
    s = random_sz0_configs(L, 1, seed=5)[0]
    with F.counting() as c:
        oracle.evaluate(A, s, L, Dc, want_delta=True)
        oracle.metropolis_sweep(A, s.copy(), L, Dc, 5, 0, 1)
    counted = c.total(exclude_tags=("rebuild", "sweep_lower_envs"))
    shape = _lib.PepsShape(L, D, Dc, 1.0, 0.5, _lib.PEPS_MIXED)
    model = lib.peps_flops_per_sample(ctypes.byref(shape), 2)
    print(L, D, Dc, "model %.4g oracle %.4g ratio %.3f" % (model, counted, model / counted))
    assert 0.5 <= model / counted <= 1.0
