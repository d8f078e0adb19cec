"""Operation counter of the FP64 oracle (the analogue of the paper's
instrumented flop counts, Sec. "Performance Measurement", which cross-checks
its DGEMM/permutation counters against PAPI).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every contraction and factorisation the oracle executes goes through the
wrappers below, which count its floating-point operations per class and then
call numpy unchanged (the oracle's arithmetic is not touched):

  contraction : a pairwise tensordot / einsum with a summed index costs
                2 * (product of all index extents); an outer product
                (no summed index) costs one multiply per output element.
  qr          : the Householder R factor of an m x n matrix,
                2 K k^2 - (2/3) k^3 with k = min(m, n), K = max(m, n).
  qr_q        : forming the thin orthogonal factor explicitly (backward
                accumulation), the same count again.
  svd         : Golub-Kahan bidiagonalisation of an m x n matrix,
                4 K k^2 - (4/3) k^3, plus the back-transformation of the
                `keep` kept singular vectors on each side,
                keep (4 m k - 2 k^2) + keep (4 n k - 2 k^2).
  other       : everything else the counter is told about (scalings,
                dot products counted by the caller).

Work can be attributed to a tag (``with tagged("rebuild"): ...``); the
oracle tags the strip rebuilds that follow an accepted exchange in its
Metropolis sweep, which an incremental sweep never needs.

    with counting() as c:
        oracle.evaluate(A, spins, L, chi, want_delta=True)
    c.flops            # {(tag, class): flops}
    c.total(exclude_tags=("rebuild",))
"""
import contextlib

import numpy as np

__all__ = ["counting", "tagged", "tensordot", "einsum", "qr", "svd", "FlopCount"]


class FlopCount:
    def __init__(self):
        self.flops = {}
        self.tags = ["main"]

    def add(self, cls, n):
        key = (self.tags[-1], cls)
        self.flops[key] = self.flops.get(key, 0.0) + float(n)

    def by_class(self, exclude_tags=()):
        out = {}
        for (tag, cls), v in self.flops.items():
            if tag in exclude_tags:
                continue
            out[cls] = out.get(cls, 0.0) + v
        return out

    def total(self, exclude_tags=(), exclude_classes=()):
        return sum(v for (tag, cls), v in self.flops.items()
                   if tag not in exclude_tags and cls not in exclude_classes)


_active = []


@contextlib.contextmanager
def counting():
    """Count the oracle's operations inside the block."""
    c = FlopCount()
    _active.append(c)
    try:
        yield c
    finally:
        _active.pop()


@contextlib.contextmanager
def tagged(tag):
    """Attribute the operations inside the block to `tag`."""
    for c in _active:
        c.tags.append(tag)
    try:
        yield
    finally:
        for c in _active:
            c.tags.pop()


def _add(cls, n):
    for c in _active:
        c.add(cls, n)


def tensordot(a, b, axes):
    """np.tensordot, counted as 2 * |output| * |contracted|."""
    if _active:
        ka = axes[0] if isinstance(axes[0], (list, tuple)) else [axes[0]]
        k = 1
        for x in ka:
            k *= a.shape[x]
        _add("contraction", 2.0 * (a.size // max(k, 1)) * (b.size // max(k, 1)) * k)
    return np.tensordot(a, b, axes=axes)


def einsum(subscripts, *ops):
    """np.einsum of explicit subscripts ('ab,bc->ac'), counted from the
    extents of every index label."""
    if _active:
        lhs, rhs = subscripts.split("->")
        dims = {}
        for spec, op in zip(lhs.split(","), ops):
            for lab, n in zip(spec, op.shape):
                dims[lab] = n
        total = 1
        for n in dims.values():
            total *= n
        summed = set(dims) - set(rhs)
        if summed:
            _add("contraction", 2.0 * total)
        else:
            _add("contraction", float(total))
    return np.einsum(subscripts, *ops)


def _householder(m, n):
    k, K = min(m, n), max(m, n)
    return 2.0 * K * k * k - (2.0 / 3.0) * k ** 3


def qr(X):
    """Thin QR (numpy, mode 'reduced'): R factor and the explicit thin Q."""
    if _active:
        m, n = X.shape
        _add("qr", _householder(m, n))
        _add("qr_q", _householder(m, n))
    return np.linalg.qr(X, mode="reduced")


def svd(X, keep):
    """Thin SVD (numpy); `keep` singular triplets are used by the caller."""
    if _active:
        m, n = X.shape
        k, K = min(m, n), max(m, n)
        f = 4.0 * K * k * k - (4.0 / 3.0) * k ** 3
        f += keep * (4.0 * m * k - 2.0 * k * k) + keep * (4.0 * n * k - 2.0 * k * k)
        _add("svd", f)
    return np.linalg.svd(X, full_matrices=False)
