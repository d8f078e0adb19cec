"""peps_amplitudes_noalloc: the amplitude entry point for callers that cannot
allocate device memory (its workspace is a fixed device array inside the
library).  Called through the C ABI and compared with peps_amplitudes, which
allocates its workspace in a context, on two calls in a row (the second with
other spins, so stale scratch contents would show).  This file is collected
last so that a failure here stops a -x run only after every other test ran."""
import ctypes

import numpy as np
import pytest

from synth import make_peps, random_sz0_configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 form's tolerance against the reference computation


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_03761_gb300 import _lib
    return _lib.load()


def _noalloc(lib, shape, A, spins):
    B = spins.shape[0]
    la = torch.empty(B, dtype=torch.float64, device="cuda")
    sg = torch.empty(B, dtype=torch.int8, device="cuda")
    rc = lib.peps_amplitudes_noalloc(ctypes.byref(shape), ctypes.c_void_p(A.data_ptr()),
                                     ctypes.c_void_p(spins.data_ptr()), B,
                                     ctypes.c_void_p(la.data_ptr()), ctypes.c_void_p(sg.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, la, sg


@pytest.mark.parametrize("L,D,Dc,kind", [(6, 3, 4, "gauss"), (8, 4, 16, "neel")])
def test_noalloc_matches_allocating_entry_point(lib, L, D, Dc, kind):
    from paper_1806_03761_gb300 import PepsContext, _lib
    A = torch.from_numpy(make_peps(L, D, seed=21, kind=kind)).cuda()
    shape = _lib.PepsShape(L, D, Dc, 1.0, 0.5, _lib.PEPS_FP64)
    ctx = PepsContext(L, D, Dc, precision="fp64")
    ctx.set_tensors(A)
    for call in range(2):  # two calls in a row, different spins
        spins = torch.from_numpy(random_sz0_configs(L, 9 + call, seed=30 + call)).cuda()
        rc, la, sg = _noalloc(lib, shape, A, spins)
        assert rc == _lib.PEPS_OK
        ref_la, ref_sg = ctx.amplitudes(spins)
        torch.cuda.synchronize()
        assert torch.equal(sg, ref_sg)
        assert float((la - ref_la).abs().max()) <= TOL
    ctx.close()


def test_noalloc_rejects_shapes_beyond_its_scratch(lib):
    from paper_1806_03761_gb300 import _lib
    A = torch.zeros(24 * 24 * 2 * 8 ** 4, dtype=torch.float64, device="cuda")
    spins = torch.zeros(1, 24 * 24, dtype=torch.uint8, device="cuda")
    big = _lib.PepsShape(24, 8, 32, 1.0, 0.5, _lib.PEPS_FP64)
    rc, _, _ = _noalloc(lib, big, A, spins)
    assert rc == _lib.PEPS_ESCRATCH
    mixed = _lib.PepsShape(4, 2, 4, 1.0, 0.5, _lib.PEPS_MIXED)
    rc, _, _ = _noalloc(lib, mixed, A, spins[:, :16])
    assert rc == _lib.PEPS_EINVAL


def test_noalloc_reuses_slots_for_more_samples_than_fit(lib):
    """More samples than the scratch holds at once: 8x8, D=4, Dc=16 fits 39
    per-sample workspaces, so 64 samples run on 39 slots, some slots taking
    two samples in turn (the grid-stride loop), twice in a row."""
    from paper_1806_03761_gb300 import PepsContext, _lib
    L, D, Dc = 8, 4, 16
    A = torch.from_numpy(make_peps(L, D, seed=2, kind="neel")).cuda()
    shape = _lib.PepsShape(L, D, Dc, 1.0, 0.5, _lib.PEPS_FP64)
    ctx = PepsContext(L, D, Dc, precision="fp64")
    ctx.set_tensors(A)
    for call in range(2):
        spins = torch.from_numpy(random_sz0_configs(L, 64, seed=40 + call)).cuda()
        rc, la, sg = _noalloc(lib, shape, A, spins)
        assert rc == _lib.PEPS_OK
        ref_la, ref_sg = ctx.amplitudes(spins)
        torch.cuda.synchronize()
        assert torch.equal(sg, ref_sg)
        assert float((la - ref_la).abs().max()) <= TOL
    ctx.close()
