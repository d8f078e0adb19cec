"""The C-ABI library builds, loads without a GPU, and exports every entry point
include/peps.h declares; host-side logic that needs no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_03761_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1806_03761_gb300 import build
        build.build()
    return _lib.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "peps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(peps_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("peps_sample_batch", "peps_amplitudes", "peps_local_energy", "peps_logderiv",
              "peps_grad_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1806_03761_gb300 import _lib
    names = declared_entry_points()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_no_torch_types_in_the_header():
    src = open(os.path.join(ROOT, "include", "peps.h")).read()
    assert "torch" not in src.lower().replace("pytorch", "")
    assert "extern \"C\"" in src


def test_workspace_and_flop_model_host_only(lib):
    import paper_1806_03761_gb300 as p
    # host-only calls: no device needed
    n1 = p.workspace_bytes(16, 6, 24, "fp64", slots=1)
    n2 = p.workspace_bytes(16, 6, 24, "fp64", slots=2)
    assert n2 > n1 > 10 * 2 ** 20
    f = p.flops_per_sample(16, 6, 24)
    assert 1e10 < f < 5e11
    fs, fv = p.flops_per_sample(16, 6, 24, what="sweep"), p.flops_per_sample(16, 6, 24, what="vmc")
    assert fv < f + fs  # the fused step reuses the lower environments
    assert p.flops_per_sample(1, 6, 24) == 0.0
    assert p.workspace_bytes(1, 6, 24) == 0  # bad shape
    assert p.workspace_bytes(16, 6, 100) == 0  # Dc*D > 256


def test_invalid_shapes_rejected_without_a_device(lib):
    from paper_1806_03761_gb300 import _lib
    h = ctypes.c_void_p()
    for shape in ((1, 2, 4), (33, 2, 4), (4, 0, 4), (4, 9, 4), (4, 2, 0), (4, 8, 40)):
        s = _lib.PepsShape(shape[0], shape[1], shape[2], 1.0, 0.5, 0)
        assert lib.peps_create(ctypes.byref(s), 0, ctypes.byref(h)) == _lib.PEPS_EINVAL
    s = _lib.PepsShape(4, 2, 4, 1.0, 0.5, 7)
    assert lib.peps_create(ctypes.byref(s), 0, ctypes.byref(h)) == _lib.PEPS_EINVAL
    assert lib.peps_destroy(None) == _lib.PEPS_EINVAL


def test_server_refuses_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_1806_03761_gb300 import _lib
    h = ctypes.c_void_p()
    assert lib.peps_server_create(0, 0, ctypes.byref(h)) == _lib.PEPS_ECUDA
    assert lib.peps_server_create(0, -1, ctypes.byref(h)) == _lib.PEPS_EINVAL
    assert lib.peps_server_destroy(None) == _lib.PEPS_EINVAL
