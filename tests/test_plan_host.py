"""CPU tests of the host plan the kernels run on (csrc/peps_plan.h, compiled
for the host by tests/host/plan_host.cpp): the bond dimensions of every
absorption step equal the site shapes of the oracle's truncated upper and
lower environments, and every matrix and temporary of the compression fits
the slot layout's capacities, in regions that do not overlap."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle.peps as op
from synth import make_peps, random_sz0_configs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1806_03761_gb300", "csrc")
SHAPES = [(4, 2, 16), (5, 2, 3), (6, 3, 4), (6, 4, 8), (7, 3, 5), (8, 4, 16), (6, 6, 24),
          (6, 8, 32), (16, 6, 24), (24, 8, 32)]


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("plan") / "plan_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(HERE, "host", "plan_host.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    I16 = ctypes.POINTER(ctypes.c_int16)
    lib.h_plan.argtypes = [ctypes.c_int] * 3 + [I16] * 6 + [ctypes.POINTER(ctypes.c_int64)]

    def get(L, D, Dc):
        arrs = [np.zeros((L - 1, L), np.int16) for _ in range(6)]
        caps = np.zeros(27, np.int64)
        rc = lib.h_plan(L, D, Dc, *[a.ctypes.data_as(I16) for a in arrs],
                        caps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        assert rc == 0
        return dict(zip(("ia", "ip", "ib", "r", "oa", "ob"), arrs)), caps
    return get


@pytest.mark.parametrize("L,D,Dc", [s for s in SHAPES if s[0] <= 8])
def test_plan_matches_the_oracle_environments(plan, L, D, Dc):
    st, _ = plan(L, D, Dc)
    A = make_peps(L, D, seed=3)
    s = random_sz0_configs(L, 1, seed=4)[0]
    up = op.upper_envs(A, s, L, Dc)
    dn = op.lower_envs(A, s, L, Dc)
    for t in range(L - 1):
        for j in range(L):
            a, p, b = up[t].sites[j].shape
            assert (a, b) == (st["oa"][t, j], st["ob"][t, j]), (t, j)
            assert p == D
            a2, p2, b2 = dn[L - 1 - t].sites[j].shape
            assert (a2, b2) == (a, b) and p2 == D
            # the step's input is the previous output
            if t > 0:
                assert (st["ia"][t, j], st["ib"][t, j]) == (st["oa"][t - 1, j], st["ob"][t - 1, j])


@pytest.mark.parametrize("L,D,Dc", SHAPES)
def test_compression_fits_the_slot_layout(plan, L, D, Dc):
    """The sizes compress_row indexes with, from the plan, against the
    capacities: input and output sites, the QR panel X_j and the
    contraction temporaries, the R factors, X_j = R Y_j and Y_j."""
    st, caps = plan(L, D, Dc)
    site_cap, env_cap, big_cap, mat_cap, env2_cap, slot_elems, _ = caps[:7]
    assert site_cap == Dc * D * Dc and env2_cap == Dc * D * D * Dc
    for t in range(L - 1):
        rprev = 1
        for j in range(L):
            a, p, b = int(st["ia"][t, j]), int(st["ip"][t, j]), int(st["ib"][t, j])
            Dl, Dr = (1 if j == 0 else D), (1 if j == L - 1 else D)
            assert a * p * b <= site_cap
            assert int(st["oa"][t, j]) * D * int(st["ob"][t, j]) <= site_cap
            assert int(st["oa"][t, j]) <= Dc and int(st["ob"][t, j]) <= Dc
            if j < L - 1:
                assert rprev * Dl * p * b <= big_cap            # S1
                assert rprev * D * b * Dr <= big_cap            # X_j (column-major panel)
                assert int(st["r"][t, j]) * b * Dr <= mat_cap   # R_j
                rprev = int(st["r"][t, j])
        cn = 1
        for j in range(L - 1, 0, -1):
            a = int(st["ia"][t, j])
            Dl = 1 if j == 0 else D
            rr, n = int(st["r"][t, j - 1]), D * cn
            assert a * Dl * n <= mat_cap                        # Y_j
            assert rr * n <= mat_cap                            # X_j = R_{j-1} Y_j
            cn = int(st["oa"][t, j])
    offs = list(caps[7:])
    used = [o for o in offs if o > 0] + [0]
    assert all(o % 32 == 0 for o in offs)
    assert len(set(used)) == len(used)          # distinct regions
    assert max(offs) < slot_elems
    assert env_cap == L * site_cap
