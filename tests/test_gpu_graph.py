"""The VMC step captured in a CUDA graph: peps_vmc_step_dc, peps_grad_step_dc
and peps_counters_advance read their Philox counters from device memory, so
one captured step replayed K times gives the chain states, energies, gradient
sums and site tensors of K steps called directly, bit for bit."""
import numpy as np
import pytest

from synth import make_peps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_equals_direct_steps(prec):
    from paper_1806_03761_gb300 import PepsContext
    L, D, Dc, n, K, seed, dt = 5, 2, 4, 6, 3, 2468, 1e-2
    A0 = torch.from_numpy(make_peps(L, D, seed=33)).cuda()
    runs = {}
    for mode in ("direct", "graph"):
        A = A0.clone()
        ctx = PepsContext(L, D, Dc, precision=prec, slots=3)
        ctx.set_tensors(A)
        state = ctx.sample(seed, n, 2, 1, 1).contiguous()
        sums = ctx.new_sums()
        out = dict(e_loc=torch.empty(n, dtype=torch.float64, device="cuda"),
                   log_abs=torch.empty(n, dtype=torch.float64, device="cuda"),
                   sign=torch.empty(n, dtype=torch.int8, device="cuda"))
        energies = []
        if mode == "direct":
            for k in range(K):
                ctx.vmc_step(seed, state, 10 + k, sums=sums, out=out)
                ctx.grad_step(sums, n, dt, seed, 100 + k, A)
                energies.append(out["e_loc"].clone())
        else:
            counters = ctx.new_counters(10, 100)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                ctx.vmc_step_dc(seed, state, counters, sums=sums, out=out)
                ctx.grad_step_dc(sums, n, dt, seed, counters, A)
                ctx.advance_counters(counters)
            for k in range(K):
                g.replay()
                torch.cuda.synchronize()
                energies.append(out["e_loc"].clone())
            assert counters.cpu().tolist() == [10 + K, 100 + K]
        torch.cuda.synchronize()
        assert ctx.sync_status()[0] == 0
        runs[mode] = (state.cpu().numpy(), [e.cpu().numpy() for e in energies], A.cpu().numpy(),
                      [x.cpu().numpy() for x in sums])
        ctx.close()
    d, gr = runs["direct"], runs["graph"]
    assert np.array_equal(d[0], gr[0])
    for a, b in zip(d[1], gr[1]):
        assert np.array_equal(a, b)
    assert np.array_equal(d[2], gr[2])
    for a, b in zip(d[3], gr[3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_host_buffer_step_equals_device_step(prec):
    """peps_vmc_step_host (chain states, energies and sum E in host memory)
    gives the device step's states, energies and sums bit for bit."""
    from paper_1806_03761_gb300 import PepsContext
    L, D, Dc, n, seed = 5, 2, 4, 7, 1357
    A = torch.from_numpy(make_peps(L, D, seed=34)).cuda()
    ctx = PepsContext(L, D, Dc, precision=prec, slots=3)
    ctx.set_tensors(A)
    state = ctx.sample(seed, n, 2, 1, 1).contiguous()
    host_state = state.cpu().pin_memory()
    dev = ctx.vmc_step(seed, state, 7)
    sums = ctx.new_sums()
    host_e = torch.empty(n, dtype=torch.float64).pin_memory()
    host_se = torch.empty(1, dtype=torch.float64).pin_memory()
    ctx.vmc_step_host(seed, host_state, 7, sums, host_e, host_se)
    torch.cuda.synchronize()
    assert torch.equal(host_state, state.cpu())
    assert torch.equal(host_e, dev["e_loc"].cpu())
    assert torch.equal(host_se, dev["sum_e"].cpu())
    for a, b in zip(sums, (dev["sum_delta"], dev["sum_delta_e"], dev["sum_e"])):
        assert torch.equal(a, b)
    assert ctx.sync_status()[0] == 0
    ctx.close()
