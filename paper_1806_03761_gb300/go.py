"""The gradient-optimisation (GO) main loop of Sec. "Process-level
parallelism" (Step B): every iteration samples configurations from on-device
Markov chains and forms the energy and its gradient (Step B-a: Eq. energy,
Eq. gradients), then applies the sign update of the GO step (Step B-b: the
update after Eq. delta with step length dt(n)), until the energy per site
changes by less than a criterion (the paper uses 1e-5) or a step budget runs
out.  Host orchestration only: every step is peps_vmc_step launches (one
evaluation and one Metropolis sweep per chain and sample), the slot reduction
and peps_grad_step.

Readings where the paper is silent: dt(n) = dt0 * decay**n; the criterion is
|E_n - E_{n-1}| / N < tol on the Monte Carlo energy of consecutive steps; a
GO step uses samples_per_step post-sweep configurations of every chain.

Checkpoint/resume: ``save`` writes the tensors, the chain states, the step
and sweep counters and the energy history (atomically: temporary file, then
rename); a loop restored with ``load`` continues bit-identically to one that
never stopped, because every random draw comes from the counter-based
generator keyed by (seed, sweep or step, chain or element) and the batch sums
are formed in a fixed order.
"""
import os

import numpy as np

from . import PepsContext
from .dist import allreduce_sums


class GOLoop:
    def __init__(self, ctx, A, seed, n_chains, samples_per_step=1, n_burn=10, dt0=1e-3,
                 decay=1.0, tol=1e-5, chain_offset=0, world=1):
        """ctx: a PepsContext; A: float64 device tensor [N,2,D,D,D,D], updated
        in place (and loaded into ctx)."""
        import torch
        self.torch = torch
        self.ctx = ctx
        self.A = A
        self.seed = int(seed)
        self.n_chains = int(n_chains)
        self.spc = int(samples_per_step)
        self.n_burn = int(n_burn)
        self.dt0, self.decay, self.tol = float(dt0), float(decay), float(tol)
        self.chain_offset = int(chain_offset)
        self.world = int(world)
        self.step = 0
        self.sweep = 0
        self.energies = []
        self.state = None
        self.sums = ctx.new_sums()
        ctx.set_tensors(A)

    def dt(self, n):
        return self.dt0 * self.decay ** n

    def _start_chains(self):
        # Fisher-Yates starts and n_burn sweeps; the last burn-in state is the
        # first configuration evaluated
        st = self.ctx.sample(self.seed, self.n_chains, max(self.n_burn - 1, 0), 1, 1,
                             chain_offset=self.chain_offset, first_sweep=1)
        self.state = st.view(self.n_chains, self.ctx.N).contiguous()
        self.sweep = max(self.n_burn, 1) + 1

    def step_once(self):
        """One GO iteration; returns the energy per site of its samples."""
        if self.state is None:
            self._start_chains()
        for s in range(self.spc):
            self.ctx.vmc_step(self.seed, self.state, self.sweep, chain_offset=self.chain_offset,
                              sums=self.sums, accumulate=s > 0)
            self.sweep += 1
        allreduce_sums(self.sums, self.world)
        M = self.n_chains * self.spc * self.world
        e = float(self.sums[2].item()) / M / self.ctx.N
        self.ctx.grad_step(self.sums, M, self.dt(self.step), self.seed, self.step, self.A)
        self.step += 1
        self.energies.append(e)
        return e

    def converged(self):
        return (len(self.energies) >= 2
                and abs(self.energies[-1] - self.energies[-2]) < self.tol)

    def run(self, max_steps, checkpoint=None, every=1):
        """Iterate until converged() or max_steps further steps; save a
        checkpoint to `checkpoint` every `every` steps (and at the end)."""
        for k in range(int(max_steps)):
            self.step_once()
            if checkpoint and (k + 1) % every == 0:
                self.save(checkpoint)
            if self.converged():
                break
        if checkpoint:
            self.save(checkpoint)
        return list(self.energies)

    # -- checkpoint / resume ------------------------------------------------
    def save(self, path):
        if self.A.is_cuda:
            self.torch.cuda.synchronize()
        c = self.ctx
        state = (self.state.cpu().numpy() if self.state is not None
                 else np.zeros((0, c.N), np.uint8))
        tmp = path + ".tmp"
        with open(tmp, "wb") as f:
            np.savez(f, A=self.A.cpu().numpy(), state=state,
                     counters=np.array([self.step, self.sweep, self.seed, self.n_chains, self.spc,
                                        self.n_burn, self.chain_offset, self.world], np.int64),
                     shape=np.array([c.L, c.D, c.Dc], np.int64),
                     precision=np.array(c.precision),
                     hyper=np.array([self.dt0, self.decay, self.tol], np.float64),
                     energies=np.array(self.energies, np.float64))
        os.replace(tmp, path)

    @classmethod
    def load(cls, path, ctx=None, slots=0, device="cuda"):
        """Restore a loop; ctx (optional) must have the saved shape."""
        import torch
        z = np.load(path)
        L, D, Dc = (int(x) for x in z["shape"])
        prec = str(z["precision"])
        if ctx is None:
            ctx = PepsContext(L, D, Dc, precision=prec, slots=slots)
        elif (ctx.L, ctx.D, ctx.Dc, ctx.precision) != (L, D, Dc, prec):
            raise ValueError("checkpoint shape %s does not match the context" % ((L, D, Dc, prec),))
        step, sweep, seed, n_chains, spc, n_burn, off, world = (int(x) for x in z["counters"])
        dt0, decay, tol = (float(x) for x in z["hyper"])
        A = torch.from_numpy(z["A"]).to(device)
        loop = cls(ctx, A, seed, n_chains, spc, n_burn, dt0, decay, tol, off, world)
        loop.step, loop.sweep = step, sweep
        loop.energies = [float(x) for x in z["energies"]]
        if z["state"].shape[0]:
            loop.state = torch.from_numpy(z["state"]).to(device).contiguous()
        return loop
