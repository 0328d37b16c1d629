"""Gradient of the time-integrated heat release with respect to the slot
burner's profile coefficients, by the discrete adjoint of the whole step.

J(c) = sum_{n=1..N} dt * sum_cells omega(level n) dV, the profile samples are
basis @ c (e.g. Gaussian bumps across the slot face), omega the flame-sheet
heat-release rate (sim_objective).  The adjoint runs through the C ABI:
sim_adjoint_step transposes one step given the state it starts from, so the
reverse sweep needs every level's state again.  Checkpointing: the forward run
keeps the restart state every `every` steps (device copies); the reverse sweep
re-runs one segment at a time from its checkpoint, keeping that segment's
states, then steps back through it.  Memory: (N / every + every) states; work:
about two forward runs plus the adjoint sweep.

Everything here is argument marshalling; every step of the computation runs in
the library's CUDA kernels.
"""

import numpy as np

from .lowmach import Simulation


class HeatReleaseProblem:
    """One simulation reused for every evaluation of J(c) and its gradient."""

    def __init__(self, prm, geo, fields, basis, nsteps, every=20, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.prm = dict(prm)
        self.geo = dict(geo)
        self.fields = fields
        self.basis = np.asarray(basis, dtype=np.float64)
        self.nsteps = int(nsteps)
        self.every = max(1, int(every))
        self.device = torch.device(device)
        self.sim = Simulation(self.prm, self._geo(np.ones(self.basis.shape[1])), device=self.device,
                              stream=stream)
        self.state_bytes = None
        self.ckpt = {}
        self.c = None

    def _geo(self, c):
        g = dict(self.geo)
        g["profile"] = list(self.basis @ np.asarray(c, dtype=np.float64))
        return g

    def _save(self):
        if self.state_bytes is None:
            self.state_bytes = self.sim.state_size()
        buf = self.torch.empty(self.state_bytes, dtype=self.torch.uint8, device=self.device)
        self.sim.state_save(buf)
        return buf

    def value(self, c, keep_checkpoints=True):
        """J(c); keeps the checkpoints for gradient()."""
        sim = self.sim
        dt = float(self.prm["dt"])
        sim.set_ibm(self._geo(c))
        sim.set_fields(self.fields)
        sim.step(0)                                   # level 0: state relation, F^0, mass
        self.ckpt = {0: self._save()} if keep_checkpoints else {}
        J = 0.0
        for n in range(self.nsteps):
            sim.step(1)
            J += dt * sim.objective()                 # level n + 1
            if keep_checkpoints and (n + 1) % self.every == 0 and n + 1 < self.nsteps:
                self.ckpt[n + 1] = self._save()
        sim.sync()
        self.c = np.array(c, dtype=np.float64)
        return J

    def gradient(self):
        """dJ/dc at the c of the last value() call (and dJ/d samples)."""
        if self.c is None or 0 not in self.ckpt:
            raise RuntimeError("value(c) must run (with checkpoints) before gradient()")
        sim = self.sim
        dt = float(self.prm["dt"])
        n_prof = self.basis.shape[0]
        sim.adjoint_begin()
        g = None
        try:
            for s0 in sorted(self.ckpt, reverse=True):
                s1 = min(s0 + self.every, self.nsteps)
                sim.state_load(self.ckpt[s0])
                seg = [self._save()]
                for _ in range(s0, s1 - 1):
                    sim.step(1)
                    seg.append(self._save())
                for n in range(s1 - 1, s0 - 1, -1):
                    sim.state_load(seg[n - s0])
                    g = sim.adjoint_step(dt, n_profile=n_prof if n == 0 else 0)
        finally:
            sim.adjoint_end()
        return self.basis.T @ g, g

    def close(self):
        self.sim.close()


def heat_release_function():
    """torch.autograd.Function: J = f(c) with the adjoint gradient."""
    import torch

    class HeatRelease(torch.autograd.Function):
        @staticmethod
        def forward(ctx, c, problem):
            ctx.problem = problem
            J = problem.value(c.detach().cpu().numpy().astype(np.float64))
            return c.new_tensor(J)

        @staticmethod
        def backward(ctx, gJ):
            gc, _ = ctx.problem.gradient()
            return gJ * torch.as_tensor(gc, dtype=gJ.dtype, device=gJ.device), None

    return HeatRelease
