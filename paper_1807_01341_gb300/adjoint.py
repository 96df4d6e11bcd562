"""Differentiable runs: the gradient of a loss on the SPH density of a run's
final state, sampled on a grid, with respect to the run's initial positions,
velocities and internal energies.

The forward steps are the library's kick-drift-kick steps; the backward pass
runs sph_step_bwd over them in reverse, with checkpoint-and-recompute: the
state before every k-th step is kept (in the caller's particle order), and
the backward pass recomputes each segment of k steps from its checkpoint,
keeping the states before each of its steps, then runs the segment's steps
backwards.  Memory: one state per checkpoint plus k + 1 states.

So that a recomputed segment repeats the original steps bit for bit, the
forward run also restarts from each checkpoint (sph_resume: the cells are
rebuilt from the checkpointed order) and uses one lane per particle.

The paper has no adjoint; this module only orchestrates library calls
(argument marshalling).  :class:`GridDensityRun` wraps it as a
torch.autograd.Function.
"""
from __future__ import annotations

import torch

from . import _lib
from .sim import Adjoint, Context, Params, Particles


class Run:
    """n_steps kick-drift-kick steps from given initial positions, velocities
    and internal energies (masses and initial h guesses fixed), then the SPH
    density of the final state on an n_grid^3 grid.

    checkpoint_every = k: states kept before steps 0, k, 2k, ...; the backward
    pass recomputes k steps at a time."""

    def __init__(self, params: Params, m, h0, n_steps: int, n_grid: int,
                 checkpoint_every: int = 5, form: int = _lib.SPH_FORM_BATCHED, device="cuda"):
        if params.threads_per_particle != 1:
            raise ValueError("differentiable runs need threads_per_particle = 1 (bitwise recompute)")
        if n_steps < 1 or checkpoint_every < 1:
            raise ValueError("n_steps and checkpoint_every must be >= 1")
        self.params = params
        self.m = torch.as_tensor(m, dtype=torch.float32, device=device)
        self.h0 = torch.as_tensor(h0, dtype=torch.float32, device=device)
        self.n = int(self.m.shape[0])
        self.n_steps, self.n_grid = int(n_steps), int(n_grid)
        self.k = int(checkpoint_every)
        self.form = form
        self.device = torch.device(device)
        self.ctx = Context(params, self.n)
        self.p = Particles(self.n, device, with_counts=False)
        self.checkpoints: dict[int, Particles] = {}
        self.ticks: list[int] = []
        self.final: Particles | None = None
        self.recomputed_final: Particles | None = None  # the last step's state, recomputed

    # -- helpers -----------------------------------------------------------
    def _new_state(self) -> Particles:
        return Particles(self.n, self.device, with_counts=False)

    def _load(self, src: Particles, ti: int, first: bool):
        """The live state becomes src (caller order), resumed at tick ti."""
        self.ctx.state_copy(src, self.p, False)
        self.ctx.resume(self.p, ti, first)

    def _snapshot(self) -> Particles:
        """The live state in the caller's order."""
        s = self._new_state()
        self.ctx.state_copy(self.p, s, True)
        return s

    def _next_tick(self) -> int:
        return self.ctx.get_time()[1]

    # -- forward -----------------------------------------------------------
    def forward(self, pos0: torch.Tensor, vel0: torch.Tensor, u0: torch.Tensor) -> torch.Tensor:
        p0 = self._new_state()
        p0.x.copy_(pos0[:, 0])
        p0.y.copy_(pos0[:, 1])
        p0.z.copy_(pos0[:, 2])
        p0.vx.copy_(vel0[:, 0])
        p0.vy.copy_(vel0[:, 1])
        p0.vz.copy_(vel0[:, 2])
        p0.m.copy_(self.m)
        p0.A.copy_(u0)  # A holds u until the first density pass
        p0.h.copy_(self.h0)
        self.ctx.begin_run()
        self.checkpoints = {}
        self.ticks = []
        ti = 0
        for k in range(self.n_steps):
            if k % self.k == 0:
                snap = p0 if k == 0 else self._snapshot()
                self.checkpoints[k] = snap
                self._load(snap, ti, k == 0)
            self.ticks.append(ti)
            self.ctx.step(self.p, self.form)
            ti = self._next_tick()
        self.final = self._snapshot()
        return self.ctx.grid_density(self.final, self.n_grid, self.ticks[-1])

    # -- backward ----------------------------------------------------------
    def backward(self, rho_bar: torch.Tensor):
        """d loss / d (pos0, vel0, u0) from d loss / d rho_grid."""
        if self.final is None:
            raise RuntimeError("forward first")
        adj = Adjoint(self.n, self.device)
        self.ctx.grid_density_bwd(self.final, self.n_grid, self.ticks[-1],
                                  rho_bar.to(device=self.device, dtype=torch.float64), adj)
        starts = sorted(self.checkpoints)
        for s in reversed(starts):
            e = min(s + self.k, self.n_steps)
            # recompute the segment, keeping the state before each step
            self._load(self.checkpoints[s], self.ticks[s], s == 0)
            tape = [self.checkpoints[s]]
            for k in range(s, e):
                self.ctx.step(self.p, self.form)
                tape.append(self._snapshot())
            if e == self.n_steps:
                self.recomputed_final = tape[-1]
            for k in range(e - 1, s - 1, -1):
                self.ctx.step_bwd(tape[k - s], tape[k - s + 1], self.ticks[k], k == 0, adj)
        gpos = torch.stack([adj.x, adj.y, adj.z], dim=1)
        gvel = torch.stack([adj.vx, adj.vy, adj.vz], dim=1)
        return gpos, gvel, adj.A.clone()

    def close(self):
        self.ctx.close()


class GridDensityRun(torch.autograd.Function):
    """rho_grid = GridDensityRun.apply(pos0, vel0, u0, run): the grid density
    of the final state of `run` (a :class:`Run`); its backward is the library's
    reverse pass."""

    @staticmethod
    def forward(fctx, pos0, vel0, u0, run: Run):
        fctx.run = run
        return run.forward(pos0.detach(), vel0.detach(), u0.detach())

    @staticmethod
    def backward(fctx, g):
        gpos, gvel, gu = fctx.run.backward(g.detach())
        return gpos, gvel, gu, None
