"""Kick-drift-kick integrator with individual power-of-two time bins (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

One call of :meth:`OracleSim.step` advances the system from the current integer
time ``ti`` to the next time at which some particle's step ends (Sec. II-A):

  (i)   drift every particle to ti (x += v_half dt; drift-all, which gives the
        same positions as drifting only the relevant particles) and predict
        v_pred = v_half + a (t - t_mid), A_pred = A + Adot (t - t_mid);
  (ii)  the active set: particles whose step ends at ti (Eq. 2, read as
        "every bin n with ti a multiple of 2^n");
  (iii) density loop with the smoothing-length iteration for the active
        particles; inactive neighbours keep their last h, rho, f and take
        P, c from their predicted entropy;
  (iv)  force loop for the active particles;
  (v)   closing half-kick of the old step: v += a dt_old/2, A += Adot dt_old/2;
  (vi)  new time-step (Eq. 1), bin (Eq. 2) and end time;
  (vii) opening half-kick of the new step: v += a dt_new/2, A += Adot dt_new/2.

The first step (ti = 0, every particle active with a zero-length old step)
sets the entropy from the initial internal energy after its density pass.
The integer timeline has ticks of dt_min; the time of tick ti is t_begin + ti dt_min.

Variants (Gadget-2's; off by default):
  predict   inactive particles' density and smoothing length are predicted
            from their last density with their velocity divergence over the
            time since then, rho exp(-div v dt), h exp(div v dt / 3) (an active
            particle starts its h iteration from its predicted h);
  balsara   the viscosity of a pair is scaled by the mean of the two
            particles' Balsara factors;
  limiter   a new bin is at most 2 above the smallest bin among the
            particle's force neighbours, and an inactive neighbour whose bin is
            more than 2 above an active particle's is woken: its step is cut to
            end at the first multiple of 2^(bin_i + 2) after the current tick
            (Saitoh & Makino 2009; the waking as Durier & Dalla Vecchia 2012
            describe it, with the bins of the step being closed).
The divergence and curl (needed by predict and balsara) are taken after the
density loop at each active particle's new h, with the step's predicted
velocities.
"""
from __future__ import annotations

import numpy as np


class OracleSim:
    def __init__(self, pos, vel, m, u, h0, *, box=1.0, eta=1.2348, gamma=5.0 / 3.0,
                 alpha=0.8, cfl=0.1, dt_min=1e-6, bin_cap=10, h_tol=1e-12, max_iter=100,
                 use_cells=True, global_step=False, predict=False, balsara=False,
                 limiter=False):
        n = pos.shape[0]
        self.n = n
        self.box, self.eta, self.gamma, self.alpha = box, eta, gamma, alpha
        self.cfl, self.dt_min, self.bin_cap = cfl, dt_min, bin_cap
        self.h_tol, self.max_iter, self.use_cells = h_tol, max_iter, use_cells
        self.global_step = global_step
        self.predict, self.balsara, self.limiter = predict, balsara, limiter
        self.divv = np.zeros(n)   # velocity divergence at the last density
        self.curl = np.zeros(n)   # |curl v| at the last density
        self.pos = np.array(pos, dtype=np.float64) % box
        self.vel = np.array(vel, dtype=np.float64)
        self.m = np.array(m, dtype=np.float64) * np.ones(n)
        self.u0 = np.array(u, dtype=np.float64) * np.ones(n)
        self.h = np.array(h0, dtype=np.float64) * np.ones(n)
        self.acc = np.zeros((n, 3))
        self.A = np.zeros(n)
        self.Adot = np.zeros(n)
        self.rho = np.zeros(n)
        self.drho_dh = np.zeros(n)
        self.f = np.ones(n)
        self.P = np.zeros(n)
        self.c = np.zeros(n)
        self.vsig = np.zeros(n)
        self.bin = np.zeros(n, dtype=np.int8)
        self.ti_begin = np.zeros(n, dtype=np.int64)
        self.ti_end = np.zeros(n, dtype=np.int64)
        self.ti = 0                               # current integer time
        self.ti_drift = np.zeros(n, dtype=np.int64)  # tick each position refers to
        self.first = True
        self.n_steps = 0
        self.pairs_density = 0
        self.pairs_force = 0
        self.last_active = None
        self.E_sync = []       # total energy at steps where every particle is synchronised

    # -- the pieces of one step --------------------------------------------
    def _drift(self, ti):
        dt = (ti - self.ti_drift) * self.dt_min
        moved = dt != 0.0
        if moved.any():
            self.pos[moved] = (self.pos[moved] + self.vel[moved] * dt[moved, None]) % self.box
        self.ti_drift[:] = ti

    def _predict(self, ti):
        """v_pred and A_pred at ti from the half-step state (the middle of
        each particle's step: its length is 2^bin, or shorter once woken)."""
        step = self.ti_end - self.ti_begin
        dtp = ((ti - self.ti_begin) - 0.5 * step) * self.dt_min
        return self.vel + self.acc * dtp[:, None], self.A + self.Adot * dtp

    def _predict_rho_h(self, ti):
        """rho and h at ti: the last values, or (predict) those advanced with
        the velocity divergence over the time since the last density."""
        if not self.predict:
            return self.rho.copy(), self.h.copy()
        import oracle as orc
        dt = (ti - self.ti_begin) * self.dt_min
        return orc.predict_inactive(self.rho, self.h, self.divv, dt)

    def step(self):
        import oracle as orc
        ti = self.ti
        g = self.gamma
        self._drift(ti)
        vpred, Apred = self._predict(ti)
        active = self.ti_end == ti
        self.last_active = active.copy()
        rho_p, h_p = self._predict_rho_h(ti)
        d = orc.density(self.pos, self.m, h_p, active, self.box, self.eta, self.h_tol,
                        self.max_iter, self.use_cells)
        self.h[active] = d["h"][active]
        self.rho[active] = d["rho"][active]
        self.drho_dh[active] = d["drho_dh"][active]
        self.pairs_density += int(d["count"][active].sum())
        self.f[active] = orc.gradh_f(self.h[active], self.rho[active], self.drho_dh[active])
        if self.first:
            self.A = orc.entropy_from_u(self.u0, self.rho, g)
            Apred = self.A.copy()
        if self.predict or self.balsara:
            gr = orc.gradient(self.pos, vpred, self.m, self.h, self.rho, active, self.box,
                              self.use_cells)
            self.divv[active] = gr["div"][active]
            self.curl[active] = np.sqrt((gr["curl"] ** 2).sum(1))[active]
        # inactive neighbours: their last (or predicted) rho and h
        h_now = np.where(active, self.h, h_p)
        rho_now = np.where(active, self.rho, rho_p)
        self.P, self.c = orc.eos(Apred, rho_now, g)
        bal = orc.balsara(self.divv, self.curl, self.c, h_now) if self.balsara else None
        fr = orc.force(self.pos, vpred, self.m, h_now, rho_now, self.f, self.P, self.c,
                       active, self.box, self.alpha, g, self.use_cells, balsara=bal,
                       bins=self.bin if self.limiter else None)
        self.acc[active] = fr["a"][active]
        self.Adot[active] = fr["Adot"][active]
        self.vsig[active] = fr["vsig"][active]
        self.pairs_force += int(fr["count"][active].sum())
        # wake requests from the force loop's pairs, with the bins of this step
        req = (orc.wake_bins(self.pos, h_now, active, self.bin, self.box, self.use_cells)
               if self.limiter else None)
        # (v) closing half-kick of the old step
        dt_old = ((self.ti_end - self.ti_begin) * self.dt_min)[active]
        self.vel[active] += self.acc[active] * (0.5 * dt_old)[:, None]
        self.A[active] += self.Adot[active] * (0.5 * dt_old)
        if active.all():
            v2 = (self.vel ** 2).sum(axis=1)
            u = orc.u_from_entropy(self.A, self.rho, g)
            self.E_sync.append(float((self.m * (0.5 * v2 + u)).sum()))
        # (vi) new time-step and bin
        cap = 0 if self.global_step else self.bin_cap
        tb = orc.timestep_bins(self.h, self.vsig, active, self.cfl, self.dt_min, cap, ti,
                               self.bin, fr["bin_ngb_min"] if self.limiter else None)
        self.n_dt_too_small = tb["n_too_small"]
        self.bin[active] = tb["bin"][active]
        self.ti_begin[active] = tb["ti_begin"][active]
        self.ti_end[active] = tb["ti_end"][active]
        # (vii) opening half-kick of the new step
        dt_new = ((self.ti_end - self.ti_begin) * self.dt_min)[active]
        self.vel[active] += self.acc[active] * (0.5 * dt_new)[:, None]
        self.A[active] += self.Adot[active] * (0.5 * dt_new)
        # (viii) limiter: inactive neighbours of much shorter steps are woken
        self.n_woken = 0
        if self.limiter:
            self.n_woken = orc.wake(ti, req, active, self.bin, self.ti_begin, self.ti_end,
                                    self.vel, self.A, self.acc, self.Adot, self.dt_min)
        self.first = False
        self.n_steps += 1
        self.ti = int(self.ti_end.min())
        return active

    @classmethod
    def from_state(cls, st, *, ti, first=False, **kw):
        """An oracle integrator holding a given state (FP64 copies of the
        arrays of a particle structure: x, y, z, vx.., ax.., A, Adot, h, rho, f,
        m, bin, ti_begin, ti_end, ti_drift) at integer time ti.  With first,
        A holds u and the next step is the initial one."""
        pos = np.stack([st["x"], st["y"], st["z"]], axis=1).astype(np.float64)
        vel = np.stack([st["vx"], st["vy"], st["vz"]], axis=1).astype(np.float64)
        s = cls(pos, vel, st["m"].astype(np.float64), st["A"].astype(np.float64),
                st["h"].astype(np.float64), **kw)
        s.pos = pos.copy()
        s.acc = np.stack([st["ax"], st["ay"], st["az"]], axis=1).astype(np.float64)
        s.A = st["A"].astype(np.float64).copy()
        s.Adot = st["Adot"].astype(np.float64).copy()
        s.rho = st["rho"].astype(np.float64).copy()
        s.f = st["f"].astype(np.float64).copy()
        s.bin = st["bin"].astype(np.int8).copy()
        s.ti_begin = st["ti_begin"].astype(np.int64).copy()
        s.ti_end = st["ti_end"].astype(np.int64).copy()
        s.ti_drift = st["ti_drift"].astype(np.int64).copy()
        if "div_v" in st:
            s.divv = st["div_v"].astype(np.float64).copy()
        if "curl_v" in st:
            s.curl = st["curl_v"].astype(np.float64).copy()
        s.ti = int(ti)
        s.first = bool(first)
        return s

    def momentum(self):
        return (self.m[:, None] * self.vel).sum(axis=0)
