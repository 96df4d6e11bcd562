"""Gradient oracle: the kick-drift-kick run of :mod:`oracle.kdk`, re-expressed
with PyTorch FP64 CPU tensors so that automatic differentiation gives the
gradient of a loss on the final state with respect to the initial positions,
velocities and internal energies.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It shares nothing with
the CUDA library; its derivative is taken by torch.autograd from the plain
formulas below, independently of any hand-derived adjoint.

The forward is the same run as ``OracleSim`` (Sec. II-A time integration with
individual power-of-two bins, Eq. 1 and Eq. 2), step by step:

  drift of every particle to the step's tick; prediction of v and A; the
  density loop with the smoothing-length solve for the active particles; the
  entropy from u on the first step; the equation of state for every
  particle; the force loop for the active particles; the closing half-kick,
  new bins, the opening half-kick.

The discrete parts (which particles are active, the bins, the integer times)
are piecewise constant in the inputs: they are taken from the FP64 values
without a derivative, through the C oracle's own bin routine.  The smoothing
length solves h^3 n(h) = eta^3; the C oracle finds the root, and one Newton
step at the root, h* - F(h*, x) / F_h(h*, x) with F_h held constant, carries
the implicit derivative dh/dx = -F_x / F_h.

The loss (the differentiation workload): the SPH density of the final state
sampled on a regular grid of n_g^3 points, rho(x_g) = sum_j m_j W(|x_g - x_j|,
h_j) (each particle's own smoothing length), compared with a target by the sum
of squared differences.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as orc

GAMMA_K = orc.GAMMA_K
KN = 8.0 / np.pi
DT = torch.float64


# ---------------------------------------------------------------------------
# kernel (cubic spline; dimensionless w(q) with w(0) = 1, W = (8/pi) H^-3 w)
# ---------------------------------------------------------------------------
def w_q(q):
    """w(q): 1 - 6q^2 + 6q^3 (q < 1/2), 2 (1 - q)^3 (q < 1), 0 beyond."""
    s = 1.0 - q
    inner = 1.0 - 6.0 * q * q + 6.0 * q * q * q
    outer = 2.0 * s * s * s
    return torch.where(q < 0.5, inner, torch.where(q < 1.0, outer, torch.zeros_like(q)))


def dw_q(q):
    """w'(q)."""
    s = 1.0 - q
    inner = -12.0 * q + 18.0 * q * q
    outer = -6.0 * s * s
    return torch.where(q < 0.5, inner, torch.where(q < 1.0, outer, torch.zeros_like(q)))


def min_image(d, box):
    return d - box * torch.round(d / box)


def _wrap_np(p, box):
    p = np.mod(p, box)
    return np.where(p >= box, p - box, p)


# ---------------------------------------------------------------------------
# neighbour pairs (no derivative: which pairs exist is piecewise constant, and
# W and W' vanish at the edge of the support)
# ---------------------------------------------------------------------------
def _tree(pos_np, box):
    from scipy.spatial import cKDTree
    return cKDTree(_wrap_np(pos_np, box), boxsize=box)


def pairs_within(pos_np, centres_idx, radius, box, tree=None):
    """(I, J): I in centres_idx, J != I with |x_I - x_J| <= radius[I]."""
    tree = tree if tree is not None else _tree(pos_np, box)
    lists = tree.query_ball_point(_wrap_np(pos_np[centres_idx], box), r=radius[centres_idx])
    I = np.repeat(centres_idx, [len(l) for l in lists])
    J = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]) if len(lists) else \
        np.zeros(0, dtype=np.int64)
    keep = I != J
    return I[keep].astype(np.int64), J[keep].astype(np.int64)


def force_pairs(pos_np, active_idx, H, box):
    """(I, J): I active, J != I with r < max(H_I, H_J)."""
    tree = _tree(pos_np, box)
    I, J = pairs_within(pos_np, active_idx, np.full(pos_np.shape[0], H.max()), box, tree)
    d = pos_np[I] - pos_np[J]
    d -= box * np.round(d / box)
    r2 = (d * d).sum(axis=1)
    keep = (r2 < H[I] ** 2) | (r2 < H[J] ** 2)
    return I[keep], J[keep]


# ---------------------------------------------------------------------------
# the pieces of one step
# ---------------------------------------------------------------------------
def _seg_sum(idx, vals, n):
    return torch.zeros(n, dtype=DT).index_add(0, idx, vals)


def _pair_geometry(pos, I, J, box):
    d = min_image(pos[I] - pos[J], box)
    r = torch.sqrt((d * d).sum(dim=1))
    return d, r


def density_active(pos, m, h_c, act_idx, box, eta):
    """h, rho, drho/dh of the active particles (index act_idx) at positions
    pos, from the converged FP64 root h_c (numpy, all particles)."""
    n = pos.shape[0]
    H_np = GAMMA_K * h_c
    I, J = pairs_within(pos.detach().numpy(), act_idx, H_np * (1.0 + 1e-12), box)
    It, Jt = torch.from_numpy(I), torch.from_numpy(J)
    _, r = _pair_geometry(pos, It, Jt, box)
    hc = torch.from_numpy(h_c)
    # implicit smoothing length: one Newton step at the root
    q0 = r / (GAMMA_K * hc[It])
    F = KN / GAMMA_K ** 3 * (1.0 + _seg_sum(It, w_q(q0), n)) - eta ** 3
    Fh = (-KN / (GAMMA_K ** 3 * hc) * _seg_sum(It, q0 * dw_q(q0), n)).detach()
    a = torch.from_numpy(act_idx)
    h_act = hc[a] - F[a] / Fh[a]
    h_full = hc.clone().index_put((a,), h_act)
    H = GAMMA_K * h_full
    q = r / H[It]
    mw = _seg_sum(It, m[Jt] * w_q(q), n) + m
    mt = _seg_sum(It, m[Jt] * (3.0 * w_q(q) + q * dw_q(q)), n) + 3.0 * m
    rho = KN * mw / H ** 3
    drho_dh = -GAMMA_K * KN * mt / H ** 4
    return h_act, rho[a], drho_dh[a], I.size


def force_active(pos, vpred, m, h, rho, f, P, c, act_idx, box, alpha, gamma):
    """a (n_act x 3), Adot, vsig (numpy, no derivative) of the active
    particles; the same per-pair formulas as the C oracle's force loop."""
    n = pos.shape[0]
    H = GAMMA_K * h
    I, J = force_pairs(pos.detach().numpy(), act_idx, H.detach().numpy(), box)
    It, Jt = torch.from_numpy(I), torch.from_numpy(J)
    d, r = _pair_geometry(pos, It, Jt, box)
    if (r.detach() == 0).any():
        raise ValueError("coincident particles: the gradient oracle has no direction for them")
    Hi, Hj = H[It], H[Jt]
    dWi = KN * dw_q(r / Hi) / Hi ** 4
    dWj = KN * dw_q(r / Hj) / Hj ** 4
    Q = f * P / (rho * rho)
    dv = vpred[It] - vpred[Jt]
    dvdr = (dv * d).sum(dim=1)
    # the switch min(0, v.r / r) is not differentiable at v.r = 0 (e.g. every
    # pair of a state at rest): its derivative is taken as 0 there, the
    # receding side's
    wij = torch.where(dvdr < 0.0, dvdr / r, torch.zeros_like(dvdr))
    vsig_ij = c[It] + c[Jt] - 3.0 * wij
    Pi = -0.5 * alpha * vsig_ij * wij / (0.5 * (rho[It] + rho[Jt]))
    dWbar = 0.5 * (dWi + dWj)
    s = m[Jt] * (Q[It] * dWi + Q[Jt] * dWj + Pi * dWbar) / r
    acc = torch.zeros((n, 3), dtype=DT).index_add(0, It, -s[:, None] * d)
    sA = _seg_sum(It, m[Jt] * Pi * (dvdr / r) * dWbar, n)
    Adot = 0.5 * (gamma - 1.0) * rho ** (1.0 - gamma) * sA
    a = torch.from_numpy(act_idx)
    vs = np.maximum(2.0 * c.detach().numpy(), 0.0)
    if I.size:
        np.maximum.at(vs, I, vsig_ij.detach().numpy())
    return acc[a], Adot[a], vs[act_idx], I.size


class TorchRun:
    """The oracle run with differentiable state.

    State tensors (FP64): pos [n, 3], vel [n, 3], acc [n, 3], A, Adot, h, rho, f;
    integer state (numpy): bin, ti_begin, ti_end, ti_drift, ti."""

    def __init__(self, m, h0, *, box=1.0, eta=1.2348, gamma=5.0 / 3.0, alpha=0.8, cfl=0.1,
                 dt_min=1e-6, bin_cap=10, h_tol=1e-12, max_iter=100):
        self.m = torch.as_tensor(np.asarray(m, dtype=np.float64))
        self.n = self.m.shape[0]
        self.h0 = np.asarray(h0, dtype=np.float64).copy()
        self.box, self.eta, self.gamma, self.alpha = box, eta, gamma, alpha
        self.cfl, self.dt_min, self.bin_cap = cfl, dt_min, bin_cap
        self.h_tol, self.max_iter = h_tol, max_iter

    def run(self, pos0, vel0, u0, n_steps, record=None):
        """Runs n_steps steps from (pos0, vel0, u0) (tensors; may require grad)
        and returns the final (pos, h) as tensors, plus the history of the
        discrete state in `record` (a list, when given)."""
        n, box, g = self.n, self.box, self.gamma
        m = self.m
        pos = torch.remainder(pos0, box)
        vel = vel0
        acc = torch.zeros((n, 3), dtype=DT)
        A = torch.zeros(n, dtype=DT)
        Adot = torch.zeros(n, dtype=DT)
        h = torch.from_numpy(self.h0.copy())
        rho = torch.zeros(n, dtype=DT)
        f = torch.ones(n, dtype=DT)
        vsig = np.zeros(n)
        bin_ = np.zeros(n, dtype=np.int8)
        ti_begin = np.zeros(n, dtype=np.int64)
        ti_end = np.zeros(n, dtype=np.int64)
        ti_drift = np.zeros(n, dtype=np.int64)
        ti = 0
        for step in range(n_steps):
            first = step == 0
            # drift every particle to ti
            dtd = torch.from_numpy((ti - ti_drift) * self.dt_min)
            pos = torch.remainder(pos + vel * dtd[:, None], box)
            ti_drift[:] = ti
            # prediction
            dtp = torch.from_numpy(((ti - ti_begin) - 0.5 * (np.int64(1) << bin_.astype(np.int64)))
                                   * self.dt_min)
            vpred = vel + acc * dtp[:, None]
            Apred = A + Adot * dtp
            active = ti_end == ti
            act = np.nonzero(active)[0].astype(np.int64)
            at = torch.from_numpy(act)
            # density and the smoothing-length solve
            d = orc.density(pos.detach().numpy(), m.numpy(), h.detach().numpy(), active, box,
                            self.eta, self.h_tol, self.max_iter)
            h_act, rho_act, drho_act, _ = density_active(pos, m, d["h"], act, box, self.eta)
            h = h.index_put((at,), h_act)
            rho = rho.index_put((at,), rho_act)
            f_act = 1.0 / (1.0 + h_act / (3.0 * rho_act) * drho_act)
            f = f.index_put((at,), f_act)
            if first:
                A = (g - 1.0) * u0 / rho ** (g - 1.0)
                Apred = A
            P = Apred * rho ** g
            c = torch.sqrt(g * P / rho)
            a_act, Adot_act, vs_act, _ = force_active(pos, vpred, m, h, rho, f, P, c, act, box,
                                                     self.alpha, g)
            acc = acc.index_put((at,), a_act)
            Adot = Adot.index_put((at,), Adot_act)
            vsig[act] = vs_act
            # closing half-kick of the old step
            dt_old = torch.from_numpy(((ti_end - ti_begin) * self.dt_min)[act])
            vel = vel.index_put((at,), vel[at] + a_act * (0.5 * dt_old)[:, None])
            A = A.index_put((at,), A[at] + Adot_act * (0.5 * dt_old))
            # new bins (Eq. 1, Eq. 2), from the FP64 values without derivative
            tb = orc.timestep_bins(h.detach().numpy(), vsig, active, self.cfl, self.dt_min,
                                   self.bin_cap, ti, bin_)
            bin_[act] = tb["bin"][act]
            ti_begin[act] = tb["ti_begin"][act]
            ti_end[act] = tb["ti_end"][act]
            # opening half-kick of the new step
            dt_new = torch.from_numpy(((ti_end - ti_begin) * self.dt_min)[act])
            vel = vel.index_put((at,), vel[at] + a_act * (0.5 * dt_new)[:, None])
            A = A.index_put((at,), A[at] + Adot_act * (0.5 * dt_new))
            if record is not None:
                record.append(dict(ti=ti, active=act.copy(), bin=bin_.copy()))
            ti = int(ti_end.min())
        self.state = dict(pos=pos, vel=vel, acc=acc, A=A, Adot=Adot, h=h, rho=rho, f=f,
                          bin=bin_.copy(), ti_begin=ti_begin.copy(), ti_end=ti_end.copy(),
                          ti_drift=ti_drift.copy(), ti=ti)
        return pos, h


# ---------------------------------------------------------------------------
# the loss: SPH density on a grid against a target
# ---------------------------------------------------------------------------
def grid_points(n_grid, box=1.0):
    """Cell centres of an n_grid^3 grid, x fastest: point (i, j, k) at index
    i + n_grid (j + n_grid k), position ((i, j, k) + 1/2) box / n_grid."""
    s = (np.arange(n_grid) + 0.5) * (box / n_grid)
    gz, gy, gx = np.meshgrid(s, s, s, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)


def grid_pairs(pos_np, H_np, n_grid, box):
    """(G, J): grid point G within the support H_J of particle J (r < H_J)."""
    from scipy.spatial import cKDTree
    pts = grid_points(n_grid, box)
    tree = cKDTree(pts, boxsize=box)
    lists = tree.query_ball_point(_wrap_np(pos_np, box), r=H_np)
    J = np.repeat(np.arange(pos_np.shape[0], dtype=np.int64), [len(l) for l in lists])
    G = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]) if len(lists) else \
        np.zeros(0, dtype=np.int64)
    return G, J, pts


def grid_density_t(pos, h, m, n_grid, box=1.0):
    """rho(x_g) = sum_j m_j W(|x_g - x_j|, h_j) (torch, differentiable)."""
    H = GAMMA_K * h
    G, J, pts = grid_pairs(pos.detach().numpy(), H.detach().numpy(), n_grid, box)
    Gt, Jt = torch.from_numpy(G), torch.from_numpy(J)
    d = min_image(torch.from_numpy(pts)[Gt] - pos[Jt], box)
    r = torch.sqrt((d * d).sum(dim=1))
    vals = m[Jt] * KN * w_q(r / H[Jt]) / H[Jt] ** 3
    return torch.zeros(n_grid ** 3, dtype=DT).index_add(0, Gt, vals)


def grid_density(pos, h, m, n_grid, box=1.0):
    """The same sampled density in numpy (the finite-difference checks)."""
    with torch.no_grad():
        return grid_density_t(torch.as_tensor(np.asarray(pos, dtype=np.float64)),
                              torch.as_tensor(np.asarray(h, dtype=np.float64)),
                              torch.as_tensor(np.asarray(m, dtype=np.float64)), n_grid, box).numpy()


def loss_from_grid(rho_g, target):
    return ((rho_g - target) ** 2).sum()


def oracle_loss(ic, n_steps, n_grid, target, pos0=None, u0=None, **kw):
    """Loss of the C-oracle run (``OracleSim``): finite differences of this
    are the reference the gradients are checked against."""
    from oracle.kdk import OracleSim
    pos0 = ic["pos"] if pos0 is None else pos0
    u0 = ic["u"] if u0 is None else u0
    sim = OracleSim(pos0, ic["vel"], ic["m"], u0, ic["h0"], **kw)
    bins = []
    for _ in range(n_steps):
        sim.step()
        bins.append(sim.bin.copy())
    rho_g = grid_density(sim.pos, sim.h, sim.m, n_grid, sim.box)
    return float(((rho_g - target) ** 2).sum()), np.stack(bins), sim


def gradient(ic, n_steps, n_grid, target, **kw):
    """Loss and its gradient with respect to the initial positions, velocities
    and internal energies, by autograd through :class:`TorchRun`."""
    pos0 = torch.tensor(np.asarray(ic["pos"], dtype=np.float64), requires_grad=True)
    vel0 = torch.tensor(np.asarray(ic["vel"], dtype=np.float64), requires_grad=True)
    u0 = torch.tensor(np.broadcast_to(np.asarray(ic["u"], dtype=np.float64),
                                      (pos0.shape[0],)).copy(), requires_grad=True)
    run = TorchRun(ic["m"], ic["h0"], **kw)
    record = []
    pos, h = run.run(pos0, vel0, u0, n_steps, record)
    rho_g = grid_density_t(pos, h, run.m, n_grid, run.box)
    L = loss_from_grid(rho_g, torch.as_tensor(target))
    gx, gv, gu = torch.autograd.grad(L, (pos0, vel0, u0), allow_unused=True)
    z = lambda t, like: torch.zeros_like(like) if t is None else t
    return dict(loss=float(L.detach()), pos=z(gx, pos0).numpy(), vel=z(gv, vel0).numpy(),
                u=z(gu, u0).numpy(), run=run, record=record, rho_grid=rho_g.detach().numpy())
