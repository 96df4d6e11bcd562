"""GPU reverse pass (sph_step_bwd, sph_grid_density, sph_grid_density_bwd and
the checkpointed differentiable run) against the gradient oracle (PyTorch FP64
autograd through the oracle's run) and against central finite differences of
the oracle's loss.

Tolerance of the gradients: element-wise |g_gpu - g_oracle| <= 1e-3 rms(g).
The GPU run is the FP32-pair-arithmetic forward with h converged to 1e-6
(relative); its trajectory differs from the FP64 oracle's by ~1e-6 relative,
and the adjoint pair terms are FP32 summed in FP64; kernel curvature
amplifies the h difference by ~10-100 in the derivatives, so 1e-3 rms bounds
both with margin (the observed worst elements are 2e-5 to 3e-4 rms).
"""
import json
import math
import os

import numpy as np
import pytest

import sph_ics

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KW = dict(cfl=0.1, dt_min=2.0 ** -24, bin_cap=12)
TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01341_gb300 import build
    build.build()
    from paper_1807_01341_gb300 import adjoint as gadj, sim, _lib
    from oracle import adjoint as oadj
    import oracle
    oracle.build()
    return dict(torch=torch, gadj=gadj, sim=sim, lib=_lib, oadj=oadj)


def _target(env, ic, n_steps, n_grid, seed=7):
    oadj = env["oadj"]
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(seed)
    icp = dict(ic)
    icp["pos"] = (ic["pos"] + rng.normal(0.0, 0.01 / round(n ** (1 / 3)), size=ic["pos"].shape)) % 1.0
    _, _, simt = oadj.oracle_loss(icp, n_steps, n_grid, np.zeros(n_grid ** 3), **KW)
    return oadj.grid_density(simt.pos, simt.h, simt.m, n_grid)


def _gpu_gradient(env, ic, n_steps, n_grid, target, k=5, leaf_max=8):
    torch, gadj, sim = env["torch"], env["gadj"], env["sim"]
    n = ic["pos"].shape[0]
    params = sim.Params(**KW, leaf_max=leaf_max, cell_margin=2.0)
    run = gadj.Run(params, np.array(np.broadcast_to(ic["m"], (n,))), ic["h0"], n_steps, n_grid,
                   checkpoint_every=k)
    pos0 = torch.tensor(ic["pos"], dtype=torch.float64, device="cuda", requires_grad=True)
    vel0 = torch.tensor(np.asarray(ic["vel"], dtype=np.float64), device="cuda", requires_grad=True)
    u0 = torch.tensor(np.broadcast_to(np.asarray(ic["u"], dtype=np.float64), (n,)).copy(),
                      device="cuda", requires_grad=True)
    rho = gadj.GridDensityRun.apply(pos0, vel0, u0, run)
    loss = ((rho - torch.as_tensor(target, device="cuda")) ** 2).sum()
    loss.backward()
    out = dict(loss=float(loss.detach()), rho=rho.detach().cpu().numpy(),
               pos=pos0.grad.cpu().numpy(), vel=vel0.grad.cpu().numpy(),
               u=u0.grad.cpu().numpy(), final=run.final.numpy(), run=run)
    return out


def _check(g, o, name, tol=TOL):
    rms = math.sqrt(float((o ** 2).mean()))
    assert rms > 0.0, name
    err = np.abs(g - o)
    assert err.max() <= tol * rms, (name, err.max() / rms, np.unravel_index(err.argmax(), err.shape))


# ---------------------------------------------------------------------------
# the loss
# ---------------------------------------------------------------------------
def _loss_state(env, n=300, seed=5):
    torch, sim = env["torch"], env["sim"]
    rng = np.random.default_rng(seed)
    p = sim.Particles(n, with_counts=False)
    pos = rng.uniform(0.0, 1.0, size=(n, 3))
    vel = rng.normal(0.0, 1.0, size=(n, 3)).astype(np.float32)
    h = rng.uniform(0.03, 0.12, size=n).astype(np.float32)
    m = rng.uniform(0.5, 1.5, size=n).astype(np.float32)
    td = rng.integers(0, 50, size=n)
    for k, name in enumerate("xyz"):
        getattr(p, name).copy_(torch.as_tensor(pos[:, k]))
        getattr(p, "v" + name).copy_(torch.as_tensor(vel[:, k]))
    p.h.copy_(torch.as_tensor(h))
    p.m.copy_(torch.as_tensor(m))
    p.ti_drift.copy_(torch.as_tensor(td))
    ti, dt_min = 64, 1e-3
    # the positions the library samples: drifted to ti in FP64 from FP32 velocities
    xt = (pos + vel.astype(np.float64) * ((ti - td) * dt_min)[:, None]) % 1.0
    return p, dict(pos=pos, vel=vel, h=h, m=m, td=td, ti=ti, dt_min=dt_min, xt=xt)


def test_grid_density_matches_oracle(env):
    """sph_grid_density equals the oracle's sampled density (both FP64) at the
    positions drifted to the requested tick."""
    sim, oadj = env["sim"], env["oadj"]
    p, s = _loss_state(env)
    ctx = sim.Context(sim.Params(dt_min=s["dt_min"]), p.n)
    ng = 12
    rho = ctx.grid_density(p, ng, s["ti"]).cpu().numpy()
    ref = oadj.grid_density(s["xt"], s["h"].astype(np.float64), s["m"].astype(np.float64), ng)
    assert np.abs(rho - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()


def test_grid_density_bwd_matches_oracle_autograd(env):
    """sph_grid_density_bwd gives d loss / d x, d h and (through the drift)
    d v of the oracle's autograd of the same sampled density."""
    torch, sim, oadj = env["torch"], env["sim"], env["oadj"]
    p, s = _loss_state(env)
    ctx = sim.Context(sim.Params(dt_min=s["dt_min"]), p.n)
    ng = 12
    rng = np.random.default_rng(3)
    rho_bar = rng.normal(size=ng ** 3)
    adj = sim.Adjoint(p.n)
    ctx.grid_density_bwd(p, ng, s["ti"], torch.as_tensor(rho_bar, device="cuda"), adj)
    x = torch.tensor(s["xt"], requires_grad=True)
    h = torch.tensor(s["h"].astype(np.float64), requires_grad=True)
    r = oadj.grid_density_t(x, h, torch.as_tensor(s["m"].astype(np.float64)), ng)
    gx, gh = torch.autograd.grad((r * torch.as_tensor(rho_bar)).sum(), (x, h))
    gx, gh = gx.numpy(), gh.numpy()
    g = np.stack([adj.x.cpu().numpy(), adj.y.cpu().numpy(), adj.z.cpu().numpy()], axis=1)
    gv = np.stack([adj.vx.cpu().numpy(), adj.vy.cpu().numpy(), adj.vz.cpu().numpy()], axis=1)
    assert np.abs(g - gx).max() <= 1e-10 * np.abs(gx).max()
    assert np.abs(adj.h.cpu().numpy() - gh).max() <= 1e-10 * np.abs(gh).max()
    dtd = (s["ti"] - s["td"]) * s["dt_min"]
    assert np.abs(gv - gx * dtd[:, None]).max() <= 1e-10 * np.abs(gx).max()
    ctx.close()


# ---------------------------------------------------------------------------
# whole differentiable runs
# ---------------------------------------------------------------------------
def _small_clumpy():
    ic = sph_ics.clumpy_lattice(8, 2, 16, seed=4)
    ic["vel"] = np.random.default_rng(12).normal(0.0, 0.05, size=ic["pos"].shape)
    return ic


def _small_lattice():
    ic = sph_ics.lattice(10, 0.2, seed=3)
    ic["vel"] = np.random.default_rng(13).normal(0.0, 0.05, size=ic["pos"].shape)
    return ic


@pytest.mark.parametrize("make_ic,n_steps", [(_small_clumpy, 1), (_small_clumpy, 2),
                                              (_small_clumpy, 5), (_small_lattice, 3)])
def test_run_gradient_matches_oracle(env, make_ic, n_steps):
    """d loss / d (x0, v0, u0) of the checkpointed GPU run against the oracle's
    autograd gradient, element by element (one step isolates the density
    adjoint with the implicit smoothing length; more steps add the force,
    kicks, prediction and drift).  The discrete trajectory (bins, step ends)
    must be the oracle's exactly."""
    oadj = env["oadj"]
    ic = make_ic()
    ng = 8
    target = _target(env, ic, n_steps, ng)
    go = oadj.gradient(ic, n_steps, ng, target, **KW)
    gg = _gpu_gradient(env, ic, n_steps, ng, target)
    st = go["run"].state
    assert (gg["final"]["bin"] == st["bin"]).all()
    assert (gg["final"]["ti_end"] == st["ti_end"]).all()
    assert abs(gg["loss"] / go["loss"] - 1.0) < 1e-4
    _check(gg["pos"], go["pos"], "pos")
    if n_steps > 1:  # one step moves nothing: v and u do not reach the loss
        _check(gg["u"], go["u"], "u")
        _check(gg["vel"], go["vel"], "vel")
    gg["run"].close()


def test_checkpoint_recompute_is_exact_and_spacing_independent(env):
    """The backward pass recomputes each segment from its checkpoint: the
    recomputed final state equals the forward's bit for bit, and the gradient
    does not depend on the checkpoint spacing beyond the rounding of the
    forward itself (restarts rebuild the cells) and of the FP64 atomics."""
    oadj = env["oadj"]
    ic = _small_clumpy()
    ng, n_steps = 8, 5
    target = _target(env, ic, n_steps, ng)
    runs = {k: _gpu_gradient(env, ic, n_steps, ng, target, k=k) for k in (1, 2, 5)}
    for k, g in runs.items():
        run = g["run"]
        a, b = run.final.arrays(), run.recomputed_final.arrays()
        for name in a:
            assert env["torch"].equal(a[name], b[name]), (k, name)
    ref = runs[5]
    for k in (1, 2):
        for name in ("pos", "vel", "u"):
            rms = math.sqrt(float((ref[name] ** 2).mean()))
            assert np.abs(runs[k][name] - ref[name]).max() <= 1e-5 * rms, (k, name)
    for g in runs.values():
        g["run"].close()


def test_step_bwd_rejects_bad_arguments(env):
    """Mismatched sizes and missing adjoint arrays are argument errors,
    reported before anything runs."""
    sim, lib = env["sim"], env["lib"]
    ic = _small_lattice()
    n = ic["pos"].shape[0]
    ctx = sim.Context(sim.Params(**KW), n)
    a = sim.Particles.from_ics(ic, with_counts=False)
    b = sim.Particles.from_ics(ic, with_counts=False)
    adj = sim.Adjoint(n)
    s = adj.struct()
    s.h = None
    import ctypes
    code = ctx.L.sph_step_bwd(ctx.h, ctypes.byref(a.struct()), ctypes.byref(b.struct()), 0, 1,
                              ctypes.byref(s), None)
    assert code == lib.SPH_ERR_ARG
    small = sim.Adjoint(n - 1)
    code = ctx.L.sph_step_bwd(ctx.h, ctypes.byref(a.struct()), ctypes.byref(b.struct()), 0, 1,
                              ctypes.byref(small.struct()), None)
    assert code == lib.SPH_ERR_ARG
    ctx.close()


# ---------------------------------------------------------------------------
# the differentiation workload: 32^3 lattice with 8 clumps, 20 steps
# ---------------------------------------------------------------------------
def test_c4_gradient_matches_finite_differences_and_oracle(env):
    """The 32,768-particle workload (8 Plummer clumps of 512 in a jittered
    32^3 lattice, 20 steps, 32^3 grid, checkpoints every 5 steps): the GPU
    gradient against the stored central finite differences of the oracle's
    loss on 64 seeded coordinates (48 positions, 16 energies), and against the
    oracle's autograd gradient for every particle."""
    import importlib.util
    oadj = env["oadj"]
    with open(os.path.join(GOLDEN, "c4_gradient_fd.json")) as f:
        gold = json.load(f)
    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLDEN,
                                                                     "make_c4_gradient_fd.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert mk.RECIPE == gold["recipe"]
    ic, kw, target = mk.workload()
    r = gold["recipe"]
    gg = _gpu_gradient(env, ic, r["n_steps"], r["n_grid"], target, k=5)
    assert abs(gg["loss"] / gold["loss"] - 1.0) < 1e-4
    go = oadj.gradient(ic, r["n_steps"], r["n_grid"], target, **kw)
    st = go["run"].state
    assert (gg["final"]["bin"] == st["bin"]).all()
    _check(gg["pos"], go["pos"], "pos")
    _check(gg["u"], go["u"], "u")
    # element-wise against the finite differences.  Positions: relative 5e-4
    # (the GPU's elements sit within 1e-4 of the oracle's, the differences
    # within 1e-5 of the oracle's autograd), with a floor of 1e-7 rms for
    # elements near 0.  Energies act only through 20 steps of FP32 pressure
    # forces (each within 1e-4 of the rms acceleration): relative 1e-3, floor
    # 1e-5 rms.
    rms_p = math.sqrt(float((go["pos"] ** 2).mean()))
    rms_u = math.sqrt(float((go["u"] ** 2).mean()))
    used = 0
    for e in gold["pos"]:
        if not e["bins_same"]:
            continue
        used += 1
        g = gg["pos"][e["i"], e["k"]]
        assert abs(g - e["fd"]) <= 5e-4 * abs(e["fd"]) + 1e-7 * rms_p, (e, g)
    for e in gold["u"]:
        if not e["bins_same"]:
            continue
        used += 1
        g = gg["u"][e["i"]]
        assert abs(g - e["fd"]) <= 1e-3 * abs(e["fd"]) + 1e-5 * rms_u, (e, g)
    assert used >= 70
    gg["run"].close()
