"""Pins of the gradient oracle (oracle/adjoint.py) and of the grid-density loss
(no GPU).

The gradient oracle re-expresses the oracle's kick-drift-kick run in PyTorch
FP64 and differentiates it with autograd.  It is pinned to things other than
itself: its forward must reproduce the C oracle's run, and its gradient must
match central finite differences of the C oracle's loss (which shares only the
neighbour-free formulas' meaning, not code, with the torch run).  A dropped
term anywhere in the chain (the implicit smoothing length, the grad-h factor,
the equation of state, the viscosity, a kick, the prediction, the drift)
changes the gradient far beyond the tolerances below.
"""
import math

import numpy as np
import pytest

import sph_ics

torch = pytest.importorskip("torch")

KW = dict(cfl=0.1, dt_min=2.0 ** -24, bin_cap=12)
N_STEPS, N_GRID = 5, 8


@pytest.fixture(scope="module")
def case(orc):
    from oracle import adjoint as adj
    ic = sph_ics.clumpy_lattice(8, 2, 16, seed=4)
    # small random initial velocities: the viscosity switch min(0, v.r / r)
    # then sees no pair exactly at v.r = 0, where it has no derivative
    ic["vel"] = np.random.default_rng(12).normal(0.0, 0.05, size=ic["pos"].shape)
    # the target: the same run from positions displaced by 1 % of the spacing
    rng = np.random.default_rng(7)
    icp = dict(ic)
    icp["pos"] = (ic["pos"] + rng.normal(0.0, 0.01 / 8, size=ic["pos"].shape)) % 1.0
    _, _, simt = adj.oracle_loss(icp, N_STEPS, N_GRID, np.zeros(N_GRID ** 3), **KW)
    target = adj.grid_density(simt.pos, simt.h, simt.m, N_GRID)
    L0, bins0, sim0 = adj.oracle_loss(ic, N_STEPS, N_GRID, target, **KW)
    g = adj.gradient(ic, N_STEPS, N_GRID, target, **KW)
    return dict(adj=adj, ic=ic, target=target, L0=L0, bins0=bins0, sim0=sim0, g=g)


def test_torch_run_reproduces_oracle_run(case):
    """The differentiable run is the C oracle's run: same final state to
    rounding, same bins and active sets (catches a step of the torch
    re-expression that differs from the integrator it stands for)."""
    st, sim = case["g"]["run"].state, case["sim0"]
    assert (st["bin"] == sim.bin).all() and (st["ti_end"] == sim.ti_end).all()
    assert np.abs(st["pos"].detach().numpy() - sim.pos).max() < 1e-13
    assert np.abs(st["vel"].detach().numpy() - sim.vel).max() < 1e-12
    for k in ("h", "A", "rho", "f"):
        a = st[k].detach().numpy()
        b = getattr(sim, k)
        assert np.abs(a / b - 1.0).max() < 1e-12, k
    assert abs(case["g"]["loss"] / case["L0"] - 1.0) < 1e-12
    # the run exercises inactive particles: some steps have few active ones
    sizes = [len(r["active"]) for r in case["g"]["record"]]
    assert min(sizes) < 0.1 * case["ic"]["pos"].shape[0] and max(sizes) == case["ic"]["pos"].shape[0]


def _fd(case, which, i, k, eps):
    adj, ic = case["adj"], case["ic"]
    base = {"pos": ic["pos"], "vel": ic["vel"],
            "u": np.broadcast_to(np.asarray(ic["u"], dtype=np.float64), (ic["pos"].shape[0],))}
    vals = []
    for s in (+1.0, -1.0):
        arr = np.array(base[which], dtype=np.float64, copy=True)
        if arr.ndim == 2:
            arr[i, k] += s * eps
        else:
            arr[i] += s * eps
        icx = dict(ic)
        if which == "vel":
            icx["vel"] = arr
            L, bins, _ = adj.oracle_loss(icx, N_STEPS, N_GRID, case["target"], **KW)
        elif which == "pos":
            L, bins, _ = adj.oracle_loss(icx, N_STEPS, N_GRID, case["target"], pos0=arr, **KW)
        else:
            L, bins, _ = adj.oracle_loss(icx, N_STEPS, N_GRID, case["target"], u0=arr, **KW)
        assert (bins == case["bins0"]).all(), "a bin changed under the perturbation"
        vals.append(L)
    return (vals[0] - vals[1]) / (2.0 * eps)


@pytest.mark.parametrize("seed", [0, 1])
def test_position_gradient_matches_finite_differences(case, seed):
    """d loss / d x0 against central differences (step 1e-6) of the C-oracle
    loss on seeded coordinates: relative error below 1e-4 (the FD truncation
    and h-convergence noise are ~1e-6 here)."""
    g = case["g"]["pos"]
    rng = np.random.default_rng(seed)
    n = g.shape[0]
    rms = math.sqrt((g ** 2).mean())
    for _ in range(6):
        i, k = int(rng.integers(n)), int(rng.integers(3))
        fd = _fd(case, "pos", i, k, 1e-6)
        assert abs(fd - g[i, k]) <= 1e-4 * abs(fd) + 1e-7 * rms, (i, k, fd, g[i, k])


def test_velocity_gradient_matches_finite_differences(case):
    """d loss / d v0 (the drift and the viscosity carry it)."""
    g = case["g"]["vel"]
    rng = np.random.default_rng(11)
    n = g.shape[0]
    rms = math.sqrt((g ** 2).mean())
    assert rms > 0.0
    for _ in range(4):
        i, k = int(rng.integers(n)), int(rng.integers(3))
        fd = _fd(case, "vel", i, k, 1e-6)
        assert abs(fd - g[i, k]) <= 1e-3 * abs(fd) + 1e-4 * rms, (i, k, fd, g[i, k])


def test_energy_gradient_matches_finite_differences(case):
    """d loss / d u0 (through the entropy, the pressure and the kicks); u is
    ~1, so the step is 1e-4 to stay above the h-convergence noise."""
    g = case["g"]["u"]
    rng = np.random.default_rng(5)
    n = g.shape[0]
    rms = math.sqrt((g ** 2).mean())
    assert rms > 0.0
    for _ in range(4):
        i = int(rng.integers(n))
        fd = _fd(case, "u", i, 0, 1e-4)
        assert abs(fd - g[i]) <= 1e-3 * abs(fd) + 1e-3 * rms, (i, fd, g[i])


def test_one_step_gradient_is_the_implicit_h_derivative(orc):
    """With one step nothing moves, so the loss depends on x0 only through W
    and the solved h: its gradient checks dh/dx = -F_x / F_h alone."""
    from oracle import adjoint as adj
    ic = sph_ics.lattice(6, 0.2, seed=3)
    target = np.zeros(N_GRID ** 3)
    g = adj.gradient(ic, 1, N_GRID, target, **KW)
    # the same loss with h frozen at the solution differs in gradient: the
    # h-dependence is not negligible, so a missing implicit term is caught
    rng = np.random.default_rng(2)
    for _ in range(4):
        i, k = int(rng.integers(ic["pos"].shape[0])), int(rng.integers(3))
        vals = []
        for s in (+1.0, -1.0):
            p = ic["pos"].copy()
            p[i, k] += s * 1e-6
            L, _, _ = adj.oracle_loss(ic, 1, N_GRID, target, pos0=p, **KW)
            vals.append(L)
        fd = (vals[0] - vals[1]) / 2e-6
        assert abs(fd - g["pos"][i, k]) <= 1e-5 * abs(fd) + 1e-9, (fd, g["pos"][i, k])


def test_grid_density_closed_form_single_particle(orc):
    """One particle: the sampled density is m W(r, h) at each grid point,
    W = (8/pi) H^-3 w(r/H) (catches a wrong normalisation, support or
    periodic image)."""
    from oracle import adjoint as adj
    ng, h, m = 8, 0.1, 0.7
    pos = np.array([[0.01, 0.5, 0.97]])
    rho = adj.grid_density(pos, np.array([h]), np.array([m]), ng)
    pts = adj.grid_points(ng)
    H = adj.GAMMA_K * h
    for g in range(ng ** 3):
        d = pts[g] - pos[0]
        d -= np.round(d)
        r = math.sqrt((d * d).sum())
        q = r / H
        w = (1 - 6 * q * q + 6 * q ** 3) if q < 0.5 else (2 * (1 - q) ** 3 if q < 1 else 0.0)
        assert abs(rho[g] - m * (8 / math.pi) * w / H ** 3) <= 1e-12 * (8 / math.pi) / H ** 3


def test_grid_density_brute_force(orc):
    """The tree-based sampling equals a double loop over all (point, particle)
    pairs (catches a missed neighbour or a wrong radius)."""
    from oracle import adjoint as adj
    rng = np.random.default_rng(9)
    n, ng = 60, 5
    pos = rng.uniform(0, 1, size=(n, 3))
    h = rng.uniform(0.05, 0.2, size=n)
    m = rng.uniform(0.5, 1.5, size=n)
    rho = adj.grid_density(pos, h, m, ng)
    pts = adj.grid_points(ng)
    ref = np.zeros(ng ** 3)
    for g in range(ng ** 3):
        for j in range(n):
            d = pts[g] - pos[j]
            d -= np.round(d)
            r = math.sqrt((d * d).sum())
            ref[g] += m[j] * orc.kernel_w([r / (adj.GAMMA_K * h[j])])[0] / (adj.GAMMA_K * h[j]) ** 3
    assert np.abs(rho - ref).max() <= 1e-12 * np.abs(ref).max()
