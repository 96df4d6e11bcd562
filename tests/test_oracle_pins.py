"""Pins of the FP64 oracle against closed forms, invariants and independent
computations (no GPU).  Each test names the part of the method it pins and the
mistake it would catch."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import sph_ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ETA = 1.2348
GAMMA = 5.0 / 3.0


# --------------------------------------------------------------------------
# Kernel
# --------------------------------------------------------------------------

def test_kernel_normalisation(orc):
    """int W dV = 1 in 3-D (catches a wrong 8/pi or a wrong piece)."""
    w = lambda q: 4.0 * math.pi * q * q * orc.kernel_w([q])[0]
    a, _ = integrate.quad(w, 0.0, 0.5, epsabs=1e-14, epsrel=1e-14)
    b, _ = integrate.quad(w, 0.5, 1.0, epsabs=1e-14, epsrel=1e-14)
    assert abs(a + b - 1.0) < 1e-12


def test_kernel_smoothness_and_support(orc):
    """w, w' continuous at q = 1/2; w(1) = w'(1) = 0; w' is the derivative of w;
    w'' (from w') continuous at 1/2 (a C^2 cubic spline)."""
    eps = 1e-7
    for q0 in (0.5, 1.0):
        wl, wr = orc.kernel_w([q0 - 1e-12])[0], orc.kernel_w([min(q0 + 1e-12, 0.999999999999)])[0]
        assert abs(wl - wr) < 1e-9
    assert orc.kernel_w([1.0])[0] == 0.0 and orc.kernel_dw([1.0])[0] == 0.0
    assert abs(orc.kernel_dw([1.0 - 1e-9])[0]) < 1e-15
    for q in np.linspace(0.01, 0.99, 37):
        num = (orc.kernel_w([q + eps])[0] - orc.kernel_w([q - eps])[0]) / (2 * eps)
        assert abs(num - orc.kernel_dw([q])[0]) < 1e-6
    d2l = (orc.kernel_dw([0.5 - 1e-6])[0] - orc.kernel_dw([0.5 - 2e-6])[0]) / 1e-6
    d2r = (orc.kernel_dw([0.5 + 2e-6])[0] - orc.kernel_dw([0.5 + 1e-6])[0]) / 1e-6
    assert abs(d2l - d2r) < 1e-4
    # monotone decreasing on [0, 1)
    q = np.linspace(0, 0.999, 200)
    assert np.all(np.diff(orc.kernel_w(q)) < 0)


def test_neighbour_number_closed_form(orc):
    """eta = 1.2348 with H = 1.825742 h encodes ~48 neighbours: (4 pi / 3)(H/h eta)^3."""
    n = 4.0 * math.pi / 3.0 * (orc.GAMMA_K * ETA) ** 3
    assert abs(n - 47.995) < 2e-3


# --------------------------------------------------------------------------
# Density and smoothing length
# --------------------------------------------------------------------------

def _lattice_vectors(reach):
    k = np.arange(-reach, reach + 1)
    v = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3).astype(float)
    return np.sqrt((v * v).sum(1))


def test_lattice_density_matches_lattice_sum(orc):
    """On a perfect periodic lattice every particle has the same h and rho, and
    they equal the root of h^3 n(h) = eta^3 found by enumerating lattice
    vectors of an infinite lattice (an independent summation, no periodic
    wrapping, brentq instead of the oracle's Newton).  Catches a wrong
    minimum-image rule, a dropped self term or a wrong Newton update."""
    nside = 12
    ic = sph_ics.lattice(nside, jitter=0.0)
    d = orc.density(ic["pos"], ic["m"], ic["h0"] * 1.1, np.ones(nside ** 3, np.uint8),
                    use_cells=True)
    assert d["n_unconverged"] == 0
    h, rho = d["h"], d["rho"]
    assert np.ptp(h) < 1e-13 * h.mean() and np.ptp(rho) < 1e-12 * rho.mean()
    dr = _lattice_vectors(4) / nside  # |lattice vector| in box units

    def F(hh):
        H = orc.GAMMA_K * hh
        q = dr[dr < H] / H
        n = orc.kernel_w(q).sum() / H ** 3
        return hh ** 3 * n - ETA ** 3

    h_ref = optimize.brentq(F, 0.5 * ETA / nside, 2.0 * ETA / nside, xtol=1e-15, rtol=1e-15)
    H = orc.GAMMA_K * h_ref
    q = dr[dr < H] / H
    rho_ref = orc.kernel_w(q).sum() / H ** 3 * ic["m"][0]
    assert abs(h[0] - h_ref) < 1e-12 * h_ref
    assert abs(rho[0] - rho_ref) < 1e-11 * rho_ref
    # a normalised kernel reproduces the mean density to within a percent
    assert abs(rho[0] - 1.0) < 0.01


def test_density_h_derivatives_numeric(orc):
    """d rho / dh and dn / dh agree with central differences of the fixed-h
    sums (catches a wrong sign or a missing GAMMA_K in dW/dh)."""
    ic = sph_ics.lattice(8, jitter=0.1, seed=11)
    n = ic["pos"].shape[0]
    h = ic["h0"] * np.random.default_rng(0).uniform(0.9, 1.1, n)
    eps = 1e-6 * h
    d0 = orc.density_fixed_h(ic["pos"], ic["m"], h)
    dp = orc.density_fixed_h(ic["pos"], ic["m"], h + eps)
    dm = orc.density_fixed_h(ic["pos"], ic["m"], h - eps)
    num_rho = (dp["rho"] - dm["rho"]) / (2 * eps)
    num_n = (dp["wn"] - dm["wn"]) / (2 * eps)
    # only where no neighbour sits within eps of the support edge
    ok = (dp["count"] == dm["count"])
    assert ok.mean() > 0.9
    scale = np.abs(d0["drho_dh"][ok]).max()
    assert np.abs(num_rho[ok] - d0["drho_dh"][ok]).max() < 1e-6 * scale
    assert np.abs(num_n[ok] - d0["dwn_dh"][ok]).max() < 1e-6 * np.abs(d0["dwn_dh"][ok]).max()


def test_h_solution_and_search_modes(orc):
    """The converged h solves h^3 n(h) = eta^3, the neighbour count matches the
    continuous estimate, and the cell-grid search visits exactly the
    brute-force neighbour sets."""
    ic = sph_ics.clumpy_lattice(nside=12, n_clumps=2, per_clump=200, seed=3)
    n = ic["pos"].shape[0]
    act = np.ones(n, np.uint8)
    a = orc.density(ic["pos"], ic["m"], ic["h0"], act, use_cells=True)
    b = orc.density(ic["pos"], ic["m"], ic["h0"], act, use_cells=False)
    assert a["n_unconverged"] == 0 and b["n_unconverged"] == 0
    resid = a["h"] ** 3 * a["wn"] - ETA ** 3
    assert np.abs(resid).max() < 1e-9
    assert np.array_equal(a["count"], b["count"])
    assert np.abs(a["h"] - b["h"]).max() < 1e-13 * a["h"].max()
    assert np.abs(a["rho"] / b["rho"] - 1).max() < 1e-12
    # on a smooth (jittered lattice) distribution the neighbour count is close
    # to the continuous estimate (4 pi / 3)(H/h eta)^3 = 48
    lat = sph_ics.lattice(12, jitter=0.1, seed=8)
    c = orc.density(lat["pos"], lat["m"], lat["h0"], np.ones(12 ** 3, np.uint8))["count"]
    assert 42 < c.mean() + 1 < 54


def test_density_active_subset(orc):
    """Inactive particles keep their h and are not written."""
    ic = sph_ics.lattice(8, seed=5)
    n = ic["pos"].shape[0]
    act = np.zeros(n, np.uint8)
    act[::7] = 1
    d = orc.density(ic["pos"], ic["m"], ic["h0"], act)
    assert np.all(d["h"][act == 0] == ic["h0"][act == 0])
    assert np.all(d["rho"][act == 0] == 0.0)
    full = orc.density(ic["pos"], ic["m"], ic["h0"], np.ones(n, np.uint8))
    assert np.allclose(d["rho"][act == 1], full["rho"][act == 1], rtol=1e-13)


# --------------------------------------------------------------------------
# Force
# --------------------------------------------------------------------------

def _hydro_state(orc, ic, A, tol=1e-14):
    n = ic["pos"].shape[0]
    d = orc.density(ic["pos"], ic["m"], ic["h0"], np.ones(n, np.uint8), tol=tol, max_iter=200,
                    use_cells=False)
    f = orc.gradh_f(d["h"], d["rho"], d["drho_dh"])
    P, c = orc.eos(A, d["rho"], GAMMA)
    return d, f, P, c


def test_force_is_minus_gradient_of_thermal_energy(orc):
    """With alpha = 0 and fixed entropies, m_k a_k = -dU/dx_k with
    U = sum_i m_i A_i rho_i^(gamma-1) / (gamma-1), where every rho_i is taken at
    its re-converged h.  This is the defining property of the grad-h
    formulation: it pins the pressure term, the grad-h factor f, the kernel
    gradient and the equation of state together (any dropped term, sign error
    or transposed i/j fails it)."""
    ic = sph_ics.lattice(7, jitter=0.15, seed=21)
    n = ic["pos"].shape[0]
    A = np.random.default_rng(1).uniform(0.5, 1.5, n)
    d, f, P, c = _hydro_state(orc, ic, A)
    fr = orc.force(ic["pos"], np.zeros((n, 3)), ic["m"], d["h"], d["rho"], f, P, c,
                   np.ones(n, np.uint8), alpha=0.0, gamma=GAMMA, use_cells=False)

    def U(pos):
        dd = orc.density(pos, ic["m"], d["h"], np.ones(n, np.uint8), tol=1e-15, max_iter=200,
                         use_cells=False)
        return float((ic["m"] * A * dd["rho"] ** (GAMMA - 1) / (GAMMA - 1)).sum())

    rng = np.random.default_rng(2)
    eps = 1e-6
    amax = np.abs(fr["a"]).max()
    for k in rng.choice(n, 6, replace=False):
        for ax in range(3):
            p1 = ic["pos"].copy(); p1[k, ax] += eps
            p2 = ic["pos"].copy(); p2[k, ax] -= eps
            grad = (U(p1) - U(p2)) / (2 * eps)
            assert abs(ic["m"][k] * fr["a"][k, ax] + grad) < 2e-6 * ic["m"][k] * amax


def test_force_zero_on_perfect_lattice(orc):
    """Uniform pressure on a perfect lattice: a = 0 to roundoff by symmetry."""
    ic = sph_ics.lattice(10, jitter=0.0)
    n = ic["pos"].shape[0]
    A = np.ones(n)
    d, f, P, c = _hydro_state(orc, ic, A, tol=1e-13)
    fr = orc.force(ic["pos"], np.zeros((n, 3)), ic["m"], d["h"], d["rho"], f, P, c,
                   np.ones(n, np.uint8))
    scale = P.mean() / (d["rho"].mean() * orc.GAMMA_K * d["h"].mean())
    assert np.abs(fr["a"]).max() < 1e-11 * scale
    assert np.all(fr["Adot"] == 0.0)


def test_force_pairwise_conservation_and_heating(orc):
    """All particles active, random velocities: total momentum change sum m a = 0
    to roundoff (pairwise antisymmetry); viscous heating is non-negative and
    balances the viscous kinetic-energy loss exactly:
    sum_i m_i v_i . a_visc,i + sum_i m_i rho_i^(gamma-1)/(gamma-1) Adot_i = 0."""
    ic = sph_ics.lattice(9, jitter=0.1, seed=31)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(4)
    A = rng.uniform(0.5, 1.5, n)
    vel = rng.normal(scale=0.5, size=(n, 3))
    d, f, P, c = _hydro_state(orc, ic, A, tol=1e-13)
    act = np.ones(n, np.uint8)
    fa = orc.force(ic["pos"], vel, ic["m"], d["h"], d["rho"], f, P, c, act, alpha=0.8)
    f0 = orc.force(ic["pos"], vel, ic["m"], d["h"], d["rho"], f, P, c, act, alpha=0.0)
    m = ic["m"]
    tot = (m[:, None] * fa["a"]).sum(0)
    assert np.abs(tot).max() < 1e-12 * (m[:, None] * np.abs(fa["a"])).sum()
    assert np.all(fa["Adot"] >= 0.0) and fa["Adot"].max() > 0
    a_visc = fa["a"] - f0["a"]
    kin = (m * (vel * a_visc).sum(1)).sum()
    heat = (m * d["rho"] ** (GAMMA - 1) / (GAMMA - 1) * fa["Adot"]).sum()
    assert abs(kin + heat) < 1e-10 * abs(heat)
    # signal velocity: at least 2 c_i (the pair with itself, Eq. 1)
    assert np.all(fa["vsig"] >= 2 * c - 1e-15)
    # same neighbour sets either way
    assert np.array_equal(fa["count"], f0["count"])


def _visc_case(orc, alpha=0.8):
    """Three particles in a box of side 10, no pressure (P = 0), so every
    acceleration and entropy rate comes from the artificial viscosity alone.

    i  at (5, 5, 5), v = (1, 0, 0), H = 1, rho = 8, c = 1
    j1 at (5.75, 5, 5), v = (-1, 0, 0), H = 1, rho = 4, c = 1 (approaching i)
    j2 at (5, 5.6, 5), v = (0, 1, 0), H = 1.2, rho = 1, c = 20 (receding from i)
    masses 1.  H = 1.825742 h is the kernel support."""
    pos = np.array([[5.0, 5.0, 5.0], [5.75, 5.0, 5.0], [5.0, 5.6, 5.0]])
    vel = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    H = np.array([1.0, 1.0, 1.2])
    rho = np.array([8.0, 4.0, 1.0])
    c = np.array([1.0, 1.0, 20.0])
    n = 3
    return orc.force(pos, vel, np.ones(n), H / orc.GAMMA_K, rho, np.ones(n), np.zeros(n), c,
                     np.ones(n, np.uint8), box=10.0, alpha=alpha, gamma=GAMMA, use_cells=False)


def test_force_viscosity_hand_computed(orc):
    """Pins the signal-velocity viscosity (Monaghan 1997, beta = 3 as inside
    Eq. 1) with numbers worked out by hand.

    Pair (i, j1): r_ij = x_i - x_j1 = (-0.75, 0, 0), r = 0.75, v_ij = (2, 0, 0),
    v_ij . r_ij / r = -2, so w = min(0, -2) = -2 and v_sig,ij = c_i + c_j - 3w
    = 8.  Mean density (8 + 4) / 2 = 6, so Pi = -(alpha/2) v_sig w / rho_bar
    = -0.4 * 8 * (-2) / 6 = 16/15.  Both supports are 1, q = 0.75, and
    w'(q) = -(8/pi) 6 (1 - q)^2 = -3/pi, so grad_i Wbar = (r_ij / r) dW/dr
    = (3/pi, 0, 0).  a_i = -m Pi grad_i Wbar = (-16/(5 pi), 0, 0): the
    approaching pair is braked.  dA_i/dt = (gamma - 1)/2 rho_i^(1 - gamma)
    m Pi v_ij . grad_i Wbar = (1/3)(1/4)(16/15)(6/pi) = 8/(15 pi).

    Pair (i, j2): v_ij . r_ij = (1, -1, 0) . (0, -0.6, 0) = 0.6 > 0, receding:
    w = 0, no viscous force or heating, v_sig,ij = c_i + c_j2 = 21.  So
    v_sig,i = max(2 c_i, 8, 21) = 21.  With P = 0 the pair adds nothing else.

    j1 and j2 approach each other too (v . r = -0.15 at r = 0.96), so only
    the total momentum is checked for them: every pair term is antisymmetric,
    sum_k m_k a_k = 0."""
    fr = _visc_case(orc)
    a_i = fr["a"][0]
    assert abs(a_i[0] - (-16.0 / (5.0 * math.pi))) < 1e-12
    assert abs(a_i[1]) < 1e-15 and abs(a_i[2]) < 1e-15
    assert abs(fr["Adot"][0] - 8.0 / (15.0 * math.pi)) < 1e-12
    assert fr["vsig"][0] == 21.0
    assert fr["count"][0] == 2
    assert np.abs(fr["a"].sum(0)).max() < 1e-14
    # no viscosity: the same configuration moves nothing (P = 0)
    f0 = _visc_case(orc, alpha=0.0)
    assert np.all(f0["a"] == 0.0) and np.all(f0["Adot"] == 0.0)
    # Pi is linear in alpha: a_i(alpha = 1.6) = 2 a_i(0.8)
    f2 = _visc_case(orc, alpha=1.6)
    assert abs(f2["a"][0, 0] - 2.0 * a_i[0]) < 1e-12


def test_force_viscosity_plausible_slips_are_distinguishable():
    """The hand-computed case above separates the plausible slips in the
    viscosity: each gives a value of a_i,x or v_sig,i that is off by far more
    than the 1e-12 tolerance of the pin (values worked out by hand)."""
    right = -16.0 / (5.0 * math.pi)
    slips = {
        "alpha for alpha/2": -32.0 / (5.0 * math.pi),          # Pi = 32/15
        "rho_i for the mean density": -2.4 / math.pi,          # Pi = 0.8
        "-w for -3w in v_sig": -1.6 / math.pi,                 # v_sig 4, Pi = 8/15
        "max(0, .) for min(0, .)": 0.0,                        # no approach seen
        "rho_j for the mean density": -4.8 / math.pi,          # Pi = 1.6
    }
    for name, val in slips.items():
        assert abs(val - right) > 0.1, name


def test_force_search_modes_agree(orc):
    ic = sph_ics.clumpy_lattice(nside=12, n_clumps=2, per_clump=200, seed=3)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(5)
    A = rng.uniform(0.5, 1.5, n)
    vel = rng.normal(size=(n, 3))
    d = orc.density(ic["pos"], ic["m"], ic["h0"], np.ones(n, np.uint8))
    f = orc.gradh_f(d["h"], d["rho"], d["drho_dh"])
    P, c = orc.eos(A, d["rho"], GAMMA)
    act = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    a = orc.force(ic["pos"], vel, ic["m"], d["h"], d["rho"], f, P, c, act, use_cells=True)
    b = orc.force(ic["pos"], vel, ic["m"], d["h"], d["rho"], f, P, c, act, use_cells=False)
    assert np.array_equal(a["count"], b["count"])
    assert np.abs(a["a"] - b["a"]).max() < 1e-12 * np.abs(b["a"]).max()
    assert np.all(a["count"][act == 0] == 0)


# --------------------------------------------------------------------------
# Time bins (Eq. 1, Eq. 2)
# --------------------------------------------------------------------------

def test_bins_golden(orc):
    g = json.load(open(os.path.join(GOLDEN, "bins_cases.json")))
    for c in g["bin_of_dt"]:
        assert orc.bin_of_dt(c["dt"], c["dt_min"], c["cap"]) == c["bin"], c
    # synchronisation of bin increases: drive timestep_bins with a dt that
    # asks for the unsynchronised bin exactly
    for c in g["sync"]["cases"]:
        dt = 2.0 ** c["new"] * 1.5
        r = orc.timestep_bins(np.array([dt]), np.array([1.0]), np.ones(1, np.uint8), 1.0, 1.0,
                              30, c["ti"], np.array([c["old"]], np.int8))
        assert int(r["bin"][0]) == c["bin"], c
        assert r["ti_end"][0] == c["ti"] + 2 ** c["bin"]
        assert r["ti_end"][0] % 2 ** c["bin"] == 0


def test_bins_cfl_and_errors(orc):
    """dt = C h / v_sig (Eq. 1); dt below dt_min is reported and put on bin 0."""
    h = np.array([0.01, 0.02, 1e-9])
    vs = np.array([1.0, 1.0, 1.0])
    r = orc.timestep_bins(h, vs, np.ones(3, np.uint8), 0.1, 1e-4, 12, 0, np.zeros(3, np.int8))
    assert np.allclose(r["dt"], 0.1 * h / vs, rtol=0, atol=0)
    assert list(r["bin"]) == [3, 4, 0] and r["n_too_small"] == 1


# --------------------------------------------------------------------------
# Cells
# --------------------------------------------------------------------------

def test_cells_golden(orc):
    g = json.load(open(os.path.join(GOLDEN, "cells_cases.json")))
    r = orc.cells(np.array(g["positions"]), g["box"], g["n_cells"])
    assert list(r["cell"]) == g["cell"]
    assert list(r["perm"]) == g["perm"]


def test_cells_order_is_stable_sort(orc):
    ic = sph_ics.clumpy_lattice(nside=10, n_clumps=2, per_clump=100, seed=7)
    r = orc.cells(ic["pos"], 1.0, 5)
    key = r["key"]
    perm = r["perm"]
    assert np.all(np.diff(key[perm].astype(np.float64)) >= 0)
    ref = np.lexsort((np.arange(len(key)), key))
    assert np.array_equal(perm, ref)
    assert np.all(r["cell"] == (key >> np.uint64(30)).astype(np.int64))


# --------------------------------------------------------------------------
# Kick-drift-kick with bins
# --------------------------------------------------------------------------

def _small_sim(orc, dt_min, alpha=0.0, seed=41, nside=6, **kw):
    ic = sph_ics.lattice(nside, jitter=0.1, seed=seed)
    rng = np.random.default_rng(seed)
    vel = rng.normal(scale=0.3, size=ic["pos"].shape)
    vel -= vel.mean(0)
    u = rng.uniform(0.8, 1.2, ic["pos"].shape[0])
    return orc.OracleSim(ic["pos"], vel, ic["m"], u, ic["h0"], alpha=alpha, dt_min=dt_min,
                         use_cells=False, **kw)


def test_kdk_energy_error_is_second_order(orc):
    """Global step, alpha = 0: the energy error after a fixed time falls by ~4
    when dt is halved (a second-order symplectic scheme; catches a kick or
    drift with the wrong weight, or a missing grad-h term)."""
    T = 0.02
    errs = []
    for dt in (2e-3, 1e-3):
        s = _small_sim(orc, dt, global_step=True)
        nsteps = int(round(T / dt)) + 1
        for _ in range(nsteps):
            s.step()
        errs.append(abs(s.E_sync[-1] - s.E_sync[0]))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.5, (errs, ratio)


def test_kdk_momentum_and_reversibility(orc):
    """Global step, alpha = 0: momentum conserved to roundoff; reversing the
    velocities retraces the trajectory (KDK is time-symmetric)."""
    dt = 1e-3
    s = _small_sim(orc, dt, global_step=True, h_tol=1e-15, max_iter=200)
    p0 = s.momentum()
    x0 = s.pos.copy()
    N = 8
    for _ in range(N):
        s.step()
    assert np.abs(s.momentum() - p0).max() < 1e-13
    # positions are at t_(N-1) and the state holds v_half = v_full + a dt/2; the
    # reversed half-step velocity is -v_full + a dt/2 = -v_half + a dt, and N-1
    # reversed steps lead back to the initial positions
    s.vel = -s.vel + s.acc * dt
    for _ in range(N - 1):
        s.step()
    d = s.pos - x0
    d -= np.round(d)
    assert np.abs(d).max() < 1e-10


def test_kdk_bins_invariants(orc):
    """Individual bins: each particle's step ends on a multiple of its step,
    the active set at each time is exactly the particles whose step ends
    there, and the integrator visits times in increasing order."""
    ic = sph_ics.clumpy_lattice(nside=8, n_clumps=1, per_clump=60, seed=9)
    s = orc.OracleSim(ic["pos"], np.zeros_like(ic["pos"]), ic["m"], ic["u"], ic["h0"],
                      dt_min=2e-6, bin_cap=8, use_cells=False)
    last = -1
    seen_partial = False
    for _ in range(12):
        ti = s.ti
        assert ti > last
        last = ti
        act = s.step()
        seen_partial |= (0 < act.sum() < s.n)
        step = 1 << s.bin.astype(np.int64)
        assert np.all(s.ti_end % step == 0)
        assert np.all(s.ti_end > ti)
        assert np.all((s.ti_end[act] - s.ti_begin[act]) == step[act])
    assert seen_partial


# --------------------------------------------------------------------------
# Sedov blast: the self-similar shock radius
# --------------------------------------------------------------------------
# Sedov-Taylor constant of a spherical point explosion for gamma = 5/3: the
# energy integral of the self-similar solution is alpha = 0.4936, so
# R = XI0 (E t^2 / rho_0)^(1/5) with XI0 = alpha^(-1/5)
XI0 = 0.4936 ** -0.2


def test_sedov_shock_radius(orc):
    """Point explosion in a cold uniform medium (24^3 jittered lattice,
    rho_0 = 1, unit energy in the 32 central particles, u = 1e-5 elsewhere,
    individual bins up to 2^3 t_min): at t = 0.0075, 0.015 and 0.03
    (R / h = 3 .. 5.5) the mass-weighted radius of the compressed shell
    (rho > 1.2) is within 5 % of the Sedov-Taylor radius, the peak of the
    binned radial density lies 0-12 % behind it (SPH smooths the front over
    ~h), the front moves as t^(2/5) (exponent 0.33-0.45 between the first and
    last time), and the total energy stays within 1 % of its initial value.
    A pressure force off by a factor 2 moves R by ~15 % (R ~ E^(1/5)); a wrong
    adiabatic index changes XI0 and the compression of the shell."""
    ic = sph_ics.sedov(24, seed=2)
    dt_min = 2.0 ** -15
    s = orc.OracleSim(ic["pos"], ic["vel"], ic["m"], ic["u"], ic["h0"], cfl=0.1,
                      dt_min=dt_min, bin_cap=3)
    E0 = float((s.m * s.u0).sum())
    edges = np.arange(0.0, 0.45, 0.005)
    shells = []
    for t_want in (0.0075, 0.015, 0.03):
        while s.ti * dt_min < t_want:
            s.step()
        t = int(s.ti_drift.max()) * dt_min  # the tick the positions refer to
        r = np.linalg.norm(s.pos - 0.5, axis=1)
        R_st = XI0 * (E0 * t * t / 1.0) ** 0.2
        sh = s.rho > 1.2
        R_shell = float((s.m[sh] * r[sh]).sum() / s.m[sh].sum())
        assert abs(R_shell / R_st - 1.0) < 0.05, (t, R_shell, R_st)
        k = np.digitize(r, edges) - 1
        prof = np.array([s.rho[k == j].mean() if (k == j).any() else 0.0
                         for j in range(len(edges) - 1)])
        R_peak = 0.5 * (edges[np.argmax(prof)] + edges[np.argmax(prof) + 1])
        assert 0.88 < R_peak / R_st <= 1.0, (t, R_peak, R_st)
        u = orc.u_from_entropy(s.A, s.rho, s.gamma)
        E = float((s.m * (0.5 * (s.vel ** 2).sum(1) + u)).sum())
        assert abs(E / E0 - 1.0) < 0.01, (t, E, E0)
        shells.append((t, R_shell))
    (t1, r1), (t2, r2) = shells[0], shells[-1]
    expo = math.log(r2 / r1) / math.log(t2 / t1)
    assert 0.33 < expo < 0.45, expo
