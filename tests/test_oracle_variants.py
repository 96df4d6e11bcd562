"""Pins of the oracle's scheme variants (no GPU): the velocity divergence and
curl, the Balsara switch, the prediction of inactive particles' density and
smoothing length, and the neighbour time-step limiter.  Each test names the
mistake it would catch."""
import math

import numpy as np

import sph_ics

ETA = 1.2348
GAMMA = 5.0 / 3.0


def _interior(pos, h, gk, margin=1.0):
    """Particles whose whole support lies inside the box (a linear velocity
    field is not periodic, so only their neighbour sets see it whole)."""
    H = gk * h
    return np.all((pos > H[:, None] * margin + 1e-9) & (pos < 1.0 - H[:, None] * margin - 1e-9),
                  axis=1)


def _lattice_state(orc, nside):
    ic = sph_ics.lattice(nside, jitter=0.0)
    n = nside ** 3
    d = orc.density(ic["pos"], ic["m"], ic["h0"] * 1.05, np.ones(n, np.uint8), tol=1e-13,
                    max_iter=200)
    return ic, d


def _lattice_sums(orc, nside, h):
    """Independent lattice-vector sums (no periodic wrap, no oracle search):
    S1 = sum |r| W'(|r|) and S2 = sum (r_x^2 + r_y^2) W'(|r|) / |r| over the
    lattice vectors within the support, W' = H^-4 w'(r / H)."""
    H = orc.GAMMA_K * h
    k = np.arange(-6, 7)
    v = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3) / nside
    r = np.sqrt((v * v).sum(1))
    ok = (r > 0) & (r < H)
    v, r = v[ok], r[ok]
    dw = orc.kernel_dw(r / H) / H ** 4
    return (r * dw).sum(), ((v[:, 0] ** 2 + v[:, 1] ** 2) * dw / r).sum()


def test_divergence_of_homologous_expansion(orc):
    """v = H0 (x - x_c) on a perfect lattice: div v = -H0 m S1 / rho (the
    independent lattice sum, ~3 H0), curl = 0; catches a wrong sign, a
    missing 1/rho or m_j, or a kernel gradient of the wrong support."""
    nside = 16
    ic, d = _lattice_state(orc, nside)
    H0 = 0.37
    vel = H0 * (ic["pos"] - 0.5)
    gr = orc.gradient(ic["pos"], vel, ic["m"], d["h"], d["rho"], None)
    inner = _interior(ic["pos"], d["h"], orc.GAMMA_K)
    assert inner.sum() > 50
    S1, _ = _lattice_sums(orc, nside, d["h"][0])
    ref = -H0 * ic["m"][0] * S1 / d["rho"][0]
    assert abs(ref / (3 * H0) - 1) < 0.02          # the SPH estimate of 3 H0
    assert np.abs(gr["div"][inner] - ref).max() < 1e-10 * abs(ref)
    assert np.abs(gr["curl"][inner]).max() < 1e-10 * abs(ref)


def test_curl_of_rigid_rotation(orc):
    """v = Omega z x (x - x_c): curl_z = -Omega m S2 / rho (~2 Omega), the
    other components and div v vanish (catches a transposed cross product)."""
    nside = 16
    ic, d = _lattice_state(orc, nside)
    Om = 1.3
    rel = ic["pos"] - 0.5
    vel = Om * np.stack([-rel[:, 1], rel[:, 0], np.zeros(len(rel))], 1)
    gr = orc.gradient(ic["pos"], vel, ic["m"], d["h"], d["rho"], None)
    inner = _interior(ic["pos"], d["h"], orc.GAMMA_K)
    _, S2 = _lattice_sums(orc, nside, d["h"][0])
    ref = -Om * ic["m"][0] * S2 / d["rho"][0]
    assert abs(ref / (2 * Om) - 1) < 0.02
    c = gr["curl"][inner]
    assert np.abs(c[:, 2] - ref).max() < 1e-10 * abs(ref)
    assert np.abs(c[:, :2]).max() < 1e-10 * abs(ref)
    assert np.abs(gr["div"][inner]).max() < 1e-10 * abs(ref)


def test_divergence_is_the_rate_of_change_of_the_density(orc):
    """The SPH continuity equation with adaptive h: d ln rho_i / dt =
    -f_i div v_i.  The density after a small drift of a jittered set with a
    smooth velocity field, re-converged h, checks the divergence against the
    density loop itself (an independent route through the oracle)."""
    ic = sph_ics.lattice(12, jitter=0.15, seed=3)
    n = ic["pos"].shape[0]
    kx = 2 * np.pi * np.array([1, 2, 1])
    vel = 0.3 * np.stack([np.sin(kx[0] * ic["pos"][:, 1]), np.cos(kx[1] * ic["pos"][:, 2]),
                          np.sin(kx[2] * ic["pos"][:, 0] + 0.4)], 1)
    act = np.ones(n, np.uint8)
    d0 = orc.density(ic["pos"], ic["m"], ic["h0"], act, tol=1e-14, max_iter=200)
    f = orc.gradh_f(d0["h"], d0["rho"], d0["drho_dh"])
    gr = orc.gradient(ic["pos"], vel, ic["m"], d0["h"], d0["rho"], act)
    eps = 1e-6
    dp = orc.density((ic["pos"] + eps * vel) % 1.0, ic["m"], d0["h"], act, tol=1e-14,
                     max_iter=200)
    dm = orc.density((ic["pos"] - eps * vel) % 1.0, ic["m"], d0["h"], act, tol=1e-14,
                     max_iter=200)
    ok = (dp["count"] == d0["count"]) & (dm["count"] == d0["count"])
    assert ok.mean() > 0.8
    rate = (np.log(dp["rho"]) - np.log(dm["rho"])) / (2 * eps)
    pred = -f * gr["div"]
    scale = np.abs(pred[ok]).max()
    assert np.abs(rate[ok] - pred[ok]).max() < 1e-5 * scale


def test_balsara_factor_closed_form(orc):
    """B = |div| / (|div| + |curl| + 1e-4 c / h): hand-computed values."""
    assert orc.balsara([1.0], [0.0], [0.0], [1.0])[0] == 1.0
    assert orc.balsara([0.0], [2.0], [1.0], [1.0])[0] == 0.0
    assert abs(orc.balsara([-3.0], [4.0], [2.0], [0.5])[0] - 3.0 / 7.0004) < 1e-15


def test_balsara_scales_the_viscosity(orc):
    """The hand-computed three-particle viscosity case (test_oracle_pins):
    with Balsara factors B = (0.5, 0.25, 1) the pair (i, j1) is scaled by
    (0.5 + 0.25) / 2 = 0.375, so a_i,x = 0.375 (-16 / (5 pi)) and dA_i/dt =
    0.375 (8 / (15 pi)); the receding pair (i, j2) adds nothing either way."""
    pos = np.array([[5.0, 5.0, 5.0], [5.75, 5.0, 5.0], [5.0, 5.6, 5.0]])
    vel = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    H = np.array([1.0, 1.0, 1.2])
    rho = np.array([8.0, 4.0, 1.0])
    c = np.array([1.0, 1.0, 20.0])
    n = 3
    fr = orc.force(pos, vel, np.ones(n), H / orc.GAMMA_K, rho, np.ones(n), np.zeros(n), c,
                   np.ones(n, np.uint8), box=10.0, alpha=0.8, gamma=GAMMA, use_cells=False,
                   balsara=np.array([0.5, 0.25, 1.0]))
    assert abs(fr["a"][0, 0] - 0.375 * (-16.0 / (5.0 * math.pi))) < 1e-12
    assert abs(fr["Adot"][0] - 0.375 * 8.0 / (15.0 * math.pi)) < 1e-12
    assert fr["vsig"][0] == 21.0  # the signal velocity is not switched


def test_prediction_closed_form(orc):
    """rho exp(-div dt) and h exp(div dt / 3): hand-computed numbers, and
    mass conservation of the prediction (rho h^3 is unchanged)."""
    rho, h = orc.predict_inactive([2.0, 1.0], [0.1, 0.2], [3.0, -1.5], [0.1, 0.2])
    assert abs(rho[0] - 2.0 * math.exp(-0.3)) < 1e-15
    assert abs(h[0] - 0.1 * math.exp(0.1)) < 1e-16
    assert abs(rho[1] - math.exp(0.3)) < 1e-15
    assert abs(h[1] - 0.2 * math.exp(-0.1)) < 1e-16
    assert np.allclose(rho * h ** 3, [2.0 * 0.1 ** 3, 0.2 ** 3], rtol=1e-14)


def test_limiter_bins_hand_computed(orc):
    """dt_i <= 4 min_j dt_j: a CFL bin of 8 next to a neighbour on bin 3 is
    capped at 5; at tick 16 the rise from bin 4 to 5 waits for a tick that 2^5
    divides (the synchronisation rule comes after the cap); a CFL bin below the
    cap is kept; without the limiter nothing is capped."""
    dt_min = 1.0
    h = np.array([1.0, 1.0, 1.0])
    vsig = np.array([0.1 / 256.5, 0.1 / 256.5, 0.1 / 8.5])  # CFL bins 8, 8, 3 (C = 0.1)
    act = np.ones(3, np.uint8)
    old = np.array([4, 4, 4], np.int8)
    ngb = np.array([3, 3, 3], np.int8)
    tb = orc.timestep_bins(h, vsig, act, 0.1, dt_min, 20, 32, old, ngb)
    assert list(tb["bin"]) == [5, 5, 3]
    assert list(tb["ti_end"]) == [64, 64, 40]
    tb = orc.timestep_bins(h, vsig, act, 0.1, dt_min, 20, 16, old, ngb)
    assert list(tb["bin"]) == [4, 4, 3]
    tb = orc.timestep_bins(h, vsig, act, 0.1, dt_min, 20, 256, old, None)
    assert list(tb["bin"]) == [8, 8, 3]


def test_limiter_neighbour_minimum_from_the_force_loop(orc):
    """The force loop reports the smallest bin among each particle's
    neighbours j != i with r < max(H_i, H_j) (the three-particle case: all
    three are mutual neighbours)."""
    pos = np.array([[5.0, 5.0, 5.0], [5.75, 5.0, 5.0], [5.0, 5.6, 5.0], [8.0, 8.0, 8.0]])
    vel = np.zeros((4, 3))
    H = np.array([1.0, 1.0, 1.2, 1.0])
    n = 4
    fr = orc.force(pos, vel, np.ones(n), H / orc.GAMMA_K, np.ones(n), np.ones(n), np.ones(n),
                   np.ones(n), np.ones(n, np.uint8), box=10.0, use_cells=False,
                   bins=np.array([5, 2, 7, 1], np.int8))
    assert list(fr["bin_ngb_min"][:3]) == [2, 5, 2]
    assert fr["bin_ngb_min"][3] == 127  # no neighbour: no cap


def test_wake_requests_hand_computed(orc):
    """The waking half of the limiter: an inactive particle whose bin is more
    than 2 above an active force-loop neighbour's is asked down to that bin
    + 2 (the smallest such request wins); active particles and particles
    with no active neighbour get no request (127).  Particles 0, 1, 2 are
    mutual neighbours, particle 3 is isolated."""
    pos = np.array([[5.0, 5.0, 5.0], [5.75, 5.0, 5.0], [5.0, 5.6, 5.0], [8.0, 8.0, 8.0]])
    H = np.array([1.0, 1.0, 1.2, 1.0])
    bins = np.array([5, 2, 7, 1], np.int8)
    act = np.array([0, 1, 0, 1], np.uint8)
    req = orc.wake_bins(pos, H / orc.GAMMA_K, act, bins, box=10.0, use_cells=False)
    assert list(req) == [4, 127, 4, 127]
    # particle 0 active too (bin 5): it asks particle 2 for 7, which is not
    # below 7; particle 1's request (4) stands
    act = np.array([1, 1, 0, 1], np.uint8)
    req = orc.wake_bins(pos, H / orc.GAMMA_K, act, bins, box=10.0, use_cells=False)
    assert list(req) == [127, 127, 4, 127]
    # out of reach: the pair must be a force-loop pair (r < max(H_i, H_j))
    far = pos.copy()
    far[1] = [6.3, 5.0, 5.0]  # 1.3 from particle 0, 1.43 from particle 2 (H <= 1.2)
    req = orc.wake_bins(far, H / orc.GAMMA_K, np.array([0, 1, 0, 0], np.uint8), bins,
                        box=10.0, use_cells=False)
    assert list(req) == [127, 127, 127, 127]


def test_wake_hand_computed(orc):
    """Waking at tick 4: a particle on bin 6 (step [0, 64)) asked down to bin
    4 now ends its step at 16, the first multiple of 16 after 4; its opening
    half-kick is cut from 32 to 8 ticks (v -= a 24 dt_min, A -= Adot 24
    dt_min).  A particle whose step already ends at the first multiple (bin 3,
    [0, 8), asked for 2: 8) and one without a request are left alone; the
    predicted velocity at the current tick does not change."""
    dt_min = 0.5
    ti = 4
    act = np.array([True, False, False, False])
    req = np.array([127, 4, 2, 127], np.int8)
    bins = np.array([2, 6, 3, 6], np.int8)
    tb = np.array([4, 0, 0, 0], np.int64)
    te = np.array([8, 64, 8, 64], np.int64)
    vel = np.array([[1.0, 0, 0], [2.0, 1.0, 0], [3.0, 0, 0], [4.0, 0, 0]])
    acc = np.array([[0.1, 0, 0], [0.5, -0.25, 0], [0.2, 0, 0], [0.3, 0, 0]])
    A = np.array([1.0, 2.0, 3.0, 4.0])
    Adot = np.array([0.0, 0.125, 0.0, 0.0])
    vpred0 = vel + acc * (((ti - tb) - 0.5 * (te - tb)) * dt_min)[:, None]
    n = orc.wake(ti, req, act, bins, tb, te, vel, A, acc, Adot, dt_min)
    assert n == 1
    assert list(bins) == [2, 4, 3, 6]
    assert list(te) == [8, 16, 8, 64]
    assert np.allclose(vel[1], [2.0 - 0.5 * 24 * 0.5, 1.0 + 0.25 * 24 * 0.5, 0.0], rtol=0,
                       atol=1e-15)
    assert A[1] == 2.0 - 0.125 * 24 * 0.5
    assert np.array_equal(vel[[0, 2, 3]], [[1.0, 0, 0], [3.0, 0, 0], [4.0, 0, 0]])
    vpred1 = vel + acc * (((ti - tb) - 0.5 * (te - tb)) * dt_min)[:, None]
    assert np.allclose(vpred1, vpred0, rtol=0, atol=1e-14)


def test_wake_invariant_in_a_kdk_step(orc):
    """After a limiter step from mixed bins (a clump on bin 2 inside a
    background on bin 6), every inactive force-loop neighbour of a particle
    active in the step ends its step within 2^(bin_i + 2) ticks of it (pairs
    found here by a brute-force periodic double loop), some particles were
    woken, and the run's later steps see them active."""
    ic = sph_ics.clumpy_lattice(nside=8, n_clumps=1, per_clump=64, seed=11)
    n = ic["pos"].shape[0]
    kw = dict(dt_min=1e-6, bin_cap=14, cfl=0.1)
    s = orc.OracleSim(ic["pos"], np.zeros((n, 3)), ic["m"], 1.0, ic["h0"], limiter=True, **kw)
    s.step()  # the first step (all active) sets h, rho, A, a
    # mixed bins: the clump (the 64 densest) on bin 2, the rest on bin 6,
    # every step starting at the current tick
    ti0 = s.ti
    t0 = ti0 - ti0 % 64
    dense = np.argsort(-s.rho)[:64]
    s.bin[:] = 6
    s.bin[dense] = 2
    s.ti_begin[:] = t0
    s.ti_end[:] = t0 + (np.int64(1) << s.bin.astype(np.int64))
    s.ti = int(s.ti_end.min())
    ti = s.ti
    bins_before = s.bin.copy()
    act = s.step()
    assert act.sum() == 64 and s.n_woken > 0
    # brute-force force-loop pairs at the step's positions and supports
    H = orc.GAMMA_K * s.h
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= np.round(d)
    r2 = (d ** 2).sum(-1)
    pair = (r2 < H[:, None] ** 2) | (r2 < H[None, :] ** 2)
    np.fill_diagonal(pair, False)
    for i in np.nonzero(act)[0]:
        for j in np.nonzero(pair[i] & ~act)[0]:
            assert s.ti_end[j] - ti <= (1 << (int(bins_before[i]) + 2)), (i, j)
    woken = (s.bin < bins_before) & ~act
    assert woken.sum() == s.n_woken
    # the woken particles are active when their shortened steps end
    t_w = int(s.ti_end[woken].min())
    while s.ti < t_w:
        s.step()
    assert s.ti == t_w
    act = s.step()
    assert act[woken & (s.ti_end > 0)].any()


def test_variants_kdk_run(orc):
    """A short run with all three variants: momentum is conserved to
    roundoff (the Balsara factor is symmetric in the pair), the predicted
    density of the inactive particles keeps rho h^3 fixed, and the variants
    change the run."""
    ic = sph_ics.clumpy_lattice(nside=10, n_clumps=1, per_clump=150, seed=9)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(9)
    ic["vel"] = rng.normal(scale=0.2, size=(n, 3))
    kw = dict(dt_min=1e-6, bin_cap=14, cfl=0.1)
    s = orc.OracleSim(ic["pos"], ic["vel"], ic["m"], 1.0, ic["h0"], predict=True, balsara=True,
                      limiter=True, **kw)
    b = orc.OracleSim(ic["pos"], ic["vel"], ic["m"], 1.0, ic["h0"], **kw)
    p0 = s.momentum()
    for _ in range(6):
        s.step()
        b.step()
    scale = (s.m[:, None] * np.abs(s.vel)).sum()
    assert np.abs(s.momentum() - p0).max() < 1e-12 * scale
    rho_p, h_p = s._predict_rho_h(s.ti)
    assert np.allclose(rho_p * h_p ** 3, s.rho * s.h ** 3, rtol=1e-12)
    # the variants change the run (Balsara damps the viscosity)
    assert not np.allclose(s.vel, b.vel)
