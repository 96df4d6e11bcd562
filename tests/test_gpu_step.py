"""Whole kick-drift-kick steps on the GPU against the oracle, and the three
execution forms (plain per-bin launches, batched persistent kernels, CUDA
graph replay) against each other."""
import numpy as np
import pytest

import sph_ics
from _gpu_helpers import gpu_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01341_gb300 import build
    build.build()
    from paper_1807_01341_gb300 import sim as S
    return S


def _lib():
    from paper_1807_01341_gb300 import _lib
    return _lib


def _ic_step(seed=13, nside=12):
    ic = sph_ics.clumpy_lattice(nside=nside, n_clumps=1, per_clump=200, seed=seed)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(seed)
    ic["vel"] = rng.normal(scale=0.1, size=(n, 3))
    ic["u"] = rng.uniform(0.5, 2.0, n)
    return ic


STEP_PARAMS = dict(dt_min=1e-6, bin_cap=14, cfl=0.1)


@pytest.mark.parametrize("heavy_factor", [0.0, 1e-9])
def test_step_parity_each_step_from_same_state(sim, orc, heavy_factor):
    """Before every GPU step the oracle integrator is loaded with the GPU's
    state and advanced one step: active sets and bins must agree exactly
    (bins up to dt values within 2e-5 of a power of two), and the floating
    point state within the hot-path tolerances.  heavy_factor 1e-9 marks every
    work group heavy (taken from the back of the queue, first)."""
    ic = _ic_step()
    n = ic["pos"].shape[0]
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS, heavy_factor=heavy_factor))
    L = _lib()
    n_partial = 0
    for k in range(10):
        st0 = p.numpy()
        _, ti = ctx.get_time()
        osim = orc.OracleSim.from_state(st0, ti=ti, first=(k == 0), use_cells=True,
                                        **STEP_PARAMS)
        act_ref = osim.step()
        ctx.step(p, L.SPH_FORM_BATCHED)
        st = p.numpy()
        act = st["active"].astype(bool)
        assert np.array_equal(act, act_ref), k
        n_partial += int(0 < act.sum() < n)
        pos = np.stack([st["x"], st["y"], st["z"]], 1)
        moved = st["ti_drift"] == ti
        assert moved[act].all()
        d = pos[moved] - osim.pos[moved]
        d -= np.round(d)
        assert np.abs(d).max() < 1e-12
        assert np.max(np.abs(st["h"][act] / osim.h[act] - 1)) < 1e-5
        assert np.max(np.abs(st["rho"][act] / osim.rho[act] - 1)) < 1e-5
        a = np.stack([st["ax"], st["ay"], st["az"]], 1)[act]
        a_ref = osim.acc[act]
        a_rms = np.sqrt((a_ref ** 2).sum(1).mean())
        assert np.max(np.abs(a - a_ref)) < 1e-4 * a_rms
        assert np.max(np.abs(st["vsig"][act] / osim.vsig[act] - 1)) < 1e-5
        # bins: exact unless the oracle's dt sits on a power-of-two edge
        q = osim.cfl * osim.h / osim.vsig / osim.dt_min
        edge = np.abs(np.log2(q) - np.round(np.log2(q))) < 2e-5
        ok = act & ~edge
        assert np.array_equal(st["bin"][ok], osim.bin[ok])
        assert np.array_equal(st["ti_end"][ok], osim.ti_end[ok])
        # velocities after both half-kicks
        v = np.stack([st["vx"], st["vy"], st["vz"]], 1)[ok]
        dt = (osim.ti_end - osim.ti_begin)[ok] * osim.dt_min
        scale = np.sqrt((osim.vel[ok] ** 2).sum(1).mean()) + a_rms * dt.max()
        assert np.max(np.abs(v - osim.vel[ok])) < 1e-4 * scale
    assert n_partial >= 3          # the run exercised individual time bins


def _run_form(sim, ic, form, steps, params):
    import torch
    ctx, p = gpu_setup(ic, sim.Params(**params))
    if form == "graph":
        ctx.step_graph(p, steps)
    else:
        L = _lib()
        f = L.SPH_FORM_PLAIN if form == "plain" else L.SPH_FORM_BATCHED_NOGRAPH
        for _ in range(steps):
            ctx.step(p, f)
    torch.cuda.synchronize()
    return p.numpy(), ctx.counters(), ctx.get_time()


@pytest.mark.parametrize("heavy_factor,coop_max_groups", [(0.0, 0), (1.0, 0), (1e-9, 0),
                                                           (0.0, 1 << 30)])
def test_plain_batched_graph_bitwise_identical(sim, heavy_factor, coop_max_groups):
    """One lane per particle: every sum's order depends on the particle only,
    whichever warp takes a group and in which order (heavy factor 1: some
    groups started first, 1e-9: all), and also when the force loop's groups
    are shared by the warps of a block (coop_max_groups: every group of every
    step).  At this size (1,728 particles, about a hundred work groups) the
    batched form splits every step's groups into slices of their active
    particles over its idle warps (density and force) or blocks (shared force
    groups), while the plain form takes each group whole: the bits still
    agree."""
    ic = _ic_step(seed=17)
    params = dict(STEP_PARAMS, heavy_factor=heavy_factor, coop_max_groups=coop_max_groups)
    res = {f: _run_form(sim, ic, f, 12, params) for f in ("plain", "batched", "graph")}
    ref, cref, tref = res["batched"]
    for f in ("plain", "graph"):
        st, c, t = res[f]
        assert t == tref, f
        for k in ref:
            assert np.array_equal(st[k], ref[k]), (f, k)
        for k in ("pairs_density", "pairs_force", "steps", "active_particles"):
            assert c[k] == cref[k], (f, k)


def test_forms_agree_with_several_lanes_per_particle(sim):
    """Four lanes per particle: the forms agree to rounding, and exactly on
    every integer result."""
    ic = _ic_step(seed=18)
    params = dict(STEP_PARAMS, threads_per_particle=4)
    a, ca, ta = _run_form(sim, ic, "plain", 6, params)
    b, cb, tb = _run_form(sim, ic, "graph", 6, params)
    assert ta == tb
    for k in ("bin", "ti_end", "active"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("h", "rho", "ax", "vx"):
        assert np.allclose(a[k], b[k], rtol=1e-5, atol=1e-5 * np.abs(b[k]).max()), k


def test_drift_all_same_result_as_relevant_drift(sim):
    """Drifting every particle each step (the ablation) gives the same state
    as drifting only the cells next to active cells (Sec. III-D), up to the
    rounding of split drifts."""
    ic = _ic_step(seed=19)
    a, ca, _ = _run_form(sim, ic, "batched", 8, dict(STEP_PARAMS, drift_all=0))
    b, cb, _ = _run_form(sim, ic, "batched", 8, dict(STEP_PARAMS, drift_all=1))
    assert ca["pairs_density"] == cb["pairs_density"]
    for k in ("bin", "ti_end", "active"):
        assert np.array_equal(a[k], b[k]), k
    # positions agree once brought to the same tick
    for k in ("h", "rho", "ax"):
        assert np.allclose(a[k], b[k], rtol=1e-5, atol=1e-6 * np.abs(b[k]).max()), k


def test_global_step_ablation(sim):
    """bin_cap = 0 puts every particle on the smallest step: every step is
    all-active."""
    ic = _ic_step(seed=23)
    n = ic["pos"].shape[0]
    params = dict(STEP_PARAMS, bin_cap=0, dt_min=1e-5)
    st, c, (ti, tn) = _run_form(sim, ic, "batched", 5, params)
    assert c["active_particles"] == 5 * n
    assert tn == 5


def test_empty_and_degenerate_sizes(sim):
    import torch
    L = _lib()
    # no particles at all
    ctx = sim.Context(sim.Params(), 1)
    p = sim.Particles(0)
    ctx.build_cells(p)
    ctx.step(p, L.SPH_FORM_BATCHED)
    ctx.step(p, L.SPH_FORM_PLAIN)
    assert ctx.status()[0] == 0
    # the smallest grid (3 cells per axis)
    ic = sph_ics.lattice(8, 0.1, seed=3)
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS))
    assert ctx.grid_info()[0] == 3
    ctx.step(p, L.SPH_FORM_BATCHED)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(p.numpy()["rho"]))
    # supports wider than a third of the box: reported, not faulted
    ic = sph_ics.lattice(4, 0.0, seed=3)
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS))
    with pytest.raises(L.SphError) as e:
        ctx.step(p, L.SPH_FORM_BATCHED)
    assert e.value.code == L.SPH_ERR_CELL_OVERFLOW


def test_h_growth_triggers_rebuild_and_redo(sim, orc):
    """Initial h guesses far too small with a coarse grid forced narrow by
    them: the h iteration outgrows the cells, the step is redone after a
    rebuild, and the result still matches the oracle."""
    ic = sph_ics.lattice(16, 0.1, seed=29)
    n = ic["pos"].shape[0]
    ic["h0"] = ic["h0"] * 0.3
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS))
    nc0 = ctx.grid_info()[0]
    L = _lib()
    ctx.step(p, L.SPH_FORM_BATCHED)
    c = ctx.counters()
    assert c["redone_steps"] >= 1 and ctx.grid_info()[0] < nc0
    st = p.numpy()
    pos = np.stack([st["x"], st["y"], st["z"]], 1)
    perm = ctx.perm_tensor(n).cpu().numpy()
    ref = orc.density(pos, st["m"].astype(np.float64),
                      np.float32(ic["h0"])[perm].astype(np.float64), np.ones(n, np.uint8))
    assert np.max(np.abs(st["h"] / ref["h"] - 1)) < 1e-5


def test_invalid_input_is_rejected(sim):
    """A non-finite position or h (NaN, inf, h <= 0): the cell build returns
    SPH_ERR_ARG before reordering anything; the context stays usable."""
    import torch
    L = _lib()
    ic = sph_ics.lattice(8, 0.1, seed=5)
    for field, value in (("x", float("nan")), ("z", float("inf")), ("h", float("nan")),
                         ("h", 0.0), ("h", -1.0)):
        ctx = sim.Context(sim.Params(**STEP_PARAMS), ic["pos"].shape[0])
        p = sim.Particles.from_ics(ic)
        getattr(p, field)[7] = value
        before = p.numpy()["y"].copy()
        with pytest.raises(L.SphError) as e:
            ctx.build_cells(p)
        assert e.value.code == L.SPH_ERR_ARG, (field, value)
        assert np.array_equal(p.numpy()["y"], before)  # not reordered
        # the same context builds and steps once the input is repaired
        p2 = sim.Particles.from_ics(ic)
        ctx.build_cells(p2)
        ctx.step(p2, L.SPH_FORM_BATCHED)
        assert ctx.status()[0] == 0
        ctx.close()
    torch.cuda.synchronize()


def test_h_nonconvergence_is_reported(sim):
    """h_max_iter = 1: the smoothing lengths cannot converge; the step
    completes and the status word reports SPH_ERR_H_NOCONV with the number
    of particles concerned (no halt, finite state)."""
    L = _lib()
    ic = _ic_step(seed=37)
    n = ic["pos"].shape[0]
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS, h_max_iter=1))
    ctx.step(p, L.SPH_FORM_BATCHED)
    code, detail = ctx.status()
    assert code == L.SPH_ERR_H_NOCONV and 0 < detail <= n
    st = p.numpy()
    assert np.all(np.isfinite(st["rho"])) and np.all(np.isfinite(st["ax"]))
    ctx.clear_status()
    assert ctx.status()[0] == 0
    ctx.close()


def test_dt_below_t_min_is_reported(sim):
    """t_min larger than every CFL step: the step completes, the particles go
    to bin 0 and the status word reports SPH_ERR_DT_TOO_SMALL for all of
    them."""
    L = _lib()
    ic = _ic_step(seed=41)
    n = ic["pos"].shape[0]
    ctx, p = gpu_setup(ic, sim.Params(**dict(STEP_PARAMS, dt_min=10.0)))
    ctx.step(p, L.SPH_FORM_BATCHED)
    code, detail = ctx.status()
    assert code == L.SPH_ERR_DT_TOO_SMALL and detail == n
    assert np.all(p.numpy()["bin"] == 0)
    ctx.close()


@pytest.mark.parametrize("coop_max_groups", [0, 1 << 30])
def test_lists_margin_and_staging_depth_do_not_change_results(sim, coop_max_groups):
    """The density loop's neighbour lists (kept across h iterations), their
    capacity, the search margin of a gather and the number of staging buffers
    change how the candidates are found, not which pairs are summed nor in
    what order: 12 steps agree bit for bit.  A list of 32 entries fills up
    for most particles (their gathers run in passes); coop_max_groups 2^30
    sends every work group to a whole block (per-warp lists)."""
    ic = _ic_step(seed=43)
    base = dict(STEP_PARAMS, coop_max_groups=coop_max_groups)
    ref, cref, tref = _run_form(sim, ic, "graph", 12,
                                dict(base, list_cap=128, search_margin=1.1, staging_depth=1))
    # a list spares most iterations their gather
    assert 0 < cref["gathers_density"] < cref["iters_density"]
    variants = [dict(list_cap=512, search_margin=1.5, staging_depth=3),
                dict(list_cap=64, search_margin=1.0, staging_depth=2),
                dict(list_cap=32, search_margin=1.1, staging_depth=2)]
    for var in variants:
        st, c, t = _run_form(sim, ic, "graph", 12, dict(base, **var))
        assert t == tref, var
        for k in ref:
            assert np.array_equal(st[k], ref[k]), (var, k)
        for k in ("pairs_density", "pairs_force", "iters_density", "active_particles"):
            assert c[k] == cref[k], (var, k)
        if var["list_cap"] == 32:
            assert c["list_overflows"] > 0
    # the plain form with three buffers is the same run too
    st, c, t = _run_form(sim, ic, "plain", 12, dict(base, list_cap=96, staging_depth=3))
    assert t == tref
    for k in ref:
        assert np.array_equal(st[k], ref[k]), ("plain", k)


@pytest.mark.parametrize("coop_max_groups", [0, 1 << 30])
def test_bounded_wait_gives_up_and_context_recovers(sim, coop_max_groups):
    """A staging barrier that no copy completes (test_stall: one warp of the
    first density launch issues no copy and never arrives): the bounded wait
    gives up after wait_limit polls, the step stops with SPH_ERR_TIMEOUT
    (status word: the timed-out waits counted), nothing traps, and after the
    status is cleared the same context completes the step and agrees with a
    run that never stalled."""
    import torch
    L = _lib()
    ic = _ic_step(seed=47)
    params = dict(STEP_PARAMS, coop_max_groups=coop_max_groups)
    ref, _, _ = _run_form(sim, ic, "batched", 1, params)
    ctx, p = gpu_setup(ic, sim.Params(**params, wait_limit=2000, test_stall=1))
    with pytest.raises(L.SphError) as e:
        ctx.step(p, L.SPH_FORM_BATCHED)
    assert e.value.code == L.SPH_ERR_TIMEOUT
    code, detail = ctx.status()
    assert code == L.SPH_ERR_TIMEOUT and detail >= 1
    assert ctx.counters()["steps"] == 0
    ctx.clear_status()
    ctx.step(p, L.SPH_FORM_BATCHED)
    torch.cuda.synchronize()
    assert ctx.status()[0] == 0 and ctx.counters()["steps"] == 1
    st = p.numpy()
    for k in ("x", "y", "z"):
        assert np.array_equal(st[k], ref[k]), k
    assert np.array_equal(st["active"], ref["active"])
    # the redone step starts its h iteration from partly updated guesses:
    # the same roots to the convergence tolerance
    for k in ("h", "rho"):
        assert np.max(np.abs(st[k] / ref[k] - 1)) < 1e-5, k
    a = np.stack([st["ax"], st["ay"], st["az"]], 1)
    a_ref = np.stack([ref["ax"], ref["ay"], ref["az"]], 1)
    assert np.max(np.abs(a - a_ref)) < 1e-4 * np.sqrt((a_ref ** 2).sum(1).mean())
    ctx.close()


VARIANTS = [dict(balsara=1, predict_inactive=1, limiter=1), dict(balsara=1),
            dict(predict_inactive=1), dict(limiter=1)]


@pytest.mark.parametrize("var", VARIANTS)
def test_variants_step_parity_each_step_from_same_state(sim, orc, var):
    """The scheme's variants (Balsara switch, Gadget-2 prediction of inactive
    rho and h, Saitoh-Makino neighbour limiter) against the oracle run with
    the same switches, step by step from the GPU's state: active sets and
    bins exact, the velocity divergence and curl within 1e-4 of their rms,
    the floating-point state within the hot-path tolerances."""
    ic = _ic_step(seed=53)
    n = ic["pos"].shape[0]
    ctx, p = gpu_setup(ic, sim.Params(**STEP_PARAMS, **var))
    L = _lib()
    okw = dict(predict=bool(var.get("predict_inactive")), balsara=bool(var.get("balsara")),
               limiter=bool(var.get("limiter")))
    n_partial = 0
    for k in range(8):
        st0 = p.numpy()
        _, ti = ctx.get_time()
        osim = orc.OracleSim.from_state(st0, ti=ti, first=(k == 0), use_cells=True,
                                        **STEP_PARAMS, **okw)
        act_ref = osim.step()
        ctx.step(p, L.SPH_FORM_BATCHED)
        st = p.numpy()
        act = st["active"].astype(bool)
        assert np.array_equal(act, act_ref), k
        n_partial += int(0 < act.sum() < n)
        assert np.max(np.abs(st["h"][act] / osim.h[act] - 1)) < 1e-5
        assert np.max(np.abs(st["rho"][act] / osim.rho[act] - 1)) < 1e-5
        if okw["predict"] or okw["balsara"]:
            for key, ref in (("div_v", osim.divv), ("curl_v", osim.curl)):
                rms = np.sqrt((ref[act] ** 2).mean()) + 1e-30
                assert np.max(np.abs(st[key][act] - ref[act])) < 1e-4 * rms, (k, key)
        a = np.stack([st["ax"], st["ay"], st["az"]], 1)[act]
        a_ref = osim.acc[act]
        a_rms = np.sqrt((a_ref ** 2).sum(1).mean())
        assert np.max(np.abs(a - a_ref)) < 1e-4 * a_rms, k
        assert np.max(np.abs(st["vsig"][act] / osim.vsig[act] - 1)) < 1e-5
        q = osim.cfl * osim.h / osim.vsig / osim.dt_min
        with np.errstate(divide="ignore", invalid="ignore"):
            edge = np.abs(np.log2(q) - np.round(np.log2(q))) < 2e-5
        ok = act & ~edge
        assert np.array_equal(st["bin"][ok], osim.bin[ok]), k
    assert n_partial >= 2          # individual bins (the limiter narrows them)


def test_limiter_wakes_inactive_neighbours(sim, orc):
    """The limiter's waking (Saitoh & Makino 2009): from a state with the
    densest particles on bin 2 and the rest on bin 6 (steps from tick 0), the
    step at tick 4 wakes the bin-6 force neighbours of the active particles:
    their steps now end at tick 16 (bin 4) and their opening half-kicks are
    cut to the shorter step.  Against the oracle from the same state, step by
    step: active sets, bins and step ends exact, the woken count equal,
    velocities within the hot-path tolerance."""
    import torch
    ic = _ic_step(seed=67)
    n = ic["pos"].shape[0]
    params = dict(STEP_PARAMS, limiter=1)
    ctx, p = gpu_setup(ic, sim.Params(**params))
    L = _lib()
    ctx.step(p, L.SPH_FORM_BATCHED)  # the first step: h, rho, entropy, a
    st = p.numpy()
    dense = np.argsort(-st["rho"])[: n // 8]
    b = np.full(n, 6, np.int64)
    b[dense] = 2
    p.bin.copy_(torch.as_tensor(b.astype(np.int8)))
    p.ti_begin.zero_()
    p.ti_end.copy_(torch.as_tensor(np.left_shift(1, b)))
    p.ti_drift.zero_()
    ctx.build_cells(p)  # (bin occupancy and leaf bins from the new bins)
    ctx.set_time(4)
    woken_total = 0
    for k in range(4):
        st0 = p.numpy()
        _, ti = ctx.get_time()
        w0 = ctx.counters()["wakes"]
        osim = orc.OracleSim.from_state(st0, ti=ti, use_cells=True, limiter=True, **STEP_PARAMS)
        act_ref = osim.step()
        ctx.step(p, L.SPH_FORM_BATCHED)
        st = p.numpy()
        assert ctx.status()[0] == 0
        act = st["active"].astype(bool)
        assert np.array_equal(act, act_ref), k
        woken = ctx.counters()["wakes"] - w0
        assert woken == osim.n_woken, (k, woken, osim.n_woken)
        woken_total += woken
        q = osim.cfl * osim.h / osim.vsig / osim.dt_min
        with np.errstate(divide="ignore", invalid="ignore"):
            edge = np.abs(np.log2(q) - np.round(np.log2(q))) < 2e-5
        ok = ~(act & edge)
        assert np.array_equal(st["bin"][ok], osim.bin[ok]), k
        assert np.array_equal(st["ti_end"][ok], osim.ti_end[ok]), k
        v = np.stack([st["vx"], st["vy"], st["vz"]], 1).astype(np.float64)
        v_rms = np.sqrt((osim.vel ** 2).sum(1).mean())
        assert np.max(np.abs(v - osim.vel)) < 1e-4 * v_rms, k
        assert np.max(np.abs(st["A"] / osim.A - 1)) < 1e-5, k
    assert woken_total > 0


def test_variants_forms_bitwise_identical(sim):
    """With all three variants the plain, batched and graph forms agree bit
    for bit (every sum of a particle still depends on the particle alone)."""
    ic = _ic_step(seed=59)
    params = dict(STEP_PARAMS, balsara=1, predict_inactive=1, limiter=1)
    res = {f: _run_form(sim, ic, f, 10, params) for f in ("plain", "batched", "graph")}
    ref, cref, tref = res["batched"]
    for f in ("plain", "graph"):
        st, c, t = res[f]
        assert t == tref, f
        for k in ref:
            assert np.array_equal(st[k], ref[k]), (f, k)


def test_variants_change_the_run_and_need_their_arrays(sim):
    """The variants act (a run with them differs from the base run) and a
    state without the divergence arrays is refused with SPH_ERR_ARG; the
    reverse pass refuses them."""
    L = _lib()
    ic = _ic_step(seed=61)
    a, _, _ = _run_form(sim, ic, "batched", 6, STEP_PARAMS)
    b, _, _ = _run_form(sim, ic, "batched", 6, dict(STEP_PARAMS, balsara=1, predict_inactive=1,
                                                     limiter=1))
    assert not np.array_equal(a["vx"], b["vx"])
    ctx = sim.Context(sim.Params(**STEP_PARAMS, balsara=1), ic["pos"].shape[0])
    p = sim.Particles.from_ics(ic, with_gradients=False)
    with pytest.raises(L.SphError) as e:
        ctx.build_cells(p)
    assert e.value.code == L.SPH_ERR_ARG
