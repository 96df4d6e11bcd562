"""FP64 diagnostics of the GPU state (sph_diagnostics): total energy and
momentum, against the oracle integrator's synchronised energy and against
momentum conservation."""
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


def _ic(seed=3, nside=10):
    ic = sph_ics.lattice(nside, 0.2, seed=seed)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(seed)
    ic["vel"] = rng.normal(scale=0.3, size=(n, 3))
    ic["u"] = rng.uniform(0.5, 1.5, n)
    return ic


def test_energy_matches_oracle_at_sync_points(sim, orc):
    """One global time step (every particle active every step): after each
    step the GPU's energy at the step's tick is the synchronised energy, equal
    to the oracle's E_sync of the same run within 1e-5 relative (kinetic and
    thermal parts alike); the momentum stays at its initial value (pairwise
    antisymmetric forces) to 1e-6 of sum m|v|."""
    ic = _ic()
    n = ic["pos"].shape[0]
    kw = dict(cfl=0.1, dt_min=1e-3)
    ctx, p = gpu_setup(ic, sim.Params(**kw, bin_cap=0))
    osim = orc.OracleSim(ic["pos"], ic["vel"], ic["m"], ic["u"], ic["h0"], bin_cap=0,
                         global_step=True, **kw)
    m = np.broadcast_to(np.asarray(ic["m"], dtype=np.float64), (n,))
    p0 = (m[:, None] * ic["vel"]).sum(0)
    L = _lib()
    for k in range(6):
        ctx.step(p, L.SPH_FORM_BATCHED)
        assert ctx.status()[0] == 0
        osim.step()
        d = ctx.diagnostics(p)
        assert d["no_density"] == 0
        assert abs(d["mass"] / m.sum() - 1.0) < 1e-6
        E_ref = osim.E_sync[-1]
        assert abs(d["E"] / E_ref - 1.0) < 1e-5, (k, d["E"], E_ref)
        v_ref = osim.vel - osim.acc * (0.5 * kw["dt_min"])  # back to the step's tick
        ek_ref = float((0.5 * m * (v_ref ** 2).sum(1)).sum())
        assert abs(d["E_kin"] / ek_ref - 1.0) < 1e-5, (k, d["E_kin"], ek_ref)
        st = p.numpy()
        scale = float((np.asarray(st["m"], np.float64) *
                       np.sqrt(np.asarray(st["vx"], np.float64) ** 2 +
                               np.asarray(st["vy"], np.float64) ** 2 +
                               np.asarray(st["vz"], np.float64) ** 2)).sum())
        assert np.abs(np.array(d["momentum"]) - p0).max() < 1e-6 * scale
    ctx.close()


def test_diagnostics_of_mixed_bins_state(sim):
    """With individual bins the diagnostics predict each particle's velocity
    and entropy to the tick from its half-step state: equal to the FP64 sum of
    that prediction over the GPU's own arrays (1e-12 relative), the same bits
    on a second call, and zero thermal terms missing after the first step."""
    ic = sph_ics.clumpy_lattice(nside=10, n_clumps=1, per_clump=150, seed=21)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(21)
    ic["vel"] = rng.normal(scale=0.1, size=(n, 3))
    params = sim.Params(cfl=0.1, dt_min=1e-6, bin_cap=14)
    ctx, p = gpu_setup(ic, params)
    L = _lib()
    for _ in range(4):
        ctx.step(p, L.SPH_FORM_BATCHED)
    assert ctx.status()[0] == 0
    ti = ctx.get_time()[0]
    st = {k: np.asarray(v) for k, v in p.numpy().items()}
    assert len(np.unique(st["bin"])) > 1  # the state really has several bins
    d1 = ctx.diagnostics(p)
    d2 = ctx.diagnostics(p, ti)
    assert d1 == d2
    f = lambda k: st[k].astype(np.float64)
    b = st["bin"].astype(np.int64)
    dtp = ((ti - st["ti_begin"]).astype(np.float64) - 0.5 * np.left_shift(1, b)) * params.dt_min
    v2 = sum((f(c) + f(a) * dtp) ** 2 for c, a in (("vx", "ax"), ("vy", "ay"), ("vz", "az")))
    g = params.gamma
    A = f("A") + f("Adot") * dtp
    ek = (0.5 * f("m") * v2).sum()
    et = (f("m") * A * f("rho") ** (g - 1.0) / (g - 1.0)).sum()
    assert abs(d1["E_kin"] / ek - 1.0) < 1e-12
    assert abs(d1["E_therm"] / et - 1.0) < 1e-12
    assert d1["no_density"] == 0
    # another tick: a different prediction of the same state
    d3 = ctx.diagnostics(p, ti + 8)
    assert d3["E_kin"] != d1["E_kin"]
    ctx.close()


def test_diagnostics_empty_and_args(sim):
    """No particles: all sums zero.  A missing output pointer: SPH_ERR_ARG."""
    import ctypes
    from paper_1807_01341_gb300 import _lib as L
    ctx = sim.Context(sim.Params(), 16)
    p = sim.Particles(0)
    d = ctx.diagnostics(p, 0)
    assert d["E"] == 0.0 and d["mass"] == 0.0 and d["momentum"] == (0.0, 0.0, 0.0)
    rc = ctx.L.sph_diagnostics(ctx.h, ctypes.byref(p.struct()), 0, None, None)
    assert rc == L.SPH_ERR_ARG
    ctx.close()
