"""The allocation-free cell ordering (sph_cell_order_noalloc) against the
ordering of sph_build_cells, through the C ABI.

Some callers cannot allocate device memory (all of it belongs to their own
pool, or allocation is not allowed in their loop); for them the library keeps
its sort buffers in one statically defined device array.  Two calls in a row
check that the shared array carries nothing from one call into the next.
This file is collected last on purpose: if it fails, every other test of a
run that stops at the first failure has already run.
"""
import ctypes

import numpy as np
import pytest

import sph_ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01341_gb300 import build
    build.build()
    from paper_1807_01341_gb300 import _lib, sim
    return torch, _lib, sim


def _noalloc_order(torch, L, pos, nc):
    n = pos.shape[0]
    x, y, z = (torch.as_tensor(np.ascontiguousarray(pos[:, k]), device="cuda") for k in range(3))
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = L.sph_cell_order_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(z.data_ptr()), n, 1.0, nc,
                                  ctypes.c_void_p(perm.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    # the positions are read only
    assert np.array_equal(x.cpu().numpy(), pos[:, 0])
    return rc, perm.cpu().numpy()


def _build_cells_order(sim, ic, nc):
    n = ic["pos"].shape[0]
    ctx = sim.Context(sim.Params(n_cells_override=nc), n)
    p = sim.Particles.from_ics(ic)
    ctx.build_cells(p)
    return ctx.perm_tensor(n).cpu().numpy()


def test_noalloc_order_matches_build_cells_twice(env, orc):
    """Two calls in a row (the shared array carries nothing over), each equal
    bit for bit to the FP64 oracle's stable (cell, Morton) order and to the
    order sph_build_cells produces."""
    torch, _lib, sim = env
    L = _lib.load()
    cases = [(sph_ics.clumpy_lattice(nside=24, n_clumps=3, per_clump=900, seed=41), 9),
             (sph_ics.clumpy_lattice(nside=40, n_clumps=2, per_clump=2000, seed=42), 17)]
    for ic, nc in cases:
        ic["pos"][::53, 2] -= 1.0        # outside the box: wrapped, as by the build
        rc, order = _noalloc_order(torch, L, ic["pos"], nc)
        assert rc == _lib.SPH_OK
        assert np.array_equal(order, orc.cells(ic["pos"], 1.0, nc)["perm"])
        assert np.array_equal(order, _build_cells_order(sim, ic, nc))


def test_noalloc_at_its_size_limit(env, orc):
    """Exactly 65,536 particles (the stated limit), with duplicates and ties."""
    torch, _lib, sim = env
    L = _lib.load()
    rng = np.random.default_rng(7)
    pos = rng.uniform(size=(65536, 3))
    pos[1000:1100] = pos[0]              # coincident particles: order by index
    rc, order = _noalloc_order(torch, L, pos, 31)
    assert rc == _lib.SPH_OK
    assert np.array_equal(order, orc.cells(pos, 1.0, 31)["perm"])


def test_noalloc_non_finite_input_returns(env):
    """A NaN position: the call (which does not check its input) returns
    SPH_OK and the context stays usable; the order of such input is not
    specified."""
    torch, _lib, sim = env
    L = _lib.load()
    pos = np.random.default_rng(8).uniform(size=(1000, 3))
    pos[17, 1] = np.nan
    rc, _ = _noalloc_order(torch, L, pos, 5)
    assert rc == _lib.SPH_OK
    clean = np.nan_to_num(pos, nan=0.5)
    rc, order = _noalloc_order(torch, L, clean, 5)
    assert rc == _lib.SPH_OK
    assert np.array_equal(np.sort(order), np.arange(1000))


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, _lib, sim = env
    L = _lib.load()
    pos = np.random.default_rng(0).uniform(size=(65537, 3))
    rc, order = _noalloc_order(torch, L, pos, 8)
    assert rc == _lib.SPH_ERR_ARG
    assert np.all(order == -1)          # nothing was launched
    rc, _ = _noalloc_order(torch, L, pos[:100], 256)
    assert rc == _lib.SPH_ERR_ARG
