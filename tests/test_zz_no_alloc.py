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


def test_noalloc_order_matches_build_cells_twice(env):
    torch, _lib, sim = env
    L = _lib.load()
    cases = [(sph_ics.clumpy_lattice(nside=24, n_clumps=3, per_clump=900, seed=41), 9),
             (sph_ics.clumpy_lattice(nside=40, n_clumps=2, per_clump=2000, seed=42), 17)]
    for ic, nc in cases:
        ic["pos"][::53, 2] -= 1.0        # outside the box: wrapped, as by the build
        rc, order = _noalloc_order(torch, L, ic["pos"], nc)
        assert rc == _lib.SPH_OK
        ref = _build_cells_order(sim, ic, nc)
        assert np.array_equal(order, ref)


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, _lib, sim = env
    L = _lib.load()
    pos = np.random.default_rng(0).uniform(size=(65537, 3))
    rc, order = _noalloc_order(torch, L, pos, 8)
    assert rc == _lib.SPH_ERR_ARG
    assert np.all(order == -1)          # nothing was launched
    rc, _ = _noalloc_order(torch, L, pos[:100], 256)
    assert rc == _lib.SPH_ERR_ARG
