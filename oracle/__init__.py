"""FP64 CPU oracle of the SWIFT SPH hot path (arXiv 1807.01341).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product library never imports this
package, and this package imports nothing from the product.

The arithmetic lives in ``sph_oracle.c`` (compiled here with gcc, FP64,
``-ffp-contract=off``); this module marshals numpy arrays into it and holds the
few elementwise formulas (grad-h factor, equation of state, kick, drift) that
read more plainly in numpy, plus the kick-drift-kick driver with individual
power-of-two time bins (Sec. II-A, Eq. 2).

Readings of the paper used here (it defers the SPH equations to "a standard SPH
scheme" and prints only Eq. 1 and Eq. 2):
  * kernel: cubic spline, support H = 1.825742 h; eta = 1.2348 gives ~48
    neighbours;
  * h solves h^3 n(h) = eta^3 with n = sum_j W (number density);
  * grad-h factor f = [1 + h/(3 rho) d rho/dh]^-1 (Springel & Hernquist 2002);
  * entropy A = (gamma-1) u / rho^(gamma-1), P = A rho^gamma, c = sqrt(gamma P/rho);
  * Monaghan signal-velocity viscosity with beta = 3 (the form inside Eq. 1),
    alpha = 0.8, no Balsara switch in the base scheme;
  * dt = C h / v_sig (Eq. 1); bin n = floor(log2(dt / dt_min)) (Eq. 2),
    increases synchronised to multiples of the new step; a particle is active
    when its step ends at the current integer time.
Variants of the scheme (off by default; Gadget-2, the paper's reference code,
uses all three): velocity divergence and curl from the density loop, the
Gadget-2 prediction of inactive particles' density and smoothing length from
their divergence, the Balsara switch on the viscosity, and the Saitoh & Makino
(2009) limit of a time step to four times its neighbours' smallest one, with
the waking of inactive neighbours on much longer steps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA_K = 1.825742


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no fused multiply-add, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i64, i32, u8, vp = (ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_uint8, ctypes.c_void_p)
            L.orc_kernel_w.restype = d
            L.orc_kernel_w.argtypes = [d]
            L.orc_kernel_dw.restype = d
            L.orc_kernel_dw.argtypes = [d]
            L.orc_gamma_k.restype = d
            L.orc_density_fixed_h.restype = None
            L.orc_density_fixed_h.argtypes = [i64, vp, vp, vp, vp, vp, vp, d, i32,
                                              vp, vp, vp, vp, vp]
            L.orc_density.restype = i64
            L.orc_density.argtypes = [i64, vp, vp, vp, vp, vp, vp, d, d, d, i32, i32,
                                      vp, vp, vp, vp, vp, vp]
            L.orc_force.restype = None
            L.orc_force.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                    vp, vp, d, d, d, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                    vp]
            L.orc_gradient.restype = None
            L.orc_gradient.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, i32,
                                       vp, vp, vp, vp]
            L.orc_balsara.restype = d
            L.orc_balsara.argtypes = [d, d, d, d]
            L.orc_bin_of_dt.restype = i32
            L.orc_bin_of_dt.argtypes = [d, d, i32]
            L.orc_timestep_bins.restype = i64
            L.orc_timestep_bins.argtypes = [i64, vp, vp, vp, d, d, i32, i64, vp, vp, vp, vp,
                                            vp]
            L.orc_wake_bins.restype = None
            L.orc_wake_bins.argtypes = [i64, vp, vp, vp, vp, vp, vp, d, i32, vp]
            L.orc_cells.restype = None
            L.orc_cells.argtypes = [i64, vp, vp, vp, d, i32, vp, vp, vp]
            L.orc_num_threads.restype = i32
            L.orc_set_num_threads.argtypes = [i32]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _mask(active, n):
    if active is None:
        return None
    a = np.ascontiguousarray(active, dtype=np.uint8)
    assert a.shape == (n,)
    return a


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


# --------------------------------------------------------------------------
# Kernel
# --------------------------------------------------------------------------

def kernel_w(q):
    """Dimensionless cubic spline w(q), W(r,h) = H^-3 w(r/H)."""
    L = lib()
    return np.array([L.orc_kernel_w(float(v)) for v in np.atleast_1d(q)])


def kernel_dw(q):
    """dw/dq of the cubic spline."""
    L = lib()
    return np.array([L.orc_kernel_dw(float(v)) for v in np.atleast_1d(q)])


# --------------------------------------------------------------------------
# Density loop and smoothing-length solve (the density and ghost tasks)
# --------------------------------------------------------------------------

def density_fixed_h(pos, m, h, active=None, box=1.0, use_cells=True):
    """Density sums at the given h: returns dict(rho, drho_dh, wn, dwn_dh, count)."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    n = x.shape[0]
    m, h = _f64(m), _f64(h)
    act = _mask(active, n)
    out = {k: np.zeros(n) for k in ("rho", "drho_dh", "wn", "dwn_dh")}
    cnt = np.zeros(n, dtype=np.int64)
    lib().orc_density_fixed_h(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), _ptr(act),
                              box, int(use_cells), _ptr(out["rho"]), _ptr(out["drho_dh"]),
                              _ptr(out["wn"]), _ptr(out["dwn_dh"]), _ptr(cnt))
    out["count"] = cnt
    return out


def density(pos, m, h0, active=None, box=1.0, eta=1.2348, tol=1e-12, max_iter=100,
            use_cells=True):
    """Density with the smoothing-length iteration for the active particles.

    Returns dict(h, rho, drho_dh, wn, dwn_dh, count, iters, n_unconverged); h of
    inactive particles is returned unchanged."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    n = x.shape[0]
    m = _f64(m)
    h = _f64(h0).copy()
    act = _mask(active, n)
    out = {k: np.zeros(n) for k in ("rho", "drho_dh", "wn", "dwn_dh")}
    cnt = np.zeros(n, dtype=np.int64)
    iters = np.zeros(n, dtype=np.int32)
    bad = lib().orc_density(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h), _ptr(act), box,
                            eta, tol, max_iter, int(use_cells), _ptr(out["rho"]),
                            _ptr(out["drho_dh"]), _ptr(out["wn"]), _ptr(out["dwn_dh"]),
                            _ptr(cnt), _ptr(iters))
    out.update(h=h, count=cnt, iters=iters, n_unconverged=int(bad))
    return out


def gradh_f(h, rho, drho_dh):
    """Grad-h factor f = [1 + h/(3 rho) d rho/dh]^-1 (Springel & Hernquist 2002)."""
    return 1.0 / (1.0 + h / (3.0 * rho) * drho_dh)


def entropy_from_u(u, rho, gamma):
    """Entropic function A = (gamma - 1) u / rho^(gamma - 1)."""
    return (gamma - 1.0) * u / rho ** (gamma - 1.0)


def u_from_entropy(A, rho, gamma):
    return A * rho ** (gamma - 1.0) / (gamma - 1.0)


def eos(A, rho, gamma):
    """Pressure P = A rho^gamma and sound speed c = sqrt(gamma P / rho)."""
    P = A * rho ** gamma
    return P, np.sqrt(gamma * P / rho)


# --------------------------------------------------------------------------
# Force loop
# --------------------------------------------------------------------------

def force(pos, vel, m, h, rho, f, P, c, active=None, box=1.0, alpha=0.8, gamma=5.0 / 3.0,
          use_cells=True, balsara=None, bins=None):
    """Hydro accelerations for the active particles: dict(a[n,3], Adot, vsig,
    count, bin_ngb_min).  balsara (optional): each particle's Balsara factor,
    the viscosity of a pair scaled by their mean; bins (optional): time bins,
    whose smallest over each particle's neighbours is returned."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    vx, vy, vz = (_f64(vel[:, k]) for k in range(3))
    n = x.shape[0]
    arrs = [_f64(a) for a in (m, h, rho, f, P, c)]
    act = _mask(active, n)
    ax, ay, az, Adot, vsig = (np.zeros(n) for _ in range(5))
    cnt = np.zeros(n, dtype=np.int64)
    bal = None if balsara is None else _f64(balsara)
    b8 = None if bins is None else np.ascontiguousarray(bins, dtype=np.int8)
    bmin = np.zeros(n, dtype=np.int8)
    lib().orc_force(n, _ptr(x), _ptr(y), _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz),
                    *[_ptr(a) for a in arrs], _ptr(act), box, alpha, gamma, int(use_cells),
                    _ptr(bal) if bal is not None else None,
                    _ptr(b8) if b8 is not None else None,
                    _ptr(ax), _ptr(ay), _ptr(az), _ptr(Adot), _ptr(vsig), _ptr(cnt),
                    _ptr(bmin))
    return dict(a=np.stack([ax, ay, az], axis=1), Adot=Adot, vsig=vsig, count=cnt,
                bin_ngb_min=bmin if b8 is not None else None)


def gradient(pos, vel, m, h, rho, active=None, box=1.0, use_cells=True):
    """Velocity divergence and curl at each active particle's h:
    dict(div[n], curl[n, 3])."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    vx, vy, vz = (_f64(vel[:, k]) for k in range(3))
    n = x.shape[0]
    m, h, rho = _f64(m), _f64(h), _f64(rho)
    act = _mask(active, n)
    dv, cx, cy, cz = (np.zeros(n) for _ in range(4))
    lib().orc_gradient(n, _ptr(x), _ptr(y), _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(m),
                       _ptr(h), _ptr(rho), _ptr(act), box, int(use_cells), _ptr(dv),
                       _ptr(cx), _ptr(cy), _ptr(cz))
    return dict(div=dv, curl=np.stack([cx, cy, cz], axis=1))


def balsara(divv, curl, c, h):
    """Balsara factor |div v| / (|div v| + |curl v| + 1e-4 c / h) (per particle)."""
    f = lib().orc_balsara
    return np.array([f(float(a), float(b), float(cc), float(hh))
                     for a, b, cc, hh in zip(np.ravel(divv), np.ravel(curl), np.ravel(c),
                                             np.ravel(h))])


def predict_inactive(rho, h, divv, dt):
    """Gadget-2 prediction of an inactive particle's density and smoothing
    length over the time dt since its last density evaluation:
    rho exp(-div v dt), h exp(div v dt / 3)."""
    rho, h, divv, dt = (np.asarray(a, dtype=np.float64) for a in (rho, h, divv, dt))
    return rho * np.exp(-divv * dt), h * np.exp(divv * dt / 3.0)


# --------------------------------------------------------------------------
# Time-step (Eq. 1) and bins (Eq. 2)
# --------------------------------------------------------------------------

def bin_of_dt(dt, dt_min, bin_cap):
    """floor(log2(dt / dt_min)) capped at bin_cap; -1 when dt < dt_min."""
    return int(lib().orc_bin_of_dt(float(dt), float(dt_min), int(bin_cap)))


def timestep_bins(h, vsig, active, cfl, dt_min, bin_cap, ti_current, bin_old,
                  bin_ngb_min=None):
    """New bins for active particles: dict(bin, ti_begin, ti_end, dt, n_too_small).

    bin_old, and ti_begin / ti_end of the inactive particles, are left as given
    (the returned ti arrays are zero for inactive particles).  bin_ngb_min
    (optional): each particle's smallest neighbour bin; a new bin is then at
    most 2 above it (the Saitoh & Makino limiter)."""
    h, vsig = _f64(h), _f64(vsig)
    n = h.shape[0]
    act = _mask(active, n)
    b = np.ascontiguousarray(bin_old, dtype=np.int8).copy()
    tb = np.zeros(n, dtype=np.int64)
    te = np.zeros(n, dtype=np.int64)
    dt = np.zeros(n)
    lim = None if bin_ngb_min is None else np.ascontiguousarray(bin_ngb_min, dtype=np.int8)
    bad = lib().orc_timestep_bins(n, _ptr(h), _ptr(vsig), _ptr(act), cfl, dt_min, bin_cap,
                                  int(ti_current), _ptr(lim) if lim is not None else None,
                                  _ptr(b), _ptr(tb), _ptr(te), _ptr(dt))
    return dict(bin=b, ti_begin=tb, ti_end=te, dt=dt, n_too_small=int(bad))


def wake_bins(pos, h, active, bins, box=1.0, use_cells=True):
    """Saitoh & Makino's waking of inactive neighbours: for each inactive
    particle j, the smallest bin_i + 2 over the active particles i whose
    force-loop pair with j (r < max(H_i, H_j)) has bin_j > bin_i + 2, else 127."""
    x, y, z = (_f64(pos[:, k]) for k in range(3))
    n = x.shape[0]
    act = _mask(active, n)
    b8 = np.ascontiguousarray(bins, dtype=np.int8)
    req = np.zeros(n, dtype=np.int8)
    lib().orc_wake_bins(n, _ptr(x), _ptr(y), _ptr(z), _ptr(_f64(h)), _ptr(act), _ptr(b8), box,
                        int(use_cells), _ptr(req))
    return req


def wake(ti, req, active, bins, ti_begin, ti_end, vel, A, acc, Adot, dt_min):
    """Wakes the inactive particles with req < bin at tick ti (in place): the
    step of such a particle j now ends at the first multiple of 2^req_j after
    ti (when that comes before its old end), its bin becomes req_j, and the
    opening half-kick of its step is cut to the shortened step:
    v -= a (D_old - D_new) / 2, A -= Adot (D_old - D_new) / 2 (D in ticks of
    dt_min).  Returns the number of particles woken."""
    woken = 0
    for j in np.nonzero((~np.asarray(active, bool)) & (req < bins))[0]:
        bw = int(req[j])
        step = 1 << bw
        tw = (int(ti) // step + 1) * step
        if tw >= ti_end[j]:
            continue
        corr = 0.5 * float(ti_end[j] - tw) * dt_min   # (D_old - D_new) / 2
        vel[j] -= acc[j] * corr
        A[j] -= Adot[j] * corr
        ti_end[j] = tw
        bins[j] = bw
        woken += 1
    return woken


# --------------------------------------------------------------------------
# Cells
# --------------------------------------------------------------------------

def cells(pos, box, n_cells):
    """Wrapped positions, cell index, (cell, Morton) key and stable order.

    Returns dict(pos (wrapped copy), cell, key, perm) with perm[k] = original
    index of the k-th particle in (key, index) order."""
    x, y, z = (_f64(pos[:, k]).copy() for k in range(3))
    n = x.shape[0]
    cell = np.zeros(n, dtype=np.int64)
    key = np.zeros(n, dtype=np.uint64)
    perm = np.zeros(n, dtype=np.int64)
    lib().orc_cells(n, _ptr(x), _ptr(y), _ptr(z), float(box), int(n_cells), _ptr(cell),
                    _ptr(key), _ptr(perm))
    return dict(pos=np.stack([x, y, z], axis=1), cell=cell, key=key, perm=perm)


def n_cells_for(hmax, box=1.0, margin=1.0, nc_max=1024):
    """Top-level grid size: the largest n_c with box / n_c >= margin * H_max, n_c >= 3."""
    import math
    nc = int(math.floor(box / (margin * (GAMMA_K * float(hmax)))))
    return max(3, min(nc, nc_max))


from .kdk import OracleSim  # noqa: E402  (driver built on the functions above)
