"""Thin Python front end over the C ABI: particle arrays as torch CUDA tensors,
a context object whose methods map one-to-one onto the sph_* calls.

Only argument marshalling happens here; every computation runs in
libsph_gb300.so.  Calls are asynchronous on the current torch CUDA stream
unless the C ABI documents a synchronisation.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields

import numpy as np
import torch

from . import _lib
from ._lib import check

_TORCH = {"f8": torch.float64, "f4": torch.float32, "i1": torch.int8, "i8": torch.int64,
          "u1": torch.uint8, "i4": torch.int32}
_NP = {"f8": np.float64, "f4": np.float32, "i1": np.int8, "i8": np.int64, "u1": np.uint8,
       "i4": np.int32}


@dataclass
class Params:
    box: float = 1.0
    eta: float = 1.2348
    gamma: float = 5.0 / 3.0
    alpha_visc: float = 0.8
    cfl: float = 0.1
    h_tol: float = 1e-6
    h_max_iter: int = 30
    bin_cap: int = 20
    dt_min: float = 1e-6
    t_begin: float = 0.0
    cell_margin: float = 2.0
    leaf_max: int = 8
    threads_per_particle: int = 1
    drift_all: int = 0
    n_cells_override: int = 0
    heavy_factor: float = 2.0
    coop_max_groups: int = -1
    list_cap: int = 512
    search_margin: float = 1.02
    staging_depth: int = 1
    wait_limit: int = 0
    test_stall: int = 0
    test_bad_group: int = 0
    balsara: int = 0
    predict_inactive: int = 0
    limiter: int = 0

    def to_c(self) -> _lib.sph_params:
        p = _lib.sph_params()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_FIELD_NAMES = frozenset(name for name, _ in _lib.PARTICLE_FIELDS)


class Particles:
    """Structure-of-arrays particle state on one CUDA device (caller-owned).

    All arrays are views into one contiguous byte buffer (`storage`, each
    array 256-byte aligned), so a whole state moves between host and device
    with a single copy."""

    ALIGN = 256

    def __init__(self, n: int, device="cuda", with_counts: bool = True,
                 with_gradients: bool = True):
        self.n = int(n)
        self.device = torch.device(device)
        fields = [(name, dt) for name, dt in _lib.PARTICLE_FIELDS
                  if (with_counts or name not in ("ngb_density", "ngb_force")) and
                  (with_gradients or name not in ("div_v", "curl_v"))]
        offs, total = {}, 0
        for name, dt in fields:
            offs[name] = total
            nbytes = self.n * np.dtype(_NP[dt]).itemsize
            total += (nbytes + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        self.storage = torch.zeros(max(total, self.ALIGN), dtype=torch.uint8, device=self.device)
        for name, dt in _lib.PARTICLE_FIELDS:
            if name not in offs:
                setattr(self, name, None)
                continue
            nbytes = self.n * np.dtype(_NP[dt]).itemsize
            view = self.storage[offs[name]:offs[name] + nbytes].view(_TORCH[dt])
            setattr(self, name, view)
        self._struct = None

    @classmethod
    def from_ics(cls, ic: dict, device="cuda", with_counts: bool = True,
                 with_gradients: bool = True):
        """Initial state: positions, velocities, masses, u (held in A until the
        first density pass converts it), h guess; every particle on bin 0 at
        tick 0."""
        n = ic["pos"].shape[0]
        p = cls(n, device, with_counts, with_gradients)
        pos = torch.as_tensor(np.ascontiguousarray(ic["pos"]), dtype=torch.float64)
        vel = torch.as_tensor(np.ascontiguousarray(ic["vel"]), dtype=torch.float32)
        p.x.copy_(pos[:, 0]); p.y.copy_(pos[:, 1]); p.z.copy_(pos[:, 2])
        p.vx.copy_(vel[:, 0]); p.vy.copy_(vel[:, 1]); p.vz.copy_(vel[:, 2])
        p.m.copy_(torch.as_tensor(ic["m"], dtype=torch.float32))
        p.A.copy_(torch.as_tensor(ic["u"], dtype=torch.float32))
        p.h.copy_(torch.as_tensor(ic["h0"], dtype=torch.float32))
        return p

    def __setattr__(self, name, value):
        # a replaced array (or count) invalidates the cached C structure
        if name == "n" or name in _FIELD_NAMES:
            self.__dict__["_struct"] = None
        super().__setattr__(name, value)

    def struct(self) -> _lib.sph_particles:
        """The sph_particles of this state (built once; rebuilt after an array
        is replaced), so a step's submission does not rebuild it."""
        s = self.__dict__.get("_struct")
        if s is None:
            s = _lib.sph_particles()
            s.n = self.n
            for name, _ in _lib.PARTICLE_FIELDS:
                t = getattr(self, name)
                setattr(s, name, None if t is None else t.data_ptr())
            self.__dict__["_struct"] = s
        return s

    def numpy(self, perm=None) -> dict:
        """Host copy of every array; with perm (int array), in the order of the
        first build (out[perm[k]] = state[k])."""
        out = {}
        for name, dt in _lib.PARTICLE_FIELDS:
            t = getattr(self, name)
            if t is None:
                continue
            a = t.cpu().numpy()
            if perm is not None:
                b = np.empty_like(a)
                b[perm] = a
                a = b
            out[name] = a
        return out

    def arrays(self):
        return {name: getattr(self, name) for name, _ in _lib.PARTICLE_FIELDS
                if getattr(self, name) is not None}


class Adjoint:
    """Adjoint of a particle state: FP64 device arrays d loss / d field."""

    def __init__(self, n: int, device="cuda"):
        self.n = int(n)
        for name in _lib.ADJOINT_FIELDS:
            setattr(self, name, torch.zeros(self.n, dtype=torch.float64, device=device))

    def struct(self) -> _lib.sph_adjoint:
        s = _lib.sph_adjoint()
        s.n = self.n
        for name in _lib.ADJOINT_FIELDS:
            setattr(s, name, getattr(self, name).data_ptr())
        self._struct = s
        return s

    def zero_(self):
        for name in _lib.ADJOINT_FIELDS:
            getattr(self, name).zero_()
        return self


class _DevArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


class Context:
    """An sph_ctx: scratch for up to n_max particles on the current device."""

    def __init__(self, params: Params, n_max: int):
        self.L = _lib.load()
        self.params = params
        self._cp = params.to_c()
        h = ctypes.c_void_p()
        check(self.L.sph_create(ctypes.byref(self._cp), int(n_max), ctypes.byref(h)), "sph_create")
        self.h = h

    def close(self):
        if self.h:
            self.L.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the C ABI, one method per call ------------------------------------
    def build_cells(self, p: Particles, stream=None):
        check(self.L.sph_build_cells(self.h, ctypes.byref(p.struct()), _stream_ptr(stream)),
              "sph_build_cells")

    def perm_tensor(self, n: int) -> torch.Tensor:
        ptr = self.L.sph_perm(self.h)
        if not ptr:
            raise RuntimeError("cells not built")
        return torch.as_tensor(_DevArray(ptr, n, "<i4"), device="cuda").clone()

    def grid_info(self):
        nc, nl = ctypes.c_int(), ctypes.c_int()
        check(self.L.sph_grid_info(self.h, ctypes.byref(nc), ctypes.byref(nl)), "sph_grid_info")
        return nc.value, nl.value

    def mark_active(self, p: Particles, ti: int = -1, stream=None):
        check(self.L.sph_mark_active(self.h, ctypes.byref(p.struct()), int(ti),
                                     _stream_ptr(stream)), "sph_mark_active")

    def kick_drift(self, p: Particles, phase: int, stream=None):
        check(self.L.sph_kick_drift(self.h, ctypes.byref(p.struct()), int(phase),
                                    _stream_ptr(stream)), "sph_kick_drift")

    def density_active(self, p: Particles, flags: int = 0, stream=None):
        check(self.L.sph_density_active(self.h, ctypes.byref(p.struct()), int(flags),
                                        _stream_ptr(stream)), "sph_density_active")

    def force_active(self, p: Particles, stream=None):
        check(self.L.sph_force_active(self.h, ctypes.byref(p.struct()), _stream_ptr(stream)),
              "sph_force_active")

    def timestep_bins(self, p: Particles, ti_next_dev: torch.Tensor | None = None, stream=None):
        ptr = None if ti_next_dev is None else ctypes.c_void_p(ti_next_dev.data_ptr())
        check(self.L.sph_timestep_bins(self.h, ctypes.byref(p.struct()), ptr,
                                       _stream_ptr(stream)), "sph_timestep_bins")

    def begin_run(self, stream=None):
        check(self.L.sph_begin_run(self.h, _stream_ptr(stream)), "sph_begin_run")

    def step_async(self, p: Particles, form: int = _lib.SPH_FORM_BATCHED, stream=None):
        check(self.L.sph_step_async(self.h, ctypes.byref(p.struct()), int(form),
                                    _stream_ptr(stream)), "sph_step_async")

    def step_sync(self, p: Particles, stream=None) -> int:
        c = ctypes.c_int()
        check(self.L.sph_step_sync(self.h, ctypes.byref(p.struct()), ctypes.byref(c),
                                   _stream_ptr(stream)), "sph_step_sync")
        return c.value

    def step(self, p: Particles, form: int = _lib.SPH_FORM_BATCHED, stream=None):
        check(self.L.sph_step(self.h, ctypes.byref(p.struct()), int(form), _stream_ptr(stream)),
              "sph_step")

    def step_graph(self, p: Particles, n_steps: int, stream=None):
        check(self.L.sph_step_graph(self.h, ctypes.byref(p.struct()), int(n_steps),
                                    _stream_ptr(stream)), "sph_step_graph")

    def get_time(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        check(self.L.sph_get_time(self.h, ctypes.byref(a), ctypes.byref(b)), "sph_get_time")
        return a.value, b.value

    def set_time(self, ti: int, stream=None):
        check(self.L.sph_set_time(self.h, int(ti), _stream_ptr(stream)), "sph_set_time")

    def bin_counts(self, n_bins: int = 64, stream=None) -> list:
        """Particles per time bin (Eq. 2) as of the last step or cell build."""
        out = (ctypes.c_int64 * n_bins)()
        check(self.L.sph_get_bin_counts(self.h, out, int(n_bins), _stream_ptr(stream)),
              "sph_get_bin_counts")
        return list(out)

    def diagnostics(self, p: Particles, ti: int = -1, stream=None) -> dict:
        """FP64 kinetic and thermal energy, momentum and mass of the state at
        tick ti (default: the current tick); see sph_diagnostics."""
        out = (ctypes.c_double * 8)()
        check(self.L.sph_diagnostics(self.h, ctypes.byref(p.struct()), int(ti), out,
                                     _stream_ptr(stream)), "sph_diagnostics")
        return {"E_kin": out[0], "E_therm": out[1], "E": out[0] + out[1],
                "momentum": (out[2], out[3], out[4]), "mass": out[5],
                "no_density": int(out[6])}

    def status(self):
        s, d = ctypes.c_int(), ctypes.c_int64()
        check(self.L.sph_get_status(self.h, ctypes.byref(s), ctypes.byref(d)), "sph_get_status")
        return s.value, d.value

    def clear_status(self, stream=None):
        check(self.L.sph_clear_status(self.h, _stream_ptr(stream)), "sph_clear_status")

    def check_report(self):
        """(site, index, bound) of the first failed device bounds check since the
        status was last cleared (site 0: none; always 0 without SPH_CHECKS)."""
        site, idx, bound = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        check(self.L.sph_get_check_report(self.h, ctypes.byref(site), ctypes.byref(idx),
                                          ctypes.byref(bound)), "sph_get_check_report")
        return site.value, idx.value, bound.value

    def counters(self) -> dict:
        c = _lib.sph_counters()
        check(self.L.sph_get_counters(self.h, ctypes.byref(c)), "sph_get_counters")
        return {k: getattr(c, k) for k, _ in c._fields_}

    def set_profiling(self, enable: bool = True):
        check(self.L.sph_set_profiling(self.h, int(bool(enable))), "sph_set_profiling")

    def kernel_times(self) -> dict:
        t = _lib.sph_kernel_times()
        check(self.L.sph_get_kernel_times(self.h, ctypes.byref(t)), "sph_get_kernel_times")
        return {k: getattr(t, k) for k, _ in t._fields_}

    def reset_kernel_times(self):
        check(self.L.sph_reset_kernel_times(self.h), "sph_reset_kernel_times")

    # -- checkpoints and the reverse pass -----------------------------------
    def state_copy(self, src: Particles, dst: Particles, to_input_order: bool, stream=None):
        check(self.L.sph_state_copy(self.h, ctypes.byref(src.struct()), ctypes.byref(dst.struct()),
                                    int(bool(to_input_order)), _stream_ptr(stream)),
              "sph_state_copy")

    def resume(self, p: Particles, ti: int, first: bool, stream=None):
        check(self.L.sph_resume(self.h, ctypes.byref(p.struct()), int(ti), int(bool(first)),
                                _stream_ptr(stream)), "sph_resume")

    def grid_density(self, p: Particles, n_grid: int, ti: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(n_grid ** 3, dtype=torch.float64, device=p.device)
        check(self.L.sph_grid_density(self.h, ctypes.byref(p.struct()), int(n_grid), int(ti),
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
              "sph_grid_density")
        return out

    def grid_density_bwd(self, p: Particles, n_grid: int, ti: int, rho_bar: torch.Tensor,
                         adj: Adjoint, stream=None):
        rho_bar = rho_bar.contiguous()
        check(self.L.sph_grid_density_bwd(self.h, ctypes.byref(p.struct()), int(n_grid), int(ti),
                                          ctypes.c_void_p(rho_bar.data_ptr()),
                                          ctypes.byref(adj.struct()), _stream_ptr(stream)),
              "sph_grid_density_bwd")

    def step_bwd(self, pre: Particles, post: Particles, ti: int, first: bool, adj: Adjoint,
                 stream=None):
        check(self.L.sph_step_bwd(self.h, ctypes.byref(pre.struct()), ctypes.byref(post.struct()),
                                  int(ti), int(bool(first)), ctypes.byref(adj.struct()),
                                  _stream_ptr(stream)), "sph_step_bwd")

    def reset_counters(self, stream=None):
        check(self.L.sph_reset_counters(self.h, _stream_ptr(stream)), "sph_reset_counters")
