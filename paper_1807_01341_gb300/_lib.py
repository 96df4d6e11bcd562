"""ctypes binding of libsph_gb300.so (include/sph.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  PyTorch provides the device memory (tensors) and the stream.
Loading fails loudly when the library has not been built: there is no CPU
fallback.  With SPH_GB300_CHECKS=1 in the environment the process loads the
build with device bounds checks (libsph_gb300_checks.so) instead.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsph_gb300.so")
CHECKS_LIB_PATH = os.path.join(HERE, "_build", "libsph_gb300_checks.so")

# status codes (include/sph.h)
SPH_OK = 0
SPH_ERR_ARG = 1
SPH_ERR_CUDA = 2
SPH_ERR_H_NOCONV = 3
SPH_ERR_CELL_OVERFLOW = 4
SPH_ERR_DT_TOO_SMALL = 5
SPH_ERR_TIMEOUT = 6
SPH_ERR_NOMEM = 7
SPH_ERR_NOT_BUILT = 8
SPH_ERR_BOUNDS = 9

# sites of the device bounds checks (sph_check_site)
SPH_CHECK_NONE, SPH_CHECK_GROUP, SPH_CHECK_GROUP_LEAVES, SPH_CHECK_GROUP_SIZE = 0, 1, 2, 3
SPH_CHECK_CELL_LEAVES, SPH_CHECK_LEAF, SPH_CHECK_PARTICLE_LEAF = 4, 5, 6
SPH_CHECK_DRIFT_CHUNK, SPH_CHECK_ACTIVE_LEAF, SPH_CHECK_SCATTER = 7, 8, 9
SPH_CHECK_WAKE = 10

SPH_DRIFT, SPH_KICK_CLOSE, SPH_KICK_OPEN = 0, 1, 2
SPH_DENSITY_INIT_ENTROPY = 1
SPH_FORM_PLAIN, SPH_FORM_BATCHED, SPH_FORM_BATCHED_NOGRAPH = 0, 1, 2

_d, _i, _i64, _vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p


class sph_params(ctypes.Structure):
    _fields_ = [("box", _d), ("eta", _d), ("gamma", _d), ("alpha_visc", _d), ("cfl", _d),
                ("h_tol", _d), ("h_max_iter", _i), ("bin_cap", _i), ("dt_min", _d),
                ("t_begin", _d), ("cell_margin", _d), ("leaf_max", _i),
                ("threads_per_particle", _i), ("drift_all", _i), ("n_cells_override", _i),
                ("heavy_factor", _d), ("coop_max_groups", _i), ("list_cap", _i),
                ("search_margin", _d), ("staging_depth", _i), ("wait_limit", _i),
                ("test_stall", _i), ("test_bad_group", _i), ("balsara", _i),
                ("predict_inactive", _i), ("limiter", _i)]


PARTICLE_FIELDS = [("x", "f8"), ("y", "f8"), ("z", "f8"), ("vx", "f4"), ("vy", "f4"),
                   ("vz", "f4"), ("ax", "f4"), ("ay", "f4"), ("az", "f4"), ("A", "f4"),
                   ("Adot", "f4"), ("h", "f4"), ("rho", "f4"), ("f", "f4"), ("P", "f4"),
                   ("c", "f4"), ("vsig", "f4"), ("m", "f4"), ("bin", "i1"), ("ti_begin", "i8"),
                   ("ti_end", "i8"), ("ti_drift", "i8"), ("active", "u1"),
                   ("ngb_density", "i4"), ("ngb_force", "i4"), ("div_v", "f4"),
                   ("curl_v", "f4")]


class sph_particles(ctypes.Structure):
    _fields_ = [("n", _i64)] + [(name, _vp) for name, _ in PARTICLE_FIELDS]


ADJOINT_FIELDS = ["x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "A", "Adot", "h", "rho", "f"]


class sph_adjoint(ctypes.Structure):
    _fields_ = [("n", _i64)] + [(name, _vp) for name in ADJOINT_FIELDS]


class sph_counters(ctypes.Structure):
    _fields_ = [(k, _i64) for k in ("pairs_density", "pairs_force", "cand_density", "cand_force",
                                    "iters_density", "active_particles", "steps", "rebuilds",
                                    "redone_steps", "kernel_launches", "gathers_density",
                                    "list_overflows", "evals_density", "wakes")]


class sph_kernel_times(ctypes.Structure):
    _fields_ = [("density_ms", _d), ("force_ms", _d), ("density_launches", _i64),
                ("force_launches", _i64)]


_lib = None


def load(path: str = None):
    """Load the library (it must have been built: paper_1807_01341_gb300.build);
    the build with device bounds checks when SPH_GB300_CHECKS=1."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = CHECKS_LIB_PATH if os.environ.get("SPH_GB300_CHECKS") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run "
                           "`python -m paper_1807_01341_gb300.build` -- there is no CPU fallback")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.sph_default_params.argtypes = [P(sph_params)]
    L.sph_default_params.restype = None
    L.sph_create.argtypes = [P(sph_params), _i64, P(_vp)]
    L.sph_destroy.argtypes = [_vp]
    L.sph_build_cells.argtypes = [_vp, P(sph_particles), _vp]
    L.sph_perm.argtypes = [_vp]
    L.sph_perm.restype = _vp
    L.sph_grid_info.argtypes = [_vp, P(_i), P(_i)]
    L.sph_mark_active.argtypes = [_vp, P(sph_particles), _i64, _vp]
    L.sph_kick_drift.argtypes = [_vp, P(sph_particles), _i, _vp]
    L.sph_density_active.argtypes = [_vp, P(sph_particles), _i, _vp]
    L.sph_force_active.argtypes = [_vp, P(sph_particles), _vp]
    L.sph_timestep_bins.argtypes = [_vp, P(sph_particles), _vp, _vp]
    L.sph_begin_run.argtypes = [_vp, _vp]
    L.sph_step_async.argtypes = [_vp, P(sph_particles), _i, _vp]
    L.sph_step_sync.argtypes = [_vp, P(sph_particles), P(_i), _vp]
    L.sph_step.argtypes = [_vp, P(sph_particles), _i, _vp]
    L.sph_step_graph.argtypes = [_vp, P(sph_particles), _i, _vp]
    L.sph_get_time.argtypes = [_vp, P(_i64), P(_i64)]
    L.sph_set_time.argtypes = [_vp, _i64, _vp]
    L.sph_get_status.argtypes = [_vp, P(_i), P(_i64)]
    L.sph_clear_status.argtypes = [_vp, _vp]
    L.sph_built_with_checks.argtypes = []
    L.sph_get_check_report.argtypes = [_vp, P(_i), P(_i64), P(_i64)]
    L.sph_get_counters.argtypes = [_vp, P(sph_counters)]
    L.sph_reset_counters.argtypes = [_vp, _vp]
    L.sph_set_profiling.argtypes = [_vp, _i]
    L.sph_get_kernel_times.argtypes = [_vp, P(sph_kernel_times)]
    L.sph_reset_kernel_times.argtypes = [_vp]
    L.sph_cell_order_noalloc.argtypes = [_vp, _vp, _vp, _i64, _d, _i, _vp, _vp]
    L.sph_cell_order_noalloc.restype = _i
    L.sph_state_copy.argtypes = [_vp, P(sph_particles), P(sph_particles), _i, _vp]
    L.sph_resume.argtypes = [_vp, P(sph_particles), _i64, _i, _vp]
    L.sph_grid_density.argtypes = [_vp, P(sph_particles), _i, _i64, _vp, _vp]
    L.sph_diagnostics.argtypes = [_vp, P(sph_particles), _i64, P(_d), _vp]
    L.sph_get_bin_counts.argtypes = [_vp, P(_i64), _i, _vp]
    L.sph_grid_density_bwd.argtypes = [_vp, P(sph_particles), _i, _i64, _vp, P(sph_adjoint), _vp]
    L.sph_step_bwd.argtypes = [_vp, P(sph_particles), P(sph_particles), _i64, _i,
                               P(sph_adjoint), _vp]
    L.sph_strerror.argtypes = [_i]
    L.sph_strerror.restype = ctypes.c_char_p
    for name in ("sph_create", "sph_destroy", "sph_build_cells", "sph_grid_info",
                 "sph_mark_active", "sph_kick_drift", "sph_density_active", "sph_force_active",
                 "sph_timestep_bins", "sph_begin_run", "sph_step_async", "sph_step_sync",
                 "sph_step", "sph_step_graph", "sph_get_time",
                 "sph_set_time", "sph_get_status", "sph_clear_status", "sph_get_counters",
                 "sph_reset_counters", "sph_set_profiling", "sph_get_kernel_times",
                 "sph_reset_kernel_times", "sph_state_copy", "sph_resume", "sph_grid_density",
                 "sph_grid_density_bwd", "sph_step_bwd", "sph_diagnostics",
                 "sph_get_bin_counts", "sph_built_with_checks", "sph_get_check_report"):
        getattr(L, name).restype = _i
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/sph.h (the tests check the library exports them)."""
    return ["sph_default_params", "sph_create", "sph_destroy", "sph_build_cells", "sph_perm",
            "sph_grid_info", "sph_mark_active", "sph_kick_drift", "sph_density_active",
            "sph_force_active", "sph_timestep_bins", "sph_begin_run", "sph_step_async",
            "sph_step_sync", "sph_step", "sph_step_graph",
            "sph_get_time", "sph_set_time", "sph_get_status", "sph_clear_status",
            "sph_get_counters", "sph_reset_counters", "sph_set_profiling",
            "sph_get_kernel_times", "sph_reset_kernel_times", "sph_cell_order_noalloc",
            "sph_state_copy", "sph_resume", "sph_grid_density", "sph_grid_density_bwd",
            "sph_step_bwd", "sph_diagnostics", "sph_get_bin_counts", "sph_strerror",
            "sph_built_with_checks", "sph_get_check_report"]


class SphError(RuntimeError):
    def __init__(self, code, where):
        msg = load().sph_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def check(code, where):
    if code != SPH_OK:
        raise SphError(code, where)
