"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/sph.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_1807_01341_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = _declared("sph.h")
    for required in ("sph_build_cells", "sph_density_active", "sph_force_active",
                     "sph_timestep_bins", "sph_kick_drift", "sph_create", "sph_destroy",
                     "sph_step", "sph_step_graph", "sph_get_status", "sph_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for header in os.listdir(os.path.join(ROOT, "include")):
        for name in _declared(header):
            assert hasattr(lib, name), name


def test_checks_library_exports_the_same_symbols_and_reports_its_build(libpath):
    """The build with device bounds checks (-DSPH_CHECKS) exports every declared
    entry point, says it was built with checks, and the plain one says it was
    not (neither call touches a GPU)."""
    from paper_1807_01341_gb300 import build
    plain = ctypes.CDLL(libpath)
    checked = ctypes.CDLL(build.CHECKS_LIB)
    for name in _declared("sph.h"):
        assert hasattr(checked, name), name
    assert plain.sph_built_with_checks() == 0
    assert checked.sph_built_with_checks() == 1


def test_plain_library_refuses_a_planted_bad_index(libpath):
    """test_bad_group plants an out-of-range work group for the bounds checks to
    catch; a library without checks must refuse it (sph_create: SPH_ERR_ARG)
    before anything reaches a GPU."""
    from paper_1807_01341_gb300 import _lib
    lib = ctypes.CDLL(libpath)
    lib.sph_default_params.argtypes = [ctypes.POINTER(_lib.sph_params)]
    lib.sph_create.argtypes = [ctypes.POINTER(_lib.sph_params), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_void_p)]
    p = _lib.sph_params()
    lib.sph_default_params(ctypes.byref(p))
    p.test_bad_group = 1
    h = ctypes.c_void_p()
    assert lib.sph_create(ctypes.byref(p), 1000, ctypes.byref(h)) == _lib.SPH_ERR_ARG
    assert not h.value


def test_binding_names_match_header(libpath):
    from paper_1807_01341_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared("sph.h")


def test_struct_layouts_match_header(libpath, tmp_path):
    """ctypes mirrors of the public structs have the C sizes and offsets."""
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_1807_01341_gb300 import _lib
    src = tmp_path / "layout.c"
    checks = []
    for cname, cls in (("sph_params", _lib.sph_params), ("sph_particles", _lib.sph_particles),
                       ("sph_counters", _lib.sph_counters), ("sph_adjoint", _lib.sph_adjoint),
                       ("sph_kernel_times", _lib.sph_kernel_times)):
        checks.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            checks.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sph.h"\nint main(void){\n'
                   + "\n".join(checks) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
               if line)
    for cname, cls in (("sph_params", _lib.sph_params), ("sph_particles", _lib.sph_particles),
                       ("sph_counters", _lib.sph_counters), ("sph_adjoint", _lib.sph_adjoint),
                       ("sph_kernel_times", _lib.sph_kernel_times)):
        assert int(out[cname]) == ctypes.sizeof(cls)
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def test_product_fails_loudly_without_library(tmp_path):
    """No CPU fallback: a missing library is an error, not a slower path."""
    from paper_1807_01341_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
