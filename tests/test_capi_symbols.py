"""The C-ABI library builds, loads without a GPU, and exports every function
that include/psm.h declares (no compute calls are made here)."""
import ctypes
import os
import re

from paper_2303_11811_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psm_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    from paper_2303_11811_gb300 import build
    build.build()
    L = ctypes.CDLL(capi.LIB_PATH)
    names = _declared("psm.h")
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    names = set(_declared("psm.h"))
    assert names == set(capi.EXPORTS), names.symmetric_difference(capi.EXPORTS)


def test_default_options_without_gpu():
    """psm_default_options is pure host code and can run here."""
    L = capi.lib()
    o = capi.PsmOptions()
    L.psm_default_options(ctypes.byref(o))
    assert abs(o.magic - 3 / 16) < 1e-15 and o.eps_n == 4 and o.dem_subcycles == 10
    assert o.weighting == capi.PSM_W_NT and o.deterministic == 1


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    """Argument checks come before any CUDA call."""
    L = capi.lib()
    o = capi.PsmOptions()
    L.psm_default_options(ctypes.byref(o))
    g = capi.PsmGrid()
    g.nx, g.ny, g.nz = 8, 8, 8
    h = ctypes.c_void_p()
    assert L.psm_create(ctypes.byref(g), 0.5, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    g.wall[0] = 1  # -x wall without +x wall
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    g.wall[0] = 0
    o.eps_n = 0
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    o.eps_n = 4
    o.deterministic = 0  # only the fixed-order reduction exists
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    assert not h.value


def test_checkpoint_entries_reject_null_arguments_without_a_gpu():
    """psm_save / psm_load / psm_get_particle_count check their arguments
    before touching a context or the GPU."""
    L = capi.lib()
    n = ctypes.c_int(-1)
    assert L.psm_save(None, b"/nonexistent/x.psm") == 1
    assert L.psm_load(None, b"/nonexistent/x.psm") == 1
    assert L.psm_get_particle_count(None, ctypes.byref(n)) == 1
    assert n.value == -1
    o = capi.PsmOptions()
    L.psm_default_options(ctypes.byref(o))
    g = capi.PsmGrid()
    g.nx, g.ny, g.nz = 8, 8, 8
    o.precision = capi.PSM_FP64_DF + 1  # not a storage form
    h = ctypes.c_void_p()
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    assert not h.value


def test_no_other_c_symbols_leak():
    """Every unmangled function the library exports is a psm_ entry point
    (internal helpers have internal linkage)."""
    import shutil
    import subprocess

    import pytest
    if not shutil.which("nm"):
        pytest.skip("nm not available")
    from paper_2303_11811_gb300 import build
    build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    names = [ln.split()[-1] for ln in out.splitlines() if " T " in ln]
    leaked = [n for n in names if not n.startswith(("psm_", "_Z", "_init", "_fini"))]
    assert not leaked, leaked
