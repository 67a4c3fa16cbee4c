"""Failure detection without a GPU fault.

- every bounded device wait (staged collision, surrogate inference, DEM grid
  barrier) gives up against a barrier that nothing completes, raises the
  timeout status, and the next call reports PSM_ERR_TIMEOUT; the context is
  usable again after psm_set_pdfs;
- a non-finite PDF in a covered cell is reported as PSM_ERR_NONFINITE by
  the step that meets it, and the context refuses to step until reset;
- an allocator callback that returns NULL makes psm_create and
  psm_set_particles return PSM_ERR_OOM (host-side fault injection).
"""
import ctypes

import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_11811_gb300 import build, capi as c
    build.build()
    return c


def test_bounded_waits_give_up_and_report_timeout(capi):
    e = capi.Engine(32, 16, 16, 0.6, relax="trt", dem=True)
    e.set_particles(np.array([[10.0, 8.0, 8.0]]), np.array([3.0]))
    f0 = e.pdfs()
    assert e.selftest_waits(2_000_000) == capi.PSM_OK        # 2 ms per wait
    assert e.step_status(1) == capi.PSM_ERR_TIMEOUT
    assert e.step_status(1) == capi.PSM_ERR_STATE
    e.set_pdfs(f0.ravel())
    assert e.step_status(3) == capi.PSM_OK                   # usable again
    e.close()


def test_nonfinite_state_is_reported(capi):
    e = capi.Engine(32, 16, 16, 0.6, relax="trt")
    e.set_particles(np.array([[16.0, 8.0, 8.0]]), np.array([4.0]), fixed=np.ones(1, np.uint8))
    clean = e.pdfs()
    f = clean.copy()
    f[:, 8, 8, 16] = np.nan                  # a cell inside the sphere
    e.set_pdfs(f.ravel())
    assert e.step_status(1) == capi.PSM_ERR_NONFINITE
    assert e.step_status(1) == capi.PSM_ERR_STATE
    e.set_pdfs(clean.ravel())               # a finite field clears the error state
    assert e.step_status(2) == capi.PSM_OK
    assert np.isfinite(e.pdfs()).all()
    e.close()


def test_allocator_failure_is_reported(capi):
    L = capi.lib()
    o = capi.PsmOptions()
    L.psm_default_options(ctypes.byref(o))
    calls = {"n": 0, "fail_after": 0}

    @capi.ALLOC_FN
    def alloc(nbytes, user):
        calls["n"] += 1
        return None if calls["n"] > calls["fail_after"] else _keep(nbytes)

    @capi.FREE_FN
    def free(p, user):
        _free(p)

    import torch
    bufs = {}

    def _keep(nbytes):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        bufs[t.data_ptr()] = t
        return t.data_ptr()

    def _free(p):
        bufs.pop(p, None)

    o.alloc = alloc
    o.free = free
    g = capi.PsmGrid()
    g.nx, g.ny, g.nz = 16, 16, 16
    h = ctypes.c_void_p()
    # the first allocation fails: psm_create reports PSM_ERR_OOM and no context
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == \
        capi.PSM_ERR_OOM
    assert not h.value
    # context buffers succeed, particle buffers fail
    calls["n"], calls["fail_after"] = 0, 10 ** 6
    assert L.psm_create(ctypes.byref(g), 0.6, 0, ctypes.byref(o), ctypes.byref(h)) == capi.PSM_OK
    calls["fail_after"] = calls["n"]
    x = np.array([8.0, 8.0, 8.0])
    r = np.array([3.0])
    z = np.zeros(3)
    d = np.array([1.0])
    dp = ctypes.POINTER(ctypes.c_double)
    st = L.psm_set_particles(h, 1, x.ctypes.data_as(dp), r.ctypes.data_as(dp),
                             z.ctypes.data_as(dp), z.ctypes.data_as(dp), d.ctypes.data_as(dp),
                             None)
    assert st == capi.PSM_ERR_OOM
    L.psm_destroy(h)
    assert not bufs
