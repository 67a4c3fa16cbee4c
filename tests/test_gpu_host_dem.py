"""The paper's coupling through the C ABI (psm_step_host_dem): the LBM part
on the device, the particle dynamics on the host cores with per-step force
and state transfers.  Its DEM is the device DEM's arithmetic, so the run
equals psm_step's (PDFs, forces, particle state) with moving spheres, DEM
contacts and walls, in the FP64, FP32 and double-float forms, and at the
settling workload's full size; without the DEM it is refused."""
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


KW = dict(tau=0.57, relax="trt", walls=(1, 1, 0, 0, 0, 0), fbody=(0.0, 1e-5, 2e-5),
          weighting="nt", eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, -3e-5),
          dem=True, kn=100.0, restitution=0.8)
SHAPE = (37, 24, 20)


def _start(capi, precision, streaming="pull", **kw):
    e = capi.Engine(*SHAPE, precision=precision, streaming=streaming, **{**KW, **kw})
    # spheres 0 and 1 overlap by 0.1 (a contact from the first sub-step),
    # sphere 2 presses on the +x wall and wraps around the z faces
    x = np.array([[6.0, 7.5, 9.2], [13.8, 7.6, 9.3], [33.95, 16.7, 3.3]])
    r = np.array([4.3, 3.6, 3.1])
    u = np.array([[-2e-3, 1e-3, 0.0], [-1e-3, 0.0, 1e-3], [5e-4, -1e-3, -2e-3]])
    e.set_particles(x, r, u=u, omega=inputs.random_velocities(3, 1e-3, 4),
                    density=np.array([2.5, 2.0, 3.0]))
    return e


def _state(e):
    F, T = e.force_torque()
    x, u, w = e.particles()
    return e.pdfs(), np.concatenate([F, T]), np.concatenate([x, u, w])


@pytest.mark.parametrize("precision,streaming", [("fp64", "pull"), ("fp64", "aa"),
                                                 ("fp32", "pull"), ("df64", "pull")])
def test_host_dem_equals_device_dem(capi, precision, streaming):
    a = _start(capi, precision, streaming)
    b = _start(capi, precision, streaming)
    a.step(12)
    host_ms = b.step_host_dem(12, threads=4)
    fa, Fa, Pa = _state(a)
    fb, Fb, Pb = _state(b)
    assert host_ms > 0.0
    # same operations in the same order on both sides: equal to the last bit
    assert np.array_equal(Pa, Pb), float(np.max(np.abs(Pa - Pb)))
    assert np.array_equal(Fa, Fb) and np.array_equal(fa, fb)
    # the device DEM picks up where the host left off
    a.step(3)
    b.step(3)
    assert np.array_equal(_state(a)[2], _state(b)[2])


def test_settle128_full_size_host_dem(capi):
    """The 128^3 settling workload (400 spheres, the bench's configuration):
    three steps with the DEM on the host equal three on the device."""
    w = inputs.settle128()
    kw = dict(tau=w.tau, relax=w.relax, gravity=w.gravity, weighting=w.weighting,
              eps_mode=w.eps_mode, eps_n=w.eps_n, dem=True, kn=w.kn, restitution=w.restitution)
    p = w.particles
    engines = []
    for _ in range(2):
        e = capi.Engine(w.nx, w.ny, w.nz, **kw)
        e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
        engines.append(e)
    engines[0].step(3)
    engines[1].step_host_dem(3)
    sa, sb = _state(engines[0]), _state(engines[1])
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y), float(np.max(np.abs(x - y)))


def test_host_dem_needs_the_dem(capi):
    e = _start(capi, "fp64", dem=False)
    with pytest.raises(capi.PsmError) as err:
        e.step_host_dem(1)
    assert err.value.status == capi.PSM_ERR_ARG
