"""Open z faces (the velocity inflow and pressure outflow of the fluidized
bed, Sec. 4.1) on the CUDA path against the FP64 oracle: side walls on x and
y, an inflow at -z with a tangential component, an outflow at +z at a density
other than 1, moving spheres with the DEM (the z faces are walls for the
particles) and gravity (no counter force with open faces), a noisy field.

FP64 (staged kernel) and the double-float form: PDFs within 1e-12 relative,
forces and torques within 1e-12 (double-float: 1e-10) of the largest
component, particle states as in the other parity tests.  FP32 deviations:
the derived bound n * 32 * 2^-24 * max|f - w| of the FP32 tests.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPE = (37, 24, 30)
KW = dict(tau=0.57, relax="trt", walls=(1, 1, 1, 1, 2, 3), weighting="nt",
          eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, -3e-5), dem=True, kn=100.0,
          restitution=0.8, bc_velocity=(2e-4, -1e-4, 3e-3), bc_density=1.004)


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_11811_gb300 import build, capi as c
    build.build()
    return c


def rel_pdf_err(fg, fo):
    return float(np.max(np.abs(fg - fo) / np.abs(fo)))


def force_err(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _pair(capi, precision, eps_mode="supersample"):
    kw = dict(KW, eps_mode=eps_mode)
    e = capi.Engine(*SHAPE, precision=precision, **kw)
    o = Oracle(*SHAPE, **kw)
    # sphere 0 presses on the inflow face, sphere 1 is next to the outflow
    # face, spheres 2 and 3 overlap (contacts from the first sub-step)
    x = np.array([[8.0, 9.5, 3.3], [20.3, 12.4, 26.1], [25.0, 8.0, 14.2], [31.4, 8.3, 14.6]])
    r = np.array([3.4, 3.0, 3.5, 3.0])
    u = np.array([[1e-3, 0.0, -2e-3], [0.0, 1e-3, 2e-3], [1e-3, 0.0, 0.0], [-1e-3, 0.0, 0.0]])
    f0 = o.pdfs()
    f0 = f0 * (1.0 + inputs.noise(f0.shape, 1e-3, 13))
    for s in (e, o):
        s.set_pdfs(f0.ravel())
        s.set_particles(x, r, u=u, omega=inputs.random_velocities(4, 1e-3, 14),
                        density=np.array([2.5, 2.0, 3.0, 1.5]))
    return e, o


@pytest.mark.parametrize("precision,eps_mode", [("fp64", "supersample"), ("fp64", "linear"),
                                                ("df64", "supersample")])
def test_open_faces_fp64_forms_match_oracle(capi, precision, eps_mode):
    e, o = _pair(capi, precision, eps_mode)
    e.step(25)
    o.step(25)
    assert rel_pdf_err(e.pdfs(), o.pdfs()) < 1e-12
    Fg, Tg = e.force_torque()
    Fo, To = o.force_torque()
    ftol = 1e-12 if precision == "fp64" else 1e-10
    assert force_err(Fg, Fo) < ftol, force_err(Fg, Fo)
    assert force_err(Tg, To) < ftol, force_err(Tg, To)
    xg, ug, wg = e.particles()
    xo, uo, wo = o.particles()
    assert np.max(np.abs(xg - xo)) < 1e-12
    assert np.max(np.abs(ug - uo)) < 1e-13 and np.max(np.abs(wg - wo)) < 1e-13
    rg, ugf = e.macroscopic()
    ro, uof = o.macroscopic()
    assert np.max(np.abs(rg - ro)) < 1e-13 and np.max(np.abs(ugf - uof)) < 1e-13
    # the face plane pushed the sphere that pressed on it back up
    assert uo[0, 2] > 0.0
    e.close()


def test_open_faces_fp32_within_derived_bound(capi):
    e, o = _pair(capi, "fp32")
    n = 20
    e.step(n)
    o.step(n)
    fo = o.pdfs()
    rest = Oracle(1, 1, 1, 0.6).pdfs()[:, 0, 0, 0]
    tol = n * 32 * 2.0 ** -24 * float(np.max(np.abs(fo - rest[:, None, None, None])))
    err = float(np.max(np.abs(e.pdfs() - fo)))
    assert err <= tol, (err, tol)
    Fg, _ = e.force_torque()
    Fo, _ = o.force_torque()
    assert np.max(np.abs(Fg - Fo)) <= 1e-4 * np.max(np.abs(Fo))
    e.close()


def test_inflow_mass_flux_on_the_device(capi):
    """Inflow at -z, wall at +z, periodic x and y: the device's mass grows by
    exactly U_z * nx * ny per step (psm_check's FP64 sums)."""
    nx, ny, nz, Uz = 40, 20, 12, 2e-3
    e = capi.Engine(nx, ny, nz, 0.6, relax="trt", walls=(0, 0, 0, 0, 2, 1),
                    bc_velocity=(1e-4, 0.0, Uz))
    m = [e.check()[0]]
    for _ in range(4):
        e.step(1)
        m.append(e.check()[0])
    assert np.max(np.abs(np.diff(m) - Uz * nx * ny)) < 1e-12 * m[-1]
    e.close()


def test_open_faces_refused_where_not_built(capi):
    """Open faces need pull streaming and sit on the z faces only."""
    with pytest.raises(capi.PsmError):
        capi.Engine(16, 16, 16, 0.6, walls=(0, 0, 0, 0, 2, 3), streaming="aa")
    with pytest.raises(capi.PsmError):
        capi.Engine(16, 16, 16, 0.6, walls=(2, 3, 0, 0, 0, 0))
    with pytest.raises(capi.PsmError):
        capi.Engine(16, 16, 16, 0.6, walls=(0, 0, 0, 0, 2, 0))
