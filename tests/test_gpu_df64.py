"""The double-float form (PDFs as FP32 pairs hi + lo, collision in
double-float arithmetic on the FP32 pipes) against the FP64 oracle, at the
bound of the FP64 path: PDFs within 1e-12 relative (max over cells and
directions of |f_gpu - f_oracle| / |f_oracle|), forces and torques within
1e-10 relative to the largest component.

The form keeps about 2^-47 relative precision on the stored deviations
f_q - w_q, which are small (|f - w| << w), so its rounding stays orders of
magnitude below the bound after 1000 steps.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu

PDF_TOL = 1e-12


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
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / scale


def test_sphere32_df64_1000_steps(capi):
    """32^3 periodic box, one fixed sphere r = 4, SRT tau = 0.6, body force
    1e-6 in x, 4^3 sampling: 1000 steps in the double-float form."""
    w = inputs.sphere32()
    kw = dict(tau=w.tau, relax=w.relax, fbody=w.fbody, weighting=w.weighting,
              eps_mode=w.eps_mode, eps_n=w.eps_n)
    e = capi.Engine(32, 32, 32, precision="df64", **kw)
    o = Oracle(32, 32, 32, **kw)
    for s in (e, o):
        s.set_particles(w.particles["x"], w.particles["r"], density=w.particles["density"],
                        fixed=w.particles["fixed"])
    e.step(1000)
    o.step(1000)
    err = rel_pdf_err(e.pdfs(), o.pdfs())
    print(f"df64 sphere32 1000 steps: max relative PDF error {err:.2e}")
    assert err < PDF_TOL
    Fg, Tg = e.force_torque()
    Fo, To = o.force_torque()
    assert force_err(Fg, Fo) < 1e-10
    assert np.max(np.abs(Tg - To)) < 1e-10 * np.max(np.abs(Fo))
    e.close()


@pytest.mark.parametrize("streaming", ["pull", "aa"])
def test_df64_moving_particles_walls_ragged_grid(capi, streaming):
    """37x24x20 cells (padded lanes), walls on the x faces, noisy initial
    field, three moving spheres with DEM contacts, gravity and body force,
    TRT, 4^3 sampling: 25 steps."""
    shape = (37, 24, 20)
    kw = dict(tau=0.57, relax="trt", walls=(1, 1, 0, 0, 0, 0), fbody=(0.0, 1e-5, 2e-5),
              weighting="nt", eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, -3e-5),
              dem=True, kn=100.0, restitution=0.8)
    e = capi.Engine(*shape, precision="df64", streaming=streaming, **kw)
    o = Oracle(*shape, **kw)
    x = np.array([[6.0, 7.5, 9.2], [13.8, 7.6, 9.3], [33.95, 16.7, 3.3]])
    r = np.array([4.3, 3.6, 3.1])
    u = np.array([[-2e-3, 1e-3, 0.0], [-1e-3, 0.0, 1e-3], [5e-4, -1e-3, -2e-3]])
    om = inputs.random_velocities(3, 1e-3, 4)
    f0 = o.pdfs()
    f0 = f0 * (1.0 + inputs.noise(f0.shape, 1e-3, 3))
    for s in (e, o):
        s.set_pdfs(f0.ravel())
        s.set_particles(x, r, u=u, omega=om, density=np.array([2.5, 2.0, 3.0]))
    e.step(25)
    o.step(25)
    assert rel_pdf_err(e.pdfs(), o.pdfs()) < PDF_TOL
    Fg, Tg = e.force_torque()
    Fo, To = o.force_torque()
    assert force_err(Fg, Fo) < 1e-10 and force_err(Tg, To) < 1e-10
    xg, ug, wg = e.particles()
    xo, uo, wo = o.particles()
    assert np.max(np.abs(xg - xo)) < 1e-12
    assert np.max(np.abs(ug - uo)) < 1e-13 and np.max(np.abs(wg - wo)) < 1e-13
    e.close()


def test_df64_aa_equals_pull_bitwise(capi):
    """The AA pattern moves where the pairs live, not what is computed."""
    shape = (33, 20, 18)
    kw = dict(tau=0.62, relax="trt", walls=(1, 1, 0, 0, 0, 0), fbody=(1e-5, 0, 0),
              weighting="nt", eps_mode="supersample", eps_n=4, precision="df64")
    a = capi.Engine(*shape, streaming="aa", **kw)
    b = capi.Engine(*shape, streaming="pull", **kw)
    x = np.array([[10.2, 9.1, 8.7], [22.4, 11.3, 9.2]])
    for s in (a, b):
        s.set_particles(x, np.array([4.0, 3.5]), u=inputs.random_velocities(2, 1e-3, 8),
                        fixed=np.ones(2, np.uint8))
    for n in (7, 6):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.pdfs(), b.pdfs())
        assert np.array_equal(a.force_torque()[0], b.force_torque()[0])
    a.close()
    b.close()


def test_df64_settle128_full_size_three_steps(capi):
    """The 128^3 settling workload of the bench in the double-float form:
    3 full steps, every PDF compared with the oracle."""
    w = inputs.settle128()
    kw = dict(tau=w.tau, relax=w.relax, gravity=w.gravity, weighting=w.weighting,
              eps_mode=w.eps_mode, eps_n=w.eps_n, dem=True, kn=w.kn, restitution=w.restitution)
    e = capi.Engine(128, 128, 128, precision="df64", **kw)
    o = Oracle(128, 128, 128, **kw)
    p = w.particles
    for s in (e, o):
        s.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    e.step(3)
    o.step(3)
    assert rel_pdf_err(e.pdfs(), o.pdfs()) < PDF_TOL
    Fg, _ = e.force_torque()
    Fo, _ = o.force_torque()
    assert force_err(Fg, Fo) < 1e-10
    xg, _, _ = e.particles()
    xo, _, _ = o.particles()
    assert np.max(np.abs(xg - xo)) < 1e-12
    e.close()


@pytest.mark.parametrize("eps_mode,eps_n", [("supersample", 8), ("mlp", 8)])
def test_df64_mapping_records(capi, eps_mode, eps_n):
    """The double-float form keeps its slot records as FP32 pairs: the same
    slots as the FP64 form and the same weights to the pairs' precision
    (surrogate mode included: its weights are written by the inference)."""
    shape = (48, 40, 36)
    kw = dict(tau=0.6, relax="srt", weighting="nt", eps_mode=eps_mode, eps_n=eps_n)
    a = capi.Engine(*shape, precision="df64", **kw)
    b = capi.Engine(*shape, precision="fp64", **kw)
    x = np.array([[1.2, 39.4, 17.9], [24.25, 20.0, 18.0], [24.25 + 9.4, 20.3, 18.5],
                  [46.9, 3.3, 35.2]])
    r = np.array([5.5, 4.0, 5.0, 3.3])
    params = capi.pack_mlp(inputs.mlp_init(4))
    for s in (a, b):
        if eps_mode == "mlp":
            s.set_mlp(params)
        s.set_particles(x, r)
        s.step(1)
    pa0, ba0, pa1, ba1 = a.slots()
    pb0, bb0, pb1, bb1 = b.slots()
    assert np.array_equal(pa0, pb0) and np.array_equal(pa1, pb1)
    assert np.max(np.abs(ba0 - bb0)) < 1e-14 and np.max(np.abs(ba1 - bb1)) < 1e-14
    assert (pa1 >= 0).sum() > 0
    a.close()
    b.close()
