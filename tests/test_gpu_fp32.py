"""FP32 deviation storage (PSM_FP32_DEV) against the FP64 oracle.

The FP32 path stores delta_q = f_q - w_q and collides in FP32.  Each step
rounds every stored value (relative 2^-24) and the collision's few dozen
operations add a few roundings of the same size, so after n steps the error
is bounded by about n * 32 * 2^-24 * max|delta|: that is the PDF tolerance.
Forces are per-cell FP32 contributions summed in FP64: 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_11811_gb300 import build, capi as c
    build.build()
    return c


def _setup(capi, streaming):
    shape = (37, 24, 20)
    kw = dict(tau=0.57, relax="trt", walls=(1, 1, 0, 0, 0, 0), fbody=(0.0, 1e-5, 2e-5),
              weighting="nt", eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, -3e-5),
              dem=True, kn=100.0, restitution=0.8)
    e = capi.Engine(*shape, precision="fp32", streaming=streaming, **kw)
    o = Oracle(*shape, **kw)
    x = np.array([[6.0, 7.5, 9.2], [13.8, 7.6, 9.3], [33.95, 16.7, 3.3]])
    r = np.array([4.3, 3.6, 3.1])
    u = np.array([[-2e-3, 1e-3, 0.0], [-1e-3, 0.0, 1e-3], [5e-4, -1e-3, -2e-3]])
    f0 = o.pdfs()
    f0 = f0 * (1.0 + inputs.noise(f0.shape, 1e-3, 3))
    for s in (e, o):
        s.set_pdfs(f0.ravel())
        s.set_particles(x, r, u=u, omega=inputs.random_velocities(3, 1e-3, 4),
                        density=np.array([2.5, 2.0, 3.0]))
    return e, o


@pytest.mark.parametrize("streaming", ["pull", "aa"])
def test_fp32_deviation_storage_within_derived_bound(capi, streaming):
    e, o = _setup(capi, streaming)
    n = 20
    e.step(n)
    o.step(n)
    fo = o.pdfs()
    rest = Oracle(1, 1, 1, 0.6).pdfs()[:, 0, 0, 0]
    delta = fo - rest[:, None, None, None]
    tol = n * 32 * 2.0 ** -24 * float(np.max(np.abs(delta)))
    err = float(np.max(np.abs(e.pdfs() - fo)))
    assert err <= tol, (err, tol)
    Fg, Tg = e.force_torque()
    Fo, To = o.force_torque()
    assert np.max(np.abs(Fg - Fo)) <= 1e-4 * np.max(np.abs(Fo))
    xg, _, _ = e.particles()
    xo, _, _ = o.particles()
    assert np.max(np.abs(xg - xo)) < 1e-6


def test_fp32_aa_equals_fp32_pull_bitwise(capi):
    a, _ = _setup(capi, "aa")
    b, _ = _setup(capi, "pull")
    a.step(9)
    b.step(9)
    assert np.array_equal(a.pdfs(), b.pdfs())


def test_fp32_drag_against_fp64_on_fixed_array(capi):
    """Fixed random array in a channel (walls at the x faces), 300 steps from
    rest: the FP32 path's drag and velocity field against the FP64 path."""
    w = inputs.channel(nx=64, ny=64, nz=96)
    res = {}
    for prec, stream in (("fp64", "pull"), ("fp32", "aa")):
        e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, fbody=w.fbody,
                        weighting=w.weighting, eps_mode=w.eps_mode, eps_n=w.eps_n,
                        precision=prec, streaming=stream)
        p = w.particles
        e.set_particles(p["x"], p["r"], fixed=p["fixed"])
        e.step(300)
        F, _ = e.force_torque()
        _, u = e.macroscopic()
        res[prec] = (F, u)
        e.close()
    F64, u64 = res["fp64"]
    F32, u32 = res["fp32"]
    assert np.linalg.norm(F32 - F64) / np.linalg.norm(F64) < 5e-3
    assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-3


@pytest.mark.parametrize("weighting,tol", [("eps", 2e-5), ("nt", 2e-4)])
def test_fp32_linear_mapping_against_the_oracle(capi, weighting, tol):
    """Linear approximation (Eqs. 25-26) with FP32 records: the same slots as
    the FP64 definition (the inside test is certified), weights within the
    FP32 evaluation of |d| (|d|^2 rounded to 2^-24 relative, r = 10: about
    1e-6 in eps; Noble-Torczynski's dB/deps reaches 1/(tau - 1/2) = 20)."""
    shape = (60, 48, 44)
    kw = dict(tau=0.55, relax="srt", walls=(1, 1, 1, 1, 0, 0), weighting=weighting,
              eps_mode="linear", eps_n=4)
    e = capi.Engine(*shape, precision="fp32", **kw)
    o = Oracle(*shape, **kw)
    x = np.array([[14.3, 12.1, 20.7], [36.25, 24.0, 21.0], [47.5, 33.9, 3.2]])
    r = np.array([10.0, 8.5, 7.25])
    for s in (e, o):
        s.set_particles(x, r, fixed=np.ones(3, np.uint8))
    assert o.map() == 0
    pg0, bg0, pg1, bg1 = e.slots()
    po0, bo0, po1, bo1 = o.slots()
    Bsum = bo0 + bo1
    over = Bsum > 1.0
    bo0 = np.where(over, bo0 / np.where(over, Bsum, 1.0), bo0)
    bo1 = np.where(over, bo1 / np.where(over, Bsum, 1.0), bo1)
    assert np.array_equal(pg0, po0) and np.array_equal(pg1, po1)
    assert np.max(np.abs(bg0 - bo0)) < tol and np.max(np.abs(bg1 - bo1)) < tol
    e.close()
