"""Full-size checks in the launch configurations the bench times, where the
oracle cannot step the whole field: sampled cells and budgets.

Sampled cells (tests/subbox.py): the engine's post-collision PDFs of a cell
after one step must equal the oracle's on a box around the cell: 1e-12
relative in FP64 and in the double-float form (which is held to the FP64
bound); in FP32 the one-step bound of tests/test_gpu_fp32.py,
32 * 2^-24 * max|delta| over the neighbourhood.

Budgets (FP64 and double-float).  Mass is conserved to rounding; in a periodic box the fluid
momentum changes per step by V_fluid f - sum_i F_i (Eqs. 1, 8, 17, 21), with
V_fluid and f the engine's own of that step (with walls, bounce-back passes
momentum to the walls): sums over all cells, any size.
"""
import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs
from tests.subbox import REST, box, oracle_cell, sample_cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_11811_gb300 import build, capi as c
    build.build()
    return c


def _engine(capi, w, precision, streaming):
    e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, fbody=w.fbody,
                    weighting=w.weighting, eps_mode=w.eps_mode, eps_n=w.eps_n,
                    gravity=w.gravity, kn=w.kn, restitution=w.restitution,
                    subcycles=w.subcycles, dem=w.dem, precision=precision, streaming=streaming,
                    bc_velocity=w.bc_velocity, bc_density=w.bc_density)
    p = w.particles
    e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    return e


def _sampled_step(e, w, cells, precision):
    """One engine step checked at the sampled cells against the oracle."""
    xs, us, oms = e.particles()
    R = w.particles["r"]
    dens = w.particles["density"]
    pre = []
    for c in cells:
        o, ext = box(w, c)
        pre.append(e.pdfs_box(*o, *ext))
    e.step(1)
    fext, _ = e.fluid_force()
    worst = 0.0
    for c, fb in zip(cells, pre):
        got = e.pdfs_box(*c, 1, 1, 1)[:, 0, 0, 0]
        want = oracle_cell(w, c, fb, fext, xs, R, us, oms, dens)
        if precision in ("fp64", "df64"):
            err = float(np.max(np.abs(got - want) / np.abs(want)))
            assert err < 1e-12, (c, err)
        else:
            o, _ = box(w, c)
            loc = [c[a] - o[a] for a in range(3)]
            nb = fb[:, max(loc[2] - 1, 0):loc[2] + 2, max(loc[1] - 1, 0):loc[1] + 2,
                    max(loc[0] - 1, 0):loc[0] + 2]
            delta = np.max(np.abs(nb - REST[:, None, None, None]))
            err = float(np.max(np.abs(got - want)))
            # plus the FP64 rounding of w_q + delta in the canonical values
            assert err <= 32 * 2.0 ** -24 * delta + 2.0 ** -50, (c, err, delta)
        worst = max(worst, err)
    return worst


def _budgets(e, steps, periodic):
    """Mass and (periodic box) fluid momentum budgets over single steps."""
    for _ in range(steps):
        m0, P0 = e.check()
        e.step(1)
        m1, P1 = e.check()
        fext, vf = e.fluid_force()
        F, _ = e.force_torque()
        expect = vf * fext - F.sum(axis=0)
        scale = vf * float(np.max(np.abs(fext))) + float(np.abs(F).sum())
        assert abs(m1 - m0) <= 1e-13 * m0, (m0, m1)
        if periodic:
            assert np.max(np.abs((P1 - P0) - expect)) <= 1e-6 + 1e-9 * scale, (P1 - P0, expect)


@pytest.mark.parametrize("precision,streaming", [("fp64", "pull"), ("fp32", "pull"),
                                                 ("fp32", "aa"), ("df64", "pull")])
def test_channel_full_size_sampled(capi, precision, streaming):
    """256x256x512 channel, walls at the x faces, 12,817 fixed spheres r=5,
    4^3 sampling: 24 sampled cells of one step after two warm-up steps; FP64
    also the mass budget of two more steps."""
    import torch
    w = inputs.channel()
    e = _engine(capi, w, precision, streaming)
    e.step(2)
    _sampled_step(e, w, sample_cells(w, 24, 11), precision)
    if precision != "fp32":
        _budgets(e, 2, periodic=False)
    e.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision,streaming", [("fp64", "pull"), ("fp32", "aa"),
                                                 ("df64", "aa")])
def test_settle512_full_size_sampled(capi, precision, streaming):
    """512x512x1024 periodic box (268M cells), 94,692 settling spheres r in
    [3, 6] at solid fraction 0.15, gravity, DEM: every step succeeds (no slot
    or neighbour-list overflow, no skin violation), 16 sampled cells of one
    step match the oracle, and in FP64 the mass and momentum budgets hold."""
    import torch
    w = inputs.settle512()
    e = _engine(capi, w, precision, streaming)
    e.step(2)
    _sampled_step(e, w, sample_cells(w, 16, 12), precision)
    if precision != "fp32":
        _budgets(e, 1, periodic=True)
    e.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("case,precision", [("dilute", "fp64"), ("dense", "fp64"),
                                            ("dilute", "fp32"), ("dense", "df64")])
def test_bed_full_size_sampled(capi, case, precision):
    """The fluidized-bed stand-ins at full size (500x200x800, side walls,
    velocity inflow at the bottom, pressure outflow at the top, spheres r=10,
    the linear approximation): 20 sampled cells of one step after two warm-up
    steps, among them cells on the inflow and outflow layers, at the side
    walls and in the packed bed, match the oracle on boxes with the same
    faces."""
    import torch
    w = inputs.bed(case)
    e = _engine(capi, w, precision, "pull")
    e.step(2)
    faces = [(250, 100, 0), (0, 0, 0), (499, 199, 0), (123, 57, 1), (250, 100, 799),
             (0, 199, 799), (331, 17, 798), (7, 150, 400)]
    _sampled_step(e, w, faces + sample_cells(w, 12, 13), precision)
    e.close()
    torch.cuda.empty_cache()
