"""The sampled-cell method of tests/subbox.py against whole-field oracle runs
(CPU): one step of a cell's box reproduces the cell's post-collision PDFs of
the whole field to rounding (within 1e-15 relative; bit for bit unless the
integer shift of a sphere centre into the box rounds it), with gravity (the box gets the field's fluid
force density as its body force), moving spheres, two spheres sharing cells,
periodic axes and walls.  This is what lets the full-size GPU tests compare
sampled cells with the oracle."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2303_11811_gb300 import inputs
from tests.subbox import box, oracle_cell, sample_cells


def _field(walls):
    w = inputs.Workload("t", 24, 20, 22, tau=0.57, relax="trt", walls=walls,
                        fbody=(1e-6, 0.0, 0.0), gravity=(0.0, 0.0, -2e-5), weighting="nt",
                        eps_mode="supersample", eps_n=4, bc_velocity=(1e-4, 0.0, 2e-3),
                        bc_density=1.003)
    x = np.array([[7.3, 9.1, 10.6], [15.2, 9.7, 11.4], [12.0, 2.0, 20.5]])
    r = np.array([4.6, 3.9, 3.2])
    u = inputs.random_velocities(3, 2e-3, 21)
    om = inputs.random_velocities(3, 1e-3, 22)
    dens = np.array([2.5, 2.0, 3.0])
    w.particles = dict(x=x, r=r, density=dens, fixed=np.zeros(3, np.uint8))
    o = Oracle(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=walls, fbody=w.fbody,
               weighting=w.weighting, eps_mode=w.eps_mode, eps_n=w.eps_n, gravity=w.gravity,
               dem=True, bc_velocity=w.bc_velocity, bc_density=w.bc_density)
    f0 = o.pdfs()
    o.set_pdfs((f0 * (1.0 + inputs.noise(f0.shape, 1e-3, 23))).ravel())
    o.set_particles(x, r, u=u, omega=om, density=dens)
    return w, o, u, om, dens


@pytest.mark.parametrize("walls", [(0, 0, 0, 0, 0, 0), (1, 1, 0, 0, 0, 0),
                                   (1, 1, 1, 1, 2, 3)])
def test_box_step_equals_field_step(walls):
    w, o, u, om, dens = _field(walls)
    o.step(2)
    xs, us, oms = o.particles()
    pre = o.pdfs()
    o.step(1)
    post = o.pdfs()
    fext = o.last_fext()
    # gravity's counter force acts, but not with open faces
    assert (np.max(np.abs(fext - np.array(w.fbody))) > 0) == (max(walls) < 2)
    cells = sample_cells(w, 24, 5) + [(0, 3, 4), (w.nx - 1, 10, 21), (5, 5, 0), (9, 12, 1),
                                      (w.nx - 1, 0, w.nz - 1), (7, 9, w.nz - 2)]
    for c in cells:
        orig, ext = box(w, c)
        idx = [np.arange(orig[a], orig[a] + ext[a]) % (w.nx, w.ny, w.nz)[a] for a in range(3)]
        fb = pre[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
        got = oracle_cell(w, c, fb, fext, xs, w.particles["r"], us, oms, dens)
        want = post[:, c[2], c[1], c[0]]
        assert np.max(np.abs(got - want) / np.abs(want)) < 1e-15, c
