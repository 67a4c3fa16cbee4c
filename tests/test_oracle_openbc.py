"""Pins of the oracle's open faces (reading V: the velocity inflow and
pressure outflow that Sec. 4.1 names for the fluidized bed).

- the inflow lets exactly U_z of mass per face cell and step into the box
  (the moving-wall bounce-back adds 6 w_q c_q.U over the five entering
  directions, whose w_q c_qz sum to 1/6);
- a uniform flow at the inflow velocity and the outflow density is a fixed
  point of the whole scheme (inflow, bulk, anti-bounce-back outflow);
- from rest, a plug flow settles to that state: the outflow holds the
  density it is given;
- between no-slip walls the flow develops into the discrete Poiseuille
  profile of TRT with Lambda = 3/16 (a parabola with zero slip at the
  faces) carrying the inflow's flux.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2303_11811_gb300 import inputs
from tests.lattice_fixture import equilibrium, uniform_field

U = 2e-3


def test_inflow_lets_in_exactly_its_mass_flux():
    nx, ny, nz = 6, 5, 7
    o = Oracle(nx, ny, nz, 0.6, relax="trt", walls=(0, 0, 0, 0, 2, 1),
               bc_velocity=(3e-4, -2e-4, U))
    f = o.pdfs()
    o.set_pdfs((f * (1.0 + inputs.noise(f.shape, 1e-3, 3))).ravel())
    for _ in range(5):
        m0 = math.fsum(o.pdfs().ravel())
        o.step(1)
        m1 = math.fsum(o.pdfs().ravel())
        # the tangential inflow components carry no mass through the face
        assert abs((m1 - m0) - U * nx * ny) < 1e-14 * m1


@pytest.mark.parametrize("rho_b", [1.0, 1.01])
def test_uniform_open_flow_is_a_fixed_point(rho_b):
    shape = (16, 3, 3)
    o = Oracle(3, 3, 16, 0.7, relax="trt", walls=(0, 0, 0, 0, 2, 3), bc_velocity=(0, 0, U),
               bc_density=rho_b)
    f0 = uniform_field(equilibrium(rho_b, (0.0, 0.0, U)), shape)
    o.set_pdfs(f0.ravel())
    o.step(5)
    assert np.max(np.abs(o.pdfs() - f0)) < 1e-15


def test_plug_flow_settles_to_the_outflow_density():
    rho_b = 1.01
    o = Oracle(3, 3, 16, 1.0, relax="trt", walls=(0, 0, 0, 0, 2, 3), bc_velocity=(0, 0, U),
               bc_density=rho_b)
    errs = []
    for _ in range(2):
        o.step(3000)
        rho, u = o.macroscopic()
        errs.append(max(np.max(np.abs(rho - rho_b)), np.max(np.abs(u[2] - U))))
        assert np.max(np.abs(u[:2])) < 1e-15
    assert errs[1] < 1e-6 and errs[1] < 0.1 * errs[0]


def test_developed_poiseuille_between_walls():
    """Walls on the x faces, uniform inflow at -z, outflow at +z: mid-channel
    the profile is u(x) = A x (H - x) at the cell centres (zero slip at the
    faces with Lambda = 3/16), with A set by the inflow's flux
    U (H - 1/3) per unit depth (the two wall cells each lose the 1/6 of
    their inflow carried by the edge link that crosses the wall)."""
    H, nz = 8, 32
    o = Oracle(H, 1, nz, 1.0, relax="trt", magic=3.0 / 16.0, walls=(1, 1, 0, 0, 2, 3),
               bc_velocity=(0.0, 0.0, U))
    o.step(10000)
    _, u = o.macroscopic()
    xc = np.arange(H) + 0.5
    prof = u[2, nz // 2, 0, :]
    exact = U * (H - 1.0 / 3.0) / np.sum(xc * (H - xc)) * xc * (H - xc)
    assert np.max(np.abs(prof - exact)) < 1e-6 * exact.max()
    assert abs(prof.sum() / (U * (H - 1.0 / 3.0)) - 1.0) < 1e-6
    # once developed no cross flow is left but the compressibility terms of
    # the scheme, of order Ma^2 = 3 U^2 = 1.2e-5 of U
    assert np.max(np.abs(u[0, nz // 2])) < 1e-4 * U
