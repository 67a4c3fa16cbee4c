"""Pins of the oracle's DEM (Sec. 2.2): velocity-Verlet exactness, the
restitution coefficient of the linear spring-dashpot, energy conservation."""
import math

import numpy as np

from oracle import Oracle


def _dem(L=64, walls=(0, 0, 0, 0, 0, 0), e=0.9, g=(0, 0, 0), sub=10):
    return Oracle(L, L, L, 0.6, walls=walls, gravity=g, kn=1e3, restitution=e,
                  subcycles=sub, dem=True)


def test_free_fall_is_integrated_exactly():
    """Eqs. 15-16 integrate a constant force exactly:
    x = x0 + u0 t + a t^2/2 with a = (1 - 1/rho_p) g (buoyancy, reading J)."""
    g = (0.0, 0.0, -2e-5)
    o = _dem(g=g)
    x0 = np.array([[20.0, 30.0, 40.0]])
    u0 = np.array([[1e-3, -2e-3, 5e-4]])
    o.set_particles(x0, np.array([3.0]), u=u0, density=np.array([2.5]))
    n = 37
    o.dem_only(n)
    x, u, _ = o.particles()
    a = (1.0 - 1.0 / 2.5) * np.array(g)
    t = float(n)
    assert np.allclose(x[0], x0[0] + u0[0] * t + 0.5 * a * t * t, rtol=0, atol=1e-12)
    assert np.allclose(u[0], u0[0] + a * t, rtol=0, atol=1e-15)


def test_constant_torque_spin_up_follows_verlet_with_zero_start():
    """Angular velocity under a constant torque: the first sub-step averages the
    initial zero torque with the new one (reading L), so after k sub-steps
    omega = (k - 1/2) dt T / I, I = 2/5 m r^2."""
    o = _dem()
    o.set_particles(np.array([[20.0, 20.0, 20.0]]), np.array([4.0]), density=np.array([2.0]))
    T = np.array([[0.0, 3e-3, -1e-3]])
    o.set_hydro(np.zeros((1, 3)), T)
    o.dem_only(5)
    _, _, om = o.particles()
    m = 2.0 * 4.0 / 3.0 * math.pi * 64.0
    I = 0.4 * m * 16.0
    k, dt = 50, 0.1
    assert np.allclose(om[0], (k - 0.5) * dt * T[0] / I, rtol=1e-13, atol=0)


def _collide(e, v=0.01, steps=40, sub=10):
    o = _dem(e=e, sub=sub)
    r = 6.0
    x = np.array([[20.0, 32.0, 32.0], [20.0 + 2 * r + 0.5, 32.0, 32.0]])
    u = np.array([[v, 0, 0], [-v, 0, 0]])
    o.set_particles(x, np.array([r, r]), u=u, density=np.array([2.5, 2.5]))
    o.dem_only(steps)
    return o


def test_head_on_restitution():
    """Normal spring-dashpot (Eq. 12) with d_n from the restitution
    coefficient (reading K): the relative normal velocity after the contact is
    -e times the one before, up to the sub-cycling error: about (omega dt)^2
    ~ 1% for ~33 sub-steps per contact, omega = sqrt(k_n / m_eff)."""
    for e in (0.9, 0.5):
        o = _collide(e)
        _, u, _ = o.particles()
        ratio = (u[0, 0] - u[1, 0]) / (0.01 - (-0.01))
        assert abs(ratio + e) < 0.02 * e, ratio
        # momentum is conserved exactly by the pair force
        assert abs(u[0, 0] + u[1, 0]) < 1e-16


def test_elastic_contact_conserves_energy():
    """With e = 1 there is no damping and the kinetic energy after the
    contact equals the one before, to the Verlet error (omega dt)^2 ~ 1% of
    ~33 sub-steps per contact."""
    o = _collide(1.0)
    _, u, _ = o.particles()
    assert abs((u[0, 0] ** 2 + u[1, 0] ** 2) / (2 * 0.01 ** 2) - 1.0) < 1e-2


def test_wall_bounce():
    """A wall face acts as a particle of infinite mass (m_eff = m_i)."""
    e = 0.8
    o = _dem(walls=(1, 1, 0, 0, 0, 0), e=e)
    r = 5.0
    o.set_particles(np.array([[r + 0.5, 30.0, 30.0]]), np.array([r]),
                    u=np.array([[-0.02, 0.0, 0.0]]), density=np.array([2.5]))
    o.dem_only(60)
    x, u, _ = o.particles()
    assert abs(u[0, 0] / 0.02 - e) < 0.02 * e
    assert x[0, 0] > r
