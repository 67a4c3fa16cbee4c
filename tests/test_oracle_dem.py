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


def _damping(meff, kn, e):
    le = math.log(e)
    return -2.0 * le * math.sqrt(meff * kn) / math.sqrt(math.pi ** 2 + le * le)


def test_tangential_history_of_a_spinning_contact():
    """Eqs. 13-14 (reading W) at a contact whose surfaces slide at a constant
    rate: two fixed, overlapping spheres, sphere 0 spinning.  The relative
    surface velocity at the contact point is U_t = omega_0 x a_0 with the arm
    a_0 = -(r_0 - delta/2) n, constant, so after S sub-steps the history is
    S dt_p U_t and the contact force on sphere 0 is k_n delta n - k_t S dt_p U_t
    - d_t U_t, with k_t = 2/7 k_n, d_t = 2/7 d_n; its torque is a_0 x F_t;
    sphere 1 gets -F and the torque a_1 x (-F_t), a_1 = (r_1 - delta/2) n."""
    kn, e, sub = 1e3, 0.9, 10
    o = _dem(e=e, sub=sub)
    x = np.array([[20.0, 21.0, 22.0], [26.7, 23.1, 21.4]])
    r = np.array([3.5, 3.6])
    rho = np.array([2.5, 1.8])
    om = np.array([[1e-3, -2e-3, 3e-3], [0.0, 0.0, 0.0]])
    o.set_particles(x, r, omega=om, density=rho, fixed=np.ones(2, np.uint8))
    steps = 3
    o.dem_only(steps)
    F, T = o.contact()
    d = x[0] - x[1]
    dist = np.linalg.norm(d)
    n = d / dist
    delta = r.sum() - dist
    assert delta > 0
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    dn = _damping(m[0] * m[1] / m.sum(), kn, e)
    a0 = -(r[0] - delta / 2) * n
    a1 = (r[1] - delta / 2) * n
    Ut = np.cross(om[0], a0)
    S = steps * sub
    Ft = -(2.0 / 7.0) * kn * (S / sub) * Ut - (2.0 / 7.0) * dn * Ut
    F0 = kn * delta * n + Ft
    assert np.max(np.abs(F[0] - F0)) < 1e-12 * np.max(np.abs(F0))
    assert np.max(np.abs(F[1] + F0)) < 1e-12 * np.max(np.abs(F0))
    assert np.max(np.abs(T[0] - np.cross(a0, Ft))) < 1e-12 * np.max(np.abs(np.cross(a0, Ft)))
    assert np.max(np.abs(T[1] - np.cross(a1, -Ft))) < 1e-12 * np.max(np.abs(np.cross(a1, Ft)))
    # the spring part grows with the slid distance: twice the steps, about
    # twice the history term
    o.dem_only(steps)
    F2, _ = o.contact()
    Ft2 = F2[0] - kn * delta * n
    assert np.allclose(Ft2, -(2.0 / 7.0) * kn * 2 * steps * Ut - (2.0 / 7.0) * dn * Ut,
                       rtol=1e-12, atol=0)


def test_tangential_contact_needs_sliding_and_balances_torques():
    """A head-on collision without spin has no tangential motion: the model
    with Eqs. 13-14 gives the normal-only result bit for bit.  In an oblique
    collision with spin the contact forces and torques of a pair balance about
    any point (the arms meet at the contact point): sum_i (x_i x F_i + T_i) = 0
    at each sub-step, and the linear momentum is conserved."""
    res = []
    for kt in (0.0, 2.0 / 7.0):
        o = Oracle(64, 64, 64, 0.6, kn=1e3, restitution=0.8, subcycles=10, dem=True,
                   kt_ratio=kt)
        o.set_particles(np.array([[20.0, 30.0, 30.0], [27.2, 30.0, 30.0]]), np.array([3.5, 3.5]),
                        u=np.array([[2e-2, 0, 0], [-2e-2, 0, 0]]), density=np.array([2.5, 2.5]))
        o.dem_only(6)
        res.append(o.particles())
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    o = Oracle(64, 64, 64, 0.6, kn=1e3, restitution=0.8, subcycles=10, dem=True)
    x = np.array([[20.0, 30.0, 30.0], [26.5, 32.1, 29.0]])
    r = np.array([3.5, 3.2])
    u = np.array([[2e-2, 4e-3, -1e-3], [-2e-2, -3e-3, 2e-3]])
    om = np.array([[1e-3, -4e-3, 2e-3], [3e-3, 1e-3, -2e-3]])
    rho = np.array([2.5, 2.0])
    m = rho * 4.0 / 3.0 * math.pi * r ** 3
    o.set_particles(x, r, u=u, omega=om, density=rho)
    P0 = (m[:, None] * u).sum(axis=0)
    touched = 0
    for _ in range(12):
        o.dem_only(1)
        F, T = o.contact()
        xp, up, wp = o.particles()
        if np.max(np.abs(F)) > 0:
            touched += 1
            tot = np.cross(xp, F).sum(axis=0) + T.sum(axis=0)
            scale = np.max(np.abs(np.cross(xp, F)))
            assert np.max(np.abs(tot)) < 1e-12 * scale
            assert np.max(np.abs(T)) > 1e-6 * np.max(np.abs(F))  # friction torques act
    assert touched >= 1
    assert np.max(np.abs((m[:, None] * up).sum(axis=0) - P0)) < 1e-14 * np.abs(m[:, None] * u).sum()
