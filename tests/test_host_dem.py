"""The host-core DEM of the hybrid coupling (psm_dem_step_host, the DEM of
psm_step_host_dem) against the oracle's DEM (Sec. 2.2, Eqs. 12-16, with the
tangential contact history carried over the steps) with
the same hydrodynamic forces: contacts between spheres and with walls, a
sphere wrapping around periodic faces, a fixed sphere; thread-count
independence; argument and skin errors.  No GPU: the library's host code runs
here."""
import numpy as np
import pytest

import oracle
from paper_2303_11811_gb300 import build, capi, inputs

SHAPE = (37, 24, 20)
WALLS = (1, 1, 0, 0, 0, 0)
KN, E, SUB = 100.0, 0.8, 10
G = (0.0, 0.0, -3e-5)


@pytest.fixture(scope="module", autouse=True)
def _libs():
    build.build()
    oracle.build()


def scene():
    # spheres 0 and 1 overlap by 0.1, sphere 2 presses on the +x wall and
    # wraps around the z faces, sphere 3 is fixed and touched by sphere 1
    x = np.array([[6.0, 7.5, 9.2], [13.8, 7.6, 9.3], [33.95, 16.7, 0.4], [13.8, 15.0, 9.3]])
    r = np.array([4.3, 3.6, 3.1, 3.8])
    u = np.array([[-2e-3, 1e-3, 0.0], [-1e-3, 0.0, 1e-3], [5e-4, -1e-3, -2e-3], [0.0, 0.0, 0.0]])
    om = inputs.random_velocities(4, 1e-3, 4)
    om[3] = 0.0
    dens = np.array([2.5, 2.0, 3.0, 2.0])
    fixed = np.array([0, 0, 0, 1], dtype=np.uint8)
    return x, r, u, om, dens, fixed


def host_state(x, r, u, om, dens, fixed):
    vol = 4.0 / 3.0 * np.pi * r ** 3
    m = dens * vol
    Fo = np.where(fixed[:, None] == 0, (m - vol)[:, None] * np.array(G)[None, :], 0.0)
    # copies: the step advances them in place
    return (np.array(x, dtype=np.float64), np.array(u, dtype=np.float64),
            np.array(om, dtype=np.float64), np.array(Fo, dtype=np.float64), np.zeros_like(Fo))


def hydro(n, k):
    """Hydrodynamic force and torque of step k (seeded, of the size the
    fluid gives these spheres)."""
    rng = np.random.default_rng(1000 + k)
    return rng.normal(0.0, 2e-3, (n, 3)), rng.normal(0.0, 5e-3, (n, 3))


def test_host_dem_matches_the_oracle_dem():
    x, r, u, om, dens, fixed = scene()
    o = oracle.Oracle(*SHAPE, 0.6, relax="srt", walls=WALLS, gravity=G, kn=KN, restitution=E,
                      subcycles=SUB, dem=True)
    o.set_particles(x, r, u=u, omega=om, density=dens, fixed=fixed)
    hx, hu, ho, Fo, To = host_state(x, r, u, om, dens, fixed)
    n = r.size
    hist = capi.dem_history(n)  # the tangential contact history, carried over the steps
    most = 0
    for k in range(30):
        Fh, Th = hydro(n, k)
        o.set_hydro(Fh.ravel(), Th.ravel())
        o.dem_only(1)
        capi.dem_step_host(SHAPE, WALLS, hx, hu, ho, Fo, To, Fh, Th, r, dens, fixed=fixed,
                           kn=KN, restitution=E, subcycles=SUB, gravity=G, threads=2,
                           history=hist)
        most = max(most, int(hist[0].sum()))
    assert most > 0  # contacts with tangential history were carried over steps
    xo, uo, wo = o.particles()
    # nearest image: sphere 2 crosses the periodic z faces
    d = hx - xo
    for a, dim in enumerate(SHAPE):
        if not WALLS[2 * a]:
            d[:, a] -= dim * np.round(d[:, a] / dim)
    assert np.max(np.abs(d)) < 1e-12
    assert np.max(np.abs(hu - uo)) < 1e-13 and np.max(np.abs(ho - wo)) < 1e-13
    # the contacts acted: sphere 0 and 1 were pushed apart, 3 stayed put
    assert hx[1, 0] - hx[0, 0] > 13.8 - 6.0
    assert np.array_equal(hx[3], x[3]) and np.array_equal(hu[3], u[3])


def test_thread_count_does_not_change_the_result():
    x, r, u, om, dens, fixed = scene()
    runs = []
    for threads in (1, 3, 4):
        hx, hu, ho, Fo, To = host_state(x, r, u, om, dens, fixed)
        hist = capi.dem_history(r.size)
        for k in range(5):
            Fh, Th = hydro(r.size, k)
            capi.dem_step_host(SHAPE, WALLS, hx, hu, ho, Fo, To, Fh, Th, r, dens, fixed=fixed,
                               kn=KN, restitution=E, subcycles=SUB, gravity=G, threads=threads,
                               history=hist)
        runs.append(np.concatenate([hx, hu, ho, Fo, To, hist[2].reshape(-1, 3)]))
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])


def test_free_fall_without_contacts_is_exact():
    """One sphere far from everything, no hydrodynamic force: velocity
    Verlet integrates constant (m - V) g exactly up to rounding."""
    r = np.array([3.0])
    dens = np.array([2.0])
    x = np.array([[18.0, 12.0, 10.0]])
    hx, hu, ho, Fo, To = host_state(x, r, np.zeros((1, 3)), np.zeros((1, 3)), dens,
                                    np.zeros(1, np.uint8))
    steps = 40
    for _ in range(steps):
        capi.dem_step_host(SHAPE, WALLS, hx, hu, ho, Fo, To, np.zeros((1, 3)), np.zeros((1, 3)),
                           r, dens, kn=KN, restitution=E, subcycles=SUB, gravity=G)
    g_eff = (dens[0] - 1.0) / dens[0] * G[2]
    z = 10.0 + 0.5 * g_eff * steps ** 2
    z = (z % SHAPE[2] + SHAPE[2]) % SHAPE[2]
    assert abs(hx[0, 2] - z) < 1e-12 and abs(hu[0, 2] - g_eff * steps) < 1e-15


def test_arguments_and_skin_are_checked():
    x, r, u, om, dens, fixed = scene()
    hx, hu, ho, Fo, To = host_state(x, r, u, om, dens, fixed)
    Fh, Th = hydro(r.size, 0)
    with pytest.raises(capi.PsmError) as e:  # one wall face of an axis only
        capi.dem_step_host(SHAPE, (1, 0, 0, 0, 0, 0), hx, hu, ho, Fo, To, Fh, Th, r, dens)
    assert e.value.status == capi.PSM_ERR_ARG
    with pytest.raises(capi.PsmError) as e:
        capi.dem_step_host(SHAPE, WALLS, hx, hu, ho, Fo, To, Fh, Th, r, dens, restitution=0.0)
    assert e.value.status == capi.PSM_ERR_ARG
    assert np.array_equal(hx, x)  # nothing changed
    fast = hu.copy()
    fast[0] = (0.8, 0.0, 0.0)  # 0.8 cells per step: beyond half the 1-cell skin
    with pytest.raises(capi.PsmError) as e:
        capi.dem_step_host(SHAPE, WALLS, hx, fast, ho, Fo, To, Fh, Th, r, dens, fixed=fixed)
    assert e.value.status == capi.PSM_ERR_STATE
    # no particles: nothing to do; zero sub-cycles or stiffness: refused
    e0 = np.zeros((0, 3))
    capi.dem_step_host(SHAPE, WALLS, e0.copy(), e0.copy(), e0.copy(), e0.copy(), e0.copy(), e0,
                       e0, np.zeros(0), np.zeros(0))
    for bad in (dict(subcycles=0), dict(kn=0.0)):
        with pytest.raises(capi.PsmError) as e:
            capi.dem_step_host(SHAPE, WALLS, hx, hu, ho, Fo, To, Fh, Th, r, dens, **bad)
        assert e.value.status == capi.PSM_ERR_ARG
