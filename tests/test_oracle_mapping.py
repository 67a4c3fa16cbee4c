"""Pins of the oracle's particle mapping (Sec. 2.3.2) against quadrature,
exact lattice counts and geometry."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
from oracle import Oracle

XG, WG = leggauss(160)


def _quad2(fn):
    """Gauss-Legendre over the unit square [-1/2, 1/2]^2."""
    x = 0.5 * XG
    w = 0.5 * WG
    X, Y = np.meshgrid(x, x, indexing="ij")
    return float(np.sum(np.outer(w, w) * fn(X, Y)))


@pytest.mark.parametrize("r", [0.9, 1.0, 2.0, 3.3, 6.0, 12.0])
def test_Va_closed_form_matches_quadrature(r):
    """Eq. 27: V_a is the integral of sqrt(r^2 - x^2 - y^2) over the unit square."""
    ref = _quad2(lambda X, Y: np.sqrt(r * r - X * X - Y * Y))
    assert abs(oracle.Va(r) - ref) < 1e-12 * ref


@pytest.mark.parametrize("r", [3.0, 5.5, 10.0])
def test_linear_approximation_exact_for_axis_aligned_cells(r):
    """Eqs. 25-26 are exact for the blue cells of Fig. 'linear_approximation':
    a cell centred on an axis through the sphere centre, cut by the surface
    only through its bottom and top faces."""
    lo = r - 0.5                   # surface at the cell centre below the top face
    hi = math.sqrt(r * r - 0.5) + 0.5  # surface at the corners above the bottom face
    for t in np.linspace(0.0, 1.0, 7):
        dist = lo + (hi - lo) * t
        exact = _quad2(lambda X, Y: np.sqrt(r * r - X * X - Y * Y) - (dist - 0.5))
        assert abs(oracle.eps_linear(dist, r) - min(max(exact, 0.0), 1.0)) < 1e-12


def _fine_lattice_count(dims, centre, r, n):
    """Brute-force count of the points ((k + 1/2)/n) of the n-times finer
    lattice inside the sphere, nearest image in a periodic box."""
    total = 0
    axes = []
    for a in range(3):
        p = (np.arange(dims[a] * n) + 0.5) / n - centre[a]
        p = np.where(p > dims[a] / 2, p - dims[a], p)
        p = np.where(p < -dims[a] / 2, p + dims[a], p)
        axes.append(p)
    X2 = axes[0] ** 2
    for z in axes[2]:
        Y2Z2 = axes[1][:, None] ** 2 + z * z
        total += int(np.count_nonzero(X2[None, :] + Y2Z2 <= r * r))
    return total


@pytest.mark.parametrize("centre,r,n", [((8.0, 8.0, 8.0), 4.0, 4),
                                        ((8.25, 7.5, 8.125), 3.5, 4),
                                        ((7.375, 8.625, 8.5), 3.0, 8),
                                        ((0.25, 15.5, 8.75), 4.25, 8)])
def test_supersampling_equals_fine_lattice_count(centre, r, n):
    """Sum over cells of eps * n^3 is the number of fine-lattice points inside
    the sphere (readings F and G) -- an exact identity for dyadic centres."""
    L = 16
    o = Oracle(L, L, L, 0.6, weighting="eps", eps_mode="supersample", eps_n=n)
    o.set_particles(np.array([centre]), np.array([r]))
    assert o.map() == 0
    p0, b0, p1, b1 = o.slots()
    assert np.all(p1 < 0)
    got = float(b0.sum()) * n ** 3
    assert got == _fine_lattice_count((L, L, L), centre, r, n)


@pytest.mark.parametrize("mode,n,tol", [("supersample", 4, 1.5e-2), ("supersample", 8, 4e-3),
                                        ("linear", 4, 5e-3)])
def test_solid_volume_of_sphere(mode, n, tol):
    """Sum of eps over all cells approximates 4/3 pi r^3 (random centres)."""
    rng = np.random.default_rng(4)
    L = 24
    for r in (3.0, 4.0, 5.5):
        for _ in range(3):
            c = 8.0 + 8.0 * rng.random(3)
            o = Oracle(L, L, L, 0.6, weighting="eps", eps_mode=mode, eps_n=n)
            o.set_particles(np.array([c]), np.array([r]))
            assert o.map() == 0
            _, b0, _, _ = o.slots()
            vol = 4.0 / 3.0 * math.pi * r ** 3
            assert abs(b0.sum() / vol - 1.0) < tol


def test_reach_and_inside_cells():
    """Cells beyond r + sqrt(3)/2 hold no slot; cells closer than
    r - sqrt(3)/2 are fully covered (eps = 1)."""
    L = 20
    c = np.array([9.3, 10.1, 10.7])
    r = 4.6
    o = Oracle(L, L, L, 0.6, weighting="eps", eps_mode="supersample", eps_n=4)
    o.set_particles(np.array([c]), np.array([r]))
    assert o.map() == 0
    p0, b0, _, _ = o.slots()
    z, y, x = np.meshgrid(np.arange(L) + 0.5, np.arange(L) + 0.5, np.arange(L) + 0.5,
                          indexing="ij")
    d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    assert np.all(p0[d >= r + math.sqrt(3) / 2] == -1)
    assert np.all(p0[d < r + math.sqrt(3) / 2 - 1e-9] == 0)
    assert np.all(b0[d <= r - math.sqrt(3) / 2] == 1.0)
    part = (d > r - math.sqrt(3) / 2) & (d < r + math.sqrt(3) / 2)
    assert np.all((b0[part] >= 0) & (b0[part] <= 1))


def test_nt_weighting_endpoints_and_order():
    """B(eps, tau) of Noble and Torczynski equals eps at 0 and 1, grows with
    eps, and for tau < 3/2 lies below eps."""
    for tau in (0.55, 0.6, 1.0):
        assert oracle.nt_weight(0.0, tau) == 0.0
        assert oracle.nt_weight(1.0, tau) == 1.0
        e = np.linspace(0.0, 1.0, 101)
        B = np.array([oracle.nt_weight(v, tau) for v in e])
        assert np.all(np.diff(B) > 0)
        assert np.all(B[1:-1] < e[1:-1])


def test_nt_weighting_closed_form_values():
    """B(eps, tau) = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)) at points
    worked by hand: B(1/2, 1) = (1/4)/(1) = 1/4, B(1/4, 0.55) =
    (1/4)(1/20)/(3/4 + 1/20) = 1/64, B(3/4, 3/2) = (3/4)/(5/4) = 3/5."""
    assert oracle.nt_weight(0.5, 1.0) == 0.25
    assert abs(oracle.nt_weight(0.25, 0.55) * 64.0 - 1.0) < 1e-14
    assert abs(oracle.nt_weight(0.75, 1.5) / 0.6 - 1.0) < 1e-14


def test_two_slots_in_index_order_and_overflow():
    """Up to two particles per cell (Sec. 3.1.1): a shared cell lists the
    lower index first; a cell within reach of three particles is an error."""
    L = 24
    o = Oracle(L, L, L, 0.6, weighting="eps", eps_mode="supersample", eps_n=4)
    x = np.array([[12.0, 12.0, 12.0], [12.0 + 2 * 3.0 + 0.6, 12.0, 12.0]])
    o.set_particles(x, np.array([3.0, 3.0]))
    assert o.map() == 0
    p0, b0, p1, b1 = o.slots()
    both = p1 >= 0
    assert both.sum() > 0 and np.all(p0[both] == 0) and np.all(p1[both] == 1)
    # three spheres touching one point
    c = np.array([12.0, 12.0, 12.0])
    x3 = np.array([c + 2.8 * np.array(v) for v in
                   ((1, 0, 0), (-0.5, 0.866, 0), (-0.5, -0.866, 0))])
    o.set_particles(x3, np.array([3.0, 3.0, 3.0]))
    assert o.map() == -2


def test_walls_clip_the_mapping():
    """With walls on the x faces the mapping does not wrap around x."""
    o = Oracle(16, 16, 16, 0.6, walls=(1, 1, 0, 0, 0, 0), weighting="eps",
               eps_mode="supersample", eps_n=4)
    o.set_particles(np.array([[1.5, 8.0, 8.0]]), np.array([3.0]))
    assert o.map() == 0
    p0, _, _, _ = o.slots()
    assert np.all(p0[:, :, 8:] == -1)
    assert np.any(p0[:, :, 0] == 0)
