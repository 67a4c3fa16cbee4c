"""The seeded workloads themselves (no GPU): counts, surface gaps, wall
clearance and solid fractions of the placements the bench and the tests use."""
import math

import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs


def _min_gap(w):
    x, r = w.particles["x"], w.particles["r"]
    dims = np.array([w.nx, w.ny, w.nz], float)
    per = np.array([not w.walls[0], not w.walls[2], not w.walls[4]])
    gap = np.inf
    for i in range(len(r)):
        d = x - x[i]
        d[:, per] -= dims[per] * np.round(d[:, per] / dims[per])
        dist = np.sqrt((d * d).sum(axis=1)) - r - r[i]
        dist[i] = np.inf
        gap = min(gap, float(dist.min()))
    return gap


@pytest.mark.parametrize("case,count", [("dilute", 627), ("dense", 8073)])
def test_fluidized_bed_stand_in(case, count):
    w = inputs.bed(case)
    x, r = w.particles["x"], w.particles["r"]
    assert (w.nx, w.ny, w.nz) == (500, 200, 800) and len(r) == count
    assert np.all(r == 10.0) and np.all(w.particles["density"] == 1.1)
    # inside the side walls with room for the sphere, any height (periodic)
    assert np.all(x[:, 0] >= r) and np.all(x[:, 0] <= w.nx - r)
    assert np.all(x[:, 1] >= r) and np.all(x[:, 1] <= w.ny - r)
    assert np.all((x[:, 2] >= 0) & (x[:, 2] < w.nz))
    assert _min_gap(w) >= 1.0 - 1e-9          # surface gap of the placements
    phi = float((4.0 / 3.0 * math.pi * r ** 3).sum() / w.cells)
    assert phi == pytest.approx(count * 4.0 / 3.0 * math.pi * 1000.0 / 8e7)
    if case == "dense":                       # a packed bed from the bottom
        assert x[:, 2].max() < 0.8 * w.nz


def test_settling_and_channel_placements():
    w = inputs.settle128()
    assert len(w.particles["r"]) == 400 and _min_gap(w) >= 1.0
    w = inputs.settle512(nx=128, ny=128, nz=128)
    r = w.particles["r"]
    assert r.min() >= 3.0 and r.max() <= 6.0 and _min_gap(w) >= 1.0
    phi = float((4.0 / 3.0 * math.pi * r ** 3).sum() / w.cells)
    assert 0.15 <= phi < 0.15 + 4.0 / 3.0 * math.pi * 6.0 ** 3 / w.cells
