"""Sampled single-cell checks against the oracle on a box around the cell
(shared by the full-size GPU tests and the CPU test of the method).

For a cell c the oracle runs one step on a box around c (16 cells along a
periodic axis or along z with open faces, the whole extent along an axis
with walls), filled with the post-collision PDFs of that box and holding the
spheres within reach of c, shifted by an integer, so that every cell-centre
offset is the same number as in the full field up to the rounding of the
shifted centre (the shift is exact unless it moves a centre across a power
of two).  Its body force is the full field's fluid force density of that
step, with no gravity and no DEM, so the collision of c sees the same
inputs.  The box wraps periodically at its own faces, which changes
cells next to those faces only; c sits 8 cells from them.
"""
import math
import os

import numpy as np

from oracle import Oracle

BOX = 16
REST = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def sample_cells(w, count, seed):
    """Cells on sphere surfaces (covered, partial), inside spheres and at
    random, as (x, y, z) triples."""
    rng = np.random.default_rng(seed)
    X, R = w.particles["x"], w.particles["r"]
    dims = np.array([w.nx, w.ny, w.nz])
    per = np.array([not w.walls[0], not w.walls[2], not w.walls[4]])
    cells = []
    for k in range(count):
        if k % 4 == 3:
            c = rng.integers(0, dims)
        else:
            i = rng.integers(0, R.size)
            v = rng.normal(size=3)
            s = R[i] * (0.5, 0.97, 1.08)[k % 4] if k % 4 < 3 else 0.0
            c = np.floor(X[i] + s * v / np.linalg.norm(v)).astype(int)
        c = np.where(per, np.mod(c, dims), np.clip(c, 0, dims - 1))
        cells.append(tuple(int(v) for v in c))
    return cells


def _open_z(w):
    return max(w.walls[4], w.walls[5]) >= 2 and w.nz > BOX


def box(w, c):
    """Origin and extent of the box around cell c: 16 cells along a periodic
    axis; along the z axis with open faces 16 cells clamped to the domain
    (c at least 7 cells from an end of the box that is not a domain face);
    the whole extent along any other axis with walls."""
    dims = (w.nx, w.ny, w.nz)
    walls = (w.walls[0], w.walls[2], w.walls[4])
    o, ext = [], []
    for a in range(3):
        if not walls[a]:
            o.append(c[a] - BOX // 2)
            ext.append(BOX)
        elif a == 2 and _open_z(w):
            o.append(min(max(c[2] - BOX // 2, 0), dims[2] - BOX))
            ext.append(BOX)
        else:
            o.append(0)
            ext.append(dims[a])
    return tuple(o), tuple(ext)


def box_faces(w, o):
    """Face types of the box: the domain's, with a wall where the box ends
    inside the domain along z (c is far enough from it for one step)."""
    if not _open_z(w):
        return tuple(int(w.walls[2 * a]) for a in range(3) for _ in range(2))
    zlo = w.walls[4] if o[2] == 0 else 1
    zhi = w.walls[5] if o[2] + BOX == w.nz else 1
    return (int(w.walls[0]), int(w.walls[1]), int(w.walls[2]), int(w.walls[3]), int(zlo),
            int(zhi))


def oracle_cell(w, c, pre, fext, X, R, U, OM, dens):
    """The oracle's post-collision PDFs of cell c after one step of the box."""
    dims = np.array([w.nx, w.ny, w.nz], dtype=float)
    walls = (w.walls[0], w.walls[2], w.walls[4])
    o, ext = box(w, c)
    d = (np.array(c) + 0.5) - X
    for a in range(3):
        if not walls[a]:
            d[:, a] -= dims[a] * np.round(d[:, a] / dims[a])
    sel = np.nonzero((d * d).sum(axis=1) < (R + math.sqrt(3.0) / 2) ** 2)[0]
    assert sel.size <= 2
    xs = X[sel] - np.array(o, dtype=float)  # integer shifts
    for a in range(3):
        if not walls[a]:
            xs[:, a] -= dims[a] * np.round((xs[:, a] - BOX / 2) / dims[a])
    orc = Oracle(ext[0], ext[1], ext[2], w.tau, relax=w.relax, walls=box_faces(w, o),
                 fbody=tuple(float(v) for v in fext), weighting=w.weighting,
                 eps_mode=w.eps_mode, eps_n=w.eps_n, bc_velocity=w.bc_velocity,
                 bc_density=w.bc_density)
    orc.set_threads(os.cpu_count() or 1)  # results do not depend on the thread count
    orc.set_pdfs(pre.ravel())
    if sel.size:
        orc.set_particles(xs, R[sel], u=U[sel], omega=OM[sel], density=dens[sel],
                          fixed=np.ones(sel.size, np.uint8))
    orc.step(1)
    f = orc.pdfs()
    return f[:, c[2] - o[2], c[1] - o[1], c[0] - o[0]]


