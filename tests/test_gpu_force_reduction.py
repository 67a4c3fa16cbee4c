"""The per-particle force and torque reduction (Eqs. 21-22) against FP64 sums
of the engine's own per-slot forces (psm_get_slot_forces), taken on the host.

- FP64 form: the fixed-order device reduction equals the sums to 1e-13 of the
  sum of the terms' magnitudes (FP64 rounding of a few hundred terms).
- Double-float form: the same bound (the reduction runs in double-float).
- FP32 form: the slot forces are FP32 numbers, summed on the device as
  compensated FP32 pairs (about 48 bits, an error-free two-sum per term):
  within 2^-40 of the magnitudes' sum of the exact FP64 sums.  Its torque
  arms and arm products are FP32 (three roundings of 2^-24 per term):
  within 2^-21 of the sum of |arm| |F| of the exact FP64 torque sums.
Checked at 128^3 with moving, touching spheres in all three forms, and at
the full 512x512x1024 settling box in the FP32 AA form the bench times.
"""
import math

import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    assert torch.cuda.is_available()
    from paper_2303_11811_gb300 import build, capi as c
    build.build()
    return c


def _exact_sums(e, w, xs):
    """FP64 sums over each particle's slots of F_c and of d x F_c, d the
    nearest-image offset of the cell centre from the particle position xs the
    last step's mapping used, with the magnitude sums that bound their
    rounding."""
    p0, p1, F0, F1 = e.slot_forces()
    n = xs.shape[0]
    dims = np.array([w.nx, w.ny, w.nz], dtype=np.float64)
    per = np.array([not w.walls[0], not w.walls[2], not w.walls[4]])
    z, y, x = np.nonzero(p0 >= 0)
    cells = np.stack([x, y, z], axis=1).astype(np.float64) + 0.5
    pids, forces, where = [p0[z, y, x]], [F0[z, y, x]], [cells]
    two = p1[z, y, x] >= 0
    pids.append(p1[z, y, x][two])
    forces.append(F1[z, y, x][two])
    where.append(cells[two])
    pid = np.concatenate(pids)
    F = np.concatenate(forces)
    c = np.concatenate(where)
    d = c - xs[pid]
    for a in range(3):
        if per[a]:
            d[:, a] -= dims[a] * np.round(d[:, a] / dims[a])
    T = np.cross(d, F)
    order = np.argsort(pid, kind="stable")
    pid, F, T, d = pid[order], F[order], T[order], d[order]
    starts = np.searchsorted(pid, np.arange(n))
    has = np.bincount(pid, minlength=n) > 0
    def seg(v):
        out = np.zeros((n,) + v.shape[1:])
        out[has] = np.add.reduceat(v, starts[has], axis=0)
        return out
    armF = np.abs(d[:, [1, 2, 0]] * F[:, [2, 0, 1]]) + np.abs(d[:, [2, 0, 1]] * F[:, [1, 2, 0]])
    return seg(F), seg(T), seg(np.abs(F)), seg(armF), has


def _check(e, w, precision, xs):
    Fx, Tx, magF, magT, has = _exact_sums(e, w, xs)
    Fg, Tg = e.force_torque()
    if precision == "fp32":
        tf, tt = 2.0 ** -40, 2.0 ** -21
    else:
        tf, tt = 1e-13, 1e-13
    errF = np.abs(Fg - Fx)[has]
    errT = np.abs(Tg - Tx)[has]
    assert np.all(errF <= tf * magF[has] + 1e-300), float(np.max(errF / (magF[has] + 1e-300)))
    assert np.all(errT <= tt * magT[has] + 1e-300), float(np.max(errT / (magT[has] + 1e-300)))
    return float(np.max(errF / magF[has])), float(np.max(errT / magT[has]))


@pytest.mark.parametrize("precision,streaming", [("fp64", "pull"), ("fp32", "aa"),
                                                 ("df64", "pull")])
def test_reduction_matches_fp64_sums_of_slot_forces(capi, precision, streaming):
    w = inputs.settle128()
    e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, gravity=w.gravity,
                    weighting=w.weighting, eps_mode=w.eps_mode, eps_n=w.eps_n, dem=True,
                    kn=w.kn, restitution=w.restitution, precision=precision,
                    streaming=streaming)
    p = w.particles
    e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    e.step(6)
    xs, _, _ = e.particles()  # the positions the next step maps (its DEM moves them after)
    e.step(1)
    ef, et = _check(e, w, precision, xs)
    print(f"{precision}: force {ef:.2e}, torque {et:.2e} of the magnitudes' sums")
    e.close()


def test_fp32_reduction_full_size_settling_box(capi):
    """The 512x512x1024 box with 94,692 settling spheres, FP32 AA, after a
    few steps: every particle's force and torque within the FP32 bounds of
    the FP64 sums of its slot forces (57M slots)."""
    import torch
    w = inputs.settle512()
    w.eps_n = 8
    e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, gravity=w.gravity,
                    weighting=w.weighting, eps_mode="supersample", eps_n=8, dem=True,
                    kn=w.kn, restitution=w.restitution, precision="fp32", streaming="aa")
    p = w.particles
    e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    e.step(2)
    xs, _, _ = e.particles()
    e.step(1)
    ef, et = _check(e, w, "fp32", xs)
    print(f"settle512 fp32: force {ef:.2e}, torque {et:.2e} of the magnitudes' sums")
    e.close()
    torch.cuda.empty_cache()
