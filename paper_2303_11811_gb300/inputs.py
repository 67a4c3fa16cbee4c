"""Seeded synthetic inputs shared by the tests, the bench and both of their legs.

This module holds no arithmetic of the method: it only draws particle
placements, random perturbations and initial network weights from seeded
NumPy generators, and names the workloads with their sizes.  Both the CUDA
path and the oracle receive what it returns as plain arrays.

Workloads (stand-ins for the paper's fluidized bed, Sec. 4.1, whose initial
particle bed is not public):

* ``sphere32``   32^3 periodic box, one fixed sphere r = 4 at the centre,
  SRT tau = 0.6, body force 1e-6 in x, 4^3 sub-division sampling, FP64.
* ``settle128``  128^3 periodic box, 400 spheres r = 6 placed by random
  sequential addition (surface gap >= 1), density ratio 2.5, gravity 2e-5 in
  -z, TRT (Lambda = 3/16) tau = 0.55, spring-dashpot DEM (k_n = 1e3, e = 0.9).
* ``channel``    256x256x512 channel, walls at the x faces, periodic y/z,
  12,817 fixed spheres r = 5 at solid fraction 0.20, TRT tau = 0.55, body
  force 1e-5 along z.
* ``settle512``  512x512x1024 periodic box, polydisperse spheres r in [3, 6]
  at solid fraction 0.15, settling under gravity 2e-5, density ratio 2.5.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 20230321


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    relax: str                     # "srt" | "trt"
    walls: tuple = (0, 0, 0, 0, 0, 0)
    fbody: tuple = (0.0, 0.0, 0.0)
    gravity: tuple = (0.0, 0.0, 0.0)
    weighting: str = "nt"          # "eps" | "nt"
    eps_mode: str = "supersample"  # "supersample" | "linear" | "mlp"
    eps_n: int = 4
    kn: float = 1e3
    restitution: float = 0.9
    subcycles: int = 10
    dem: bool = False
    density: float = 2.5
    steps: int = 1000
    bc_velocity: tuple = (0.0, 0.0, 0.0)  # fluid velocity of an inflow face
    bc_density: float = 1.0               # fluid density of an outflow face
    particles: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def rsa_spheres(dims, walls, radii, gap, seed, max_tries=100000):
    """Random sequential addition of non-overlapping spheres.

    ``radii`` is the list of radii in placement order; each sphere is drawn
    uniformly in the box (kept r away from wall faces) and accepted when its
    surface is at least ``gap`` from every sphere already placed (nearest image
    along periodic axes).  Returns centres (n x 3).  The candidates come from
    one generator stream, three uniforms per try; the overlap test runs on
    plain floats over a bucket grid of edge >= 2 r_max + gap.
    """
    rng = np.random.default_rng(seed)
    dims = [float(v) for v in dims]
    per = [not walls[0], not walls[2], not walls[4]]
    radii = np.asarray(radii, dtype=np.float64)
    rmax = float(radii.max()) if radii.size else 1.0
    h = 2.0 * rmax + gap
    ncell = [max(1, int(np.floor(dims[a] / h))) for a in range(3)]
    csize = [dims[a] / ncell[a] for a in range(3)]
    half = [0.5 * dims[a] for a in range(3)]
    # neighbour buckets per axis offset, wrapped or clipped, without repeats
    def around(c, a):
        out = []
        for o in (-1, 0, 1):
            k = c + o
            if k < 0 or k >= ncell[a]:
                if not per[a]:
                    continue
                k %= ncell[a]
            if k not in out:
                out.append(k)
        return out
    grid: dict = {}
    pos = []          # accepted centres as float triples
    out = np.zeros((radii.size, 3))
    for i, r in enumerate(radii.tolist()):
        lo = [0.0 if per[a] else r for a in range(3)]
        hi = [dims[a] if per[a] else dims[a] - r for a in range(3)]
        for _ in range(max_tries):
            u = rng.random(3)
            p = [lo[a] + (hi[a] - lo[a]) * float(u[a]) for a in range(3)]
            c = [min(int(p[a] // csize[a]), ncell[a] - 1) for a in range(3)]
            ok = True
            for kz in around(c[2], 2):
                for ky in around(c[1], 1):
                    for kx in around(c[0], 0):
                        for j in grid.get((kx, ky, kz), ()):
                            q = pos[j]
                            d2 = 0.0
                            for a in range(3):
                                d = p[a] - q[a]
                                if per[a]:
                                    if d > half[a]:
                                        d -= dims[a]
                                    elif d < -half[a]:
                                        d += dims[a]
                                d2 += d * d
                            s = r + radii[j] + gap
                            if d2 < s * s:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                out[i] = p
                pos.append(p)
                grid.setdefault(tuple(c), []).append(i)
                break
        else:
            raise RuntimeError(f"random sequential addition stalled at sphere {i}")
    return out


def sphere32() -> Workload:
    w = Workload("sphere32", 32, 32, 32, tau=0.6, relax="srt", fbody=(1e-6, 0.0, 0.0),
                 weighting="nt", eps_mode="supersample", eps_n=4, steps=1000)
    w.particles = dict(x=np.array([[16.0, 16.0, 16.0]]), r=np.array([4.0]),
                       density=np.array([1.0]), fixed=np.array([1], np.uint8))
    return w


def settle128(n=128, count=400, radius=6.0, seed=DEFAULT_SEED) -> Workload:
    w = Workload("settle128", n, n, n, tau=0.55, relax="trt", gravity=(0.0, 0.0, -2e-5),
                 weighting="nt", eps_mode="supersample", eps_n=4, dem=True,
                 density=2.5, steps=2000)
    r = np.full(count, radius)
    x = rsa_spheres((n, n, n), w.walls, r, 1.0, seed)
    w.particles = dict(x=x, r=r, density=np.full(count, 2.5),
                       fixed=np.zeros(count, np.uint8))
    return w


def channel(nx=256, ny=256, nz=512, phi=0.20, radius=5.0, seed=DEFAULT_SEED,
            eps_mode="supersample", eps_n=4) -> Workload:
    w = Workload("channel", nx, ny, nz, tau=0.55, relax="trt", walls=(1, 1, 0, 0, 0, 0),
                 fbody=(0.0, 0.0, 1e-5), weighting="nt", eps_mode=eps_mode, eps_n=eps_n,
                 dem=False, steps=5000)
    count = int(round(phi * nx * ny * nz / (4.0 / 3.0 * math.pi * radius ** 3)))
    r = np.full(count, radius)
    x = rsa_spheres((nx, ny, nz), w.walls, r, 1.0, seed)
    w.particles = dict(x=x, r=r, density=np.full(count, 2.5),
                       fixed=np.ones(count, np.uint8))
    return w


def settle512(nx=512, ny=512, nz=1024, phi=0.15, rmin=3.0, rmax=6.0,
              seed=DEFAULT_SEED) -> Workload:
    w = Workload("settle512", nx, ny, nz, tau=0.55, relax="trt", gravity=(0.0, 0.0, -2e-5),
                 weighting="nt", eps_mode="supersample", eps_n=4, dem=True, steps=1000)
    rng = np.random.default_rng(seed + 1)
    target = phi * nx * ny * nz
    radii = []
    vol = 0.0
    while vol < target:
        r = rmin + (rmax - rmin) * rng.random()
        radii.append(r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    r = np.array(radii)
    x = rsa_spheres((nx, ny, nz), w.walls, r, 1.0, seed)
    w.particles = dict(x=x, r=r, density=np.full(r.size, 2.5),
                       fixed=np.zeros(r.size, np.uint8))
    return w


def bed(case="dilute", nx=500, ny=200, nz=800, radius=10.0, seed=DEFAULT_SEED) -> Workload:
    """Stand-in for the paper's fluidized bed (Sec. 4.1): 500 x 200 x 800
    cells, no-slip walls on the four side faces, spheres of radius 10 (20
    cells per diameter), particle/fluid density ratio 1.1, ten DEM
    sub-cycles, SRT, the linear approximation of Eqs. 25-27 with B = eps.
    A velocity inflow at the bottom face and a pressure outflow (density 1)
    at the top, as in the paper; the inflow velocity 8.33e-4 gives the
    paper's particle Reynolds number 1.0 (U d / nu, nu = (tau - 1/2)/3 at
    tau = 0.55, d = 20).  Gravity 2.75e-5 (Galileo number about 8.9).  The
    faces are walls for the particles.  ``dilute``: 627 spheres by random
    sequential addition over the whole box; ``dense``: 8,073 spheres in
    hexagonal close-packed layers from the bottom (surface gap 1), a packed
    bed."""
    tau, d = 0.55, 2.0 * radius
    u_in = ((tau - 0.5) / 3.0) / d  # particle Reynolds number 1
    w = Workload(f"bed_{case}", nx, ny, nz, tau=tau, relax="srt", walls=(1, 1, 1, 1, 2, 3),
                 gravity=(0.0, 0.0, -2.75e-5), weighting="eps", eps_mode="linear", eps_n=4,
                 dem=True, density=1.1, steps=500, bc_velocity=(0.0, 0.0, u_in),
                 bc_density=1.0)
    if case == "dilute":
        count = 627
        r = np.full(count, radius)
        x = rsa_spheres((nx, ny, nz), w.walls, r, 1.0, seed)
    else:
        count = 8073
        d = 2.0 * radius + 1.0               # centre spacing: surface gap 1
        dy, dz = d * math.sqrt(3.0) / 2.0, d * math.sqrt(2.0 / 3.0)
        pts = []
        layer = 0
        while len(pts) < count:
            z = radius + 0.5 + layer * dz
            if z > nz - radius:
                raise RuntimeError("packed bed does not fit")
            sx = 0.5 * d if layer % 3 == 1 else 0.0
            sy = dy / 3.0 * (layer % 3)
            j = 0
            while True:
                y = radius + 0.5 + sy + j * dy
                if y > ny - radius - 0.5:
                    break
                i = 0
                while True:
                    xx = radius + 0.5 + sx + (0.5 * d if j % 2 else 0.0) + i * d
                    if xx > nx - radius - 0.5:
                        break
                    pts.append((xx, y, z))
                    i += 1
                j += 1
            layer += 1
        x = np.array(pts[:count])
        r = np.full(count, radius)
    w.particles = dict(x=x, r=r, density=np.full(count, 1.1), fixed=np.zeros(count, np.uint8))
    return w


def slab(w: Workload, z0: int, nz: int) -> Workload:
    """The cells z0 .. z0+nz-1 of a workload that is periodic in z, as a
    periodic box of its own: the spheres whose centres lie at least r + 1/2
    inside the slab's faces, shifted down by z0 (an integer, so every
    cell-centre offset is the same number as in the full box).  Two spheres
    next to opposite faces then keep the placement gap of 1 across the new
    periodic wrap.  A bounded sample of a workload too large for a quick CPU
    run."""
    assert not w.walls[4] and 0 <= z0 and z0 + nz <= w.nz
    x, r = w.particles["x"], w.particles["r"]
    zr = x[:, 2] - z0
    keep = (zr >= r + 0.5) & (zr <= nz - r - 0.5)
    out = Workload(f"{w.name}_slab{nz}", w.nx, w.ny, nz, tau=w.tau, relax=w.relax,
                   walls=w.walls, fbody=w.fbody, gravity=w.gravity, weighting=w.weighting,
                   eps_mode=w.eps_mode, eps_n=w.eps_n, kn=w.kn, restitution=w.restitution,
                   subcycles=w.subcycles, dem=w.dem, density=w.density, steps=w.steps)
    xs = x[keep].copy()
    xs[:, 2] -= z0
    out.particles = {k: (xs if k == "x" else np.asarray(v)[keep].copy())
                     for k, v in w.particles.items()}
    return out


def noise(shape, scale, seed):
    """Uniform noise in [-scale, scale) of the given shape."""
    rng = np.random.default_rng(seed)
    return scale * (2.0 * rng.random(shape) - 1.0)


def random_velocities(n, scale, seed):
    rng = np.random.default_rng(seed)
    return scale * (2.0 * rng.random((n, 3)) - 1.0)


def mlp_init(seed):
    """He-uniform initial weights for the 4-32-32-1 network (FP64 arrays).

    The radius input (range 2..12) enters the first layer as (r - 7)/5; that
    fixed affine map is folded into W1 and b1.  The output layer starts small
    (the network predicts a correction)."""
    rng = np.random.default_rng(seed)

    def lin(fan_out, fan_in):
        b = math.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, (fan_out, fan_in)), np.zeros(fan_out)

    W1, b1 = lin(32, 4)
    W2, b2 = lin(32, 32)
    W3, b3 = lin(1, 32)
    b1 += 0.01 - W1[:, 3] * 7.0 / 5.0
    W1[:, 3] /= 5.0
    b2 += 0.01
    W3 *= 0.01
    return [W1, b1, W2, b2, W3, b3]
