"""psm_field_sums_noalloc: the mass/momentum check for callers that cannot
allocate device memory at the point of the check (a fixed memory pool owned
by a host code, a hook inside another solver's loop where an allocation would
synchronise the device, a fully committed memory budget).

It must give the same sums as psm_check, which allocates, on two calls in a
row, and the sums of the field itself: math.fsum of the host copy (correctly
rounded), and, for a field of dyadic values whose every partial sum is exact
in FP64, the exact integer sum.  The sizes cover one block part, many parts
with a ragged tail, and more parts than the final kernel has threads (its
stride loop).  The test allocates its own input and output buffers with torch;
the entry point under test allocates nothing.  This file is collected last so
a run that stops at the first failure has run every other test already.
"""
import math

import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs
from tests.lattice_fixture import C

pytestmark = pytest.mark.gpu

PART = 65536  # cells per block part of the entry point


def _fsum_sums(f):
    """Correctly rounded mass and momentum of a host field f[19][cells], and
    the sums of the absolute values of their terms (the scale a summation
    error is bounded by)."""
    mass = math.fsum(f.ravel())
    P, A = [], [float(np.abs(f).sum())]
    for a in range(3):
        pos = [f[q] for q in range(19) if C[q, a] > 0]
        neg = [-f[q] for q in range(19) if C[q, a] < 0]
        terms = np.concatenate(pos + neg)
        P.append(math.fsum(terms))
        A.append(float(np.abs(terms).sum()))
    return mass, np.array(P), np.array(A)


def _call(capi, f, out, stream):
    rc = capi.field_sums_noalloc(f.data_ptr(), f.shape[1], out.data_ptr(), stream.cuda_stream)
    assert rc == capi.PSM_OK
    stream.synchronize()
    return out.cpu().numpy().copy()


def _engine_field_case(capi, torch, shape, stream, out):
    """An engine's PDF field after 3 and then 7 more steps: two calls in a row."""
    e = capi.Engine(*shape, 0.6, relax="trt", walls=(1, 1, 0, 0, 0, 0),
                    fbody=(0.0, 1e-5, 2e-5), weighting="nt")
    c = np.array(shape, np.float64) / 2
    e.set_particles(np.array([c * 0.6, c * 1.3]), np.array([4.2, 3.7]),
                    u=inputs.random_velocities(2, 1e-3, 1), fixed=np.ones(2, np.uint8))
    for steps in (3, 7):
        e.step(steps)
        host = e.pdfs().reshape(19, -1).copy()
        f = torch.from_numpy(host).cuda()
        got = _call(capi, f, out, stream)
        mass, P = e.check()
        assert abs(got[0] - mass) <= 1e-12 * abs(mass)
        assert np.max(np.abs(got[1:] - P)) <= 1e-12 * max(1.0, float(np.max(np.abs(P))))
        # a sum of n FP64 terms in any order errs by at most about n * 2^-53
        # of the sum of their magnitudes; blocked sums stay far below that
        fm, fP, A = _fsum_sums(host)
        assert np.all(np.abs(got - np.concatenate([[fm], fP])) <= 1e-15 * A), (got, fm, fP)
        assert abs(mass - host.shape[1]) < 1e-2 * host.shape[1]  # a real field, not zeros
        del f
    e.close()
    return host.shape[1]


def test_noalloc_sums_match_psm_check_and_host_sums():
    import torch
    from paper_2303_11811_gb300 import build, capi
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # one block part, then 33 parts with a ragged last part
    assert _engine_field_case(capi, torch, (40, 24, 20), stream, out) < PART
    n = _engine_field_case(capi, torch, (130, 127, 128), stream, out)
    assert n // PART == 32 and n % PART != 0
    # sizes beyond the array's capacity are refused before any GPU work
    f = torch.zeros((19, 1), dtype=torch.float64, device="cuda")
    too_many = 4096 * 65536 + 1
    assert capi.field_sums_noalloc(f.data_ptr(), too_many, out.data_ptr(),
                                   stream.cuda_stream) == capi.PSM_ERR_ARG


def test_noalloc_sums_exact_on_dyadic_field_beyond_256_parts():
    """273 parts (more than the 256 threads of the final kernel, ragged
    tail): values k * 2^-20 with 0 <= k < 2^19 make every partial sum an
    integer multiple of 2^-20 below 2^28, exact in FP64 in any order, so the
    result must equal the integer sum exactly.  Two calls in a row on two
    different fields."""
    import torch
    from paper_2303_11811_gb300 import build, capi
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    ncells = 272 * PART + 12345
    g = torch.Generator(device="cuda")
    for seed in (5, 6):
        g.manual_seed(seed)
        k = torch.randint(0, 1 << 19, (19, ncells), generator=g, device="cuda",
                          dtype=torch.int64)
        f = k.to(torch.float64) * 2.0 ** -20
        got = _call(capi, f, out, stream)
        kh = k.cpu().numpy()
        del k, f
        mass = int(kh.sum(dtype=np.int64))
        P = [int(sum(int(C[q, a]) * int(kh[q].sum(dtype=np.int64)) for q in range(19)))
             for a in range(3)]
        want = np.array([mass] + P, dtype=np.float64) * 2.0 ** -20
        assert np.array_equal(got, want), (got, want)
        del kh
    torch.cuda.empty_cache()
