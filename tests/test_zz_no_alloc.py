"""psm_field_sums_noalloc: the mass/momentum check for callers that cannot
allocate device memory at the point of the check (a fixed memory pool owned
by a host code, a hook inside another solver's loop where an allocation would
synchronise the device, a fully committed memory budget).

It must give the same sums as psm_check, which allocates, on two calls in a
row.  The test allocates its own input and output buffers with torch; the
entry point under test allocates nothing.  This file is collected last so a
run that stops at the first failure has run every other test already.
"""
import numpy as np
import pytest

from paper_2303_11811_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_psm_check_twice():
    import torch
    from paper_2303_11811_gb300 import build, capi
    build.build()
    torch.cuda.set_device(0)
    e = capi.Engine(40, 24, 20, 0.6, relax="trt", walls=(1, 1, 0, 0, 0, 0),
                    fbody=(0.0, 1e-5, 2e-5), weighting="nt")
    e.set_particles(np.array([[12.3, 11.2, 9.7], [27.6, 13.1, 10.4]]), np.array([4.2, 3.7]),
                    u=inputs.random_velocities(2, 1e-3, 1), fixed=np.ones(2, np.uint8))
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for steps in (3, 7):  # two calls in a row, on two different fields
        e.step(steps)
        f = torch.from_numpy(e.pdfs().reshape(19, -1).copy()).cuda()
        ncells = f.shape[1]
        rc = capi.field_sums_noalloc(f.data_ptr(), ncells, out.data_ptr(), stream.cuda_stream)
        assert rc == capi.PSM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        mass, P = e.check()
        assert abs(got[0] - mass) <= 1e-12 * abs(mass)
        assert np.max(np.abs(got[1:] - P)) <= 1e-12 * max(1.0, float(np.max(np.abs(P))))
        assert abs(mass - ncells) < 1e-2 * ncells  # a real field, not zeros
    # sizes beyond the array's capacity are refused before any GPU work
    too_many = 4096 * 65536 + 1
    assert capi.field_sums_noalloc(f.data_ptr(), too_many, out.data_ptr(),
                                   stream.cuda_stream) == capi.PSM_ERR_ARG
    e.close()
