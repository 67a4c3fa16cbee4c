"""Checkpoint and restart through the C ABI (psm_save / psm_load): a run
stepped past a checkpoint and a fresh context loaded from it continue bit
for bit (PDFs, forces, particle state), in the FP64, FP32 and double-float
forms, with moving spheres, DEM contacts and walls; a context of another
configuration, a foreign and a truncated file are refused."""
import os

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


KW = dict(tau=0.57, relax="trt", walls=(1, 1, 0, 0, 0, 0), fbody=(0.0, 1e-5, 2e-5),
          weighting="nt", eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, -3e-5),
          dem=True, kn=100.0, restitution=0.8)
SHAPE = (37, 24, 20)


def _start(capi, precision, streaming):
    e = capi.Engine(*SHAPE, precision=precision, streaming=streaming, **KW)
    x = np.array([[6.0, 7.5, 9.2], [13.8, 7.6, 9.3], [33.95, 16.7, 3.3]])
    r = np.array([4.3, 3.6, 3.1])
    u = np.array([[-2e-3, 1e-3, 0.0], [-1e-3, 0.0, 1e-3], [5e-4, -1e-3, -2e-3]])
    e.set_particles(x, r, u=u, omega=inputs.random_velocities(3, 1e-3, 4),
                    density=np.array([2.5, 2.0, 3.0]))
    return e


@pytest.mark.parametrize("precision,streaming", [("fp64", "pull"), ("fp32", "aa"),
                                                 ("df64", "pull"), ("fp64", "aa")])
def test_restart_continues_bit_for_bit(capi, precision, streaming, tmp_path):
    path = str(tmp_path / "state.psm")
    a = _start(capi, precision, streaming)
    a.step(7)                     # odd: the AA buffer holds the odd-step layout
    a.save(path)
    a.step(9)
    b = capi.Engine(*SHAPE, precision=precision, streaming=streaming, **KW)
    b.load(path)
    b.step(9)
    assert np.array_equal(a.pdfs(), b.pdfs())
    for ga, gb in zip(a.force_torque(), b.force_torque()):
        assert np.array_equal(ga, gb)
    for ga, gb in zip(a.particles(), b.particles()):
        assert np.array_equal(ga, gb)
    a.close()
    b.close()


def test_surrogate_parameters_travel_with_the_checkpoint(capi, tmp_path):
    path = str(tmp_path / "mlp.psm")
    kw = dict(KW, eps_mode="mlp", eps_n=8)
    a = capi.Engine(*SHAPE, **kw)
    a.set_mlp(capi.pack_mlp(inputs.mlp_init(4)))
    a.set_particles(np.array([[12.0, 11.0, 9.5]]), np.array([4.2]), fixed=np.ones(1, np.uint8))
    a.step(3)
    a.save(path)
    b = capi.Engine(*SHAPE, **kw)
    b.load(path)
    assert np.array_equal(a.get_mlp(), b.get_mlp())
    a.step(4)
    b.step(4)
    assert np.array_equal(a.pdfs(), b.pdfs())
    a.close()
    b.close()


def test_load_refuses_other_configurations_and_bad_files(capi, tmp_path):
    path = str(tmp_path / "state.psm")
    a = _start(capi, "fp64", "pull")
    a.step(2)
    a.save(path)
    f0 = a.pdfs()
    for other in (dict(precision="fp32"), dict(streaming="aa"), dict(tau=0.6)):
        kw = dict(KW, **{k: v for k, v in other.items() if k == "tau"})
        opts = {k: v for k, v in other.items() if k != "tau"}
        c = capi.Engine(*SHAPE, **opts, **kw)
        with pytest.raises(capi.PsmError):
            c.load(path)
        c.close()
    c = capi.Engine(38, 24, 20, **KW)
    with pytest.raises(capi.PsmError):
        c.load(path)
    c.close()
    junk = str(tmp_path / "junk.psm")
    with open(junk, "wb") as fh:
        fh.write(b"not a checkpoint" * 8)
    with pytest.raises(capi.PsmError):
        a.load(junk)
    short = str(tmp_path / "short.psm")
    with open(path, "rb") as fh, open(short, "wb") as gh:
        gh.write(fh.read()[: os.path.getsize(path) // 2])
    with pytest.raises(capi.PsmError):
        a.load(short)
    # the refused loads left the context as it was
    assert np.array_equal(a.pdfs(), f0)
    a.close()
