"""Failure detection on the GPU without any GPU fault: bad data and a capped
solver end in status codes the host reads at the next synchronising call,
and the context stays usable."""
import numpy as np
import pytest

import pp_synth
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as m
    return m


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_fields_flag_enan_and_context_survives(pp, precision):
    L = pp_synth.random_particles((16, 16, 16), (0.5, 0.5, 0.5), 0.25, 2000, seed=9)
    sim = H.gpu_sim(pp, L, precision, 3)
    E, B = pp_synth.random_fields(L.n, 4, 0.01)
    E[0][3, 4, 5] = np.nan
    sim.load_fields(E, B)
    sim.step(1)                                   # enqueues; particles near the NaN are skipped
    with pytest.raises(pp.PPError) as ei:
        sim.sync()
    assert ei.value.code == pp.PP_ENAN
    sim.sync()                                    # the status word was cleared; device still answers
    n = sim.count(0)
    assert n == 2000
    p = sim.particles(0)
    assert np.isfinite(p["x"]).all()              # skipped particles keep their last finite state


def test_relaxation_cap_reports_enoconv(pp):
    L = pp_synth.two_stream(n=(8, 8, 8))
    sim = H.gpu_sim(pp, L, pp.PP_FP64, 2, relax_tol=1e-15, relax_max_iter=1)
    sim.step(2)
    d = sim.diagnostics()
    assert d["relax_iters"] == 1
    assert d["status"] == pp.PP_ENOCONV
    assert d["relax_residual"] > 1e-15


def test_capacity_and_species_limits(pp):
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.25, precision=pp.PP_MIXED32)
    for _ in range(pp.PP_MAX_SPECIES):
        sim.add_species(-1.0, 1.0, 1.0, 1)
    with pytest.raises(pp.PPError) as ei:
        sim.add_species(-1.0, 1.0, 1.0, 1)
    assert ei.value.code == pp.PP_EINVAL
    with pytest.raises(pp.PPError) as ei:
        sim.load_particles(0, *[np.zeros(2)] * 6)
    assert ei.value.code == pp.PP_ENOMEM


def test_staging_wait_runs_out_into_etimeout_and_context_survives(pp):
    """The per-step sorted kernel stages each tile's E/B window with TMA tensor
    copies and waits on an mbarrier for at most a second.  The same bounded
    wait run once on a barrier whose phase completes returns PP_OK; on one
    that waits for 16 bytes no copy delivers it runs out and returns
    PP_ETIMEOUT after about twice its limit (the CTA waits once more for
    copies in flight), with no fault: the context then steps on as one that
    never met the timeout."""
    import time
    L = pp_synth.thermal(n=(16, 16, 16), ppc=4, seed=31)
    a = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=pp.PP_DEPOSIT_CELLS)
    b = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=pp.PP_DEPOSIT_CELLS)
    a.step(1)
    b.step(1)
    assert a.check_bounded_wait(True, 1_000_000) == pp.PP_OK
    t0 = time.perf_counter()
    rc = a.check_bounded_wait(False, 5_000_000)
    dt = time.perf_counter() - t0
    assert rc == pp.PP_ETIMEOUT
    assert 0.009 <= dt < 5.0
    assert a.check_bounded_wait(True, 1_000_000) == pp.PP_OK   # the status word was cleared
    assert a.check_bounded_wait(False, 0) == pp.PP_EINVAL
    a.step(3)
    b.step(3)
    a.sync()
    b.sync()
    for s in range(2):
        pa, pb = a.particles(s), b.particles(s)
        assert a.count(s) == b.count(s) == len(L.species[s]["x"])
        for k in ("ux", "uy", "uz"):
            np.testing.assert_allclose(np.sort(pa[k]), np.sort(pb[k]), rtol=0, atol=1e-5)
    da, db = a.diagnostics(), b.diagnostics()
    assert da["status"] == pp.PP_OK
    ea, eb = da["energy_E"] + da["energy_B"], db["energy_E"] + db["energy_B"]
    assert abs(ea - eb) <= 1e-4 * abs(eb)
