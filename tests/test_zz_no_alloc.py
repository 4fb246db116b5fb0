"""The allocation-free field-energy entry point (pp_field_energy_noalloc).

Some callers of this library cannot allocate device memory when they need the
field energies (loops that forbid allocation after start-up, hosts that own
all device memory and only hand over pre-allocated buffers).  This entry point
keeps its scratch in a fixed array inside the library.  Its results must equal
the energies pp_diagnostics computes for the same fields, on two calls in a
row (the second call reuses the array the first one left behind), and a call
after the first must leave the device's free memory unchanged.

Kept in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

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


def _evolved(pp):
    import pp_synth
    L = pp_synth.two_stream(n=(16, 12, 8))
    sim = pp.Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=2, precision=pp.PP_FP64,
                        relax_tol=1e-14, relax_max_iter=400)
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]))
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    sim.step(5)
    return L, sim


def test_noalloc_energies_match_diagnostics_twice(pp):
    import torch
    L, sim = _evolved(pp)
    d = sim.diagnostics()
    E, B, _ = sim.fields()
    dev = torch.device("cuda", torch.cuda.current_device())
    Et = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in E]
    Bt = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in B]
    out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
    dV = L.d[0] * L.d[1] * L.d[2]
    lib = pp.lib()
    pe = (C.c_void_p * 3)(*[t.data_ptr() for t in Et])
    pb = (C.c_void_p * 3)(*[t.data_ptr() for t in Bt])
    stream = torch.cuda.current_stream().cuda_stream
    expect = np.array([d["energy_E"], d["energy_B"], d["energy_Ex"]])
    assert expect.min() > 0.0
    free = []
    for _ in range(2):
        rc = lib.pp_field_energy_noalloc(pe, pb, L.n[0], L.n[1], L.n[2], dV, out.data_ptr(), stream)
        assert rc == pp.PP_OK, lib.pp_field_energy_noalloc_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = out.cpu().numpy()
        assert np.allclose(got, expect, rtol=1e-12, atol=0.0), (got, expect)
        out.fill_(-1.0)
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
    # the first call may load the module's code; the second allocates nothing
    assert free[1] == free[0] and free[2] == free[0], free
    # a different mesh afterwards: the shared scratch carries nothing over
    half = [t[:, :, : L.n[0] // 2].contiguous() for t in Et + Bt]
    pp.field_energy_noalloc(half[:3], half[3:], dV, out)
    torch.cuda.synchronize()
    ref = 0.5 * dV * sum(float((t.double() ** 2).sum()) for t in half[:3])
    assert out[0].item() == pytest.approx(ref, rel=1e-12)


def test_noalloc_rejects_oversized_mesh(pp):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.zeros(8, dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    lib = pp.lib()
    pe = (C.c_void_p * 3)(*([t.data_ptr()] * 3))
    rc = lib.pp_field_energy_noalloc(pe, pe, 2000, 1024, 1024, 1.0, out.data_ptr(), None)
    assert rc == pp.PP_EINVAL
    assert b"outside" in lib.pp_field_energy_noalloc_error()
