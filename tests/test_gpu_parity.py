"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

FP64 form: norm-wise relative error <= 1e-12 on E, B, J and momenta after a
step, positions within 1e-12 of the box (the bar the method's FP64 path sets).
Mixed form (int32 cell + FP32 offset, FP32 fields and current): tolerances
derived from FP32 arithmetic, stated per test.
"""
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
    import paper_1211_4575_gb300 as m
    from paper_1211_4575_gb300 import build
    build.build()
    return m


def _seed_fields(gpu, orc_sim, L, seed=99, amp=0.05):
    E, B = pp_synth.random_fields(L.n, seed, amp)
    gpu.load_fields(E, B)
    orc_sim.load_fields(E, B)


def _compare(gpu, osim, L, tol_f, tol_x, tol_u):
    fe = H.field_errors(gpu, osim)
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(gpu.particles(s), osim.species[s], H.box(L))
        assert dpos <= tol_x, (s, dpos)
        assert du <= tol_u, (s, du)
    for k, v in fe.items():
        assert v <= tol_f, (k, v, fe)
    return fe


# --------------------------------------------------------------------------
# FP64 form
# --------------------------------------------------------------------------

def test_fp64_two_stream_one_step(pp, orc):
    """16^3 two-stream pair plasma (65,536 particles), TSC, 6th order, Vay."""
    L = pp_synth.two_stream()
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 2)
    osim = H.oracle_sim(orc, L, 2)
    gpu.step(1)
    osim.step(1)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("forder", [2, 4, 6])
@pytest.mark.parametrize("pusher", [0, 1])
def test_fp64_random_fields_one_step(pp, orc, shape, forder, pusher):
    """Random particles (ragged count 3001) in random E, B on a non-cubic
    20x12x9 grid: exercises gather, both pushers, deposit and field solve."""
    L = pp_synth.random_particles((20, 12, 9), (0.5, 0.4, 0.45), 0.2, 3001, seed=shape * 10 + forder + pusher)
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, shape, field_order=forder, pusher=pusher)
    osim = H.oracle_sim(orc, L, shape, field_order=forder, pusher=pusher)
    _seed_fields(gpu, osim, L)
    gpu.step(1)
    osim.step(1)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


def test_fp64_two_stream_many_steps_and_invariants(pp, orc):
    L = pp_synth.two_stream()
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 2, sort_interval=5)
    osim = H.oracle_sim(orc, L, 2)
    for _ in range(4):
        gpu.step(5)
        osim.step(5)
        d = gpu.diagnostics()
        od = osim.diagnostics()
        assert d["status"] == 0
        assert d["gauss_drift_max"] <= 1e-12 * max(d["rho_max"], 1e-30)
        assert d["divB_max"] <= 1e-12
        assert d["energy_E"] == pytest.approx(od["energy_E"], rel=1e-10)
        assert d["kinetic_total"] == pytest.approx(od["kinetic"], rel=1e-12)
    _compare(gpu, osim, L, 1e-10, 1e-10, 1e-10)


def test_fp64_deposit_and_field_update_halves(pp, orc):
    """pp_deposit + pp_field_update is the same as pp_step; the current after
    the deposit half matches the oracle's J^{n+1}."""
    L = pp_synth.random_particles((16, 8, 8), (0.5, 0.5, 0.5), 0.25, 777, seed=3)
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 3)
    osim = H.oracle_sim(orc, L, 3)
    _seed_fields(gpu, osim, L, seed=5)
    gpu.deposit(-1)
    osim.deposit()
    _, _, J = gpu.fields()
    assert max(H.rel_err(J[a], osim.J[a]) for a in range(3)) <= 1e-12
    gpu.field_update()
    osim.field_update()
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


def test_fp64_continuity_on_gpu(pp):
    """(rho^{n+1} - rho^n)/dt + div^- J = 0 to round-off with the GPU's own J
    (6th-order divergence evaluated here in numpy from the operator's Fourier
    symbol, independent of the library's stencils)."""
    L = pp_synth.random_particles((16, 12, 10), (0.5, 0.5, 0.5), 0.25, 2000, seed=8, u_scale=1.0)
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 3)
    rho0 = gpu.rho()
    gpu.deposit(-1)
    rho1 = gpu.rho()
    _, _, J = gpu.fields()
    k = (75 / 64, -25 / 384, 3 / 640)
    div = np.zeros_like(rho0)
    for a in range(3):
        n, h = L.n[a], L.d[a]
        kk = 2 * np.pi * np.fft.fftfreq(n, d=h)
        K = (2 / h) * sum(k[m] * np.sin((2 * m + 1) * kk * h / 2) for m in range(3))
        sym = 1j * K * np.exp(-0.5j * kk * h)
        sh = [1, 1, 1]
        sh[2 - a] = n
        div += np.real(np.fft.ifft(np.fft.fft(J[a], axis=2 - a) * sym.reshape(sh), axis=2 - a))
    res = (rho1 - rho0) / L.dt + div
    assert np.abs(res).max() <= 1e-12 * np.abs((rho1 - rho0) / L.dt).max()


# --------------------------------------------------------------------------
# Mixed form (int32 cell + FP32 offset)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("mode", [1, 2])
def test_mixed_random_fields_one_step(pp, orc, shape, mode):
    """Global (mode 1) and shared-memory tiled (mode 2) deposits on a 24x16x16
    grid (3x2x2 tiles), ragged particle count."""
    L = pp_synth.random_particles((24, 16, 16), (0.5, 0.4, 0.45), 0.2, 3001, seed=40 + shape)
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, shape, deposit_mode=mode)
    osim = H.oracle_sim(orc, L, shape)
    _seed_fields(gpu, osim, L)
    gpu.step(1)
    osim.step(1)
    # FP32: positions to a few ulp of a cell offset (times dx), momenta and
    # fields to ~1e-5 relative (FP32 gather, FP32 current sums, 1e-6 relaxation)
    _compare(gpu, osim, L, 3e-5, 2e-6, 2e-6)


def test_mixed_thermal_pcs_steps_and_invariants(pp, orc):
    """Thermal PCS pair plasma on 24^3, 8 per cell per species: GPU mixed vs the
    FP64 oracle over 10 steps; Gauss drift and div B at FP32 round-off."""
    L = pp_synth.thermal(n=(24, 24, 24), ppc=8, u_th=0.1, dx=0.1, dt=0.05, seed=1212)
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
    osim = H.oracle_sim(orc, L, 3)
    for _ in range(2):
        gpu.step(5)
        osim.step(5)
        d = gpu.diagnostics()
        assert d["status"] == 0
        assert d["gauss_drift_max"] <= 2e-5 * max(d["rho_max"], 1e-30)
        od = osim.diagnostics()
        assert d["energy_E"] == pytest.approx(od["energy_E"], rel=1e-3)
        assert d["kinetic_total"] == pytest.approx(od["kinetic"], rel=1e-6)


# --------------------------------------------------------------------------
# Edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [0, 1])
def test_empty_and_single_particle_species(pp, orc, precision):
    L = pp_synth.single_particle((12, 12, 12), (0.5, 0.5, 0.5), 0.25, (0.0, 5.999999999, 2.5), (0.7, -0.2, 0.1))
    L.species.append(dict(q=1.0, m=1.0, w=1.0, x=np.zeros(0), y=np.zeros(0), z=np.zeros(0), ux=np.zeros(0),
                          uy=np.zeros(0), uz=np.zeros(0)))
    gpu = H.gpu_sim(pp, L, precision, 3)
    osim = H.oracle_sim(orc, L, 3)
    gpu.step(3)
    osim.step(3)
    tol = 1e-12 if precision == 0 else 1e-5
    _compare(gpu, osim, L, tol, tol, tol)
    assert gpu.count(1) == 0


def test_particles_on_cell_faces_and_box_edge(pp, orc):
    """Positions exactly on cell faces, at 0 and just below L; outside the box
    on load (wrapped periodically)."""
    n, d = (8, 8, 8), (0.5, 0.5, 0.5)
    xs = np.array([0.0, 0.5, 3.999999999999, 1.0, 2.25, -0.25, 4.25])
    L = pp_synth.Load(n=n, d=d, dt=0.25, species=[dict(q=-1.0, m=1.0, w=0.3, x=xs, y=xs[::-1].copy(),
                                                        z=np.roll(xs, 2), ux=np.linspace(-2, 2, 7),
                                                        uy=np.linspace(1, -1, 7), uz=np.zeros(7))])
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 2)
    Lw = pp_synth.Load(n=n, d=d, dt=0.25, species=[dict(L.species[0])])
    for k in ("x", "y", "z"):
        Lw.species[0][k] = np.mod(Lw.species[0][k], 4.0)
    osim = H.oracle_sim(orc, Lw, 2)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, Lw, 1e-12, 1e-12, 1e-12)


def test_sort_keeps_particle_set(pp):
    L = pp_synth.random_particles((16, 16, 16), (0.5, 0.5, 0.5), 0.25, 5000, seed=2)
    for precision in (0, 1):
        gpu = H.gpu_sim(pp, L, precision, 2)
        before = gpu.particles(0)
        gpu.sort()
        after = gpu.particles(0)
        dpos, du = H.particle_errors(after, before, H.box(L))
        assert dpos == 0.0 and du == 0.0
        cells = [np.floor(after[k] / 0.5).astype(int) for k in ("x", "y", "z")]
        tile = [c // 8 for c in cells]
        key = ((tile[2] * 2 + tile[1]) * 2 + tile[0]) * 512 + ((cells[2] % 8) * 8 + cells[1] % 8) * 8 + cells[0] % 8
        assert np.all(np.diff(key) >= 0)


def test_save_restore_roundtrip(pp, tmp_path):
    L = pp_synth.two_stream(n=(8, 8, 8))
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 2)
    gpu.step(3)
    path = str(tmp_path / "ck.bin")
    gpu.save(path)
    other = pp.Simulation.restore(path)
    gpu.step(2)
    other.step(2)
    E1, B1, _ = gpu.fields()
    E2, B2, _ = other.fields()
    assert max(H.rel_err(E1[a], E2[a]) for a in range(3)) <= 1e-12
    assert max(H.rel_err(B1[a], B2[a]) for a in range(3)) <= 1e-12
    assert other.diagnostics()["step"] == 5


def test_invalid_inputs_fail_loudly(pp):
    with pytest.raises(pp.PPError):
        pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.6)        # c dt / dx > 1
    sim = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.25, precision=pp.PP_FP64)
    sid = sim.add_species(-1.0, 1.0, 1.0, 4)
    with pytest.raises(pp.PPError):
        sim.load_particles(sid, *[np.array([np.nan, 0.1])] * 6)
    with pytest.raises(pp.PPError):
        sim.load_particles(sid, *[np.zeros(5)] * 6)          # above the requested capacity of 4
    assert sim.count(sid) == 0


def test_mixed_tiled_drift_fallback(pp, orc):
    """No re-sort after the load and fast particles: many drift more than the
    tiled kernel's margin from their tile and go through the global-mesh
    fallback; the result still matches the oracle and the global form."""
    L = pp_synth.random_particles((16, 16, 16), (0.5, 0.5, 0.5), 0.25, 4000, seed=77, u_scale=3.0)
    tiled = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2, sort_interval=0)
    glob = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=1, sort_interval=0)
    osim = H.oracle_sim(orc, L, 3)
    for sim in (tiled, glob):
        E, B = pp_synth.random_fields(L.n, 3, 0.02)
        sim.load_fields(E, B)
    osim.load_fields(*pp_synth.random_fields(L.n, 3, 0.02))
    for _ in range(12):
        tiled.step(1)
        glob.step(1)
        osim.step(1)
    d = tiled.diagnostics()
    assert d["status"] == 0 and d["n_slow"] > 100
    _compare(tiled, osim, L, 2e-4, 2e-5, 2e-5)
    Et, Bt, Jt = tiled.fields()
    Eg, Bg, Jg = glob.fields()
    assert max(H.rel_err(Et[a], Eg[a]) for a in range(3)) <= 1e-4
    assert max(H.rel_err(Jt[a], Jg[a]) for a in range(3)) <= 1e-4


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("n", [(20, 12, 9), (6, 5, 4), (24, 16, 16)])
def test_mixed_rho_against_oracle(pp, orc, shape, n):
    """The mixed form's charge density (eq:rho2, per-tile frames summed in
    shared memory) against the oracle's FP64 deposit of the same positions:
    tiles of every size (padded, smaller than 8, exact), and particles that
    left their sorted cell (three steps without a re-sort).  FP32 weights:
    5e-6 of max|rho|."""
    L = pp_synth.random_particles(n, (0.5, 0.4, 0.45), 0.2, 3001, seed=40 + shape, u_scale=1.0)
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, shape, sort_interval=0)
    gpu.step(3)
    rho = gpu.rho()
    p = gpu.particles(0)
    s = L.species[0]
    o = orc.Simulation(L.n, L.d, L.dt, shape_order=shape)
    o.add_species(s["q"], s["m"], s["w"], p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"])
    ro = o.rho()
    assert np.abs(rho - ro).max() <= 5e-6 * np.abs(ro).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_kinetic_energy_against_its_definition(pp, precision):
    """The kinetic energy reduction (w m dV sum of gamma - 1 per species, FP64)
    against the plain FP64 sum over the momenta read back from the device,
    for |u| log-uniform over 1e-4 .. 1e3 (non-relativistic terms, where
    gamma - 1 ~ u^2 / 2, to ultra-relativistic ones)."""
    rng = np.random.default_rng(77)
    n, count = (16, 16, 16), 20000
    L = pp_synth.random_particles(n, (0.5, 0.5, 0.5), 0.2, count, seed=5)
    mag = 10.0 ** rng.uniform(-4, 3, count)
    dirs = rng.normal(size=(3, count))
    dirs /= np.linalg.norm(dirs, axis=0)
    sp = L.species[0]
    sp["ux"], sp["uy"], sp["uz"] = mag * dirs[0], mag * dirs[1], mag * dirs[2]
    sim = H.gpu_sim(pp, L, precision, 3)
    p = sim.particles(0)
    u2 = p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2
    want = sp["w"] * sp["m"] * 0.125 * np.sum(u2 / (np.sqrt(1.0 + u2) + 1.0))
    got = sim.diagnostics()["kinetic"][0]
    assert got == pytest.approx(want, rel=1e-13)
