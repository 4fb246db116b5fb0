"""GPU parity of the reflecting walls (Sec. V "Boundary conditions",
boundary_x = PP_BOUNDARY_WALLS) against the oracle's virtual-image system.

The library deposits the particles alone, folds the images' share into the
mirror-extended mesh and reflects the particles that crossed; the oracle
carries every image as a particle and reflects nothing.  Both see the same
unsymmetrised random fields and project them by their own code."""
import math

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


def _pair(pp, orc, L, precision, shape, pusher=0, mode=0, fields_seed=31, gpu_kw=None, orc_kw=None, setup=None,
          walls=(True, False, False)):
    W = pp.PP_BOUNDARY_WALLS
    gpu = H.gpu_sim(pp, L, precision, shape, pusher=pusher, deposit_mode=mode, boundary_x=W if walls[0] else 0,
                    boundary_y=W if walls[1] else 0, boundary_z=W if walls[2] else 0, **(gpu_kw or {}))
    if setup:
        setup(gpu)
    osim = orc.WallSimulation(L.n, L.d, L.dt, walls=walls, shape_order=shape, pusher=pusher, relax_tol=1e-14,
                              relax_max_iter=2000, **(orc_kw or {}))
    for s in L.species:
        osim.add_species(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    E, B = pp_synth.random_fields(tuple(2 * L.n[a] if walls[a] else L.n[a] for a in range(3)), fields_seed, 0.05)
    gpu.load_fields(E, B)
    osim.load_fields(E, B)
    return gpu, osim


def _box(L, walls=(True, False, False)):
    return tuple((2 if walls[a] else 1) * L.n[a] * L.d[a] for a in range(3))


def _compare(gpu, osim, L, tol_f, tol_x, tol_u, walls=(True, False, False)):
    assert gpu.diagnostics()["status"] == 0
    for s in range(len(L.species)):
        p = gpu.particles(s)
        for a in range(3):
            if walls[a]:
                assert p["xyz"[a]].min() >= 0.0 and p["xyz"[a]].max() <= L.n[a] * L.d[a]
        dpos, du = H.particle_errors(p, osim.particles(s), _box(L, walls))
        assert dpos <= tol_x and du <= tol_u, (s, dpos, du)
    fe = H.field_errors(gpu, osim)
    for k, v in fe.items():
        assert v <= tol_f, (k, v, fe)


def _load(n=(10, 12, 9), count=3001, seed=140, u_scale=0.6):
    # particles fast enough that many cross a wall in a few steps
    return pp_synth.random_particles(n, (0.5, 0.4, 0.45), 0.2, count, seed=seed, u_scale=u_scale)


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("pusher", [0, 1])
def test_walls_fp64_parity(pp, orc, shape, pusher):
    """Ragged 3001 random particles between walls on 10x12x9 (mesh 20x12x9),
    random fields, four steps: FP64 to 1e-12 against the oracle's images."""
    L = _load(seed=140 + shape + 3 * pusher)
    gpu, osim = _pair(pp, orc, L, pp.PP_FP64, shape, pusher)
    gpu.step(4)
    osim.step(4)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_walls_mixed_parity(pp, orc, mode):
    """Mixed form, global (1) and tiled (2) deposits, 12x16x16 between walls
    (mesh 24x16x16), three steps: fields 3e-5, positions and momenta 2e-6."""
    L = _load((12, 16, 16), seed=151)
    gpu, osim = _pair(pp, orc, L, pp.PP_MIXED32, 3, mode=mode)
    gpu.step(3)
    osim.step(3)
    _compare(gpu, osim, L, 3e-5, 2e-6, 2e-6)


@pytest.mark.parametrize("variant", ["explicit", "direct_filter", "step4"])
def test_walls_with_the_variants(pp, orc, variant):
    """The walls under the explicit FDTD solver, the direct current with the
    divergence filter, and the 4th-order step: FP64 to 1e-12."""
    L = _load(seed=160)
    if variant == "explicit":
        L.dt = 0.1
        setup = lambda g: g.set_field_solver(pp.PP_FIELD_EXPLICIT)
        okw = dict(field_solver=orc.EXPLICIT)
    elif variant == "direct_filter":
        def setup(g):
            g.set_current_deposit(pp.PP_CURRENT_DIRECT)
            g.set_divergence_filter(2, 1)
        okw = dict(current_mode=orc.DIRECT, filter_passes=2, filter_interval=1)
    else:
        setup = lambda g: g.set_integrator(4)
        okw = dict(integrator=4)
    gpu, osim = _pair(pp, orc, L, pp.PP_FP64, 3, setup=setup, orc_kw=okw)
    gpu.step(2)
    osim.step(2)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_free_particle_bounces_on_gpu(pp, precision):
    """One light particle per wall in empty fields, 100 steps: the folded
    straight path, u_x reversed on the odd legs (closed form)."""
    n, d, dt = (16, 8, 8), (0.5, 0.5, 0.5), 0.2
    Lx = n[0] * d[0]
    sim = pp.Simulation(n, d, dt, shape_order=3, precision=precision, boundary_x=pp.PP_BOUNDARY_WALLS,
                        relax_tol=1e-14 if precision == 0 else 1e-6)
    x0 = np.array([6.7, 1.1])
    u0 = np.array([[2.0, 0.3, -0.1], [-1.5, -0.2, 0.4]])
    sid = sim.add_species(-1.0, 1.0, 1e-13, 2)
    sim.load_particles(sid, x0, np.array([1.3, 2.2]), np.array([0.7, 3.1]), u0[:, 0], u0[:, 1], u0[:, 2])
    v = u0 / np.sqrt(1.0 + (u0 ** 2).sum(1))[:, None]
    tol = 1e-9 if precision == 0 else 2e-4
    for k in range(10, 101, 10):
        sim.step(10)
        p = sim.particles(sid)
        o = np.argsort(p["uy"])[::-1]   # uy 0.3 first, -0.2 second
        X = x0 + k * dt * v[:, 0]
        s = np.mod(X, 2 * Lx)
        xe = np.where(s <= Lx, s, 2 * Lx - s)
        uxe = np.where(s <= Lx, u0[:, 0], -u0[:, 0])
        assert np.abs(p["x"][o] - xe).max() < tol, (k, p["x"][o], xe)
        assert np.abs(p["ux"][o] - uxe).max() < tol, (k, p["ux"][o], uxe)


def test_walls_keep_symmetry_and_charge_tiled(pp):
    """Thermal pair plasma between walls, tiled mixed form, 30 steps: the
    extended mesh stays mirror-symmetric (E_x odd, E_y even, B_x even, B_y odd),
    the charge equals the particles' and the Gauss drift stays at FP32 level."""
    L = pp_synth.thermal(n=(16, 16, 16), ppc=8, u_th=0.3, dx=0.1, dt=0.05, seed=1217)
    sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=2, boundary_x=pp.PP_BOUNDARY_WALLS)
    sim.step(30)
    d = sim.diagnostics()
    assert d["status"] == 0
    q = sum(s["q"] * s["w"] * len(s["x"]) for s in L.species) * 0.1 ** 3
    qe = sum(abs(s["q"]) * s["w"] * len(s["x"]) for s in L.species) * 0.1 ** 3
    assert abs(d["charge"] - q) <= 1e-6 * qe
    assert d["gauss_drift_max"] <= 1e-4 * d["rho_max"]
    E, B, J = sim.fields()
    N = E[0].shape[-1]
    i = np.arange(N)
    for F, half, sign in ((E[0], True, -1), (E[1], False, 1), (B[0], False, 1), (B[1], True, -1), (J[0], True, -1),
                          (J[2], False, 1)):
        img = sign * F[..., (N - 1 - i) if half else (-i) % N]
        assert np.abs(F - img).max() <= 1e-4 * np.abs(F).max()
    for s in range(2):
        p = sim.particles(s)
        assert p["x"].min() >= 0.0 and p["x"].max() <= 1.6


def test_walls_arguments_and_checkpoint(pp, tmp_path):
    with pytest.raises(pp.PPError):   # mesh 2 * 600 > 1023
        pp.Simulation((600, 8, 8), (0.5, 0.5, 0.5), 0.2, boundary_x=pp.PP_BOUNDARY_WALLS)
    with pytest.raises(pp.PPError):
        pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2, boundary_x=2)
    with pytest.raises(pp.PPError):   # mesh 2 * 12 = 24 is a multiple of 8, 2 * 10 is not
        pp.Simulation((10, 8, 8), (0.5, 0.5, 0.5), 0.2, precision=pp.PP_MIXED32, deposit_mode=pp.PP_DEPOSIT_TILED,
                      boundary_x=pp.PP_BOUNDARY_WALLS)
    sim = pp.Simulation((12, 8, 8), (0.5, 0.5, 0.5), 0.2, precision=pp.PP_FP64, boundary_x=pp.PP_BOUNDARY_WALLS)
    sid = sim.add_species(-1.0, 1.0, 0.1, 10)
    one = np.array([1.0])
    with pytest.raises(pp.PPError):   # x beyond the upper wall at 6
        sim.load_particles(sid, np.array([6.5]), one, one, one, one, one)
    with pytest.raises(ValueError):   # field arrays of the physical box instead of the extended one
        sim.load_fields([np.zeros((8, 8, 12))] * 3, [np.zeros((8, 8, 12))] * 3)
    assert sim.count(sid) == 0
    L = _load((12, 8, 8), count=500, seed=171)
    s = L.species[0]
    a = pp.Simulation(L.n, L.d, L.dt, shape_order=2, precision=pp.PP_FP64, boundary_x=pp.PP_BOUNDARY_WALLS,
                      relax_tol=1e-14)
    sid = a.add_species(s["q"], s["m"], s["w"], 500)
    a.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    a.step(2)
    path = str(tmp_path / "walls.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    assert b.walls and b.mesh_shape == (8, 8, 24)
    a.step(2)
    b.step(2)
    Ea, _, _ = a.fields()
    Eb, _, _ = b.fields()
    assert max(H.rel_err(Eb[k], Ea[k]) for k in range(3)) <= 1e-12


# --------------------------------------------------------------------------
# Open lower end, injectors and sliding window
# --------------------------------------------------------------------------

def _boundary_pair(pp, orc, L, precision, mode=0, window=0.0, steps=6, shape=3, inj=True, open_end=True):
    gpu, osim = _pair(pp, orc, L, precision, shape, mode=mode, gpu_kw=dict(capacity_extra=4000))
    # a second, positive species so that the inflow is neutral
    sp = L.species[0]
    e = np.zeros(0)
    sid_g = gpu.add_species(-sp["q"], sp["m"], sp["w"], 4000)
    sid_o = osim.add_species(-sp["q"], sp["m"], sp["w"], e, e, e, e, e, e)
    assert sid_g == sid_o == 1
    if open_end:
        gpu.set_open_boundary(6, 0.2, 2.0)
        osim.set_open_boundary(6, 0.2, 2.0)
    if inj:
        for sid in (0, 1):
            gpu.set_injector(sid, 1.5, (0.8, 0.1, -0.05), 0.05, 77)
            osim.set_injector(sid, 1.5, (0.8, 0.1, -0.05), 0.05, 77)
    if window:
        gpu.set_sliding_window(window)
        osim.set_window(window)
    gpu.step(steps)
    osim.step(steps)
    return gpu, osim


def _compare_all(gpu, osim, L, nsp, tol_f, tol_x, tol_u):
    assert gpu.diagnostics()["status"] == 0
    for s in range(nsp):
        p = gpu.particles(s)
        o = osim.particles(s)
        assert len(p["x"]) == len(o["x"]), (s, len(p["x"]), len(o["x"]))
        assert p["x"].min() >= 0.0 and p["x"].max() <= L.n[0] * L.d[0]
        dpos, du = H.particle_errors(p, o, _box(L))
        assert dpos <= tol_x and du <= tol_u, (s, dpos, du)
    fe = H.field_errors(gpu, osim)
    for k, v in fe.items():
        assert v <= tol_f, (k, v, fe)


def test_open_end_and_injector_fp64_parity(pp, orc):
    """Open lower end (6-cell layer, escape 2 cells) with neutral injection of
    two species, fast random particles that reach the open end, random fields,
    six steps: counts equal, FP64 to 1e-12 against the oracle."""
    L = _load(seed=181)
    gpu, osim = _boundary_pair(pp, orc, L, pp.PP_FP64)
    assert osim.counts[1] > 0 and osim.counts[0] != len(L.species[0]["x"])
    _compare_all(gpu, osim, L, 2, 1e-12, 1e-12, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_open_end_and_injector_mixed_parity(pp, orc, mode):
    """The same in the mixed form, global (1) and tiled (2, injected particles
    in the unsorted tail, escaped ones skipped until the next sort)."""
    L = _load((12, 16, 16), seed=182)
    gpu, osim = _boundary_pair(pp, orc, L, pp.PP_MIXED32, mode=mode)
    _compare_all(gpu, osim, L, 2, 3e-5, 2e-6, 2e-6)


@pytest.mark.parametrize("precision,mode", [(0, 0), (1, 2)])
def test_sliding_window_parity(pp, orc, precision, mode):
    """Window at v = 0.6 (a shift every few steps) with the open end and the
    injectors filling each new layer, ten steps: FP64 to 1e-12, mixed tiled to
    its tolerance."""
    L = _load((12, 16, 16), seed=183)
    gpu, osim = _boundary_pair(pp, orc, L, precision, mode=mode, window=0.6, steps=10)
    assert osim.shifts >= 2
    tol = (1e-12, 1e-12, 1e-12) if precision == 0 else (3e-5, 2e-6, 2e-6)
    _compare_all(gpu, osim, L, 2, *tol)


def test_boundary_state_in_checkpoint_and_errors(pp, orc, tmp_path):
    L = _load((12, 8, 8), count=600, seed=184)
    a, _ = _boundary_pair(pp, orc, L, pp.PP_FP64, window=0.6, steps=3)
    path = str(tmp_path / "open.ckpt")
    a.save(path)
    b = pp.Simulation.restore(path)
    for s in (a, b):
        s.step(4)
    for sid in (0, 1):
        pa, pb = a.particles(sid), b.particles(sid)
        assert len(pa["x"]) == len(pb["x"])
        dpos, du = H.particle_errors(pb, pa, _box(L))
        assert dpos <= 1e-12 and du <= 1e-12
    Ea, _, _ = a.fields()
    Eb, _, _ = b.fields()
    assert max(H.rel_err(Eb[k], Ea[k]) for k in range(3)) <= 1e-12
    # errors
    per = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2)
    per.add_species(-1.0, 1.0, 0.1, 10)
    with pytest.raises(pp.PPError):
        per.set_open_boundary(4, 0.1, 1.0)
    with pytest.raises(pp.PPError):
        per.set_injector(0, 1.0, (0.5, 0, 0))
    with pytest.raises(pp.PPError):
        per.set_sliding_window(0.5)
    w = pp.Simulation((8, 8, 8), (0.5, 0.5, 0.5), 0.2, boundary_x=pp.PP_BOUNDARY_WALLS)
    sid = w.add_species(-1.0, 1.0, 0.1, 10)
    for args in ((9, 0.1, 1.0), (4, 1.5, 1.0), (4, 0.1, -1.0), (4, 0.1, 1.0, 64)):
        with pytest.raises(pp.PPError):
            w.set_open_boundary(*args)
    with pytest.raises(pp.PPError):
        w.set_injector(sid, 1.0, (-0.5, 0, 0))
    with pytest.raises(pp.PPError):
        w.set_sliding_window(1.0)
    # an injection beyond the capacity fails the step
    w.set_injector(sid, 4.0, (0.9, 0, 0))
    with pytest.raises(pp.PPError):
        w.step(3)


# --------------------------------------------------------------------------
# Walls on y and z, and on all three axes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("walls", [(False, True, False), (False, False, True), (True, True, True)])
def test_other_walls_fp64_parity(pp, orc, walls):
    """Walls on y, on z, or on every axis (a closed box), random fast particles
    in unsymmetrised random fields, four steps: FP64 to 1e-12."""
    L = _load((10, 12, 9), seed=190 + sum(walls) + 2 * walls[2])
    gpu, osim = _pair(pp, orc, L, pp.PP_FP64, 3, walls=walls)
    gpu.step(4)
    osim.step(4)
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12, walls)


@pytest.mark.parametrize("walls", [(False, True, False), (True, True, True)])
def test_other_walls_mixed_tiled_parity(pp, orc, walls):
    """The tiled kernel with walls on y and in a closed box (meshes of 16 on
    walled axes): mixed tolerances."""
    L = _load((8, 8, 16) if walls[0] else (16, 8, 16), seed=195 + sum(walls))
    gpu, osim = _pair(pp, orc, L, pp.PP_MIXED32, 3, mode=2, walls=walls)
    gpu.step(3)
    osim.step(3)
    _compare(gpu, osim, L, 3e-5, 2e-6, 2e-6, walls)


def test_open_end_with_walls_on_y(pp, orc):
    """The open x end and the injectors in a box that also has walls on y:
    FP64 to 1e-12 with equal counts."""
    L = _load((10, 12, 9), count=1500, seed=198)
    walls = (True, True, False)
    gpu, osim = _pair(pp, orc, L, pp.PP_FP64, 3, walls=walls, gpu_kw=dict(capacity_extra=4000))
    e = np.zeros(0)
    sp = L.species[0]
    gpu.add_species(-sp["q"], sp["m"], sp["w"], 4000)
    osim.add_species(-sp["q"], sp["m"], sp["w"], e, e, e, e, e, e)
    gpu.set_open_boundary(6, 0.2, 2.0)
    osim.set_open_boundary(6, 0.2, 2.0)
    for sid in (0, 1):
        gpu.set_injector(sid, 1.5, (0.8, 0.1, -0.05), 0.05, 78)
        osim.set_injector(sid, 1.5, (0.8, 0.1, -0.05), 0.05, 78)
    gpu.step(6)
    osim.step(6)
    for sid in (0, 1):
        assert len(gpu.particles(sid)["x"]) == len(osim.particles(sid)["x"])
    _compare(gpu, osim, L, 1e-12, 1e-12, 1e-12, walls)


@pytest.mark.parametrize("precision", [0, 1])
def test_free_particle_in_a_closed_box_on_gpu(pp, precision):
    n, d, dt = (8, 8, 8), (0.5, 0.5, 0.5), 0.2
    Ls = np.array([n[a] * d[a] for a in range(3)])
    W = pp.PP_BOUNDARY_WALLS
    sim = pp.Simulation(n, d, dt, shape_order=2, precision=precision, boundary_x=W, boundary_y=W, boundary_z=W,
                        relax_tol=1e-14 if precision == 0 else 1e-6)
    assert sim.mesh_shape == (16, 16, 16)
    x0 = np.array([2.7, 1.1, 0.6])
    u0 = np.array([1.5, -0.9, 0.7])
    sid = sim.add_species(-1.0, 1.0, 1e-13, 1)
    sim.load_particles(sid, *[np.array([v]) for v in x0], *[np.array([v]) for v in u0])
    v = u0 / np.sqrt(1.0 + (u0 ** 2).sum())
    sim.step(40)
    p = sim.particles(sid)
    tol = 1e-9 if precision == 0 else 1e-4
    for a in range(3):
        s_ = np.mod(x0[a] + 40 * dt * v[a], 2 * Ls[a])
        xe = s_ if s_ <= Ls[a] else 2 * Ls[a] - s_
        ue = u0[a] if s_ <= Ls[a] else -u0[a]
        assert abs(p["xyz"[a]][0] - xe) < tol and abs(p["u" + "xyz"[a]][0] - ue) < tol, a


def test_walls_step_graphs_and_eager_boundary_steps(pp, orc):
    """Closed walls step through captured graphs like eagerly (FP64 1e-12);
    with an open end the steps run eagerly even when graphs are enabled."""
    import torch
    L = _load((10, 12, 9), count=1200, seed=199)
    sims = []
    for graphs in (False, True):
        st = torch.cuda.Stream()
        g = H.gpu_sim(pp, L, pp.PP_FP64, 3, sort_interval=3, stream=st.cuda_stream, boundary_x=pp.PP_BOUNDARY_WALLS,
                      boundary_y=pp.PP_BOUNDARY_WALLS)
        g._keep = st
        if graphs:
            g.set_graphs(True)
        g.step(8)
        sims.append(g)
    E0, B0, _ = sims[0].fields()
    E1, B1, _ = sims[1].fields()
    assert max(H.rel_err(E1[a], E0[a]) for a in range(3)) <= 1e-12
    assert max(H.rel_err(B1[a], B0[a]) for a in range(3)) <= 1e-12
    cap, rep = sims[1].graph_stats()
    assert cap + rep == 8 and rep >= 2, (cap, rep)
    sims[1].set_open_boundary(4, 0.1, 1.0)
    sims[1].step(3)
    assert sims[1].graph_stats() == (cap, rep)   # eager: no capture, no replay


@pytest.mark.parametrize("precision", [0, 1])
def test_injector_draws_equal_the_oracle_generator_bit_for_bit(pp, orc, precision):
    """The GPU injector's Philox4x32-10 words are the oracle's, bit for bit.
    With unit cell sizes across x and ny = nz = 4, a particle's y and z are
    4 (r + 1/2) 2^-32 exactly, so the words r1, r2 of its counter can be read
    back from them; the set of (r1, r2) over one injection equals the words of
    orc_draws (seed, step 1, position stream 0) at counters 0 .. count-1.  x is
    thick u0 to rounding, and the Box-Muller momenta of the velocity stream
    (1 + species) agree to libm-versus-CUDA rounding.  The oracle's generator itself is pinned to the published
    known-answer vectors."""
    seed, ppc, u, u_th = 0x1234_5678_9ABC_DEF0, 20.0, (0.8, 0.1, -0.05), 0.05
    n, d, dt = (16, 4, 4), (0.5, 1.0, 1.0), 0.2
    sim = pp.Simulation(n, d, dt, shape_order=3, precision=precision, boundary_x=pp.PP_BOUNDARY_WALLS,
                        relax_tol=1e-6 if precision else 1e-12, relax_max_iter=400)
    sid = sim.add_species(-1.0, 1.0, 1e-9, 4096)
    sim.set_injector(sid, ppc, u, u_th, seed)
    sim.step(1)
    p = sim.particles(sid)
    vx = u[0] / math.sqrt(1.0 + sum(v * v for v in u))
    count = int(math.floor(ppc * n[1] * n[2] * vx * dt / d[0]))
    assert len(p["x"]) == count and count > 50
    D = orc.draws(seed, 1, 0, count)
    words = np.floor(D * 2.0 ** 32).astype(np.int64)
    ry = p["y"] * 2.0 ** 30 - 0.5
    rz = p["z"] * 2.0 ** 30 - 0.5
    if precision == 0:
        # FP64 positions: the words themselves
        assert np.all(ry == np.floor(ry)) and np.all(rz == np.floor(rz))
        got = sorted(zip(ry.astype(np.int64).tolist(), rz.astype(np.int64).tolist()))
        want = sorted(zip(words[:, 1].tolist(), words[:, 2].tolist()))
        assert got == want
        order = np.lexsort((rz, ry))
        ref = np.lexsort((words[:, 2], words[:, 1]))
        thick = vx * dt
        assert np.abs(p["x"][order] - thick * D[ref, 0]).max() <= 4e-16 * thick
        # proper velocities: Box-Muller on the draws of the velocity stream 1 + species
        G = orc.gaussians(orc.draws(seed, 1, 1, count))[ref]
        for a, k in enumerate(("ux", "uy", "uz")):
            assert np.abs(p[k][order] - (u[a] + u_th * G[:, a])).max() <= 1e-14
    else:
        # mixed form: int32 cell + FP32 offset of the same draws (offset
        # rounded to FP32, 2^-24 of a cell)
        got = np.sort(p["y"] + 4.0 * p["z"])
        want = np.sort(4.0 * D[:, 1] + 16.0 * D[:, 2])
        assert np.abs(got - want).max() <= 4.0 * 2.0 ** -22
