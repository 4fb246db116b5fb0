"""Seeded synthetic plasma loads for the Photon-Plasma particle step.

This module only draws random numbers (numpy ``Generator(PCG64(seed))``) and lays
out particle arrays.  It contains none of the method's arithmetic, and it is the
one module that both the FP64 oracle's tests and the CUDA path's tests and
benchmark use, so that both sides see identical inputs.

Normalisation: c = eps0 = mu0 = 1, electron charge -1 and mass 1, lengths in
c/omega_pe where omega_pe is set by the TOTAL electron density n_e = 1.  The
weight ``w`` of a macro-particle is its number density, n_s / ppc_s.

Velocity recipe: proper velocity u = gamma*v.  A drifting thermal population
has u = Gamma_d * beta_d * e_drift + u_th * N(0, 1)^3.  A relativistic cold beam
(Gamma >= 2) draws the thermal part in its rest frame and is Lorentz-boosted
along x.  Positions are uniform inside each cell (a fixed number per cell), and
every negative particle is placed on top of a positive partner of the same
population, so that the initial charge density is exactly zero and E = B = 0
is a consistent initial condition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
import numpy as np


@dataclass
class Population:
    """One drifting Maxwellian population of a neutral pair of species."""
    ppc: int                 # macro-particles per cell for each of the two species
    density: float           # number density of each of the two species
    beta_drift: float = 0.0  # drift 3-velocity along x (units of c)
    u_th: float = 0.0        # thermal spread of the proper velocity per component
    boost: bool = False      # draw thermal part in the rest frame, then boost along x


@dataclass
class Load:
    n: tuple                 # cells (nx, ny, nz)
    d: tuple                 # cell size
    dt: float
    species: list            # list of dicts: q, m, w, x, y, z, ux, uy, uz (float64 arrays)
    params: dict = field(default_factory=dict)

    @property
    def n_particles(self) -> int:
        return int(sum(len(s["x"]) for s in self.species))


def _draw_u(rng, n, pop: Population):
    ux = rng.standard_normal(n) * pop.u_th
    uy = rng.standard_normal(n) * pop.u_th
    uz = rng.standard_normal(n) * pop.u_th
    b = pop.beta_drift
    if b == 0.0:
        return ux, uy, uz
    G = 1.0 / math.sqrt(1.0 - b * b)
    if not pop.boost:
        return ux + G * b, uy, uz
    # rest-frame proper velocity -> lab frame, boost with velocity b along x
    g_rest = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    return G * (ux + b * g_rest), uy, uz


def pair_plasma(n, d, dt, populations, seed, masses=(1.0, 1.0), cells=None) -> Load:
    """Neutral two-species load: species 0 has charge -1 and mass masses[0],
    species 1 has charge +1 and mass masses[1].

    ``cells`` optionally restricts the load to a subset of linear cell indices
    (x fastest); the draws for a cell do not depend on which other cells are
    loaded, so a subset equals the corresponding part of the full load.
    """
    nx, ny, nz = n
    ncell = nx * ny * nz
    cells = np.arange(ncell, dtype=np.int64) if cells is None else np.asarray(cells, dtype=np.int64)
    parts = {0: [], 1: []}
    for ip, pop in enumerate(populations):
        # one independent stream per (population, cell block) keeps subsets reproducible
        block = 4096
        for b0 in range(0, ncell, block):
            sel = cells[(cells >= b0) & (cells < b0 + block)]
            if sel.size == 0:
                continue
            rng = np.random.Generator(np.random.PCG64([seed, ip, b0 // block]))
            # draw the whole block so that the stream position of a cell is fixed
            nb = min(block, ncell - b0)
            c = np.arange(b0, b0 + nb, dtype=np.int64).repeat(pop.ppc)
            ri = rng.random((3, c.size))
            u0 = _draw_u(rng, c.size, pop)
            u1 = _draw_u(rng, c.size, pop)
            keep = np.isin(c, sel) if sel.size < nb else np.ones(c.size, dtype=bool)
            c = c[keep]
            ix = c % nx
            iy = (c // nx) % ny
            iz = c // (nx * ny)
            x = (ix + ri[0][keep]) * d[0]
            y = (iy + ri[1][keep]) * d[1]
            z = (iz + ri[2][keep]) * d[2]
            for sp, u in ((0, u0), (1, u1)):
                parts[sp].append((x, y, z, u[0][keep], u[1][keep], u[2][keep], pop))
    species = []
    for sp, q in ((0, -1.0), (1, 1.0)):
        chunks = parts[sp]
        if chunks:
            cols = [np.concatenate([ch[k] for ch in chunks]) for k in range(6)]
        else:
            cols = [np.zeros(0) for _ in range(6)]
        # weight: number density per macro-particle of the population it came from
        w = populations[0].density / populations[0].ppc
        for pop in populations:
            if abs(pop.density / pop.ppc - w) > 1e-15 * w:
                raise ValueError("populations of one species must share the macro-particle weight")
        species.append(dict(q=q, m=float(masses[sp]), w=w, x=cols[0], y=cols[1], z=cols[2],
                            ux=cols[3], uy=cols[4], uz=cols[5]))
    return Load(n=tuple(n), d=tuple(float(v) for v in d), dt=float(dt), species=species)


# --------------------------------------------------------------------------
# The paper-style workloads (sizes and distributions of its test problems).
# --------------------------------------------------------------------------

def two_stream(n=(16, 16, 16), seed=1211, ppc=8, beta=0.2, u_th=0.05) -> Load:
    """Counter-streaming neutral pair beams along x (+/-beta), TSC / 6th order,
    dx = 0.5, dt = 0.25; ppc macro-particles per cell per species split evenly
    between the two beams (16^3 cells, 65,536 particles at the defaults)."""
    half = ppc // 2
    pops = [Population(half, 0.5, +beta, u_th), Population(half, 0.5, -beta, u_th)]
    L = pair_plasma(n, (0.5, 0.5, 0.5), 0.25, pops, seed)
    L.params = dict(workload="two-stream", shape_order=2, field_order=6, alpha=0.55, beta=beta, u_th=u_th)
    return L


def thermal(n=(128, 128, 128), seed=1212, ppc=32, u_th=0.1, dx=0.1, dt=0.05, cells=None) -> Load:
    """Drift-free isotropic pair plasma for the numerical-heating test: PCS /
    6th order, dx = 0.1, dt = 0.05 (128^3 cells x 32 per cell per species =
    134,217,728 particles at the defaults)."""
    pops = [Population(ppc, 1.0, 0.0, u_th)]
    L = pair_plasma(n, (dx, dx, dx), dt, pops, seed, cells=cells)
    L.params = dict(workload="thermal", shape_order=3, field_order=6, alpha=0.55, u_th=u_th, sort_interval=20)
    return L


def weibel(n=(128, 128, 128), seed=1213, ppc=32, beta=0.5, u_th=0.1, dx=0.1, dt=0.05, cells=None) -> Load:
    """Counter-streaming pair beams (+/-beta along x, half of the macro-particles
    in each) for the filamentation variant."""
    half = ppc // 2
    pops = [Population(half, 0.5, +beta, u_th), Population(half, 0.5, -beta, u_th)]
    L = pair_plasma(n, (dx, dx, dx), dt, pops, seed, cells=cells)
    L.params = dict(workload="weibel", shape_order=3, field_order=6, alpha=0.55, beta=beta, u_th=u_th,
                    sort_interval=20)
    return L


def beam_background(n=(256, 128, 128), seed=1214, ppc=16, gamma_b=10.0, u_th_bg=0.01, mass_ratio=25.0,
                    cells=None) -> Load:
    """Electron-ion plasma (m_i/m_e = 25): a cold Gamma = 10 beam along +x through
    a background at rest with u_th = 0.01; each population has ppc macro-particles
    per cell per species and half of the electron density."""
    beta = math.sqrt(1.0 - 1.0 / (gamma_b * gamma_b))
    pops = [Population(ppc, 0.5, 0.0, u_th_bg), Population(ppc, 0.5, beta, 0.0, boost=True)]
    L = pair_plasma(n, (0.5, 0.5, 0.5), 0.25, pops, seed, masses=(1.0, mass_ratio), cells=cells)
    L.params = dict(workload="beam-background", shape_order=3, field_order=6, alpha=0.55, gamma_b=gamma_b)
    return L


def wall_beam(n=(256, 128, 128), seed=1218, ppc=32, gamma_b=10.0, mass_ratio=25.0, cells=None) -> Load:
    """The beam of the wall-shock setup: a cold Gamma = 10 electron-ion beam
    (m_i/m_e = 25) along +x filling a box between walls, ppc macro-particles
    per cell per species, dx = 0.5, dt = 0.25.  The inflow through the open
    end continues it: params hold the drift proper velocity and the seed."""
    beta = math.sqrt(1.0 - 1.0 / (gamma_b * gamma_b))
    pops = [Population(ppc, 1.0, beta, 0.0, boost=True)]
    L = pair_plasma(n, (0.5, 0.5, 0.5), 0.25, pops, seed, masses=(1.0, mass_ratio), cells=cells)
    L.params = dict(workload="wall-shock", shape_order=3, field_order=6, alpha=0.55, gamma_b=gamma_b,
                    u_drift=math.sqrt(gamma_b * gamma_b - 1.0), ppc=ppc, seed=seed)
    return L


def single_particle(n, d, dt, x, u, q=-1.0, m=1.0, w=1.0) -> Load:
    """One macro-particle (used by the deposit pins and the edge cases)."""
    arr = lambda v: np.array([float(v)])
    sp = dict(q=q, m=m, w=w, x=arr(x[0]), y=arr(x[1]), z=arr(x[2]), ux=arr(u[0]), uy=arr(u[1]), uz=arr(u[2]))
    return Load(n=tuple(n), d=tuple(d), dt=dt, species=[sp])


def random_particles(n, d, dt, count, seed, u_scale=0.3, q=-1.0, m=1.0, w=0.05) -> Load:
    """Particles at uniform random positions with Gaussian proper velocities
    (a generic, non-neutral load for ragged and edge-case parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = [n[a] * d[a] for a in range(3)]
    sp = dict(q=q, m=m, w=w,
              x=rng.random(count) * L[0], y=rng.random(count) * L[1], z=rng.random(count) * L[2],
              ux=rng.standard_normal(count) * u_scale, uy=rng.standard_normal(count) * u_scale,
              uz=rng.standard_normal(count) * u_scale)
    for k in ("x", "y", "z"):
        a = "xyz".index(k)
        sp[k] = np.minimum(sp[k], np.nextafter(L[a], 0.0))
    return Load(n=tuple(n), d=tuple(d), dt=dt, species=[sp])


def random_fields(n, seed, amp=0.05):
    """Random E and B, each component a sum of three random low Fourier modes
    plus 10% white noise, shape (nz, ny, nx).  B is not divergence-free;
    callers that need div B = 0 build B from a curl themselves."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for _ in range(6):
        f = np.zeros((nz, ny, nx))
        for _m in range(3):
            k = rng.integers(0, 3, size=3)
            ph = rng.random() * 2 * np.pi
            f += rng.standard_normal() * np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + ph)
        f += 0.1 * rng.standard_normal((nz, ny, nx))
        out.append(amp * f)
    return out[:3], out[3:]


def quiet_two_stream(nx=32, ntr=2, dx=0.25, dt=0.125, ppc=8, beta=0.2, mode=2, eps=1e-6) -> Load:
    """Noise-free (quiet-start) cold two-stream load: four co-located populations
    (electrons and positrons of a +beta and a -beta beam along x, density 1/2
    each) on a regular lattice, ppc per cell along x and one per cell in y and z,
    with a seeded velocity perturbation eps*sin(k x) on the +beta electrons,
    k = 2*pi*mode/(nx*dx).  Transverse uniformity makes the problem
    one-dimensional; the charge density starts exactly at zero."""
    Lx = nx * dx
    G = 1.0 / math.sqrt(1.0 - beta * beta)
    i = np.arange(nx).repeat(ppc)
    s = np.tile(np.arange(ppc), nx)
    x1 = (i + (s + 0.5) / ppc) * dx
    xs, ys, zs = [], [], []
    for k in range(ntr):
        for j in range(ntr):
            xs.append(x1)
            ys.append(np.full(x1.size, (j + 0.5) * dx))
            zs.append(np.full(x1.size, (k + 0.5) * dx))
    x = np.concatenate(xs); y = np.concatenate(ys); z = np.concatenate(zs)
    kx = 2.0 * np.pi * mode / Lx
    pert = eps * np.sin(kx * x)
    zero = np.zeros_like(x)
    w = 0.5 / ppc
    species = []
    for q in (-1.0, 1.0):
        for sgn in (+1.0, -1.0):
            ux = sgn * G * beta + (pert if (q < 0 and sgn > 0) else 0.0)
            species.append(dict(q=q, m=1.0, w=w, x=x.copy(), y=y.copy(), z=z.copy(),
                                ux=np.asarray(ux, dtype=np.float64) + zero, uy=zero.copy(), uz=zero.copy()))
    L = Load(n=(nx, ntr, ntr), d=(dx, dx, dx), dt=dt, species=species)
    L.params = dict(workload="quiet-two-stream", beta=beta, mode=mode, k=kx)
    return L


def quiet_weibel(ny=32, ntr=8, dx=0.25, dt=0.1, ppc=4, beta=0.5, mode=2, eps=1e-6) -> Load:
    """Noise-free (quiet-start) cold filamentation (Weibel) load: four co-located
    populations (electrons and positrons of a +beta and a -beta beam along x,
    density 1/2 each) on a regular lattice, ppc per cell along y and one per
    cell in x and z, on ntr x ny x ntr cells, with a seeded velocity
    perturbation eps*sin(k y) on the +beta electrons (a current modulation
    across the beams), k = 2*pi*mode/(ny*dx).  Uniform along the beams and
    along z, the problem is one-dimensional in y; the charge density starts
    exactly at zero."""
    Ly = ny * dx
    G = 1.0 / math.sqrt(1.0 - beta * beta)
    j = np.arange(ny).repeat(ppc)
    s = np.tile(np.arange(ppc), ny)
    y1 = (j + (s + 0.5) / ppc) * dx
    xs, ys, zs = [], [], []
    for k in range(ntr):
        for i in range(ntr):
            ys.append(y1)
            xs.append(np.full(y1.size, (i + 0.5) * dx))
            zs.append(np.full(y1.size, (k + 0.5) * dx))
    x = np.concatenate(xs); y = np.concatenate(ys); z = np.concatenate(zs)
    ky = 2.0 * np.pi * mode / Ly
    pert = eps * np.sin(ky * y)
    zero = np.zeros_like(x)
    w = 0.5 / ppc
    species = []
    for q in (-1.0, 1.0):
        for sgn in (+1.0, -1.0):
            ux = sgn * G * beta + (pert if (q < 0 and sgn > 0) else 0.0)
            species.append(dict(q=q, m=1.0, w=w, x=x.copy(), y=y.copy(), z=z.copy(),
                                ux=np.asarray(ux, dtype=np.float64) + zero, uy=zero.copy(), uz=zero.copy()))
    L = Load(n=(ntr, ny, ntr), d=(dx, dx, dx), dt=dt, species=species)
    L.params = dict(workload="quiet-weibel", beta=beta, mode=mode, k=ky)
    return L


def heating_plasma(n=(32, 32, 32), ppc=8, u_th=0.1, mass_ratio=16.0, dx=0.1, dt=0.05, seed=1219) -> Load:
    """The numerical-heating set-up (Sec. VIII) in 3D: electrons and ions of
    mass ratio 16 at rest, both with thermal proper velocity u_th per component,
    ten cells per skin depth, ppc per cell per species (pair-co-located)."""
    pops = [Population(ppc, 1.0, 0.0, u_th)]
    L = pair_plasma(n, (dx, dx, dx), dt, pops, seed, masses=(1.0, mass_ratio))
    L.params = dict(workload="heating", ppc=ppc, u_th=u_th, mass_ratio=mass_ratio)
    return L


# --------------------------------------------------------------------------
# Independent-run workloads of the batched and served forms.
# --------------------------------------------------------------------------

def run_load(req) -> Load:
    """The seeded load of one independent run described by a request dict
    (kind, n, ppc, plasma, seed; see batched_runs / serving_trace)."""
    n = (req["n"],) * 3
    masses = (1.0, 25.0) if req.get("plasma") == "ion" else (1.0, 1.0)
    ppc = max(2, int(req["ppc"]) // 2 * 2)
    # two-stream and Weibel loads are both counter-streaming neutral beams along x;
    # they differ in drift and temperature (set by the request)
    pops = [Population(ppc // 2, 0.5, +req["beta"], req["u_th"]), Population(ppc // 2, 0.5, -req["beta"], req["u_th"])]
    dx = req.get("dx", 0.5)
    L = pair_plasma(n, (dx, dx, dx), 0.5 * dx, pops, req["seed"], masses=masses)
    L.params = dict(workload=req["kind"], shape_order=req.get("shape", 3), field_order=6, alpha=0.55)
    return L


def run_counts(req) -> list:
    """Particles per species of the load run_load(req) builds (without building it)."""
    ppc = max(2, int(req["ppc"]) // 2 * 2)
    return [int(req["n"]) ** 3 * ppc] * 2


def batched_runs(n_runs=64, seed=1215, edges=tuple(range(16, 97, 8)), ppc=(8, 64), steps=300):
    """64 independent runs of uneven size: cubic edge uniform in {16, 24, .., 96},
    ppc per species uniform in [8, 64], drift 0.05..0.5 c, u_th 0.01..0.1 c,
    TSC or PCS by coin flip (two-stream pair plasmas)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_runs):
        out.append(dict(kind="two-stream", n=int(rng.choice(edges)), ppc=int(rng.integers(ppc[0], ppc[1] + 1)),
                        beta=float(rng.uniform(0.05, 0.5)), u_th=float(rng.uniform(0.01, 0.1)),
                        shape=int(rng.choice([2, 3])), plasma="pair", steps=int(steps), seed=seed * 1000 + k))
    return out


def serving_trace(n_requests=256, rate=20.0, seed=1216, edges=tuple(range(32, 193, 16)), ppc=(8, 32),
                  steps=(200, 1000)):
    """Poisson arrivals (mean `rate` per second) of two-stream and Weibel runs:
    cubic edge from `edges`, ppc per species in [ppc], pair or mass-ratio-25
    plasma, steps uniform in [steps]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        kind = "two-stream" if rng.random() < 0.5 else "weibel"
        out.append(dict(arrival=t, kind=kind, n=int(rng.choice(edges)), ppc=int(rng.integers(ppc[0], ppc[1] + 1)),
                        beta=0.2 if kind == "two-stream" else 0.5, u_th=0.05 if kind == "two-stream" else 0.1,
                        plasma="pair" if rng.random() < 0.5 else "ion", shape=3,
                        steps=int(rng.integers(steps[0], steps[1] + 1)), seed=seed * 1000 + k))
    return out
