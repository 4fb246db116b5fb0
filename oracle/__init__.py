"""FP64 CPU oracle of the Photon-Plasma particle step (arXiv:1211.4575).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never imports, links or calls it, and it imports nothing from
the product package.

The arithmetic lives in ``pp_oracle.c`` (plain C, one literal loop per
definition of the paper, cited per function).  This module compiles that
file with gcc and marshals numpy arrays to it with ctypes.  The one piece of
method written here, in numpy, is the reflecting wall's construction by
virtual images (WallSimulation, at the end): it adds particles and mirrors
arrays, and every step still runs in the C code.

Array conventions: fields are numpy float64 arrays of shape (nz, ny, nx)
(x fastest in memory), with the Yee staggering of the paper's Sec. III:
E_x, J_x at (i+1/2, j, k), B_x at (i, j+1/2, k+1/2), cyclic for y and z.
Positions are physical, in [0, n*dx).  c = eps0 = mu0 = 1.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pp_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")

VAY, BORIS = 0, 1


def build(force: bool = False) -> str:
    """Compile pp_oracle.c into oracle/_build/liboracle.so (gcc -O2, with
    OpenMP where gcc has it: the particle loop then runs on set_threads(n)
    threads, one by default)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(base)
    os.replace(tmp, _OUT)
    return _OUT


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double),
                ("field_order", C.c_int), ("alpha", C.c_double), ("shape_order", C.c_int),
                ("pusher", C.c_int), ("relax_max_iter", C.c_int), ("relax_tol", C.c_double),
                ("field_solver", C.c_int), ("current_mode", C.c_int)]


class Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("w", C.c_double), ("n", C.c_int64),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p), ("rad", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("energy_E", C.c_double), ("energy_B", C.c_double), ("energy_Ex", C.c_double),
                ("kinetic", C.c_double), ("charge", C.c_double), ("gauss_max", C.c_double),
                ("rho_max", C.c_double), ("divB_max", C.c_double), ("relax_iters", C.c_int),
                ("relax_residual", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.orc_weight.restype = C.c_double
        L.orc_weight.argtypes = [C.c_int, C.c_double]
        L.orc_fd_coeffs.argtypes = [C.c_int, P]
        L.orc_diff.argtypes = [C.POINTER(Grid), C.c_int, C.c_int, C.c_int, P, P]
        L.orc_gather.argtypes = [C.POINTER(Grid), P, P, P, P, P]
        L.orc_push_vay.argtypes = [C.c_double, P, P, P]
        L.orc_push_boris.argtypes = [C.c_double, P, P, P]
        L.orc_radiate.argtypes = [C.c_double, C.c_double, P, P]
        L.orc_deposit_particle.argtypes = [C.POINTER(Grid), C.c_double, C.c_double, P, P, P, P]
        L.orc_current_from_drho.argtypes = [C.POINTER(Grid), P, P, P]
        L.orc_field_update.argtypes = [C.POINTER(Grid), P, P, P, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.orc_particles_deposit.argtypes = [C.POINTER(Grid), P, P, C.POINTER(Species), C.c_int, P]
        L.orc_step4.argtypes = [C.POINTER(Grid), P, P, P, C.POINTER(Species), C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.orc_step4_coeffs.argtypes = [P, P]
        L.orc_step.argtypes = [C.POINTER(Grid), P, P, P, C.POINTER(Species), C.c_int,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.orc_rho.argtypes = [C.POINTER(Grid), C.POINTER(Species), C.c_int, P]
        L.orc_div_minus.argtypes = [C.POINTER(Grid), P, P]
        L.orc_div_plus.argtypes = [C.POINTER(Grid), P, P]
        L.orc_divergence_filter.argtypes = [C.POINTER(Grid), P, P, P, C.c_int]
        L.orc_diagnostics.argtypes = [C.POINTER(Grid), P, P, C.POINTER(Species), C.c_int, C.POINTER(Diag)]
        L.orc_philox4x32.argtypes = [P, P, P]
        L.orc_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, P]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def _ptr3(arrs):
    """Array of three double* (for the C functions taking double *F[3])."""
    t = (C.c_void_p * 3)(*[a.ctypes.data for a in arrs])
    return t


IMPLICIT, EXPLICIT = 0, 1
CHARGE_CONSERVING, DIRECT = 0, 1


def make_grid(n, d, dt, field_order=6, alpha=0.55, shape_order=2, pusher=VAY,
              relax_max_iter=200, relax_tol=1e-14, field_solver=IMPLICIT, current_mode=CHARGE_CONSERVING) -> Grid:
    g = Grid()
    g.n[:] = list(n)
    g.d[:] = [float(v) for v in d]
    g.dt = float(dt)
    g.field_order = int(field_order)
    g.alpha = float(alpha)
    g.shape_order = int(shape_order)
    g.pusher = int(pusher)
    g.relax_max_iter = int(relax_max_iter)
    g.relax_tol = float(relax_tol)
    g.field_solver = int(field_solver)
    g.current_mode = int(current_mode)
    return g


def weight(order: int, delta: float) -> float:
    """W^order(delta) exactly as printed in Sec. II."""
    return lib().orc_weight(int(order), float(delta))


def fd_coeffs(order: int) -> np.ndarray:
    k = np.zeros(3)
    lib().orc_fd_coeffs(int(order), _ptr(k))
    return k


def diff(g: Grid, f: np.ndarray, axis: int, direction: int, order: int | None = None) -> np.ndarray:
    """Staggered derivative of a (nz, ny, nx) array along axis 0=x,1=y,2=z."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().orc_diff(C.byref(g), int(order if order is not None else g.field_order), int(axis),
                   int(direction), _ptr(f), _ptr(out))
    return out


def gather(g: Grid, E, B, xp):
    xp = np.asarray(xp, dtype=np.float64)
    Ep, Bp = np.zeros(3), np.zeros(3)
    Ec = [np.ascontiguousarray(a, dtype=np.float64) for a in E]
    Bc = [np.ascontiguousarray(a, dtype=np.float64) for a in B]
    lib().orc_gather(C.byref(g), _ptr3(Ec), _ptr3(Bc), _ptr(xp), _ptr(Ep), _ptr(Bp))
    return Ep, Bp


def push(qmdt: float, E, B, u, pusher=VAY) -> np.ndarray:
    E = np.asarray(E, dtype=np.float64).copy()
    B = np.asarray(B, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).copy()
    f = lib().orc_push_vay if pusher == VAY else lib().orc_push_boris
    f(float(qmdt), _ptr(E), _ptr(B), _ptr(u))
    return u


def radiate(K: float, dt: float, um, u) -> np.ndarray:
    """Radiative cooling of one push: p- = um, p+^EM = u; returns p+."""
    um = np.asarray(um, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64).copy()
    lib().orc_radiate(float(K), float(dt), _ptr(um), _ptr(u))
    return u


def step4_coeffs():
    """Drift (a) and kick (b) fractions of the four substeps of the 4th-order step."""
    a = np.zeros(4)
    b = np.zeros(4)
    lib().orc_step4_coeffs(_ptr(a), _ptr(b))
    return a, b


def deposit_particle(g: Grid, q, w, x0, x1, Drho=None, lsum=None):
    """Accumulate one particle's D rho (3 mesh arrays) and line sums."""
    nx, ny, nz = g.n
    if Drho is None:
        Drho = [np.zeros((nz, ny, nx)) for _ in range(3)]
    if lsum is None:
        # lsum[a] is indexed [t_c, t_b] with b = a+1, c = a+2 (mod 3), t_b fastest
        n = (nx, ny, nz)
        lsum = [np.zeros((n[(a + 2) % 3], n[(a + 1) % 3])) for a in range(3)]
    x0 = np.asarray(x0, dtype=np.float64)
    x1 = np.asarray(x1, dtype=np.float64)
    lib().orc_deposit_particle(C.byref(g), float(q), float(w), _ptr(x0), _ptr(x1), _ptr3(Drho), _ptr3(lsum))
    return Drho, lsum


def current_from_drho(g: Grid, Drho, lsum):
    nx, ny, nz = g.n
    J = [np.zeros((nz, ny, nx)) for _ in range(3)]
    lib().orc_current_from_drho(C.byref(g), _ptr3(Drho), _ptr3(lsum), _ptr3(J))
    return J


def field_update(g: Grid, E, B, J):
    """Advance E, B (lists of 3 arrays, modified in place). Returns (iters, residual)."""
    it = C.c_int(0)
    res = C.c_double(0.0)
    lib().orc_field_update(C.byref(g), _ptr3(E), _ptr3(B), _ptr3(J), C.byref(it), C.byref(res))
    return it.value, res.value


def div_minus(g: Grid, F) -> np.ndarray:
    out = np.zeros_like(F[0])
    lib().orc_div_minus(C.byref(g), _ptr3(F), _ptr(out))
    return out


def div_plus(g: Grid, F) -> np.ndarray:
    out = np.zeros_like(F[0])
    lib().orc_div_plus(C.byref(g), _ptr3(F), _ptr(out))
    return out


class Simulation:
    """The oracle's whole step over numpy-held state (one FP64 copy per array)."""

    def __init__(self, n, d, dt, field_order=6, alpha=0.55, shape_order=2, pusher=VAY,
                 relax_max_iter=200, relax_tol=1e-14, integrator=2, field_solver=IMPLICIT,
                 current_mode=CHARGE_CONSERVING, filter_passes=0, filter_interval=1):
        """integrator 2: leap-frog step; 4: the four-substep 4th-order step.
        field_solver IMPLICIT (eq:EllipticB) or EXPLICIT (6th-order FDTD).
        current_mode CHARGE_CONSERVING (eq:jj6) or DIRECT (eq:jj2).  After every
        filter_interval-th step, filter_passes divergence-filter passes."""
        self.filter_passes = int(filter_passes)
        self.filter_interval = max(1, int(filter_interval))
        if integrator not in (2, 4):
            raise ValueError("integrator must be 2 or 4")
        self.integrator = integrator
        self.g = make_grid(n, d, dt, field_order, alpha, shape_order, pusher, relax_max_iter, relax_tol,
                           field_solver, current_mode)
        nx, ny, nz = n
        self.E = [np.zeros((nz, ny, nx)) for _ in range(3)]
        self.B = [np.zeros((nz, ny, nx)) for _ in range(3)]
        self.J = [np.zeros((nz, ny, nx)) for _ in range(3)]
        self.species: list[dict] = []
        self.relax_iters = 0
        self.relax_residual = 0.0
        self.nstep = 0

    def add_species(self, q, m, w, x, y, z, ux, uy, uz, rad=0.0) -> int:
        """rad: coefficient mu0 q^2 / (6 pi m c) of radiative cooling (0 = off)."""
        arrs = {k: np.ascontiguousarray(v, dtype=np.float64).copy()
                for k, v in dict(x=x, y=y, z=z, ux=ux, uy=uy, uz=uz).items()}
        self.species.append(dict(q=float(q), m=float(m), w=float(w), rad=float(rad), **arrs))
        return len(self.species) - 1

    def _sp(self):
        arr = (Species * max(1, len(self.species)))()
        for i, s in enumerate(self.species):
            arr[i].q, arr[i].m, arr[i].w, arr[i].n = s["q"], s["m"], s["w"], len(s["x"])
            arr[i].rad = s["rad"]
            for k in ("x", "y", "z", "ux", "uy", "uz"):
                setattr(arr[i], k, s[k].ctypes.data)
        return arr

    def load_fields(self, E, B):
        for a in range(3):
            self.E[a][...] = E[a]
            self.B[a][...] = B[a]

    def deposit(self):
        """Gather, push, move and deposit every particle; J receives J^{n+1}."""
        lib().orc_particles_deposit(C.byref(self.g), _ptr3(self.E), _ptr3(self.B), self._sp(),
                                    len(self.species), _ptr3(self.J))

    def field_update(self):
        self.relax_iters, self.relax_residual = field_update(self.g, self.E, self.B, self.J)

    def step(self, n: int = 1):
        it = C.c_int(0)
        res = C.c_double(0.0)
        f = lib().orc_step4 if self.integrator == 4 else lib().orc_step
        for _ in range(n):
            f(C.byref(self.g), _ptr3(self.E), _ptr3(self.B), _ptr3(self.J), self._sp(),
              len(self.species), C.byref(it), C.byref(res))
            self.nstep += 1
            if self.filter_passes and self.nstep % self.filter_interval == 0:
                self.divergence_filter(self.filter_passes)
        self.relax_iters, self.relax_residual = it.value, res.value

    def divergence_filter(self, passes: int):
        """passes smoothing steps of E towards div E = rho and of B towards div B = 0."""
        lib().orc_divergence_filter(C.byref(self.g), _ptr3(self.E), _ptr3(self.B), _ptr(self.rho()), int(passes))

    def rho(self) -> np.ndarray:
        nx, ny, nz = self.g.n
        out = np.zeros((nz, ny, nx))
        lib().orc_rho(C.byref(self.g), self._sp(), len(self.species), _ptr(out))
        return out

    def diagnostics(self) -> dict:
        d = Diag()
        lib().orc_diagnostics(C.byref(self.g), _ptr3(self.E), _ptr3(self.B), self._sp(), len(self.species),
                              C.byref(d))
        out = {k: getattr(d, k) for k, _ in Diag._fields_}
        out["relax_iters"] = self.relax_iters
        out["relax_residual"] = self.relax_residual
        return out


# ---------------------------------------------------------------------------
# Reflecting walls (Sec. V "Boundary conditions"): walls at x = 0 and
# x = L = n_x dx, both on integer (charge-density) nodes.  The paper defines
# the wall through virtual particles: every particle inside has a mirror
# image outside, x -> 2 x_b - x with the normal momentum reversed, and the
# fields obey the symmetries of the Maxwell equations across the wall.  Taken
# literally, that is the periodic system of the particles and their images in
# the mirror-extended box of 2 n_x cells in x (mirror planes at 0 and L;
# periodicity 2L makes each one the image of the other).  This oracle runs
# exactly that system: the images are real particles of the periodic oracle,
# nothing is folded or reflected.  A physical particle is, after any step, the
# member of its pair that lies in [0, L].
#
# Parities across a wall with normal x (the paper's table): quantities
# staggered in x (E_x, J_x at i+1/2; B_y, B_z at i+1/2) are odd, quantities on
# integer x nodes (rho, E_y, E_z, J_y, J_z, B_x) are even.
# ---------------------------------------------------------------------------
WALL_PARITY = {"E": ((True, -1.0), (False, 1.0), (False, 1.0)),
               "B": ((False, 1.0), (True, -1.0), (True, -1.0)),
               "J": ((True, -1.0), (False, 1.0), (False, 1.0))}


def mirror_x(f: np.ndarray, half: bool, sign: float) -> np.ndarray:
    """The mirror image across x = 0 of a mesh array of the extended box: node i
    maps to -i, node i+1/2 to -(i+1/2), i.e. index -1-i (all mod 2 n_x)."""
    N = f.shape[-1]
    i = np.arange(N)
    idx = (N - 1 - i) if half else (-i) % N
    return sign * f[..., idx]


def wall_parity(kind: str, comp: int, axis: int):
    """(staggered along the normal, sign) of component comp of E, B or J across
    a wall with normal `axis`: E_a and J_a are staggered along a, B_b along
    every axis but b; staggered components are odd, the others even.  For
    axis 0 this is WALL_PARITY."""
    half = (comp == axis) if kind in ("E", "J") else (comp != axis)
    return half, (-1.0 if half else 1.0)


def mirror(f: np.ndarray, axis: int, half: bool, sign: float) -> np.ndarray:
    """mirror_x along mesh axis `axis` (0 = x, the last array axis)."""
    return np.moveaxis(mirror_x(np.moveaxis(np.asarray(f, dtype=np.float64), 2 - axis, -1), half, sign), -1, 2 - axis)


def wall_symmetrise(F, kind: str, axes=(0,)):
    """Projection of three mesh arrays of the extended box onto the mirror-
    symmetric state, f -> (f + P f(mirror)) / 2, across each walled axis in turn
    (the projections commute)."""
    out = [np.asarray(F[a], dtype=np.float64) for a in range(3)]
    for ax in axes:
        out = [0.5 * (out[a] + mirror(out[a], ax, *wall_parity(kind, a, ax))) for a in range(3)]
    return out


def philox4x32(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (reading R23)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32(C.cast(c, C.c_void_p), C.cast(k, C.c_void_p), C.cast(o, C.c_void_p))
    return tuple(o)


def set_threads(n: int) -> int:
    """Threads of the oracle's particle loop (per-thread deposit copies, added
    after the loop); returns the number in effect (1 without OpenMP).  One by
    default: the parity tests use the oracle single-threaded."""
    return int(lib().orc_set_threads(int(n)))


def draws(seed: int, step: int, stream: int, n: int) -> np.ndarray:
    """(n, 4) uniforms in (0, 1): draw i = Philox of counter (i, 0, step, stream)."""
    out = np.zeros((max(int(n), 0), 4))
    if n > 0:
        lib().orc_draws(int(seed) & (2 ** 64 - 1), int(step) & 0xFFFFFFFF, int(stream) & 0xFFFFFFFF, int(n),
                        _ptr(out))
    return out


def gaussians(D: np.ndarray) -> np.ndarray:
    """Three standard normals per row of four uniforms (Box-Muller on (u0, u1)
    and (u2, u3))."""
    r0 = np.sqrt(-2.0 * np.log(D[:, 0]))
    r1 = np.sqrt(-2.0 * np.log(D[:, 2]))
    return np.stack([r0 * np.cos(2 * np.pi * D[:, 1]), r0 * np.sin(2 * np.pi * D[:, 1]),
                     r1 * np.cos(2 * np.pi * D[:, 3])], 1)


# Damped components of the outflow layer, bit a for E_a and 3 + a for B_a:
# by default those transverse to the wall normal x (reading R22).
TRANSVERSE = (1 << 1) | (1 << 2) | (1 << 4) | (1 << 5)


class WallSimulation:
    """Reflecting walls at 0 and L_a = n[a] d[a] on each axis a with walls[a]
    (x only by default; the others periodic): the periodic oracle on the
    mirror-extended box (2 n[a] cells on each walled axis), with every
    particle's virtual images (one per subset of the walled axes) loaded as
    particles.  Mesh arrays (fields, J, rho) are those of the extended box.
    Energies, charge and kinetic energy in diagnostics() are those of the
    physical box (the extended box's sums over 2^k, k walled axes).  The open
    end, the injector and the window act on x and need walls on x."""

    def __init__(self, n, d, dt, walls=(True, False, False), **kw):
        self.walls = tuple(bool(w) for w in walls)
        self.axes = [a for a in range(3) if self.walls[a]]
        if not self.axes:
            raise ValueError("at least one walled axis")
        self.Ls = [n[a] * float(d[a]) for a in range(3)]
        ext = tuple(2 * n[a] if self.walls[a] else n[a] for a in range(3))
        nx, ny, nz = n
        self.nx = int(nx)
        self.L = nx * float(d[0])
        self.sim = Simulation(ext, d, dt, **kw)
        self.counts: list[int] = []
        self.d = tuple(float(v) for v in d)
        self.dt = float(dt)
        self.nyz = (int(ny), int(nz))
        self.nstep = 0
        self.open = None
        self.injectors: dict = {}
        self.window = None
        self.shifts = 0

    @property
    def g(self):
        return self.sim.g

    @property
    def E(self):
        return self.sim.E

    @property
    def B(self):
        return self.sim.B

    @property
    def J(self):
        return self.sim.J

    @property
    def species(self):
        """Physical particles of each species (see particles())."""
        return [self.particles(s) for s in range(len(self.counts))]

    def add_species(self, q, m, w, x, y, z, ux, uy, uz, rad=0.0) -> int:
        phys = {k: np.asarray(v, dtype=np.float64).copy()
                for k, v in dict(x=x, y=y, z=z, ux=ux, uy=uy, uz=uz).items()}
        for a in self.axes:
            p = phys["xyz"[a]]
            if np.any(p < 0.0) or np.any(p > self.Ls[a]):
                raise ValueError("positions must lie between the walls")
        self.sim.add_species(q, m, w, *[np.zeros(0)] * 6, rad=rad)
        self.counts.append(0)
        sid = len(self.counts) - 1
        self._set_pairs(sid, phys)
        return sid

    def load_fields(self, E, B):
        """Extended-box arrays, projected onto the mirror-symmetric state."""
        self.sim.load_fields(wall_symmetrise(E, "E", self.axes), wall_symmetrise(B, "B", self.axes))

    # -- open lower end, injector, sliding window (readings R22-R24) ---------
    def set_open_boundary(self, cells: int, damping: float, escape: float, components: int = TRANSVERSE):
        """Outflow layer of `cells` cells at x = 0 (the other wall stays)."""
        if not self.walls[0]:
            raise ValueError("the open end needs walls on x")
        self.open = dict(cells=int(cells), damping=float(damping), escape=float(escape), mask=int(components))

    def set_injector(self, sid: int, ppc: float, u, u_th: float, seed: int):
        """Inflow through x = 0 of species sid: ppc particles per cell, drift
        proper velocity u (u[0] > 0), thermal spread u_th, Philox seed."""
        if not self.walls[0]:
            raise ValueError("the injector needs walls on x")
        self.injectors[sid] = dict(ppc=float(ppc), u=np.asarray(u, dtype=np.float64), u_th=float(u_th),
                                   seed=int(seed), k0=self.nstep)

    def set_window(self, v: float):
        """Sliding window at speed v against x (content moves one cell up)."""
        if not self.walls[0]:
            raise ValueError("the window needs walls on x")
        self.window = dict(v=float(v), k0=self.nstep)

    def _set_pairs(self, sid, phys: dict, keep=None):
        """Replace species sid by the given physical particles and their images:
        copy s (s = 0 .. 2^k - 1) mirrors the walled axes whose bit is set in s,
        x_a -> 2 L_a - x_a and u_a -> -u_a; copy 0 is the particles themselves."""
        if keep is not None:
            phys = {k: v[keep] for k, v in phys.items()}
        copies = []
        for sub in range(1 << len(self.axes)):
            c = {k: v.copy() for k, v in phys.items()}
            for bit, a in enumerate(self.axes):
                if (sub >> bit) & 1:
                    p = c["xyz"[a]]
                    c["xyz"[a]] = np.where(p > 0.0, 2.0 * self.Ls[a] - p, 0.0)
                    c["u" + "xyz"[a]] = -c["u" + "xyz"[a]]
            copies.append(c)
        s = self.sim.species[sid]
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            s[k] = np.concatenate([c[k] for c in copies])
        self.counts[sid] = len(phys["x"])

    def _damp(self):
        o = self.open
        N = 2 * self.nx
        for kind, F in (("E", self.sim.E), ("B", self.sim.B)):
            for a in range(3):
                if not (o["mask"] >> (a + (3 if kind == "B" else 0))) & 1:
                    continue
                pos = np.arange(N) + (0.5 if WALL_PARITY[kind][a][0] else 0.0)
                dist = np.minimum(pos, N - pos)
                f = np.where(dist < o["cells"], 1.0 - o["damping"] * ((o["cells"] - dist) / o["cells"]) ** 2, 1.0)
                F[a] *= f

    def _escape(self):
        lim = self.open["escape"] * self.d[0]
        for sid in range(len(self.counts)):
            p = self.particles(sid)
            self._set_pairs(sid, p, keep=~((p["x"] < lim) & (p["ux"] < 0.0)))

    def _append(self, sid, new: dict):
        p = self.particles(sid)
        self._set_pairs(sid, {k: np.concatenate([p[k], new[k]]) for k in p})

    def _draw_particles(self, inj, sid, count, step, stream, thick):
        D = draws(inj["seed"], step, stream, count)
        G = gaussians(draws(inj["seed"], step, stream + 1 + sid, count))
        ny, nz = self.nyz
        return dict(x=thick * D[:, 0], y=(ny * self.d[1]) * D[:, 1], z=(nz * self.d[2]) * D[:, 2],
                    ux=inj["u"][0] + inj["u_th"] * G[:, 0], uy=inj["u"][1] + inj["u_th"] * G[:, 1],
                    uz=inj["u"][2] + inj["u_th"] * G[:, 2])

    def _inject(self, sid):
        inj = self.injectors[sid]
        k = self.nstep - inj["k0"]
        u = inj["u"]
        vx = u[0] / np.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
        ny, nz = self.nyz
        rate = inj["ppc"] * ny * nz * vx * self.dt / self.d[0]
        count = int(np.floor(k * rate) - np.floor((k - 1) * rate))
        self._append(sid, self._draw_particles(inj, sid, count, self.nstep, 0, vx * self.dt))

    def _slide(self):
        w = self.window
        k = self.nstep - w["k0"]
        step_frac = w["v"] * self.dt / self.d[0]
        if np.floor(k * step_frac) <= np.floor((k - 1) * step_frac):
            return
        self.shifts += 1
        nx, N = self.nx, 2 * self.nx
        for kind, F in (("E", self.sim.E), ("B", self.sim.B)):
            for a in range(3):
                half, sign = WALL_PARITY[kind][a]
                top = nx - 1 if half else nx          # last node of the physical half
                f = F[a]
                f[..., 1:top + 1] = f[..., 0:top].copy()
                f[..., 0] = 0.0
                i = np.arange(0 if half else 1, nx)
                f[..., (N - 1 - i) if half else (N - i)] = sign * f[..., i]
        for sid in range(len(self.counts)):
            p = self.particles(sid)
            p["x"] = p["x"] + self.d[0]
            self._set_pairs(sid, p, keep=p["x"] <= self.L)
        ny, nz = self.nyz
        for sid in sorted(self.injectors):
            inj = self.injectors[sid]
            count = int(np.floor(inj["ppc"] * ny * nz + 0.5))
            self._append(sid, self._draw_particles(inj, sid, count, self.shifts, 16, self.d[0]))

    def step(self, n: int = 1):
        """Each step: the periodic step of the extended box, then the particles
        that left through the open end go (they moved out in this step's push),
        then the divergence filter when due (its rho without them), the layer's
        damping, the inflow, and the window shift."""
        for _ in range(n):
            passes = self.sim.filter_passes
            self.sim.filter_passes = 0
            self.sim.step(1)
            self.sim.filter_passes = passes
            self.nstep += 1
            if self.open is not None:
                self._escape()
            if passes and self.sim.nstep % self.sim.filter_interval == 0:
                self.sim.divergence_filter(passes)
            if self.open is not None:
                self._damp()
            for sid in sorted(self.injectors):
                self._inject(sid)
            if self.window is not None:
                self._slide()

    def particles(self, sid: int) -> dict:
        """The member of each particle's set of images that lies between the
        walls on every walled axis."""
        s = self.sim.species[sid]
        n = self.counts[sid]
        ncopy = 1 << len(self.axes)
        out = {k: s[k][:n].copy() for k in ("x", "y", "z", "ux", "uy", "uz")}
        found = np.zeros(n, dtype=bool)
        for c in range(ncopy):
            blk = slice(c * n, (c + 1) * n)
            inside = ~found
            for a in self.axes:
                inside &= s["xyz"[a]][blk] <= self.Ls[a]
            for k in out:
                out[k] = np.where(inside, s[k][blk], out[k])
            found |= inside
        return out

    def rho(self) -> np.ndarray:
        return self.sim.rho()

    def diagnostics(self) -> dict:
        d = self.sim.diagnostics()
        for k in ("energy_E", "energy_B", "energy_Ex", "kinetic", "charge"):
            d[k] *= 0.5 ** len(self.axes)
        return d
