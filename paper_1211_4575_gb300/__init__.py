"""Python binding of the GB300 Photon-Plasma particle step (libpp_gb300.so).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels (``csrc/``), reached through the C ABI of ``include/pp.h``.  The binding
raises ``RuntimeError`` when the library has not been built; there is no other
code path.

Arrays: fields are numpy float64 arrays of shape (nz, ny, nx) (x fastest), with
the Yee staggering of the paper's Sec. III (E_x, J_x at (i+1/2, j, k); B_x at
(i, j+1/2, k+1/2); cyclic).  Particle positions are physical; proper velocities
u = gamma*v at t - dt/2.  c = eps0 = mu0 = 1.
"""
from __future__ import annotations

import ctypes as C
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PP_GB300_CHECKED=1 selects the bounds-checked build (python -m
# paper_1211_4575_gb300.build --checked), whose kernels report an index that
# leaves its array as PP_EBOUNDS instead of touching memory outside it.
LIB_PATH = os.path.join(_HERE, "lib", "libpp_gb300_checked.so" if os.environ.get("PP_GB300_CHECKED") == "1"
                        else "libpp_gb300.so")

PP_OK, PP_EINVAL, PP_ENOMEM, PP_EBUSY, PP_ECUDA, PP_ETIMEOUT, PP_ENOCONV, PP_ECFL, PP_ENAN, PP_WSTAB, PP_EBOUNDS = range(11)
PP_VAY, PP_BORIS = 0, 1
PP_FP64, PP_MIXED32 = 0, 1
PP_DEPOSIT_AUTO, PP_DEPOSIT_GLOBAL, PP_DEPOSIT_TILED, PP_DEPOSIT_CELLS = 0, 1, 2, 3
PP_FIELD_IMPLICIT, PP_FIELD_EXPLICIT = 0, 1
PP_CURRENT_CONSERVING, PP_CURRENT_DIRECT = 0, 1
PP_BOUNDARY_PERIODIC, PP_BOUNDARY_WALLS = 0, 1
TRANSVERSE = 0x36   # damped components of the outflow layer: E_y, E_z, B_y, B_z
PP_MAX_SPECIES = 8
PP_BATCH_FREE, PP_BATCH_RUNNING, PP_BATCH_DONE, PP_BATCH_FAILED = 0, 1, 2, 3
_CODES = {1: "EINVAL", 2: "ENOMEM", 3: "EBUSY", 4: "ECUDA", 5: "ETIMEOUT", 6: "ENOCONV", 7: "ECFL", 8: "ENAN",
          9: "WSTAB", 10: "EBOUNDS"}


class PPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"PP_{_CODES.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("c", C.c_double), ("eps0", C.c_double), ("field_order", C.c_int), ("alpha", C.c_double),
                ("shape_order", C.c_int), ("pusher", C.c_int), ("precision", C.c_int),
                ("sort_interval", C.c_int), ("relax_max_iter", C.c_int), ("relax_tol", C.c_double),
                ("deposit_mode", C.c_int), ("stream", C.c_void_p), ("boundary_x", C.c_int),
                ("boundary_y", C.c_int), ("boundary_z", C.c_int)]


class SpeciesDesc(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("w", C.c_double), ("capacity", C.c_int64)]


class Diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("time", C.c_double), ("energy_E", C.c_double), ("energy_B", C.c_double),
                ("energy_Ex", C.c_double), ("kinetic", C.c_double * PP_MAX_SPECIES), ("kinetic_total", C.c_double),
                ("charge", C.c_double), ("rho_max", C.c_double), ("gauss_max", C.c_double),
                ("gauss_drift_max", C.c_double), ("divB_max", C.c_double), ("relax_residual", C.c_double),
                ("relax_iters", C.c_int), ("status", C.c_int), ("n_particles", C.c_int64), ("n_slow", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("particle_ms", C.c_double), ("particle_launches", C.c_int64), ("current_ms", C.c_double),
                ("field_ms", C.c_double), ("sort_ms", C.c_double), ("steps", C.c_int64),
                ("kernel_launches", C.c_int64)]


# Every entry point declared in include/pp.h: name -> (restype, argtypes)
_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "pp_init_grid": (C.c_int, [_PP, C.POINTER(GridDesc)]),
    "pp_init_species": (C.c_int, [_P, C.POINTER(SpeciesDesc), C.POINTER(C.c_int)]),
    "pp_set_radiative_cooling": (C.c_int, [_P, C.c_int, C.c_double]),
    "pp_set_integrator": (C.c_int, [_P, C.c_int]),
    "pp_set_field_solver": (C.c_int, [_P, C.c_int]),
    "pp_set_current_deposit": (C.c_int, [_P, C.c_int]),
    "pp_set_divergence_filter": (C.c_int, [_P, C.c_int, C.c_int]),
    "pp_set_open_boundary": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int]),
    "pp_set_injector": (C.c_int, [_P, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_double, C.c_uint64]),
    "pp_set_sliding_window": (C.c_int, [_P, C.c_double]),
    "pp_set_graphs": (C.c_int, [_P, C.c_int]),
    "pp_get_graph_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pp_load_particles": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_int]),
    "pp_load_fields": (C.c_int, [_P, _PP, _PP, C.c_int]),
    "pp_step": (C.c_int, [_P, C.c_int]),
    "pp_deposit": (C.c_int, [_P, C.c_int]),
    "pp_field_update": (C.c_int, [_P]),
    "pp_sort": (C.c_int, [_P]),
    "pp_sync": (C.c_int, [_P]),
    "pp_check_bounded_wait": (C.c_int, [_P, C.c_int, C.c_longlong]),
    "pp_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "pp_diagnostics": (C.c_int, [_P, C.POINTER(Diag)]),
    "pp_get_fields": (C.c_int, [_P, _PP, _PP, _PP]),
    "pp_get_rho": (C.c_int, [_P, _P]),
    "pp_get_grid": (C.c_int, [_P, C.POINTER(GridDesc), C.POINTER(C.c_int)]),
    "pp_get_count": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64)]),
    "pp_get_particles": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "pp_profile_enable": (C.c_int, [_P, C.c_int]),
    "pp_profile_read": (C.c_int, [_P, C.POINTER(Profile)]),
    "pp_save": (C.c_int, [_P, C.c_char_p]),
    "pp_restore": (C.c_int, [_PP, C.c_char_p, _P]),
    "pp_set_slab": (C.c_int, [_P, C.c_double, C.c_double]),
    "pp_get_current": (C.c_int, [_P, _PP, C.c_int]),
    "pp_set_current": (C.c_int, [_P, _PP, C.c_int]),
    "pp_extract_particles": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_int,
                                       C.POINTER(C.c_int64)]),
    "pp_field_energy_noalloc": (C.c_int, [_PP, _PP, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P]),
    "pp_field_energy_noalloc_error": (C.c_char_p, []),
    "pp_device_bytes": (C.c_int64, [_P]),
    "pp_estimate_device_bytes": (C.c_int64, [C.POINTER(GridDesc), C.c_int, C.POINTER(C.c_int64)]),
    "pp_batch_create": (C.c_int, [_PP, C.c_int64, C.c_int]),
    "pp_batch_admit": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_int)]),
    "pp_batch_advance": (C.c_int, [_P, C.c_int]),
    "pp_batch_set_fused": (C.c_int, [_P, C.c_int]),
    "pp_batch_poll": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "pp_batch_used": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "pp_batch_last_error": (C.c_char_p, [_P]),
    "pp_batch_destroy": (C.c_int, [_P]),
    "pp_destroy": (C.c_int, [_P]),
    "pp_last_error": (C.c_char_p, [_P]),
}

_lib = None


def lib():
    """Load libpp_gb300.so (built by ``python -m paper_1211_4575_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1211_4575_gb300.build` "
                               "(the CUDA library is the only implementation)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != PP_OK:
        msg = lib().pp_last_error(ctx).decode(errors="replace")
        if rc == PP_WSTAB:
            warnings.warn(msg)
            return
        raise PPError(rc, msg)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # torch missing: the legacy default stream
        pass
    return None


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr_array(arrs):
    return (C.c_void_p * 3)(*[a.ctypes.data if a is not None else None for a in arrs])


def field_energy_noalloc(E, B, dV, out, stream=None):
    """Field energies of caller-owned CUDA FP64 tensors E[3], B[3] (each shaped
    (nz, ny, nx), contiguous) written into the CUDA FP64 tensor ``out`` of 3
    values, through the allocation-free entry point (no device memory is
    allocated by the call)."""
    for t in list(E) + list(B):
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
            raise ValueError("E and B must be contiguous CUDA float64 tensors")
    nz, ny, nx = E[0].shape
    pe = (C.c_void_p * 3)(*[t.data_ptr() for t in E])
    pb = (C.c_void_p * 3)(*[t.data_ptr() for t in B])
    rc = lib().pp_field_energy_noalloc(pe, pb, nx, ny, nz, float(dV), out.data_ptr(),
                                       stream if stream is not None else _current_stream())
    if rc != PP_OK:
        raise PPError(rc, lib().pp_field_energy_noalloc_error().decode(errors="replace"))


def estimate_device_bytes(n, capacities, precision=PP_MIXED32, boundary=(PP_BOUNDARY_PERIODIC,) * 3) -> int:
    """Device bytes a Simulation of this mesh with species of these capacities
    will hold once built (pp_estimate_device_bytes), before building it."""
    g = GridDesc(nx=n[0], ny=n[1], nz=n[2], precision=precision, boundary_x=boundary[0], boundary_y=boundary[1],
                 boundary_z=boundary[2])
    caps = (C.c_int64 * max(1, len(capacities)))(*[int(c) for c in capacities])
    return int(lib().pp_estimate_device_bytes(C.byref(g), len(capacities), caps))


class Simulation:
    """One periodic 3D plasma on the GPU (a ``pp_ctx``)."""

    def __init__(self, n, d, dt, field_order=6, alpha=0.55, shape_order=3, pusher=PP_VAY, precision=PP_FP64,
                 sort_interval=20, relax_max_iter=200, relax_tol=1e-6, deposit_mode=PP_DEPOSIT_AUTO, stream=None,
                 boundary_x=PP_BOUNDARY_PERIODIC, boundary_y=PP_BOUNDARY_PERIODIC, boundary_z=PP_BOUNDARY_PERIODIC,
                 _handle=None):
        """boundary_a = PP_BOUNDARY_WALLS: reflecting walls at 0 and n[a] d[a] on
        axis a; mesh arrays (fields(), rho(), load_fields()) then span the
        mirror-extended box, twice the cells on each walled axis."""
        self._ctx = C.c_void_p()
        if _handle is not None:
            self._ctx = _handle
        else:
            g = GridDesc(nx=n[0], ny=n[1], nz=n[2], dx=d[0], dy=d[1], dz=d[2], dt=dt, c=1.0, eps0=1.0,
                         field_order=field_order, alpha=alpha, shape_order=shape_order, pusher=pusher,
                         precision=precision, sort_interval=sort_interval, relax_max_iter=relax_max_iter,
                         relax_tol=relax_tol, deposit_mode=deposit_mode,
                         stream=stream if stream is not None else _current_stream(), boundary_x=boundary_x,
                         boundary_y=boundary_y, boundary_z=boundary_z)
            rc = lib().pp_init_grid(C.byref(self._ctx), C.byref(g))
            _check(rc, self._ctx if self._ctx.value else None)
        self.n = tuple(n)
        self.wall_axes = tuple(b == PP_BOUNDARY_WALLS for b in (boundary_x, boundary_y, boundary_z))
        self.walls = self.wall_axes[0]
        self.nspecies = 0

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if self._ctx is not None and self._ctx.value:
            lib().pp_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, rc):
        _check(rc, self._ctx)

    # -- setup ------------------------------------------------------------
    def add_species(self, q, m, w, capacity) -> int:
        sid = C.c_int(-1)
        self._c(lib().pp_init_species(self._ctx, C.byref(SpeciesDesc(q, m, w, int(capacity))), C.byref(sid)))
        self.nspecies += 1
        return sid.value

    def set_integrator(self, order):
        """2: leap-frog step; 4: four-substep 4th-order symplectic step (u synchronous with x)."""
        self._c(lib().pp_set_integrator(self._ctx, int(order)))

    def set_graphs(self, enable=True):
        """Capture steps as CUDA graphs and replay them (needs a non-default stream)."""
        self._c(lib().pp_set_graphs(self._ctx, int(bool(enable))))

    def graph_stats(self):
        """(captures, replays) of the step graphs."""
        cap, rep = C.c_int64(0), C.c_int64(0)
        self._c(lib().pp_get_graph_stats(self._ctx, C.byref(cap), C.byref(rep)))
        return cap.value, rep.value

    def set_field_solver(self, solver):
        """PP_FIELD_IMPLICIT (eq:EllipticB, default) or PP_FIELD_EXPLICIT (FDTD leap-frog)."""
        self._c(lib().pp_set_field_solver(self._ctx, int(solver)))

    def set_current_deposit(self, mode):
        """PP_CURRENT_CONSERVING (default) or PP_CURRENT_DIRECT (eq:jj2)."""
        self._c(lib().pp_set_current_deposit(self._ctx, int(mode)))

    def set_divergence_filter(self, passes, interval=1):
        """passes filter passes on E and B after every interval-th step (0 = off)."""
        self._c(lib().pp_set_divergence_filter(self._ctx, int(passes), int(interval)))

    def set_open_boundary(self, cells, damping, escape, components=TRANSVERSE):
        """Outflow layer of `cells` cells at x = 0 between walls (0 = closed)."""
        self._c(lib().pp_set_open_boundary(self._ctx, int(cells), float(damping), float(escape), int(components)))

    def set_injector(self, sid, ppc, u, u_th=0.0, seed=0):
        """Inflow of species sid through x = 0: ppc per cell, drift proper
        velocity u (u[0] > 0), thermal spread u_th, Philox seed (0 ppc = off)."""
        uu = (C.c_double * 3)(*[float(v) for v in u])
        self._c(lib().pp_set_injector(self._ctx, int(sid), float(ppc), uu, float(u_th), int(seed) & (2 ** 64 - 1)))

    def set_sliding_window(self, v):
        """Sliding window at speed v against x (0 = off)."""
        self._c(lib().pp_set_sliding_window(self._ctx, float(v)))

    def set_radiative_cooling(self, sid, coef):
        """Radiative cooling coefficient mu0 q^2 / (6 pi m c) of species sid (0 = off)."""
        self._c(lib().pp_set_radiative_cooling(self._ctx, int(sid), float(coef)))

    def load_particles(self, sid, x, y, z, ux, uy, uz):
        """Append particles: numpy arrays (host) or CUDA torch tensors (device)."""
        arrs = [x, y, z, ux, uy, uz]
        if hasattr(x, "is_cuda") and x.is_cuda:
            import torch
            arrs = [a.to(torch.float64).contiguous() for a in arrs]
            ptrs = [a.data_ptr() for a in arrs]
            self._c(lib().pp_load_particles(self._ctx, sid, int(arrs[0].numel()), *ptrs, 1))
            return
        arrs = [_f64(a) for a in arrs]
        n = arrs[0].size
        if any(a.size != n for a in arrs):
            raise ValueError("particle arrays differ in length")
        self._c(lib().pp_load_particles(self._ctx, sid, n, *[a.ctypes.data for a in arrs], 0))

    def load_fields(self, E, B):
        E = [_f64(a) for a in E]
        B = [_f64(a) for a in B]
        size = int(np.prod(self.mesh_shape))
        if any(a.size != size for a in E + B):
            raise ValueError(f"field arrays must hold {size} values (mesh shape {self.mesh_shape})")
        self._c(lib().pp_load_fields(self._ctx, _ptr_array(E), _ptr_array(B), 0))

    # -- the step -----------------------------------------------------------
    def step(self, n: int = 1):
        self._c(lib().pp_step(self._ctx, int(n)))

    def deposit(self, sid: int = -1):
        self._c(lib().pp_deposit(self._ctx, int(sid)))

    def field_update(self):
        self._c(lib().pp_field_update(self._ctx))

    def sort(self):
        self._c(lib().pp_sort(self._ctx))

    def sync(self):
        self._c(lib().pp_sync(self._ctx))

    def check_bounded_wait(self, deliver: bool, limit_ns: int) -> int:
        """Run the particle kernel's bounded staging wait once on the
        context's stream (pp_check_bounded_wait): PP_OK when its barrier
        phase completes (deliver), PP_ETIMEOUT when it waits for bytes that
        never come and the limit runs out."""
        return int(lib().pp_check_bounded_wait(self._ctx, 1 if deliver else 0, int(limit_ns)))

    def set_tuning(self, sort_interval: int, deposit_mode: int):
        self._c(lib().pp_set_tuning(self._ctx, int(sort_interval), int(deposit_mode)))

    # -- readback -----------------------------------------------------------
    def diagnostics(self) -> dict:
        d = Diag()
        self._c(lib().pp_diagnostics(self._ctx, C.byref(d)))
        out = {k: getattr(d, k) for k, _ in Diag._fields_}
        out["kinetic"] = list(d.kinetic)[: self.nspecies]
        return out

    @property
    def mesh_shape(self):
        """(nz, ny, nx) of the mesh arrays; doubled on each walled axis."""
        m = [2 * self.n[a] if self.wall_axes[a] else self.n[a] for a in range(3)]
        return (m[2], m[1], m[0])

    def _mesh(self):
        return np.zeros(self.mesh_shape)

    def fields(self):
        E = [self._mesh() for _ in range(3)]
        B = [self._mesh() for _ in range(3)]
        J = [self._mesh() for _ in range(3)]
        self._c(lib().pp_get_fields(self._ctx, _ptr_array(E), _ptr_array(B), _ptr_array(J)))
        return E, B, J

    def rho(self) -> np.ndarray:
        r = self._mesh()
        self._c(lib().pp_get_rho(self._ctx, r.ctypes.data))
        return r

    def count(self, sid: int) -> int:
        n = C.c_int64(0)
        self._c(lib().pp_get_count(self._ctx, sid, C.byref(n)))
        return n.value

    def particles(self, sid: int) -> dict:
        n = self.count(sid)
        out = {k: np.zeros(n) for k in ("x", "y", "z", "ux", "uy", "uz")}
        self._c(lib().pp_get_particles(self._ctx, sid, *[out[k].ctypes.data for k in ("x", "y", "z", "ux", "uy", "uz")]))
        return out

    # -- z-slab decomposition (parallel.py) ---------------------------------
    def set_slab(self, z_lo: float, z_hi: float):
        self._c(lib().pp_set_slab(self._ctx, float(z_lo), float(z_hi)))

    def get_current(self, out=None):
        """J on the mesh as three FP64 arrays: numpy (host) by default, or into
        the given CUDA torch tensors (enqueued on the context's stream)."""
        if out is not None:
            ptrs = (C.c_void_p * 3)(*[t.data_ptr() for t in out])
            self._c(lib().pp_get_current(self._ctx, ptrs, 1))
            return out
        J = [self._mesh() for _ in range(3)]
        self._c(lib().pp_get_current(self._ctx, _ptr_array(J), 0))
        return J

    def set_current(self, J):
        """Replace J on the mesh: three FP64 numpy arrays or CUDA torch tensors."""
        if hasattr(J[0], "is_cuda") and J[0].is_cuda:
            ptrs = (C.c_void_p * 3)(*[t.data_ptr() for t in J])
            self._c(lib().pp_set_current(self._ctx, ptrs, 1))
            return
        J = [_f64(a) for a in J]
        self._c(lib().pp_set_current(self._ctx, _ptr_array(J), 0))

    def extract_particles(self, sid: int) -> dict:
        """Remove and return (host FP64 arrays) the particles of species sid
        that left the slab."""
        cap = self.count(sid)
        out = {k: np.zeros(max(cap, 1)) for k in ("x", "y", "z", "ux", "uy", "uz")}
        n = C.c_int64(0)
        self._c(lib().pp_extract_particles(self._ctx, int(sid), cap,
                                           *[out[k].ctypes.data for k in ("x", "y", "z", "ux", "uy", "uz")],
                                           0, C.byref(n)))
        return {k: v[: n.value].copy() for k, v in out.items()}

    def device_bytes(self) -> int:
        return int(lib().pp_device_bytes(self._ctx))

    def profile_enable(self, enable: bool = True):
        self._c(lib().pp_profile_enable(self._ctx, 1 if enable else 0))

    def profile_read(self) -> dict:
        pr = Profile()
        self._c(lib().pp_profile_read(self._ctx, C.byref(pr)))
        return {k: getattr(pr, k) for k, _ in Profile._fields_}

    def save(self, path: str):
        self._c(lib().pp_save(self._ctx, os.fsencode(path)))

    @classmethod
    def restore(cls, path: str, stream=None) -> "Simulation":
        h = C.c_void_p()
        rc = lib().pp_restore(C.byref(h), os.fsencode(path), stream if stream is not None else _current_stream())
        _check(rc, None)
        sim = cls.__new__(cls)
        sim._ctx = h
        g, ns = sim.grid()
        sim.n = (g.nx, g.ny, g.nz)
        sim.wall_axes = tuple(b == PP_BOUNDARY_WALLS for b in (g.boundary_x, g.boundary_y, g.boundary_z))
        sim.walls = sim.wall_axes[0]
        sim.nspecies = ns
        return sim

    def grid(self):
        """(GridDesc, number of species) of this context."""
        g = GridDesc()
        ns = C.c_int(0)
        self._c(lib().pp_get_grid(self._ctx, C.byref(g), C.byref(ns)))
        return g, ns.value


class Batch:
    """Slots of independent runs advanced together (pp_batch_*)."""

    def __init__(self, budget_bytes: int, max_slots: int = 64):
        self._b = C.c_void_p()
        rc = lib().pp_batch_create(C.byref(self._b), int(budget_bytes), int(max_slots))
        if rc != PP_OK:
            raise PPError(rc, "pp_batch_create failed")
        self.max_slots = max_slots

    def admit(self, sim: "Simulation", steps: int):
        """Slot index, or None when the batch is full (PP_EBUSY)."""
        slot = C.c_int(-1)
        rc = lib().pp_batch_admit(self._b, sim._ctx, int(steps), C.byref(slot))
        if rc == PP_EBUSY:
            return None
        if rc != PP_OK:
            raise PPError(rc, lib().pp_batch_last_error(self._b).decode(errors="replace"))
        return slot.value

    def set_fused(self, enable: bool = True):
        """Fused rounds: the particle kernels of all running slots as one
        persistent launch per group of compatible runs."""
        rc = lib().pp_batch_set_fused(self._b, 1 if enable else 0)
        if rc != PP_OK:
            raise PPError(rc, lib().pp_batch_last_error(self._b).decode(errors="replace"))

    def advance(self, max_steps: int):
        rc = lib().pp_batch_advance(self._b, int(max_steps))
        if rc != PP_OK:
            raise PPError(rc, lib().pp_batch_last_error(self._b).decode(errors="replace"))

    def poll(self, slot: int):
        """(state, steps enqueued) of a slot; DONE/FAILED are reported once."""
        done = C.c_int64(0)
        state = C.c_int(0)
        rc = lib().pp_batch_poll(self._b, int(slot), C.byref(done), C.byref(state))
        if rc != PP_OK and state.value != PP_BATCH_FAILED:
            raise PPError(rc, lib().pp_batch_last_error(self._b).decode(errors="replace"))
        return state.value, done.value

    def used(self):
        b = C.c_int64(0)
        a = C.c_int(0)
        lib().pp_batch_used(self._b, C.byref(b), C.byref(a))
        return b.value, a.value

    def close(self):
        if self._b is not None and self._b.value:
            lib().pp_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
