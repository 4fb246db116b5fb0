"""z-slab decomposition of one run over ranks (Sec. IX: the paper splits a
run into domains, moves the particles that leave a domain to its neighbour
and combines what the domains deposit on shared mesh nodes).

Every rank holds the whole mesh and the particles of one slab of cells in z.
A step is:

1. the particle pass of every rank (``deposit``: gather, push, move, the
   charge-conserving current of its own particles, the ghost fold and the
   high-order current solve, which is linear, so per-rank currents add up);
2. the sum of the ranks' currents (an allreduce of three FP64 mesh arrays),
   handed back to every rank (``set_current``);
3. the field update on every rank: identical inputs give identical fields, so
   no field halo has to be exchanged (the mesh is small next to the particle
   state, and the particle pass is most of a step);
4. migration: each rank removes the particles that left its slab
   (``extract_particles``) and sends them to the rank that owns their new z.

The compute of a rank is any object with the methods of
``paper_1211_4575_gb300.Simulation`` used here (deposit, get_current,
set_current, field_update, extract_particles, load_particles, count); the
library's Simulation is the one this package uses.  Communicators:
``TorchComm`` (one slab per process over torch.distributed: NCCL between GPUs,
gloo between CPU processes) and ``LocalComm`` (several slabs in one process).
The driver only moves arrays; every step of the method runs in the compute
objects.
"""
from __future__ import annotations

import numpy as np

_KEYS = ("x", "y", "z", "ux", "uy", "uz")


def slab_bounds(nz: int, dz: float, world: int):
    """[z_lo, z_hi) of each rank: nz cells split into world slabs of whole
    cells (the first nz % world slabs one cell thicker)."""
    if world < 1 or world > nz:
        raise ValueError(f"{world} slabs of {nz} cells")
    base, extra = divmod(nz, world)
    out, c = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((c * dz, (c + k) * dz))
        c += k
    return out


def owner(z, bounds):
    """Rank owning each z (physical, inside the periodic box)."""
    hi = np.array([b[1] for b in bounds])
    return np.minimum(np.searchsorted(hi, np.asarray(z), side="right"), len(bounds) - 1)


def select(species: dict, z_lo: float, z_hi: float) -> dict:
    """The particles of one species (dict of arrays) with z in [z_lo, z_hi)."""
    m = (species["z"] >= z_lo) & (species["z"] < z_hi)
    return {k: np.ascontiguousarray(species[k][m]) for k in _KEYS}


class LocalComm:
    """Every slab in this process: the collectives act on lists indexed by slab."""

    def __init__(self, world: int):
        self.world = world
        self.ranks = list(range(world))

    def allreduce_sum(self, per_slab):
        """per_slab[s] = list of arrays (numpy or torch) of slab s; each becomes
        the sum over slabs."""
        total = [sum(arrs[a] for arrs in per_slab) for a in range(len(per_slab[0]))]
        for arrs in per_slab:
            for a in range(len(arrs)):
                arrs[a][...] = total[a]

    def exchange(self, outgoing):
        """outgoing[s][d] = dict of arrays from slab s to slab d; returns
        incoming[d] = list of those dicts."""
        incoming = [[] for _ in range(self.world)]
        for s in range(self.world):
            for d, arrs in outgoing[s].items():
                incoming[d].append(arrs)
        return incoming

    def allreduce_scalars(self, per_slab, op="sum"):
        v = np.array(per_slab, dtype=np.float64)
        r = v.sum(0) if op == "sum" else v.max(0)
        return [r.copy() for _ in per_slab]


class TorchComm:
    """One slab per process over torch.distributed (NCCL for CUDA tensors,
    gloo for CPU ones).  Arrays handed to allreduce_sum are torch tensors on
    the backend's device; migrants travel as one (n, 6) FP64 tensor per pair of
    ranks after an all_gather of the counts."""

    def __init__(self, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.world = dist.get_world_size()
        self.rank = dist.get_rank()
        self.ranks = [self.rank]
        self.device = device

    def _dev(self):
        import torch
        return self.device if self.device is not None else torch.device("cpu")

    def allreduce_sum(self, per_slab):
        import torch
        (arrs,) = per_slab
        for a in range(len(arrs)):
            t = arrs[a]
            if isinstance(t, np.ndarray):
                tt = torch.from_numpy(t)
                self.dist.all_reduce(tt)
            else:
                self.dist.all_reduce(t)

    def exchange(self, outgoing):
        import torch
        (out,) = outgoing
        W, me = self.world, self.rank
        dev = self._dev()
        counts = torch.zeros(W, dtype=torch.int64, device=dev)
        for d, arrs in out.items():
            counts[d] = len(arrs["x"])
        table = [torch.zeros(W, dtype=torch.int64, device=dev) for _ in range(W)]
        self.dist.all_gather(table, counts)
        table = [t.cpu().numpy() for t in table]
        reqs, recv = [], {}
        for s in range(W):
            n = int(table[s][me])
            if s != me and n > 0:
                buf = torch.empty((n, 6), dtype=torch.float64, device=dev)
                recv[s] = buf
                reqs.append(self.dist.irecv(buf, src=s))
        for d, arrs in out.items():
            if d == me or len(arrs["x"]) == 0:
                continue
            pack = torch.from_numpy(np.stack([arrs[k] for k in _KEYS], 1)).to(dev)
            reqs.append(self.dist.isend(pack, dst=d))
        for r in reqs:
            r.wait()
        incoming = [out[me]] if me in out and len(out[me]["x"]) else []
        for s in sorted(recv):
            m = recv[s].cpu().numpy()
            incoming.append({k: np.ascontiguousarray(m[:, i]) for i, k in enumerate(_KEYS)})
        return [incoming]

    def allreduce_scalars(self, per_slab, op="sum"):
        import torch
        (v,) = per_slab
        t = torch.tensor(np.asarray(v, dtype=np.float64), device=self._dev())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM if op == "sum" else self.dist.ReduceOp.MAX)
        return [t.cpu().numpy()]


class Slab:
    """One rank's share: its compute object and slab bounds."""

    def __init__(self, sim, rank: int, bounds, nspecies: int):
        self.sim = sim
        self.rank = rank
        self.bounds = bounds
        self.nspecies = nspecies
        z_lo, z_hi = bounds[rank]
        sim.set_slab(z_lo, z_hi)


def load(slabs, species):
    """Give every slab the particles of its z-range: species[s] = dict with
    q, m, w and the six FP64 arrays (the whole run's particles)."""
    for sl in slabs:
        z_lo, z_hi = sl.bounds[sl.rank]
        for sid, sp in enumerate(species):
            part = select(sp, z_lo, z_hi)
            if len(part["x"]):
                sl.sim.load_particles(sid, *[part[k] for k in _KEYS])


def _current_buffers(sl, device):
    if device is None:
        return sl.sim.get_current()
    import torch
    shape = sl.sim.mesh_shape
    out = [torch.empty(shape, dtype=torch.float64, device=device) for _ in range(3)]
    return sl.sim.get_current(out)


def step(slabs, comm, device=None):
    """One step of the decomposed run over the slabs of this process."""
    for sl in slabs:
        sl.sim.deposit()
    Js = [_current_buffers(sl, device) for sl in slabs]
    comm.allreduce_sum(Js)
    for sl, J in zip(slabs, Js):
        sl.sim.set_current(J)
        sl.sim.field_update()
    migrate(slabs, comm)


def migrate(slabs, comm):
    """Move every particle that left its slab to the slab that owns its z."""
    for sid in range(slabs[0].nspecies):
        outgoing = []
        for sl in slabs:
            left = sl.sim.extract_particles(sid)
            dest = owner(left["z"], sl.bounds) if len(left["x"]) else np.zeros(0, dtype=int)
            out = {}
            for d in np.unique(dest):
                m = dest == d
                out[int(d)] = {k: np.ascontiguousarray(left[k][m]) for k in _KEYS}
            outgoing.append(out)
        incoming = comm.exchange(outgoing)
        for sl, arrivals in zip(slabs, incoming):
            for arrs in arrivals:
                if len(arrs["x"]):
                    sl.sim.load_particles(sid, *[arrs[k] for k in _KEYS])


def kinetic_and_count(slabs, comm):
    """Run-wide kinetic energy per species and particle count (sums over ranks)."""
    per = []
    for sl in slabs:
        d = sl.sim.diagnostics()
        per.append(list(d["kinetic"]) + [float(d["n_particles"])])
    tot = comm.allreduce_scalars(per, "sum")[0]
    return list(tot[:-1]), int(round(tot[-1]))
