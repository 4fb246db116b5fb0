"""The FP64 oracle behind the compute interface of paper_1211_4575_gb300.parallel
(test infrastructure: lets CPU ranks over gloo run the z-slab decomposition
with the oracle as each rank's compute)."""
import numpy as np

_KEYS = ("x", "y", "z", "ux", "uy", "uz")


class OracleSlab:
    def __init__(self, orc, n, d, dt, **kw):
        self.o = orc.Simulation(n, d, dt, **kw)
        self.mesh_shape = (n[2], n[1], n[0])
        self.lo, self.hi = 0.0, n[2] * d[2]

    def set_slab(self, z_lo, z_hi):
        self.lo, self.hi = float(z_lo), float(z_hi)

    def add_species(self, q, m, w):
        e = np.zeros(0)
        return self.o.add_species(q, m, w, e, e, e, e, e, e)

    def load_particles(self, sid, x, y, z, ux, uy, uz):
        sp = self.o.species[sid]
        for k, v in zip(_KEYS, (x, y, z, ux, uy, uz)):
            sp[k] = np.ascontiguousarray(np.concatenate([sp[k], np.asarray(v, dtype=np.float64)]))

    def count(self, sid):
        return len(self.o.species[sid]["x"])

    def deposit(self):
        self.o.deposit()

    def get_current(self):
        return [a.copy() for a in self.o.J]

    def set_current(self, J):
        for a in range(3):
            self.o.J[a][...] = J[a]

    def field_update(self):
        self.o.field_update()

    def extract_particles(self, sid):
        sp = self.o.species[sid]
        out_m = (sp["z"] < self.lo) | (sp["z"] >= self.hi)
        left = {k: np.ascontiguousarray(sp[k][out_m]) for k in _KEYS}
        for k in _KEYS:
            sp[k] = np.ascontiguousarray(sp[k][~out_m])
        return left

    def diagnostics(self):
        d = self.o.diagnostics()
        return {"kinetic": [d["kinetic"]], "n_particles": sum(len(s["x"]) for s in self.o.species)}
