"""Serving loop over the batched C ABI (pp_batch_*): requests for independent
plasma runs arrive over time, are admitted into slots as device memory and
slots allow, advance together on the GPU (each on its own stream), and report
their time to result.  `sequential` runs the same requests one at a time.

Host-side work here is orchestration only (building each run's seeded load,
admission, polling); every step of every run executes in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import PP_BATCH_DONE, PP_BATCH_FAILED, PP_MIXED32, Batch, PPError, Simulation, estimate_device_bytes


def _make_load(req):
    import pp_synth
    return pp_synth.run_load(req)


def _build(req, precision, stream, L=None):
    """The run of a request on the device: its seeded load (built here unless
    given), a context on `stream`, the particles uploaded."""
    if L is None:
        L = _make_load(req)
    sim = Simulation(L.n, L.d, L.dt, field_order=6, alpha=0.55, shape_order=req.get("shape", 3),
                     precision=precision, sort_interval=20, relax_max_iter=100,
                     relax_tol=1e-6 if precision == PP_MIXED32 else 1e-12, stream=stream)
    for s in L.species:
        sid = sim.add_species(s["q"], s["m"], s["w"], len(s["x"]))
        sim.load_particles(sid, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
    return sim, L.n_particles


class _Loads:
    """Host worker threads that build the seeded loads of arrived requests
    (the server's input preparation), at most `ahead` at a time, in arrival
    order; both the batched and the one-at-a-time server use it."""

    def __init__(self, workers=4, ahead=4):
        from concurrent.futures import ThreadPoolExecutor
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.ahead = ahead
        self.fut = {}

    def feed(self, pending, now):
        for req in pending:
            if len(self.fut) >= self.ahead or req.get("arrival", 0.0) > now:
                break
            key = id(req)
            if key not in self.fut:
                self.fut[key] = self.pool.submit(_make_load, req)

    def ready(self, req):
        f = self.fut.get(id(req))
        return f is not None and f.done()

    def take(self, req):
        return self.fut.pop(id(req)).result()

    def close(self):
        self.pool.shutdown(wait=True)


def admissible(used, need, budget_bytes, nact, max_slots, running_particles, req_particles,
               max_active_particles=None):
    """Whether the next request in arrival order may enter now: its device
    bytes fit the budget beside the running requests', a slot is free, and,
    with a particle budget, the running requests' particles plus its own stay
    within it (a request over the budget enters only an idle GPU)."""
    if used + need > budget_bytes or nact >= max_slots:
        return False
    if max_active_particles is not None and running_particles > 0 and \
            running_particles + req_particles > max_active_particles:
        return False
    return True


def _summary(lat, work, makespan):
    lat = np.asarray(lat, dtype=float)
    return {"requests": int(lat.size), "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None, "makespan_s": makespan,
            "particle_steps_per_s": work / makespan if makespan > 0 else None}


def serve(requests, budget_bytes, max_slots=16, chunk=8, precision=PP_MIXED32, keep=False, loaders=4, fused=False,
          max_active_particles=None):
    """Continuous batching.  Returns (summary, per-request results); with keep
    the finished Simulations are returned too (for comparisons).  fused: the
    batch's fused rounds (one persistent particle launch per round).

    Requests are admitted in arrival order while device memory and slots
    allow, and, with max_active_particles, while the particles of the running
    requests plus the next one stay within that budget (a request over it is
    admitted only onto an idle GPU).  Runs of a few million particles cannot
    fill the GPU alone and gain most from overlapping; a run that fills it
    gains nothing from company and would only be slowed by the runs admitted
    after it, so under the budget the largest requests run as they would one
    at a time."""
    import torch
    import pp_synth
    pending = sorted(requests, key=lambda r: r.get("arrival", 0.0))
    batch = Batch(budget_bytes, max_slots)
    if fused:
        batch.set_fused(True)
    loads = _Loads(workers=loaders, ahead=loaders)
    active = {}
    lat, work, results = [], 0, []
    t0 = time.perf_counter()
    while pending or active:
        now = time.perf_counter() - t0
        loads.feed(pending, now)
        while pending and pending[0].get("arrival", 0.0) <= now and loads.ready(pending[0]):
            req = pending[0]
            # admit by the run's device bytes, known before anything is built on
            # the device: a run that does not fit waits until a slot's memory returns
            counts = pp_synth.run_counts(req)
            need = estimate_device_bytes((req["n"],) * 3, counts, precision)
            used, nact = batch.used()
            running = sum(v[2] for v in active.values())
            if not admissible(used, need, budget_bytes, nact, max_slots, running, sum(counts), max_active_particles):
                break
            stream = torch.cuda.Stream()
            sim, npart = _build(req, precision, stream.cuda_stream, loads.take(req))
            loads.feed(pending[1:], now)
            slot = batch.admit(sim, req["steps"])
            if slot is None:          # cannot happen after the check above; keep the request
                sim.close()
                break
            pending.pop(0)
            active[slot] = (req, sim, npart, stream)
        if not active:
            if pending:
                time.sleep(max(0.001, min(0.01, pending[0].get("arrival", 0.0) - now)))
            continue
        batch.advance(chunk)
        for slot in list(active):
            state, _ = batch.poll(slot)
            if state in (PP_BATCH_DONE, PP_BATCH_FAILED):
                req, sim, npart, stream = active.pop(slot)
                t = time.perf_counter() - t0
                if state == PP_BATCH_FAILED:
                    raise PPError(state, f"request {req.get('seed')} failed")
                lat.append(t - req.get("arrival", 0.0))
                work += npart * req["steps"]
                results.append((req, sim if keep else None))
                if not keep:
                    sim.close()
    makespan = time.perf_counter() - t0
    batch.close()
    loads.close()
    return _summary(lat, work, makespan), results


def sequential(requests, precision=PP_MIXED32, keep=False, loaders=4):
    """The same requests one at a time, in arrival order, on one stream (loads
    prepared by the same host workers as the batched server)."""
    import torch
    pending = sorted(requests, key=lambda r: r.get("arrival", 0.0))
    loads = _Loads(workers=loaders, ahead=loaders)
    lat, work, results = [], 0, []
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    for i, req in enumerate(pending):
        while True:
            now = time.perf_counter() - t0
            loads.feed(pending[i:], now)
            if req.get("arrival", 0.0) <= now and loads.ready(req):
                break
            time.sleep(0.002)
        sim, npart = _build(req, precision, stream, loads.take(req))
        loads.feed(pending[i + 1:], time.perf_counter() - t0)
        sim.step(req["steps"])
        sim.sync()
        t = time.perf_counter() - t0
        lat.append(t - req.get("arrival", 0.0))
        work += npart * req["steps"]
        results.append((req, sim if keep else None))
        if not keep:
            sim.close()
    makespan = time.perf_counter() - t0
    loads.close()
    return _summary(lat, work, makespan), results


def build_all(requests, precision=PP_MIXED32):
    """Build every run of a batched workload (seeded load, resident on the
    device), each with its own stream: [(request, Simulation, particles, stream)]."""
    import torch
    built = []
    for req in requests:
        stream = torch.cuda.Stream()
        sim, npart = _build(req, precision, stream.cuda_stream)
        built.append((req, sim, npart, stream))
    torch.cuda.synchronize()
    return built


def batched(built, budget_bytes, max_slots=64, chunk=4, graphs=True, fused=False):
    """Batched form on runs already resident (build_all): all runs admitted
    into slots as budget and slots allow and advanced together, one stream
    each, each step replayed from a captured CUDA graph unless graphs=False,
    or (fused) with the particle kernels of all runs as one persistent launch
    per round, until every run has taken its steps.  Summary of the timed
    region."""
    batch = Batch(budget_bytes, max_slots)
    if fused:
        batch.set_fused(True)
    waiting = list(built)
    active = {}
    lat, work = [], 0
    t0 = time.perf_counter()
    while waiting or active:
        while waiting:
            req, sim, npart, stream = waiting[0]
            slot = batch.admit(sim, req["steps"])
            if slot is None:
                break
            if not graphs:
                sim.set_graphs(False)
            waiting.pop(0)
            active[slot] = (req, sim, npart, stream)
        batch.advance(chunk)
        for slot in list(active):
            state, _ = batch.poll(slot)
            if state in (PP_BATCH_DONE, PP_BATCH_FAILED):
                req, sim, npart, stream = active.pop(slot)
                if state == PP_BATCH_FAILED:
                    raise PPError(state, f"run {req.get('seed')} failed")
                lat.append(time.perf_counter() - t0)
                work += npart * req["steps"]
    makespan = time.perf_counter() - t0
    batch.close()
    return _summary(lat, work, makespan)


def one_at_a_time(built):
    """The same resident runs stepped one after another with plain (uncaptured)
    steps, each run to its end before the next starts."""
    lat, work = [], 0
    t0 = time.perf_counter()
    for req, sim, npart, _ in built:
        sim.set_graphs(False)
        sim.step(req["steps"])
        sim.sync()
        lat.append(time.perf_counter() - t0)
        work += npart * req["steps"]
    makespan = time.perf_counter() - t0
    return _summary(lat, work, makespan)
