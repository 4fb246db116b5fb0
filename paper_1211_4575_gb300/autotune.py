"""Autotuner for the per-run knobs that change only speed: the deposit mode
(the per-step sorted kernel, the tiled shared-memory kernel with a cell sort
every `interval` steps, or the one-thread-per-particle global kernel) and,
for the tiled and global modes, the sort interval.

Trials are real steps of the caller's own run (the physics advances normally
while it is being tuned).  Each candidate is timed over one whole sort period
with the library's per-phase CUDA events: the sort that starts the period is
inside the timed window, so a shorter interval pays for its extra sorts.
Choices are cached per (grid, particles per cell, shape, precision) so later
runs of the same kind start tuned.
"""
from __future__ import annotations

from . import PP_DEPOSIT_CELLS, PP_DEPOSIT_GLOBAL, PP_DEPOSIT_TILED, PP_FP64, PPError

_cache: dict = {}


def key_of(sim) -> tuple:
    g, ns = sim.grid()
    n = sum(sim.count(s) for s in range(ns))
    cells = g.nx * g.ny * g.nz
    return (g.nx, g.ny, g.nz, round(n / max(1, cells)), g.shape_order, g.precision)


def candidates(sim, sort_intervals=(5, 10, 20, 40)):
    """(sort interval, deposit mode) pairs the run can use.  The per-step
    sorted mode sorts every pass whatever the interval: one candidate."""
    g, _ = sim.grid()
    out = []
    if g.precision != PP_FP64 and g.nx % 8 == 0 and g.ny % 8 == 0 and g.nz % 8 == 0:
        out.append((1, PP_DEPOSIT_CELLS))
        out += [(si, PP_DEPOSIT_TILED) for si in sort_intervals]
    out += [(si, PP_DEPOSIT_GLOBAL) for si in sort_intervals]
    return out


def _trial(sim, sort_interval, mode, steps):
    """ms per step over `steps` steps that start with a sort, the sort
    included (one whole sort period when steps == sort_interval)."""
    sim.set_tuning(sort_interval, mode)
    sim.sync()
    sim.profile_enable(True)
    sim.sort()
    sim.step(steps)
    prof = sim.profile_read()
    sim.profile_enable(False)
    total = prof["particle_ms"] + prof["current_ms"] + prof["field_ms"] + prof["sort_ms"]
    return total / steps


def autotune(sim, sort_intervals=(5, 10, 20, 40), steps=None, use_cache=True):
    """Pick and apply the fastest (sort interval, deposit mode); returns
    (choice, {candidate: ms per step})."""
    k = key_of(sim)
    if use_cache and k in _cache:
        si, m = _cache[k]
        sim.set_tuning(si, m)
        return (si, m), {}
    timings = {}
    for si, m in candidates(sim, sort_intervals):
        n = steps if steps is not None else (3 if m == PP_DEPOSIT_CELLS else si)
        try:
            timings[(si, m)] = _trial(sim, si, m, n)
        except PPError:
            continue
    best = min(timings, key=timings.get)
    sim.set_tuning(*best)
    _cache[k] = best
    return best, timings
