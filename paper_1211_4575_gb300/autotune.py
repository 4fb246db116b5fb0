"""Autotuner for the per-run knobs that change only speed: the cell-sort
interval and the deposit mode (tiled shared-memory or global).

Trials are real steps of the caller's own run (the physics advances normally
while it is being tuned); each candidate starts from a freshly sorted state and
is timed with the library's per-phase CUDA events.  Choices are cached per
(grid, particles per cell, shape, precision) so later runs of the same kind
start tuned.
"""
from __future__ import annotations

from . import PP_DEPOSIT_GLOBAL, PP_DEPOSIT_TILED, PP_FP64, PPError

_cache: dict = {}


def key_of(sim) -> tuple:
    g, ns = sim.grid()
    n = sum(sim.count(s) for s in range(ns))
    cells = g.nx * g.ny * g.nz
    return (g.nx, g.ny, g.nz, round(n / max(1, cells)), g.shape_order, g.precision)


def candidates(sim, sort_intervals=(5, 10, 20, 40)):
    g, _ = sim.grid()
    modes = [PP_DEPOSIT_GLOBAL]
    if g.precision != PP_FP64 and g.nx % 8 == 0 and g.ny % 8 == 0 and g.nz % 8 == 0:
        modes = [PP_DEPOSIT_TILED, PP_DEPOSIT_GLOBAL]
    return [(si, m) for m in modes for si in sort_intervals]


def _trial(sim, sort_interval, mode, steps):
    sim.set_tuning(sort_interval, mode)
    sim.sort()
    sim.profile_enable(True)
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
        n = steps if steps is not None else max(si, 5)
        try:
            timings[(si, m)] = _trial(sim, si, m, n)
        except PPError:
            continue
    best = min(timings, key=timings.get)
    sim.set_tuning(*best)
    _cache[k] = best
    return best, timings
