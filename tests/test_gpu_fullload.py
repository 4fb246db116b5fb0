"""Element-wise parity of the mixed form at the benchmark's per-cell load.

The benchmark workloads put 32 macro-particles per cell per species (thermal
128^3, PCS) or 16 per cell per species per population (the Gamma = 10 beam
through an electron-ion background on 256 x 128 x 128).  These tests take the
same per-cell load, the same parameters and the same seeded generator on a
16^3 box the FP64 oracle steps in about a second, and compare E, B, J,
positions and momenta element by element (particles matched one to one as
periodic nearest neighbours) after the first step and after 25 steps, across
the cell sort of step 20.  At this load the tiled kernel runs full
1024-particle chunks with the lanes 32 sorted places apart, its queue of
support-crossing particles fills, and (beam) particles that drift out of their
tile's margin between sorts take the global-mesh path.

Tolerances (mixed form: FP32 offsets, momenta, fields and current; FP64
reductions; relaxation to 1e-6):
* one step: the per-step bars of the other mixed parity tests, fields 3e-5,
  positions 2e-6 (physical units), momenta 2e-6 relative;
* 25 steps: the FP32 rounding of each step adds up, at most linearly over the
  steps (the fields are integrals of the current over time): fields 25 x 3e-5
  = 7.5e-4, positions and momenta 25 x 2e-6 = 5e-5.
Field errors are relative to max|oracle array|, except where the net current
is a small difference of large species currents: FP32 rounds each species'
contribution relative to that species' own current, so the error of J is
bounded relative to the largest single-species current density
J_s = sum over its populations of |q| n |v| (the beam: 0.5 x 0.995), and E
and B, integrals of J over the elapsed time t, relative to J_s t.  The
Gauss drift of the mixed form (discrete continuity in FP32) is bounded by
2e-5 of the charge density of one species after 25 steps.
"""
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


def _loads():
    return {
        "thermal": pp_synth.thermal(n=(16, 16, 16), ppc=32, u_th=0.1, dx=0.1, dt=0.05, seed=1212),
        "beam": pp_synth.beam_background(n=(16, 16, 16), ppc=16, seed=1214),
    }


def _field_errors(gpu, osim, js, t):
    """max|GPU - oracle| per field over max(max|oracle|, floor): floor J_s for
    J and J_s t for E and B (0 where no cancelling species currents)."""
    E, B, J = gpu.fields()
    out = {}
    for name, G, O, floor in (("E", E, osim.E, js * t), ("B", B, osim.B, js * t), ("J", J, osim.J, js)):
        num = max(np.abs(G[a] - O[a]).max() for a in range(3))
        den = max(max(np.abs(O[a]).max() for a in range(3)), floor)
        out[name] = num / den
    return out


def _check(gpu, osim, L, tol_f, tol_x, tol_u, where, js=0.0, t=0.0):
    d = gpu.diagnostics()
    assert d["status"] == 0, where
    fe = _field_errors(gpu, osim, js, t)
    for k, v in fe.items():
        assert v <= tol_f, (where, k, v, fe)
    for s in range(len(L.species)):
        dpos, du = H.particle_errors(gpu.particles(s), osim.species[s], H.box(L))
        assert dpos <= tol_x and du <= tol_u, (where, s, dpos, du)
    return d, fe


@pytest.mark.parametrize("workload,mode", [("thermal", "cells"), ("beam", "cells"), ("thermal", "tiled")])
def test_mixed_at_benchmark_load(pp, orc, workload, mode):
    """The per-step sorted kernel (the benchmark's) on both loads; the tiled
    kernel with a sort every 20 steps on the thermal load.  (The tiled
    kernel's int32 fixed-point current window takes its unit from the whole
    chunk's motion: on the beam load, whose electron and ion beam currents
    cancel, its rounding reaches 4e-4 of the net current after one step,
    measured, so it is not run there.)"""
    L = _loads()[workload]
    assert L.n_particles == 262144
    dm = pp.PP_DEPOSIT_CELLS if mode == "cells" else pp.PP_DEPOSIT_TILED
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, 3, deposit_mode=dm, sort_interval=20)
    osim = H.oracle_sim(orc, L, 3)
    # largest single-species current density of the load (0: relative errors only)
    js = 0.5 * math.sqrt(1.0 - 1.0 / L.params["gamma_b"] ** 2) if workload == "beam" else 0.0
    gpu.step(1)
    osim.step(1)
    _check(gpu, osim, L, 3e-5, 2e-6, 2e-6, "step 1", js, L.dt)
    gpu.step(24)
    osim.step(24)
    d, _ = _check(gpu, osim, L, 7.5e-4, 5e-5, 5e-5, "step 25", js, 25 * L.dt)
    # one species' charge density: |q| w ppc per cell = 1 (thermal) or 1/2 per population (beam)
    assert d["gauss_drift_max"] <= 2e-5, d["gauss_drift_max"]
