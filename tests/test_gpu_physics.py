"""Config-level physics on the GPU against the FP64 oracle.

* Two-stream growth (the paper's linear-growth diagnostic, Sec. VIII): the
  field-energy growth rate of the GPU path is within 2% of the oracle's, in
  FP64 and in the mixed form, on a quiet start whose growth the oracle pins to
  the cold closed form.
* The noisy 16^3 two-stream load: the E_x energy series of the FP64 GPU path
  follows the oracle's step by step.
* Filamentation (Weibel, the config-2 variant's instability): the magnetic
  energy growth rate of the GPU path on a quiet start is within 2% of the
  oracle's, in FP64 and in the mixed form (the oracle is pinned to the
  cold-fluid dispersion relation).
* Numerical heating (Sec. VIII): an electron-ion plasma at rest (mass ratio
  16, v_th = 0.1c for both, ten cells per skin depth) heats its electrons at
  a rate proportional to 1/ppc on the GPU (8, 16 and 32 per cell per species),
  and the GPU's rate at the smallest size agrees with the oracle's.
* A relativistic beam (Gamma = 10) through an electron-ion background
  (m_i/m_e = 25): the mixed form against the oracle on a small periodic box
  with the beam-background per-cell load.
"""
import numpy as np
import pytest

import pp_synth
from tests import gpu_helpers as H
from tests import theory

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_4575_gb300 import build
    build.build()
    import paper_1211_4575_gb300 as m
    return m


def _series(sim, steps, diag):
    out = []
    for _ in range(steps):
        sim.step(1)
        out.append(diag(sim))
    return np.array(out)


@pytest.mark.parametrize("precision,eps", [(0, 1e-6), (1, 1e-4)])
def test_two_stream_growth_rate_gpu_within_2pct_of_oracle(pp, orc, precision, eps):
    L = pp_synth.quiet_two_stream(nx=32, dx=0.25, dt=0.125, mode=2, eps=eps)
    nst = 240
    gpu = H.gpu_sim(pp, L, precision, 2, relax_tol=1e-12 if precision == 0 else 1e-6)
    osim = H.oracle_sim(orc, L, 2, relax_tol=1e-13)
    Wg = _series(gpu, nst, lambda s: s.diagnostics()["energy_Ex"])
    Wo = _series(osim, nst, lambda s: s.diagnostics()["energy_Ex"])
    t = np.arange(1, nst + 1) * L.dt
    rg, ng = theory.fit_growth(t, Wg)
    ro, no = theory.fit_growth(t, Wo)
    assert ng >= 30 and no >= 30
    assert rg == pytest.approx(ro, rel=0.02)
    assert rg == pytest.approx(theory.cold_two_stream(L.params["k"], 0.2), rel=0.03)


_WEIBEL_ORACLE = {}


def _weibel_oracle_rate(orc, L, nst):
    if "rate" not in _WEIBEL_ORACLE:
        osim = H.oracle_sim(orc, L, 2, relax_tol=1e-13)
        Wo = _series(osim, nst, lambda s: s.diagnostics()["energy_B"])
        _WEIBEL_ORACLE["rate"] = theory.fit_growth(np.arange(1, nst + 1) * L.dt, Wo)
    return _WEIBEL_ORACLE["rate"]


@pytest.mark.parametrize("precision,eps", [(0, 1e-6), (1, 1e-4)])
def test_weibel_growth_rate_gpu_within_2pct_of_oracle(pp, orc, precision, eps):
    """Quiet cold +-0.5c pair beams with a seeded transverse current mode on
    8 x 32 x 8 cells (the mixed form runs the per-step sorted kernel): the
    growth rate of the magnetic energy, GPU against oracle.  The mixed form
    starts from a larger seed so that its linear phase clears FP32 noise."""
    L = pp_synth.quiet_weibel(eps=eps)
    nst = 240
    gpu = H.gpu_sim(pp, L, precision, 2, relax_tol=1e-12 if precision == 0 else 1e-6)
    Wg = _series(gpu, nst, lambda s: s.diagnostics()["energy_B"])
    t = np.arange(1, nst + 1) * L.dt
    rg, ng = theory.fit_growth(t, Wg)
    Lo = pp_synth.quiet_weibel(eps=eps)
    ro, no = _weibel_oracle_rate(orc, Lo, nst) if eps == 1e-6 else theory.fit_growth(
        t, _series(H.oracle_sim(orc, Lo, 2, relax_tol=1e-13), nst, lambda s: s.diagnostics()["energy_B"]))
    assert ng >= 20 and no >= 20, (ng, no)
    assert rg == pytest.approx(ro, rel=0.02), (rg, ro)
    assert gpu.diagnostics()["status"] == 0


def _electron_kinetic_gpu(sim):
    return sim.diagnostics()["kinetic"][0]


def _electron_kinetic_oracle(sim):
    # sum over the electrons of w m (gamma - 1) dV (the kinetic energy pp_diagnostics reports)
    s = sim.species[0]
    g = np.sqrt(1.0 + s["ux"] ** 2 + s["uy"] ** 2 + s["uz"] ** 2)
    dV = float(np.prod([sim.g.d[a] for a in range(3)]))
    return s["w"] * s["m"] * float((g - 1.0).sum()) * dV


def _heating_slope(sim, steps, every=10, ke_of=_electron_kinetic_gpu):
    """Least-squares slope, per step, of the electron kinetic energy over its
    initial value (the heating rate)."""
    ke = []
    for _ in range(steps // every):
        sim.step(every)
        ke.append(ke_of(sim))
    ke = np.array(ke)
    t = np.arange(1, len(ke) + 1) * every
    return np.polyfit(t, ke / ke[0], 1)[0]


def test_numerical_heating_scales_as_one_over_ppc(pp, orc):
    """Mixed form (the per-step sorted kernel) on 32^3 cells: the electron
    heating rate halves when the particles per cell double (8 -> 16 -> 32),
    each ratio within 25% of 2; at 16^3 x 8 ppc the GPU's rate is within 25%
    of the oracle's (FP64, same seeded particles; heating is a statistical
    property of the noise, so the two runs agree in rate, not step by step)."""
    rates = {}
    for ppc in (8, 16, 32):
        L = pp_synth.heating_plasma(n=(32, 32, 32), ppc=ppc)
        sim = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
        rates[ppc] = _heating_slope(sim, 400)
        assert sim.diagnostics()["status"] == 0
    assert rates[8] > 0.0
    assert rates[8] / rates[16] == pytest.approx(2.0, rel=0.25), rates
    assert rates[16] / rates[32] == pytest.approx(2.0, rel=0.25), rates
    L = pp_synth.heating_plasma(n=(16, 16, 16), ppc=8)
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
    rg = _heating_slope(gpu, 300)
    import os
    orc.set_threads(os.cpu_count() or 1)
    try:
        osim = H.oracle_sim(orc, L, 3, relax_tol=1e-10)
        ro = _heating_slope(osim, 300, ke_of=_electron_kinetic_oracle)
    finally:
        orc.set_threads(1)
    assert rg == pytest.approx(ro, rel=0.25), (rg, ro)


def test_noisy_two_stream_energy_series_fp64(pp, orc):
    L = pp_synth.two_stream()
    gpu = H.gpu_sim(pp, L, pp.PP_FP64, 2)
    osim = H.oracle_sim(orc, L, 2)
    Wg = _series(gpu, 30, lambda s: s.diagnostics()["energy_Ex"])
    Wo = _series(osim, 30, lambda s: s.diagnostics()["energy_Ex"])
    assert np.abs(Wg / Wo - 1).max() <= 1e-8


def test_beam_background_mixed_vs_oracle(pp, orc):
    L = pp_synth.beam_background(n=(16, 16, 16), ppc=2, seed=1214)
    gpu = H.gpu_sim(pp, L, pp.PP_MIXED32, 3)
    osim = H.oracle_sim(orc, L, 3)
    for _ in range(3):
        gpu.step(1)
        osim.step(1)
    d = gpu.diagnostics()
    assert d["status"] == 0
    # the load is a neutral beam (each electron moves with an ion), so rho stays
    # near zero while every species carries a large current: the round-off of
    # those currents is measured against one species' charge density |q| n
    cells = float(np.prod(L.n))
    rho_species = max(abs(sp["q"]) * sp["w"] * len(sp["x"]) / cells for sp in L.species)
    assert d["gauss_drift_max"] <= 2e-5 * rho_species
    # fields likewise: absolute errors against one species' current |q| n c
    # (and that current times the elapsed time for E and B)
    E, B, J = gpu.fields()
    j_species = rho_species * 1.0
    t = 3 * L.dt
    errJ = max(np.abs(J[a] - osim.J[a]).max() for a in range(3))
    errE = max(np.abs(E[a] - osim.E[a]).max() for a in range(3))
    errB = max(np.abs(B[a] - osim.B[a]).max() for a in range(3))
    assert errJ <= 5e-5 * j_species, errJ
    assert errE <= 5e-5 * j_species * t and errB <= 5e-5 * j_species * t, (errE, errB)
    for s in range(2):
        dpos, du = H.particle_errors(gpu.particles(s), osim.species[s], H.box(L))
        assert dpos <= 2e-6 and du <= 5e-6, (s, dpos, du)
