"""Admission of the serving loop (host logic, no device): device bytes,
slots, and the particle budget of the running requests."""
from paper_1211_4575_gb300.serving import admissible

GiB = 1 << 30


def test_bytes_and_slots_bound_admission():
    assert admissible(10 * GiB, 5 * GiB, 16 * GiB, 1, 8, 0, 0)
    assert not admissible(12 * GiB, 5 * GiB, 16 * GiB, 1, 8, 0, 0)        # bytes over the budget
    assert not admissible(0, 1, 16 * GiB, 8, 8, 0, 0)                       # no free slot
    assert admissible(0, 16 * GiB, 16 * GiB, 0, 8, 0, 0)                    # exactly the budget


def test_particle_budget_keeps_a_gpu_filling_run_alone():
    budget = 48_000_000
    # small runs overlap while their particles fit together
    assert admissible(0, 1, GiB, 2, 8, 20_000_000, 10_000_000, budget)
    assert not admissible(0, 1, GiB, 2, 8, 40_000_000, 10_000_000, budget)
    # a run over the budget waits for an idle GPU, then enters alone
    assert not admissible(0, 1, GiB, 1, 8, 1_000_000, 200_000_000, budget)
    assert admissible(0, 1, GiB, 0, 8, 0, 200_000_000, budget)
    # no particle budget: only bytes and slots count
    assert admissible(0, 1, GiB, 3, 8, 400_000_000, 200_000_000, None)
