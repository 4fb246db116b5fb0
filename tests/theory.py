"""Closed-form growth rates used by the physics pins (test helper).

cold_two_stream: two symmetric, cold, neutral beams at +/-beta (each of total
plasma frequency omega_b^2 = omega_pe^2 / Gamma^3 for longitudinal motion) obey
1 = omega_b^2/(omega - k v)^2 + omega_b^2/(omega + k v)^2, whose unstable root
has growth omega_b * sqrt(sqrt(1 + 4K^2) - K^2 - 1), K = k v / omega_b.

bret_*: the mixed-mode, filamentation and two-stream estimates quoted in the
paper's Sec. VIII "Relativistic two-stream instability" (eq:mmigrowth,
eq:figrowth, eq:tsigrowth).
"""
import math


def cold_two_stream(k, beta, omega_pe=1.0):
    G = 1.0 / math.sqrt(1.0 - beta * beta)
    wb = omega_pe * G ** -1.5
    K = k * beta / wb
    y = math.sqrt(1.0 + 4.0 * K * K) - K * K - 1.0
    return wb * math.sqrt(y) if y > 0 else 0.0


def bret_mmi(alpha, gamma_b):
    return 2.0 ** (-4.0 / 3.0) * math.sqrt(3.0) * alpha ** (1.0 / 3.0) * gamma_b ** (-1.0 / 3.0)


def bret_fi(alpha, gamma_b):
    beta = math.sqrt(1.0 - 1.0 / gamma_b ** 2)
    return beta * math.sqrt(alpha) / math.sqrt(gamma_b)


def bret_tsi(alpha, gamma_b):
    return 2.0 ** (-4.0 / 3.0) * math.sqrt(3.0) * alpha ** (1.0 / 3.0) / gamma_b


def fit_growth(t, W, lo_factor=1e3, hi_factor=1e-3):
    """Amplitude growth rate from a field-energy series: half the least-squares
    slope of ln W over the window where W has risen lo_factor above its early
    minimum and is still below hi_factor times its maximum (before the peak)."""
    import numpy as np
    t = np.asarray(t, dtype=float)
    W = np.asarray(W, dtype=float)
    ipk = int(np.argmax(W))
    floor = W[: max(5, len(W) // 10)].min()
    sel = (W > lo_factor * floor) & (W < hi_factor * W.max()) & (np.arange(len(W)) < ipk)
    if sel.sum() < 5:
        raise ValueError("no linear-growth window in the series")
    p = np.polyfit(t[sel], np.log(W[sel]), 1)
    return 0.5 * p[0], int(sel.sum())
