"""Closed-form growth rates used by the physics pins (test helper).

cold_two_stream: two symmetric, cold, neutral beams at +/-beta (each of total
plasma frequency omega_b^2 = omega_pe^2 / Gamma^3 for longitudinal motion) obey
1 = omega_b^2/(omega - k v)^2 + omega_b^2/(omega + k v)^2, whose unstable root
has growth omega_b * sqrt(sqrt(1 + 4K^2) - K^2 - 1), K = k v / omega_b.

cold_filamentation: cold beams along x with a transverse mode along y (E_x,
B_z ~ exp(i k y - i w t)): the linearised cold-fluid and Maxwell equations
give w^4 - (k^2 + A) w^2 - k^2 C = 0 with A = sum_s w_ps^2 / gamma_s^3 (the
longitudinal response, mass gamma^3 m) and C = sum_s w_ps^2 v_s^2 / gamma_s
(the transverse deflection of the beams by v x B, mass gamma m, feeding back
through the density modulation); the unstable root has growth
sqrt((sqrt((k^2 + A)^2 + 4 k^2 C) - (k^2 + A)) / 2), which tends to the
known cold limit beta w_p / sqrt(gamma) for k c >> w_p.

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


def cold_filamentation(k, beams):
    """Growth rate of the transverse mode k (c = 1) for cold beams given as
    (w_ps^2, beta_s) pairs."""
    A = sum(w2 * (1.0 - b * b) ** 1.5 for w2, b in beams)
    C = sum(w2 * b * b * math.sqrt(1.0 - b * b) for w2, b in beams)
    kA = k * k + A
    return math.sqrt(0.5 * (math.sqrt(kA * kA + 4.0 * k * k * C) - kA))


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
