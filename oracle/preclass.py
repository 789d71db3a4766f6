"""Pre-classification of pixels before the L1 solve (the hybrid strategy the paper
recommends in Sec. I and Sec. V) -- TEST INFRASTRUCTURE ONLY, plain numpy in FP64.

The paper's text: a cheap linear estimator serves the pixels that need no
super-resolution, and only the remaining pixels are solved by L1 (its conclusion
expects a further speed-up of about 50 from this).  It does not define the
classifier; the reading taken here, stated once so the GPU path can be checked
against it:

  u = A^H g                          beamforming (the classic linear estimator) on the grid
  class 0  2 max_l |u_l| <= lambda   x* = 0 exactly: 0 satisfies Eq. 6's optimality
                                     conditions, so the pixel holds no scatterer (K = 0)
  otherwise the single-scatterer linear estimate:
           l^ = argmax_l |u_l| (first index on ties),
           s^ = argmax |a(s)^H g| over [s_{l^-1}, s_{l^+1}] (clipped to the grid's extent),
           gamma^ = a(s^)^H g / N,   r = g - gamma^ a(s^)      (a(s)_n = exp(-j 2 pi xi_n s))
  class 1  2 max_l |a_l^H r| <= lambda   the residual would itself be screened out: one
                                     scatterer, reported as K = 1 with (s^, gamma^)
  class 2  everything else: BPDN (Eq. 6) with the refit and the model selection.

Class 0 is exact for Eq. 6.  Class 1 is the linear estimator's answer, not the BPDN
minimiser.  Here s^ is found by golden-section search on |a(s)^H g|^2 (no derivatives),
an algorithm unrelated to the library's.
"""
from __future__ import annotations

import math

import numpy as np

GOLD = (math.sqrt(5.0) - 1.0) / 2.0


def steering(xi: np.ndarray, s: float) -> np.ndarray:
    """a(s)_n = exp(-j 2 pi xi_n s) (Eq. 5 at a continuous elevation)."""
    return np.exp(-2j * np.pi * xi * s)


def beam_power(xi: np.ndarray, g: np.ndarray, s: float) -> float:
    """|a(s)^H g|^2."""
    return float(abs(np.vdot(steering(xi, s), g)) ** 2)


def refine_peak(xi: np.ndarray, g: np.ndarray, lo: float, hi: float, tol: float = 1e-12) -> float:
    """Golden-section search for the largest |a(s)^H g|^2 on [lo, hi]."""
    a, b = lo, hi
    c = b - GOLD * (b - a)
    d = a + GOLD * (b - a)
    fc, fd = beam_power(xi, g, c), beam_power(xi, g, d)
    while b - a > tol * max(1.0, abs(a) + abs(b)):
        if fc >= fd:
            b, d, fd = d, c, fc
            c = b - GOLD * (b - a)
            fc = beam_power(xi, g, c)
        else:
            a, c, fc = c, d, fd
            d = a + GOLD * (b - a)
            fd = beam_power(xi, g, d)
    s = 0.5 * (a + b)
    # the end points win if the beam is largest there (the peak at the edge of the extent)
    best = max(((beam_power(xi, g, t), t) for t in (lo, s, hi)), key=lambda v: v[0])
    return best[1]


def classify(A: np.ndarray, xi: np.ndarray, s_grid: np.ndarray, g: np.ndarray, lam: float) -> dict:
    """Class of one pixel and, for classes 0 and 1, its estimates (see the module text).

    Returns dict(cls, khat, s_hat, gamma_hat, umax, rmax): umax = 2 max|A^H g| / lambda and
    rmax = 2 max|A^H r| / lambda (the two decision ratios; NaN where not computed)."""
    g = np.asarray(g, np.complex128)
    N, L = A.shape
    u = A.conj().T @ g
    umax = 2.0 * np.max(np.abs(u)) / lam
    out = {"cls": 2, "khat": -1, "s_hat": math.nan, "gamma_hat": 0j, "umax": umax, "rmax": math.nan}
    if umax <= 1.0:
        out.update(cls=0, khat=0)
        return out
    l_hat = int(np.argmax(np.abs(u)))
    lo = s_grid[max(l_hat - 1, 0)]
    hi = s_grid[min(l_hat + 1, L - 1)]
    s_hat = refine_peak(xi, g, lo, hi) if hi > lo else float(s_grid[l_hat])
    a = steering(xi, s_hat)
    gamma = np.vdot(a, g) / N
    r = g - gamma * a
    rmax = 2.0 * np.max(np.abs(A.conj().T @ r)) / lam
    out["rmax"] = rmax
    if rmax <= 1.0:
        out.update(cls=1, khat=1, s_hat=s_hat, gamma_hat=complex(gamma))
    return out


def classify_batch(A, xi, s_grid, G, lam) -> dict:
    P = G.shape[0]
    lam_v = np.broadcast_to(np.asarray(lam, np.float64), (P,))
    rows = [classify(A, xi, s_grid, G[p], float(lam_v[p])) for p in range(P)]
    return {k: np.array([r[k] for r in rows]) for k in rows[0]} if rows else {}
