"""SL1MMER model selection and parameter estimation in FP64 -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may
import this module.  It shares no code with the CUDA implementation.

Sec. III-A lists SL1MMER's three steps: (1) the L1 minimisation of Eq. 6, (2) model
selection and (3) parameter estimation.  The paper defines steps (2) and (3) only by
reference to the original SL1MMER publication, so this module writes out the reading
the library implements (its readings are listed beside the CUDA kernel too):

  clusters      A scatterer candidate is a maximal run of adjacent nonzero grid
                points of the minimiser x.  Its elevation is the modulus-weighted
                centroid sum |x_l| s_l / sum |x_l| and its energy sum |x_l|^2 (sums in
                ascending grid order).  Candidates are ranked by energy, largest first
                (ties: lower first grid index first); at most kmax are kept.
  select        For K = 0 .. K_c (K_c = number of kept candidates) the model with the
                first K candidates is fitted by least squares with off-grid steering
                vectors a(s)_n = exp(-j 2 pi xi_n s) (Eq. 5 at the candidate elevations):
                gamma_K = argmin ||g - A_K gamma||^2, RSS_K its residual.  The model
                order minimises the Bayesian information criterion of a circular
                complex Gaussian likelihood with unknown noise power,
                    C(K) = 2 N ln RSS_K + K * penalty,   penalty = 3 ln(2N)
                (three real parameters per scatterer, 2N real observations; the
                constant -2N ln N is dropped).  The first minimum wins.  Estimated
                elevations and the amplitudes of that fit are returned in ascending
                elevation.
  detected      A realisation with two true scatterers counts as a detection when
                K_hat = 2 and each sorted estimate lies closer than half the true
                separation to its sorted true elevation.
"""
from __future__ import annotations

import math

import numpy as np

KMAX = 4


def clusters(x, s_grid):
    """[(first, last, centroid, energy)] of the runs of adjacent nonzeros of x, ranked."""
    x = np.asarray(x, np.complex128)
    nz = np.flatnonzero(x != 0)
    out = []
    i = 0
    while i < nz.size:
        j = i
        while j + 1 < nz.size and nz[j + 1] == nz[j] + 1:
            j += 1
        sw = sws = e = 0.0
        for l in nz[i:j + 1]:
            w = math.sqrt(x[l].real * x[l].real + x[l].imag * x[l].imag)
            sw += w
            sws += w * float(s_grid[l])
            e += w * w
        out.append((int(nz[i]), int(nz[j]), sws / sw, e))
        i = j + 1
    out.sort(key=lambda c: (-c[3], c[0]))
    return out


def steering(xi, s):
    """exp(-j 2 pi xi_n s_k) -> [N, K] (Eq. 5 at arbitrary elevations)."""
    return np.exp(-2j * np.pi * np.outer(np.asarray(xi, np.float64), np.atleast_1d(np.asarray(s, np.float64))))


def default_penalty(N: int) -> float:
    return 3.0 * math.log(2.0 * N)


def select(g, x, xi, s_grid, kmax: int = KMAX, penalty: float | None = None):
    """Model order, elevations and amplitudes of one pixel (steps (2) and (3)).

    Returns dict: khat, s_hat [khat] ascending, gamma_hat [khat], crit [K_c + 1],
    rss [K_c + 1], fits (list of gamma_K), centroids [K_c] in rank order."""
    g = np.asarray(g, np.complex128)
    N = g.size
    pen = default_penalty(N) if penalty is None or penalty <= 0 else float(penalty)
    cl = clusters(x, s_grid)[:kmax]
    kc = len(cl)
    cen = np.array([c[2] for c in cl], np.float64)
    A = steering(xi, cen)
    rss = np.empty(kc + 1)
    fits = [np.zeros(0, np.complex128)]
    rss[0] = float(np.vdot(g, g).real)
    for K in range(1, kc + 1):
        AK = A[:, :K]
        gam = np.linalg.solve(AK.conj().T @ AK, AK.conj().T @ g)
        r = g - AK @ gam
        rss[K] = float(np.vdot(r, r).real)
        fits.append(gam)
    with np.errstate(divide="ignore"):
        crit = 2.0 * N * np.log(rss) + pen * np.arange(kc + 1)
    khat = int(np.argmin(crit))
    order = np.argsort(cen[:khat], kind="stable")
    return {"khat": khat, "s_hat": cen[:khat][order], "gamma_hat": fits[khat][order], "crit": crit,
            "rss": rss, "fits": fits, "centroids": cen}


def select_batch(G, X, xi, s_grid, kmax: int = KMAX, penalty: float | None = None):
    """select() for every row: (khat [P], s_hat [P, kmax] NaN padded, gamma_hat [P, kmax] 0 padded)."""
    G, X = np.asarray(G), np.asarray(X)
    P = G.shape[0]
    khat = np.zeros(P, np.int32)
    s_hat = np.full((P, kmax), np.nan)
    gam = np.zeros((P, kmax), np.complex128)
    for p in range(P):
        r = select(G[p], X[p], xi, s_grid, kmax, penalty)
        k = r["khat"]
        khat[p] = k
        s_hat[p, :k] = r["s_hat"]
        gam[p, :k] = r["gamma_hat"]
    return khat, s_hat, gam


def detected(khat: int, s_hat, s_true) -> bool:
    """The detection rule for two true scatterers (see the module header)."""
    if khat != 2:
        return False
    st = np.sort(np.asarray(s_true, np.float64))
    se = np.sort(np.asarray(s_hat, np.float64)[:2])
    half = 0.5 * (st[1] - st[0])
    return bool(np.all(np.abs(se - st) < half))
