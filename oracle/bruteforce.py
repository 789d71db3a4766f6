"""Brute-force minimiser of Eq. 6 for tiny problems -- TEST INFRASTRUCTURE ONLY.

For N <= 4, L <= 8 every candidate support T is enumerated.  On each T the
restricted problem  min_z ||A_T z - g||^2 + lambda sum_i |z_i|  is convex; it is
solved by damped Newton on the smoothed objective with |z| replaced by
sqrt(|z|^2 + eps^2) (smooth and strictly convex, so damped Newton converges from
any start), for eps = 1e-1, 1e-2, ..., 1e-15 in turn, each level warm-started
from the previous one.  A support is admissible when the restricted minimiser
has every |z_i| > 0 and the off-support optimality condition
|2 a_l^H (A z - g)| <= lambda holds; the minimiser of Eq. 6 is the admissible
point of least objective.  Written in numpy, apart from the C oracle.
"""
from __future__ import annotations

import itertools

import numpy as np


def _F(A, g, lam, x):
    r = A @ x - g
    return float(np.vdot(r, r).real + lam * np.abs(x).sum())


def _smoothed_newton(AT, g, lam, eps, z, iters=200):
    """Damped Newton for ||A_T z - g||^2 + lam sum sqrt(|z_i|^2 + eps^2)."""
    m = AT.shape[1]
    G = AT.conj().T @ AT
    c = AT.conj().T @ g
    realG = np.block([[G.real, -G.imag], [G.imag, G.real]])

    def Fs(zz):
        r = AT @ zz - g
        return float(np.vdot(r, r).real + lam * np.sqrt(np.abs(zz) ** 2 + eps ** 2).sum())

    for _ in range(iters):
        q = np.sqrt(np.abs(z) ** 2 + eps ** 2)
        gc = 2.0 * (G @ z - c) + lam * z / q
        grad = np.concatenate([gc.real, gc.imag])
        H = 2.0 * realG
        for i in range(m):
            v = np.array([z[i].real, z[i].imag])
            H[np.ix_([i, m + i], [i, m + i])] += (lam / q[i]) * (np.eye(2) - np.outer(v, v) / q[i] ** 2)
        d = np.linalg.solve(H, -grad)
        slope = float(grad @ d)
        if -slope <= 1e-30:
            break
        dz = d[:m] + 1j * d[m:]
        f0 = Fs(z)
        t = 1.0
        while t > 1e-20 and Fs(z + t * dz) > f0 + 1e-4 * t * slope:
            t *= 0.5
        z = z + t * dz
        if t * np.max(np.abs(dz)) <= 1e-16 * max(1.0, np.max(np.abs(z))):
            break
    return z


def _restricted_min(AT, g, lam):
    """Minimiser of the restricted problem on T (exact zeros where it has them), or None
    when A_T has dependent columns."""
    m = AT.shape[1]
    G = AT.conj().T @ AT
    if np.linalg.matrix_rank(G) < m:
        return None
    z = np.linalg.solve(G, AT.conj().T @ g)
    for k in range(1, 16):
        z = _smoothed_newton(AT, g, lam, 10.0 ** (-k), z)
    scale = max(1.0, float(np.max(np.abs(z))))
    z = np.where(np.abs(z) <= 1e-9 * scale, 0, z)
    return z


def bruteforce_min(A: np.ndarray, g: np.ndarray, lam: float):
    """Exact minimiser of ||A x - g||^2 + lam ||x||_1 by enumeration of supports."""
    A = np.asarray(A, np.complex128)
    g = np.asarray(g, np.complex128)
    N, L = A.shape
    # zero solution: admissible iff |2 a_l^H g| <= lambda for all l
    best_x = np.zeros(L, np.complex128)
    best_F = np.inf
    if np.max(np.abs(2.0 * A.conj().T @ g)) <= lam:
        best_x, best_F = np.zeros(L, np.complex128), _F(A, g, lam, np.zeros(L))
    for m in range(1, min(N, L) + 1):
        for T in itertools.combinations(range(L), m):
            T = list(T)
            z = _restricted_min(A[:, T], g, lam)
            if z is None or np.any(z == 0):
                continue
            x = np.zeros(L, np.complex128)
            x[T] = z
            zfull = 2.0 * A.conj().T @ (A @ x - g)
            off = [l for l in range(L) if l not in T]
            if off and np.max(np.abs(zfull[off])) > lam * (1.0 + 1e-9):
                continue
            F = _F(A, g, lam, x)
            if F < best_F:
                best_F, best_x = F, x
    return best_x, best_F
