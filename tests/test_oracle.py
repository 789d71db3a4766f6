"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it pins.  The oracle is checked against hand-derived
values, closed forms, brute force and invariances -- never against itself.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.bruteforce import bruteforce_min
from paper_1805_01759_gb300 import synth

WL, RG = 0.031, 7.0e5


def _geom(b, s_min, s_max, L, wl=WL, rg=RG):
    return synth.StackGeometry(np.asarray(b, np.float64), wl, rg, s_min, s_max, L)


# ------------------------------------------------------------------ Eq. 5

def test_grid_includes_both_ends():
    """Eq. 5: gamma sampled uniformly at s_l on the elevation extent (both ends kept)."""
    s = oracle.grid(-100.0, 100.0, 201)
    assert s[0] == -100.0 and s[-1] == 100.0
    np.testing.assert_allclose(np.diff(s), 1.0, rtol=0, atol=1e-12)
    assert oracle.grid(3.0, 7.0, 1)[0] == 3.0


def test_operator_hand_values():
    """Eq. 5 with xi_n = 2 b_n / (wavelength r) (Sec. II): a baseline with xi = 0.01/m gives
    A = exp(-j 2 pi 0.01 s): s=25 -> -j, s=50 -> -1, s=-25 -> +j, b=0 -> 1."""
    b1 = 0.01 * WL * RG / 2.0  # xi = 0.01 per metre
    geom = _geom([0.0, b1], -100.0, 100.0, 201)  # s_l = -100 + l
    A = oracle.operator(geom)
    i = lambda s: int(s + 100)
    np.testing.assert_allclose(A[0], 1.0, atol=1e-15)
    np.testing.assert_allclose(A[1, i(25)], -1j, atol=1e-13)
    np.testing.assert_allclose(A[1, i(50)], -1.0, atol=1e-13)
    np.testing.assert_allclose(A[1, i(-25)], 1j, atol=1e-13)
    np.testing.assert_allclose(A[1, i(0)], 1.0, atol=1e-15)
    np.testing.assert_allclose(np.abs(A), 1.0, atol=1e-14)


def test_gram_toeplitz_matches_direct_product():
    """On the uniform grid of Eq. 5, (A^H A)_{lm} depends on l-m only: h(l-m)."""
    st = synth.workload_small(P=1)
    A = oracle.operator(st.geom)
    h = oracle.gram_toeplitz(st.geom)
    G = A.conj().T @ A  # numpy product, independent of the oracle's h
    L = st.geom.L
    l, m = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    np.testing.assert_allclose(h[l - m + L - 1], G, atol=1e-10)
    np.testing.assert_allclose(h[L - 1], st.geom.N, atol=1e-12)


def test_aah_dirichlet_closed_form():
    """(A A^H)_{nm} = sum_l exp(-j2pi(xi_n - xi_m)(s0 + l ds)), a geometric series."""
    st = synth.workload_small(P=1)
    geom = st.geom
    A = oracle.operator(geom)
    M = oracle.aah(A)
    x = 2.0 * geom.baselines_m / (geom.wavelength_m * geom.range_m)
    L = geom.L
    ds = (geom.s_max_m - geom.s_min_m) / (L - 1)
    dxi = x[:, None] - x[None, :]
    w = np.exp(-2j * np.pi * dxi * ds)
    with np.errstate(invalid="ignore", divide="ignore"):
        geo = np.where(np.abs(dxi) > 0, (1 - w ** L) / (1 - w), L)
    ref = np.exp(-2j * np.pi * dxi * geom.s_min_m) * geo
    np.testing.assert_allclose(M, ref, atol=1e-9)


def test_lipschitz_closed_forms():
    """L_f = 2 lambda_max(A^H A): DFT geometry has A^H A = N I (L_f = 2N); one acquisition
    (N = 1) has A A^H = L (L_f = 2L)."""
    for N in (4, 16, 25):
        A = oracle.operator(synth.dft_geometry(N))
        np.testing.assert_allclose(A.conj().T @ A, N * np.eye(N), atol=1e-10)
        assert abs(oracle.lipschitz(A) - 2 * N) < 1e-9
    A1 = oracle.operator(_geom([37.0], -50.0, 50.0, 77))
    assert abs(oracle.lipschitz(A1) - 2 * 77) < 1e-9


# ------------------------------------------------------------------ Eq. 10

def test_soft_threshold_closed_form():
    """Eq. 10 for complex values: S_tau(v) = v (1 - tau/|v|) if |v| > tau else 0.
    On the real line it gives Eq. 10's three cases (x - a, 0, x + a)."""
    out = oracle.soft(np.array([3 + 4j, 3 + 4j, 3 + 4j, 0j, 2.0, -2.0, 0.5, -0.5]), 1.0)
    np.testing.assert_allclose(out[0], 2.4 + 3.2j, atol=1e-15)
    np.testing.assert_allclose(out[4:], [1.0, -1.0, 0.0, 0.0], atol=1e-15)
    assert oracle.soft(3 + 4j, 5.0)[0] == 0  # |v| == tau -> exactly zero
    assert oracle.soft(3 + 4j, 4.999)[0] != 0
    assert oracle.soft(0j, 0.1)[0] == 0
    np.testing.assert_allclose(oracle.soft(1j * 3, 1.0)[0], 2j, atol=1e-15)


# ------------------------------------------------------------- Algorithm 1

def test_first_iteration_closed_form():
    """Algorithm 1 at k=1 from x^0 = 0: y = 0, grad f(0) = -2 A^H g, so
    xbar = S_{alpha lambda}(2 alpha A^H g) with the alpha left by backtracking (Eq. 15);
    it is accepted iff F(xbar) <= F(0)."""
    st = synth.workload_small(P=8)
    A = oracle.operator(st.geom)
    a0 = oracle.default_alpha0(A)
    assert abs(a0 - 1.0 / (2 * st.geom.N)) < 1e-15
    for p in range(8):
        g = st.g[p].astype(np.complex128)
        r = oracle.rbpg(A, g, st.lam, max_iter=1, trace=True)
        alpha = r["alpha"][0]
        assert alpha == a0 * 0.5 ** r["n_bt"][0]
        v = 2.0 * alpha * (A.conj().T @ g)
        a = np.abs(v)
        xbar = np.where(a > alpha * st.lam, v * (1 - alpha * st.lam / np.maximum(a, 1e-300)), 0)
        F0 = float(np.vdot(g, g).real)
        Fb = float(np.vdot(A @ xbar - g, A @ xbar - g).real + st.lam * np.abs(xbar).sum())
        np.testing.assert_allclose(r["F"][0], Fb, rtol=1e-12)
        expect = xbar if Fb <= F0 else np.zeros_like(xbar)
        np.testing.assert_allclose(r["x"], expect, atol=1e-12)
        # Eq. 15 with base point y = 0 holds for the alpha that was kept
        d = xbar
        assert np.vdot(A @ d, A @ d).real <= np.vdot(d, d).real / (2 * alpha) * (1 + 1e-12)


def test_momentum_weight_second_and_third_iteration():
    """theta_k = 2/(k+1) gives y^{k} = x^k + (k-2)/(k+1) (x^k - x^{k-1}) (Eqs. 11-12):
    beta = 0 at k=2 and 1/4 at k=3.  Re-run iteration 3 by hand from the oracle's
    x^1, x^2 and alpha and compare."""
    st = synth.workload_small(P=16)
    A = oracle.operator(st.geom)
    lam = st.lam
    checked = 0
    for p in range(16):
        g = st.g[p].astype(np.complex128)
        r1 = oracle.rbpg(A, g, lam, max_iter=1, tol=0.0, trace=True)
        r2 = oracle.rbpg(A, g, lam, max_iter=2, tol=0.0, trace=True)
        r3 = oracle.rbpg(A, g, lam, max_iter=3, tol=0.0, trace=True)
        if r3["iters"] < 3 or not (r2["accepted"][1] and r1["accepted"][0]):
            continue
        if r3["n_bt"][2] != 0:
            continue
        x1, x2 = r1["x"], r2["x"]
        y = x2 + 0.25 * (x2 - x1)
        alpha = r3["alpha"][2]
        v = y - alpha * 2.0 * (A.conj().T @ (A @ y - g))
        xb = oracle.soft(v, alpha * lam)
        F2 = r2["F"][1]
        Fb = float(np.vdot(A @ xb - g, A @ xb - g).real + lam * np.abs(xb).sum())
        expect = xb if Fb <= F2 else x2
        np.testing.assert_allclose(r3["x"], expect, atol=1e-11)
        checked += 1
    assert checked >= 4


def test_orthogonal_columns_closed_form():
    """DFT geometry (A^H A = N I): x* = S_{lambda/2}(A^H g) / N, reached by Algorithm 1
    in one step (alpha_0 = 1/(2N) = 1/L_f) and by the exact minimiser."""
    rng = np.random.default_rng(7)
    N = 16
    A = oracle.operator(synth.dft_geometry(N))
    for _ in range(5):
        g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        lam = 0.5 * np.max(np.abs(2 * A.conj().T @ g))
        c = A.conj().T @ g
        a = np.abs(c)
        xs = np.where(a > lam / 2, c * (1 - (lam / 2) / a), 0) / N
        r = oracle.minimise(A, g, lam)
        np.testing.assert_allclose(r["x"], xs, atol=1e-12)
        ra = oracle.rbpg(A, g, lam, tol=1e-12, max_iter=50)
        np.testing.assert_allclose(ra["x"], xs, atol=1e-12)
        assert ra["iters"] <= 3


def test_single_column_closed_form():
    """L = 1: x* = S_{lambda/2}(a^H g) / ||a||^2."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        N = 7
        a = np.exp(-2j * np.pi * rng.uniform(0, 1, N))
        A = a[:, None]
        g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        lam = rng.uniform(0.1, 2.0) * abs(a.conj() @ g)
        c = a.conj() @ g
        xs = (c * max(0.0, 1 - (lam / 2) / abs(c))) / N
        r = oracle.minimise(A, g, lam)
        np.testing.assert_allclose(r["x"][0], xs, atol=1e-13)
        ra = oracle.rbpg(A, g, lam, tol=1e-13, max_iter=2000)
        np.testing.assert_allclose(ra["x"][0], xs, atol=1e-12)


def test_zero_solution():
    """lambda >= 2 ||A^H g||_inf  =>  x* = 0; Algorithm 1 returns 0 at k = 1."""
    st = synth.workload_small(P=4)
    A = oracle.operator(st.geom)
    for p in range(4):
        g = st.g[p].astype(np.complex128)
        lam = 2.0 * np.max(np.abs(A.conj().T @ g)) * 1.0001
        r = oracle.minimise(A, g, lam)
        assert np.all(r["x"] == 0)
        ra = oracle.rbpg(A, g, lam)
        assert np.all(ra["x"] == 0) and ra["iters"] == 1
        assert ra["status"] & oracle.STATUS_ZERO_SOLUTION
        assert not ra["status"] & oracle.STATUS_NOT_CONVERGED


def test_nonfinite_input():
    st = synth.workload_small(P=1)
    A = oracle.operator(st.geom)
    g = st.g[0].astype(np.complex128)
    g[3] = np.nan
    ra = oracle.rbpg(A, g, st.lam)
    assert ra["status"] & oracle.STATUS_NONFINITE and np.all(ra["x"] == 0) and ra["iters"] == 0


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_tiny(seed):
    """N <= 4, L <= 8: enumerate supports; the minimiser found matches the exact
    minimiser (CD + Newton) and the end point of Algorithm 1."""
    rng = np.random.default_rng(100 + seed)
    N = int(rng.integers(2, 5))
    L = int(rng.integers(3, 9))
    b = rng.uniform(-250, 250, N)
    geom = _geom(b, -60.0, 60.0, L)
    A = oracle.operator(geom)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    lam = rng.uniform(0.2, 0.8) * np.max(np.abs(2 * A.conj().T @ g))
    xb, Fb = bruteforce_min(A, g, lam)
    r = oracle.minimise(A, g, lam)
    np.testing.assert_allclose(r["x"], xb, atol=1e-9)
    assert np.array_equal(r["x"] != 0, xb != 0)
    ra = oracle.rbpg(A, g, lam, tol=1e-13, max_iter=100000)
    np.testing.assert_allclose(ra["x"], xb, atol=1e-5 * max(1.0, np.abs(xb).max()))
    assert oracle.objective(A, g, lam, ra["x"]) >= Fb - 1e-9


@pytest.mark.parametrize("seed", range(6))
def test_repair_from_an_unconverged_descent(seed):
    """Coordinate descent stopped after one sweep leaves a wrong support; the exact
    minimiser must still come out (through the working-set repair), equal to the
    brute-force enumeration of supports, with a clean certificate."""
    rng = np.random.default_rng(300 + seed)
    N = int(rng.integers(3, 5))
    L = 8
    b = rng.uniform(-250, 250, N)
    geom = _geom(b, -30.0, 30.0, L)  # 8.6 m bins: strongly coherent neighbouring columns
    A = oracle.operator(geom)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    lam = rng.uniform(0.3, 0.6) * np.max(np.abs(2 * A.conj().T @ g))
    xb, Fb = bruteforce_min(A, g, lam)
    assert np.isfinite(Fb)
    x1, sweeps, rc = oracle.cd(A, g, lam, max_sweeps=1)
    on, off, _, _ = oracle.kkt(A, g, lam, x1)
    assert rc == 1 and (on > 1e-6 or off > 1 + 1e-6)  # one sweep is not the minimiser
    r = oracle.minimise(A, g, lam, max_sweeps=1)
    assert r["flags"] == 0 and r["sweeps"] == 1
    np.testing.assert_allclose(r["x"], xb, atol=1e-9 * max(1.0, np.abs(xb).max()))
    assert np.array_equal(r["x"] != 0, xb != 0)


def test_repair_on_workload_pixels():
    """On the small workload, three descent sweeps plus the repair give the same
    minimiser as descent run to convergence."""
    st = synth.workload_small(P=16, seed=3)
    A = oracle.operator(st.geom)
    full = oracle.minimise_batch(A, st.g, st.lam)
    short = oracle.minimise_batch(A, st.g, st.lam, max_sweeps=3)
    assert np.all(full["flags"] == 0) and np.all(short["flags"] == 0)
    np.testing.assert_allclose(short["x"], full["x"], atol=1e-9 * np.abs(full["x"]).max())


def test_stopping_trace_matches_the_stop():
    """Algorithm 1 stops at the first iteration whose relative candidate step
    ||xbar - x^k|| / ||xbar|| is at most tol; from x^0 = 0 the first step is exactly 1."""
    st = synth.workload_small(P=24, seed=4)
    A = oracle.operator(st.geom)
    for tol in (1e-2, 1e-4):
        for p in range(st.g.shape[0]):
            r = oracle.rbpg(A, st.g[p], st.lam, tol=tol, max_iter=300, trace=True)
            step = r["step"]
            if np.all(r["x"] == 0):
                continue
            assert step[0] == 1.0
            small = np.nonzero(step <= tol)[0]
            if r["status"] & oracle.STATUS_NOT_CONVERGED:
                assert small.size == 0 and r["iters"] == 300
            else:
                assert small.size >= 1 and r["iters"] == small[0] + 1


def test_certificate_on_workload():
    """Eq. 6 optimality at every oracle output of the small workload: on the support
    2 a_l^H (A x - g) = -lambda x_l/|x_l|, off it |2 a_l^H (A x - g)| <= lambda."""
    st = synth.workload_small(P=64)
    A = oracle.operator(st.geom)
    r = oracle.minimise_batch(A, st.g, st.lam)
    assert np.all(r["on_res"] <= 1e-9)
    assert np.all(r["off_max"] <= 1.0 + 1e-9)
    # and the certificate really detects a non-minimiser
    x = r["x"][np.argmax(r["nS"])].copy()
    x[np.nonzero(x)[0][0]] *= 1.01
    on, off, _, _ = oracle.kkt(A, st.g[np.argmax(r["nS"])], st.lam, x)
    assert on > 1e-4


def test_rbpg_and_cd_agree_well_conditioned():
    """Two unrelated algorithms, one unique minimiser: on a coarse grid (columns far
    from coherent) Algorithm 1 run to a tight tolerance meets coordinate descent."""
    rng = np.random.default_rng(11)
    geom = synth.make_geometry(rng, 25, 9, 250.0, 100.0)  # 25 m bins vs ~45 m resolution
    A = oracle.operator(geom)
    for _ in range(4):
        g = A[:, [2, 6]] @ (rng.standard_normal(2) + 1j * rng.standard_normal(2))
        g = g + 0.1 * (rng.standard_normal(25) + 1j * rng.standard_normal(25))
        lam = 0.2 * np.max(np.abs(2 * A.conj().T @ g))
        r = oracle.minimise(A, g, lam)
        ra = oracle.rbpg(A, g, lam, tol=1e-12, max_iter=50000)
        np.testing.assert_allclose(ra["x"], r["x"], atol=1e-7 * np.abs(r["x"]).max())


def test_invariances():
    """Global phase, scale (g, lambda) -> (c g, |c| lambda), row permutation and grid
    shift (g -> D g with D = diag(exp(-j2pi xi_n s0))) leave the minimiser's
    structure unchanged (Eq. 6)."""
    st = synth.workload_small(P=6)
    geom = st.geom
    A = oracle.operator(geom)
    rng = np.random.default_rng(5)
    for p in range(6):
        g = st.g[p].astype(np.complex128)
        lam = st.lam
        x0 = oracle.minimise(A, g, lam)["x"]
        ph = np.exp(1j * 0.7)
        np.testing.assert_allclose(oracle.minimise(A, ph * g, lam)["x"], ph * x0, atol=1e-10)
        c = 2.5 * np.exp(-1j * 1.1)
        np.testing.assert_allclose(oracle.minimise(A, c * g, abs(c) * lam)["x"], c * x0,
                                   atol=1e-9)
        perm = rng.permutation(geom.N)
        np.testing.assert_allclose(oracle.minimise(A[perm], g[perm], lam)["x"], x0, atol=1e-10)
        s0 = 17.0
        gs = geom.baselines_m
        geom2 = _geom(gs, geom.s_min_m + s0, geom.s_max_m + s0, geom.L)
        xi = 2 * gs / (WL * RG)
        g2 = np.exp(-2j * np.pi * xi * s0) * g
        np.testing.assert_allclose(oracle.minimise(oracle.operator(geom2), g2, lam)["x"], x0,
                                   atol=1e-9)


def test_monotone_objective_and_step():
    """Algorithm 1's accept test keeps F(x^k) non-increasing; backtracking only shrinks
    alpha (Eq. 15), and every kept alpha satisfies it."""
    st = synth.workload_small(P=8)
    A = oracle.operator(st.geom)
    for p in range(8):
        r = oracle.rbpg(A, st.g[p], st.lam, max_iter=300, trace=True)
        F_acc = []
        Fx = float(np.vdot(st.g[p], st.g[p]).real)
        for k in range(r["iters"]):
            if r["accepted"][k]:
                assert r["F"][k] <= Fx
                Fx = r["F"][k]
            F_acc.append(Fx)
        assert np.all(np.diff(F_acc) <= 0)
        assert np.all(np.diff(r["alpha"]) <= 0)


def test_newton_polish_one_component_closed_form():
    """|S| = 1: the restricted optimality system has x = u (|a^H g| - lambda/2)/N,
    u the phase of a^H g."""
    st = synth.workload_small(P=1)
    A = oracle.operator(st.geom)
    g = st.g[0].astype(np.complex128)
    l = 57
    c = A[:, l].conj() @ g
    lam = abs(c)  # < 2|c|, so the one-column solution is nonzero
    expect = (c / abs(c)) * (abs(c) - lam / 2) / st.geom.N
    z, rc, res = oracle.newton_polish(A, g, lam, [l], [c / st.geom.N])
    assert rc == 0
    np.testing.assert_allclose(z[0], expect, atol=1e-13)


# ------------------------------------------------- adjoint (implicit differentiation)

def _loss(c, x):
    """L(x) = Re <c, x> = sum_l Re(conj(c_l) x_l): dL/dRe x + j dL/dIm x = c."""
    return float(np.real(np.vdot(c, x)))


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_matches_finite_differences(seed):
    """Derivatives of the minimiser of Eq. 6 in g and lambda: central differences of
    the exact minimiser (CD + Newton, no Jacobian involved) against the adjoint."""
    rng = np.random.default_rng(300 + seed)
    N = int(rng.integers(5, 11))
    L = int(rng.integers(12, 31))
    geom = _geom(rng.uniform(-250, 250, N), -60.0, 60.0, L)
    A = oracle.operator(geom)
    for _ in range(50):
        g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        lam = rng.uniform(0.2, 0.6) * np.max(np.abs(2 * A.conj().T @ g))
        r = oracle.minimise(A, g, lam)
        if (r["nS"] >= 1 and r["margin"] > 1e-2
                and r["min_abs_on"] > 1e-2 * np.abs(r["x"]).max()):
            break
    else:
        raise AssertionError("no non-degenerate problem drawn")
    c = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    dg, dl, rc = oracle.adjoint(A, lam, r["x"], c)
    assert rc == 0
    h = 1e-6 * max(1.0, np.abs(g).max())
    fd = np.zeros(N, np.complex128)
    for n in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            gp, gm = g.copy(), g.copy()
            gp[n] += h * unit
            gm[n] -= h * unit
            d = (_loss(c, oracle.minimise(A, gp, lam)["x"]) - _loss(c, oracle.minimise(A, gm, lam)["x"])) / (2 * h)
            fd[n] += d if part == 0 else 1j * d
    np.testing.assert_allclose(dg, fd, rtol=0, atol=1e-6 * np.abs(fd).max())
    hl = 1e-6 * lam
    fdl = (_loss(c, oracle.minimise(A, g, lam + hl)["x"]) - _loss(c, oracle.minimise(A, g, lam - hl)["x"])) / (2 * hl)
    assert abs(dl - fdl) <= 1e-6 * max(abs(fdl), np.abs(fd).max() * np.abs(g).max() / lam)


def test_adjoint_orthogonal_columns_closed_form():
    """DFT geometry (A^H A = N I): x_l = w_l (1 - lambda / (2|w_l|)) / N for |w_l| > lambda/2,
    w = A^H g.  Differentiating that formula by hand: dx_l/dlambda = -u_l / (2N) and
    dx_l/dw_l = (I - lambda/(2|w_l|) (I - u_l u_l^T)) / N (real 2x2, u_l = w_l/|w_l|), and
    dL/dg = sum_l a_l (dL/dw_l) since w_l = a_l^H g is complex linear."""
    rng = np.random.default_rng(11)
    N = 16
    A = oracle.operator(synth.dft_geometry(N))
    for _ in range(4):
        g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        w = A.conj().T @ g
        lam = 0.6 * np.max(np.abs(2 * w))
        r = oracle.minimise(A, g, lam)
        c = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        act = np.abs(w) > lam / 2
        assert np.array_equal(act, r["x"] != 0)
        dl_ref = 0.0
        dg_ref = np.zeros(N, np.complex128)
        for l in np.nonzero(act)[0]:
            u = np.array([w[l].real, w[l].imag]) / abs(w[l])
            cl = np.array([c[l].real, c[l].imag])
            Jx = (np.eye(2) - lam / (2 * abs(w[l])) * (np.eye(2) - np.outer(u, u))) / N
            dLdw = Jx.T @ cl
            dg_ref += A[:, l] * (dLdw[0] + 1j * dLdw[1])
            dl_ref += -(cl @ u) / (2 * N)
        dg, dl, rc = oracle.adjoint(A, lam, r["x"], c)
        assert rc == 0
        np.testing.assert_allclose(dg, dg_ref, rtol=0, atol=1e-10 * np.abs(dg_ref).max())
        assert abs(dl - dl_ref) <= 1e-10 * max(1.0, abs(dl_ref))


def test_adjoint_zero_solution():
    """x* = 0 (lambda >= 2 ||A^H g||_inf) does not move under small changes: zero derivatives."""
    st = synth.workload_small(P=2)
    A = oracle.operator(st.geom)
    g = st.g[0].astype(np.complex128)
    lam = 2.5 * np.max(np.abs(A.conj().T @ g))
    x = oracle.minimise(A, g, lam)["x"]
    assert np.all(x == 0)
    dg, dl, rc = oracle.adjoint(A, lam, x, np.ones(st.geom.L, np.complex128))
    assert rc == 0 and np.all(dg == 0) and dl == 0.0


# ------------------------------------------------ multi-component operator (Eq. 4)

def test_operator_md_without_motion_is_the_elevation_operator():
    """One motion point at p = 0: Eq. 4 reduces to Eq. 5 (the C oracle's operator)."""
    rng = np.random.default_rng(4)
    geom = synth.MotionGeometry(rng.uniform(-250, 250, 20), 0.031, 7e5, -50.0, 50.0, 40,
                                eta=rng.uniform(0, 300, (1, 20)), p_min=np.zeros(1), p_max=np.zeros(1),
                                L_p=np.array([1]))
    np.testing.assert_allclose(oracle.operator_md(geom), oracle.operator(geom), rtol=0, atol=1e-13)


def test_operator_md_folds_onto_a_longer_elevation_grid():
    """With eta = c * xi the phase xi s + eta p = xi (s + c p): on an elevation grid of 8
    points spaced 1 m and a motion grid spaced 8/c, column (l_s, l_v) is the elevation
    column at s_{l_s} + 8 l_v, so the whole operator equals the elevation-only operator
    (C oracle) on a 24-point grid, column for column."""
    rng = np.random.default_rng(5)
    b = rng.uniform(-250, 250, 16)
    x = oracle.xi(b, 0.031, 7e5)
    c = 3.5
    geom = synth.MotionGeometry(b, 0.031, 7e5, 0.0, 7.0, 8, eta=(c * x)[None, :], p_min=np.zeros(1),
                                p_max=np.array([16.0 / c]), L_p=np.array([3]))
    long = synth.StackGeometry(b, 0.031, 7e5, 0.0, 23.0, 24)
    np.testing.assert_allclose(oracle.operator_md(geom), oracle.operator(long), rtol=0, atol=1e-12)


OPERATOR_MD_MUTANTS = {
    "motion_sign": ("phase = (phase[:, None, :] + part[:, :, None])", "phase = (phase[:, None, :] - part[:, :, None])"),
    "elevation_slowest": ("phase = (phase[:, None, :] + part[:, :, None]).reshape(N, -1)",
                          "phase = (phase[:, :, None] + part[:, None, :]).reshape(N, -1)"),
    "grid_open_end": ("np.linspace(geom.p_min[m], geom.p_max[m], int(geom.L_p[m]))",
                      "np.linspace(geom.p_min[m], geom.p_max[m], int(geom.L_p[m]), endpoint=False)"),
    "phase_sign": ("return np.exp(-2j * np.pi * phase)", "return np.exp(2j * np.pi * phase)"),
}


@pytest.mark.parametrize("name", sorted(OPERATOR_MD_MUTANTS))
def test_operator_md_mutant_caught(name, monkeypatch):
    """Planted mistakes in oracle.operator_md each fail one of its two pins."""
    import inspect
    import textwrap
    old, new = OPERATOR_MD_MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(oracle.operator_md))
    assert src.count(old) == 1, name
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), ns)
    monkeypatch.setattr(oracle, "operator_md", ns["operator_md"])
    caught = False
    for pin in (test_operator_md_without_motion_is_the_elevation_operator,
                test_operator_md_folds_onto_a_longer_elevation_grid):
        try:
            pin()
        except AssertionError:
            caught = True
    assert caught, f"no pin catches the planted mistake {name}"


# ------------------------------------------------- randomized blocks (Eqs. 13-14)

def test_splitmix64_published_outputs():
    """The block draws' generator against its published first outputs (tests/golden)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    assert [int(v) for v in oracle.splitmix64(0, len(want))] == want


def test_blocks_one_block_is_algorithm_1():
    """With J = 1 the block reading is Algorithm 1: identical iterates and counts."""
    st = synth.workload_small(P=16, seed=1)
    A = oracle.operator(st.geom)
    r1 = oracle.rbpg_batch(A, st.g, st.lam, tol=1e-6)
    rb = oracle.rbpg_block_batch(A, st.g, st.lam, 1, 5, tol=1e-6)
    assert np.array_equal(r1["x"], rb["x"]) and np.array_equal(r1["iters"], rb["iters"])
    assert np.array_equal(r1["status"], rb["status"])


@pytest.mark.parametrize("seed", range(3))
def test_blocks_dft_closed_form(seed):
    """Orthogonal columns (DFT geometry): every block has L_j = 2N, so the draw is uniform,
    and one block step with alpha = 1/(2N) lands on that block's part of the closed form
    x* = S_{lambda/2}(A^H g)/N, so the iterate equals x* once every block was drawn.  Eq. 15
    holds with equality there (||A d||^2 = N ||d||^2), so rounding can halve alpha on a
    block, which then converges geometrically: compared at 1e-10."""
    N = 16
    A = oracle.operator(synth.dft_geometry(N))
    Pj, cum = oracle.block_probabilities(A, 4)
    np.testing.assert_allclose(Pj, 0.25, rtol=0, atol=1e-12)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=N) + 1j * rng.normal(size=N)
    lam = float(rng.uniform(0.5, 2.0)) * float(np.abs(A.conj().T @ g).max()) / 2
    xs = oracle.soft(A.conj().T @ g, lam / 2) / N
    x, it, st, trace = oracle.rbpg_block(A, g, lam, 4, 100 + seed, 0, tol=1e-15, max_iter=400)
    assert set(trace.tolist()) == {0, 1, 2, 3}
    assert np.abs(x - xs).max() <= 1e-10 * max(1.0, np.abs(xs).max())


def test_blocks_draw_frequencies():
    """Eq. 14: the drawn blocks follow P_j = L_j / sum L_j (chi-square over 12,800 draws of
    64 pixels' streams).  On a uniform grid equal blocks have equal constants (shifting a
    block is a unitary diagonal similarity of A_j A_j^H), so the grid here has L = 13 points
    in blocks of 3, 3, 3 and 4, whose constants differ."""
    rng = np.random.default_rng(8)
    geom = synth.make_geometry(rng, 12, 13, 250.0, 100.0)
    A = oracle.operator(geom)
    Pj, _ = oracle.block_probabilities(A, 4)
    assert Pj.max() / Pj.min() > 1.05
    g = np.zeros(12, np.complex128)
    counts = np.zeros(4)
    for p in range(64):
        _, it, _, trace = oracle.rbpg_block(A, g + 1.0, 1e6, 4, 21, p, tol=-1.0, max_iter=50)
        counts += np.bincount(trace, minlength=4)
    n = counts.sum()
    assert n == 64 * 50 * 4
    chi2 = float(np.sum((counts - n * Pj) ** 2 / (n * Pj)))
    assert chi2 < 16.3, (chi2, counts / n, Pj)  # 3 degrees of freedom, p = 0.001


@pytest.mark.parametrize("seed", range(3))
def test_blocks_converge_to_minimiser(seed):
    """Tiny problems (N = 4, L = 8; J = 2, and J = 3, which does not divide L): the block
    iteration reaches the exact minimiser of Eq. 6 (coordinate-descent oracle) to 1e-6."""
    rng = np.random.default_rng(seed)
    geom = synth.make_geometry(rng, 4, 8, 250.0, 100.0)
    A = oracle.operator(geom)
    g = rng.normal(size=4) + 1j * rng.normal(size=4)
    lam = 0.5 * float(np.abs(A.conj().T @ g).max())
    ref = oracle.minimise(A, g, lam)
    for J in (2, 3):
        x, it, st, _ = oracle.rbpg_block(A, g, lam, J, 9, seed, tol=1e-12, max_iter=30000)
        assert np.linalg.norm(x - ref["x"]) <= 1e-6 * max(np.linalg.norm(ref["x"]), 1e-30), J


@pytest.mark.parametrize("seed", range(3))
def test_blocks_phase_invariance(seed):
    """g -> e^{j phi} g rotates every iterate (the draws do not depend on g); 200 block
    iterations without the stopping test."""
    st = synth.workload_small(P=4, seed=1)
    A = oracle.operator(st.geom)
    phi = 0.3 + seed
    g = st.g[seed % 4].astype(np.complex128)
    a = oracle.rbpg_block(A, g, st.lam, 4, 3, 7, tol=-1.0, max_iter=50)
    b = oracle.rbpg_block(A, np.exp(1j * phi) * g, st.lam, 4, 3, 7, tol=-1.0, max_iter=50)
    assert a[1] == b[1] == 200 and np.array_equal(a[3], b[3])
    np.testing.assert_allclose(b[0], np.exp(1j * phi) * a[0], rtol=0, atol=1e-9 * max(np.abs(a[0]).max(), 1e-30))


# ------------------------------------------------------------------ stored answers

def _read_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "small_minimiser.txt")
    lam, rows = None, []
    for line in open(path):
        if line.startswith("# lambda"):
            lam = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return lam, rows


def test_oracle_reproduces_stored_minimiser():
    """tests/golden/small_minimiser.txt (written by make_golden.py from this oracle): the
    oracle must keep producing the same supports and values (to 1e-12 relative)."""
    lam, rows = _read_golden()
    st = synth.workload_small(P=8, seed=1)
    assert lam == st.lam
    A = oracle.operator(st.geom)
    r = oracle.minimise_batch(A, st.g, st.lam)
    want = np.zeros((8, st.geom.L), np.complex128)
    for row in rows:
        if row[1] != "zero":
            want[int(row[0]), int(row[1])] = float(row[2]) + 1j * float(row[3])
    assert np.array_equal(r["x"] != 0, want != 0)
    np.testing.assert_allclose(r["x"], want, rtol=0, atol=1e-12 * np.abs(want).max())


def _torch_bf16(a):
    """bfloat16 rounding by torch's own conversion (binary32 first), as float64."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(torch.float32)
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_rounding_matches_torch():
    """The oracle's bfloat16 rounding against torch's conversion on random values, on exact
    ties (low 16 bits 0x8000: ties to even) and on bfloat16 values themselves."""
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [0.0, -0.0, 1.0, -3.5, 1e-30, 3e30]])
    bits = rng.integers(0, 1 << 16, 200).astype(np.uint32) << 16
    ties = (bits | 0x8000).view(np.float32).astype(np.float64)
    exact = bits.view(np.float32).astype(np.float64)
    for arr, dist in ((v, None), (ties, 0.0), (exact, 0.5)):
        arr = arr[np.isfinite(arr)]
        ref = _torch_bf16(arr)
        for a, r in zip(arr, ref):
            got, d = oracle.bf16_round(float(a))
            assert got == r, (a, got, r)
            if dist is not None:
                assert d == dist, (a, d)


def test_bf16_operand_first_iteration_closed_form():
    """Algorithm 1 with BF16 operands at k = 1 (x = 0, y = 0, r = -g): x^1 is the soft
    threshold of -2 alpha Ab^H bf16(-g) at alpha lambda (alpha after the step cuts of that
    iteration), or 0 if the step was rejected, with the rounding taken by torch."""
    st = synth.workload_small(P=24, seed=2)
    A = oracle.operator(st.geom)
    Ab = _torch_bf16(A.real) + 1j * _torch_bf16(A.imag)
    for p in range(st.g.shape[0]):
        g = st.g[p].astype(np.complex128)
        r = oracle.rbpg(A, g, st.lam, max_iter=1, tol=0.0, trace=True, bf16_operands=True)
        alpha = r["alpha"][0]
        gb = _torch_bf16(-g.real) + 1j * _torch_bf16(-g.imag)
        ref = oracle.soft(-2.0 * alpha * (Ab.conj().T @ gb), alpha * st.lam)
        if not r["accepted"][0]:
            ref = np.zeros_like(ref)
        np.testing.assert_allclose(r["x"], ref, atol=1e-12 * max(1.0, np.abs(ref).max()))
        # and it differs from the FP64-operand iteration by the BF16 rounding only
        r64 = oracle.rbpg(A, g, st.lam, max_iter=1, tol=0.0)
        assert np.linalg.norm(r["x"] - r64["x"]) <= 2e-2 * max(np.linalg.norm(r64["x"]), 1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_working_set_minimiser_from_zero(seed):
    """The working-set minimiser from x = 0 (the path for large grids) against brute-force
    supports on tiny problems and against coordinate descent on the small workload."""
    rng = np.random.default_rng(700 + seed)
    N = int(rng.integers(3, 5))
    L = 8
    b = rng.uniform(-250, 250, N)
    A = oracle.operator(_geom(b, -40.0, 40.0, L))
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    lam = rng.uniform(0.3, 0.6) * np.max(np.abs(2 * A.conj().T @ g))
    xb, Fb = bruteforce_min(A, g, lam)
    r = oracle.minimise_ws(A, g, lam)
    assert r["flags"] == 0 and np.isfinite(Fb)
    np.testing.assert_allclose(r["x"], xb, atol=1e-9 * max(1.0, np.abs(xb).max()))
    st = synth.workload_small(P=4, seed=10 + seed)
    A = oracle.operator(st.geom)
    for p in range(4):
        a = oracle.minimise(A, st.g[p], st.lam)
        w = oracle.minimise_ws(A, st.g[p], st.lam)
        assert w["flags"] == 0
        np.testing.assert_allclose(w["x"], a["x"], atol=1e-9 * max(1.0, np.abs(a["x"]).max()))
