"""Pins of the SL1MMER model-selection oracle (oracle/select.py), CPU only.

Each pin checks the oracle against something fixed independently of it: exact
recovery of noise-free on-grid scatterers (Eq. 5 steering vectors, least squares
exact), the closed form of the criterion at K = 0 and of the one-scatterer least
squares amplitude (a^H g / N, since |a_n| = 1), the modulus-weighted centroid of a
hand-built cluster, the energy ranking, nested least squares (residual orthogonal to
the fitted columns, RSS non-increasing in K), invariances of the model (global phase,
scale) and the two penalty extremes.  The last test plants mistakes in a copy of the
module and checks that some pin catches each one."""
import math
import types

import numpy as np
import pytest

from oracle import select as osel


def _geom(seed=0, N=29, L=201):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, N)
    b = (u - u.min()) / (u.max() - u.min()) * 269.5 - 134.75
    xi = 2.0 * b / (0.031 * 7.0e5)
    s = -100.0 + np.arange(L) * (200.0 / (L - 1))
    return xi, s


def _a(xi, s):
    return np.exp(-2j * np.pi * xi * s)


def pin_single_on_grid(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 10)
    l0 = int(rng.integers(20, 180))
    gam = complex(rng.normal(), rng.normal()) + 1.0
    g = gam * _a(xi, s[l0])
    x = np.zeros(s.size, np.complex128)
    x[l0] = gam * 0.9  # any nonzero value: the single-atom support of the minimiser
    r = sel.select(g, x, xi, s)
    assert r["khat"] == 1
    assert abs(r["s_hat"][0] - s[l0]) <= 1e-12 * 100
    assert abs(r["gamma_hat"][0] - gam) <= 1e-12 * abs(gam)


def pin_two_on_grid(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 20)
    l1 = int(rng.integers(10, 90))
    l2 = int(rng.integers(110, 190))
    g1, g2 = complex(*rng.normal(size=2)), complex(*rng.normal(size=2))
    g = g1 * _a(xi, s[l1]) + g2 * _a(xi, s[l2])
    x = np.zeros(s.size, np.complex128)
    x[l1], x[l2] = 1.0, 2.0
    r = sel.select(g, x, xi, s)
    assert r["khat"] == 2
    assert np.allclose(r["s_hat"], [s[l1], s[l2]], rtol=0, atol=1e-10)
    assert np.allclose(r["gamma_hat"], [g1, g2], rtol=0, atol=1e-9)


def pin_zero_and_k0_closed_form(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 30)
    g = rng.normal(size=xi.size) + 1j * rng.normal(size=xi.size)
    r = sel.select(g, np.zeros(s.size, np.complex128), xi, s)
    assert r["khat"] == 0 and r["s_hat"].size == 0
    assert abs(r["crit"][0] - 2 * xi.size * math.log(float(np.sum(np.abs(g) ** 2)))) <= 1e-9
    # g = 0: every residual is 0 and every criterion -inf; ties go to the smaller model
    x = np.zeros(s.size, np.complex128)
    x[40], x[140] = 1.0, 1.0
    r = sel.select(np.zeros(xi.size, np.complex128), x, xi, s)
    assert r["khat"] == 0 and np.all(np.isneginf(r["crit"]))


def pin_centroid_modulus_weighted(sel, seed=0):
    xi, s = _geom(seed)
    x = np.zeros(s.size, np.complex128)
    x[50] = 1.0j          # |x| = 1
    x[51] = 3.0           # |x| = 3
    x[120] = 0.5 - 0.5j   # a second, weaker run
    x[122] = 0.1          # one zero bin apart: a run of its own
    cl = sel.clusters(x, s)
    assert [(c[0], c[1]) for c in cl] == [(50, 51), (120, 120), (122, 122)]
    assert abs(cl[0][2] - (s[50] + 0.75 * (s[51] - s[50]))) <= 1e-12
    assert abs(cl[0][3] - 10.0) <= 1e-12 and abs(cl[1][3] - 0.5) <= 1e-12


def pin_rank_and_kmax(sel, seed=0):
    xi, s = _geom(seed)
    x = np.zeros(s.size, np.complex128)
    x[10] = 1.0          # energy 1
    x[60] = 3.0          # energy 9
    x[130] = 2.0         # energy 4
    x[131] = 0.0
    cl = sel.clusters(x, s)
    assert [c[0] for c in cl] == [60, 130, 10]
    g = _a(xi, s[60]) + _a(xi, s[130]) + _a(xi, s[10])
    r = sel.select(g, x, xi, s, kmax=2)
    assert np.allclose(r["centroids"], [s[60], s[130]])
    assert r["crit"].size == 3


def pin_one_scatterer_amplitude(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 40)
    g = rng.normal(size=xi.size) + 1j * rng.normal(size=xi.size)
    x = np.zeros(s.size, np.complex128)
    x[77] = 1.0
    r = sel.select(g, x, xi, s, penalty=1e-9)
    a = _a(xi, s[77])
    assert abs(r["fits"][1][0] - np.vdot(a, g) / xi.size) <= 1e-12 * abs(np.vdot(a, g))


def pin_nested_least_squares(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 50)
    g = rng.normal(size=xi.size) + 1j * rng.normal(size=xi.size)
    x = np.zeros(s.size, np.complex128)
    for l, v in ((30, 2.0), (31, 1.0), (90, 1.5), (150, 0.7), (170, 0.3)):
        x[l] = v
    r = sel.select(g, x, xi, s)
    assert np.all(np.diff(r["rss"]) <= 1e-12 * r["rss"][0])
    for K in range(1, r["rss"].size):
        A = np.exp(-2j * np.pi * np.outer(xi, r["centroids"][:K]))
        res = g - A @ r["fits"][K]
        assert np.max(np.abs(A.conj().T @ res)) <= 1e-9 * np.linalg.norm(g) * math.sqrt(xi.size)
        assert abs(float(np.vdot(res, res).real) - r["rss"][K]) <= 1e-12 * r["rss"][0]


def pin_invariances(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 60)
    g = 1.3 * _a(xi, -10.3) + 0.8 * _a(xi, 12.6) + 0.2 * (rng.normal(size=xi.size) + 1j * rng.normal(size=xi.size))
    x = np.zeros(s.size, np.complex128)
    x[89], x[90], x[112], x[113] = 0.4, 0.9, 0.6, 0.2
    r0 = sel.select(g, x, xi, s)
    c = 2.5 * np.exp(0.7j)
    r1 = sel.select(c * g, c * x, xi, s)
    assert r1["khat"] == r0["khat"]
    assert np.allclose(r1["s_hat"], r0["s_hat"], rtol=0, atol=1e-12)
    assert np.allclose(r1["gamma_hat"], c * r0["gamma_hat"], rtol=1e-10, atol=1e-12)
    assert np.allclose(r1["crit"] - r0["crit"], 2 * xi.size * math.log(abs(c) ** 2), rtol=0, atol=1e-8)


def pin_penalty_extremes(sel, seed=0):
    xi, s = _geom(seed)
    rng = np.random.default_rng(seed + 70)
    g = rng.normal(size=xi.size) + 1j * rng.normal(size=xi.size)
    x = np.zeros(s.size, np.complex128)
    x[20], x[80], x[160] = 1.0, 1.0, 1.0
    assert sel.select(g, x, xi, s, penalty=1e-12)["khat"] == 3
    assert sel.select(g, x, xi, s, penalty=1e6)["khat"] == 0
    assert abs(sel.default_penalty(xi.size) - 3.0 * math.log(2 * xi.size)) < 1e-15


def pin_detection_rule(sel, seed=0):
    st = [-5.0, 5.0]
    assert sel.detected(2, [4.9, -4.1], st)
    assert not sel.detected(2, [0.1, 5.0], st)       # one estimate at the midpoint
    assert not sel.detected(1, [-5.0], st)
    assert not sel.detected(3, [-5.0, 5.0, 9.0], st)


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_select_pins(pin, seed):
    pin(osel, seed)


MUTANTS = {
    "centroid_energy_weight": ("sws += w * float(s_grid[l])", "sws += w * w * float(s_grid[l])"),
    "rank_ascending": ("out.sort(key=lambda c: (-c[3], c[0]))", "out.sort(key=lambda c: (c[3], c[0]))"),
    "steering_sign": ("np.exp(-2j * np.pi * np.outer(", "np.exp(2j * np.pi * np.outer("),
    "penalty_factor": ("return 3.0 * math.log(2.0 * N)", "return 2.0 * math.log(2.0 * N)"),
    "loglik_factor": ("crit = 2.0 * N * np.log(rss)", "crit = N * np.log(rss)"),
    "normal_eq_no_conj": ("np.linalg.solve(AK.conj().T @ AK, AK.conj().T @ g)",
                          "np.linalg.solve(AK.T @ AK, AK.T @ g)"),
    "adjacency_gap": ("nz[j + 1] == nz[j] + 1", "nz[j + 1] <= nz[j] + 2"),
    "detect_full_sep": ("half = 0.5 * (st[1] - st[0])", "half = (st[1] - st[0])"),
    "last_minimum": ("khat = int(np.argmin(crit))", "khat = int(crit.size - 1 - np.argmin(crit[::-1]))"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_select_mutant_caught(name):
    old, new = MUTANTS[name]
    src = open(osel.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"select_{name}")
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    caught = []
    for pin in PINS:
        for seed in range(3):
            try:
                pin(mod, seed)
            except (AssertionError, np.linalg.LinAlgError, ValueError, IndexError):
                caught.append(pin.__name__)
                break
    assert caught, f"no pin catches the planted mistake {name}"
