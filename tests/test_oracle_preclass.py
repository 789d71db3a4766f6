"""Pins of the oracle's pre-classification (oracle/preclass.py), CPU only.

What fixes each part independently of the code under test:
  class 0      the zero solution of Eq. 6: x* = 0 iff 2 ||A^H g||_inf <= lambda, checked
               against the exact minimiser (coordinate descent + Newton + certificate);
  s^, gamma^   a noise-free scatterer at an off-grid elevation s0 with amplitude gamma0
               gives s^ = s0 and gamma^ = gamma0 (the beam peak of one steering vector is at
               its own elevation, and a(s0)^H a(s0) = N), a zero residual and class 1;
  the search   s^ maximises |a(s)^H g| against a dense scan of its bracket;
  class 2      two equal scatterers one resolution cell apart are not one scatterer;
  invariances  a common phase rotates gamma^ only; (g, lambda) -> (c g, |c| lambda) scales it.
Planted mistakes in a copy of the module must each fail one pin."""
import math
import types

import numpy as np
import pytest

import oracle
from oracle import preclass as opc
from paper_1805_01759_gb300 import synth


def _setup(seed):
    rng = np.random.default_rng(500 + seed)
    geom = synth.make_geometry(rng, 25, 200, 250.0, 100.0)
    A = oracle.operator(geom)
    xi = oracle.xi(geom.baselines_m, geom.wavelength_m, geom.range_m)
    s = oracle.grid(geom.s_min_m, geom.s_max_m, geom.L)
    return rng, geom, A, xi, s


def pin_zero_class_is_the_zero_solution(pc, seed=0):
    rng, geom, A, xi, s = _setup(seed)
    for _ in range(6):
        g = 0.3 * (rng.standard_normal(25) + 1j * rng.standard_normal(25))
        lam0 = 2.0 * np.max(np.abs(A.conj().T @ g))
        for lam in (0.97 * lam0, 1.03 * lam0):
            c = pc.classify(A, xi, s, g, lam)
            x = oracle.minimise(A, g, lam)["x"]
            assert (c["cls"] == 0) == bool(np.all(x == 0)), (lam / lam0, c["cls"])
            if c["cls"] == 0:
                assert c["khat"] == 0


def pin_noise_free_scatterer(pc, seed=0):
    rng, geom, A, xi, s = _setup(seed)
    for _ in range(4):
        s0 = rng.uniform(-80.0, 80.0)
        gam0 = rng.uniform(0.5, 2.0) * np.exp(1j * rng.uniform(0, 2 * np.pi))
        g = gam0 * np.exp(-2j * np.pi * xi * s0)
        c = pc.classify(A, xi, s, g, 1.0)
        assert c["cls"] == 1 and c["khat"] == 1, c
        assert abs(c["s_hat"] - s0) < 1e-6, (c["s_hat"], s0)
        assert abs(c["gamma_hat"] - gam0) < 1e-8 * abs(gam0)
        assert c["rmax"] < 1e-4  # the flat peak limits a derivative-free search to ~1e-7 m


def pin_search_finds_the_bracket_maximum(pc, seed=0):
    rng, geom, A, xi, s = _setup(seed)
    for _ in range(4):
        g = (np.exp(-2j * np.pi * xi * rng.uniform(-80, 80))
             + 0.2 * (rng.standard_normal(25) + 1j * rng.standard_normal(25)))
        l_hat = int(np.argmax(np.abs(A.conj().T @ g)))
        lo, hi = s[max(l_hat - 1, 0)], s[min(l_hat + 1, s.size - 1)]
        sh = pc.refine_peak(xi, g, lo, hi)
        ts = np.linspace(lo, hi, 20001)
        best = ts[np.argmax(np.abs(np.exp(2j * np.pi * np.outer(ts, xi)) @ g))]
        assert abs(sh - best) < 2e-3, (sh, best)
        # and classify reports that elevation with the least-squares amplitude
        c = pc.classify(A, xi, s, g, 2.0 * 1.05 * np.max(np.abs(A.conj().T @ (g - np.vdot(
            np.exp(-2j * np.pi * xi * sh), g) / 25 * np.exp(-2j * np.pi * xi * sh)))))
        assert c["cls"] == 1 and abs(c["s_hat"] - sh) < 1e-12
        a = np.exp(-2j * np.pi * xi * sh)
        assert abs(c["gamma_hat"] - np.vdot(a, g) / 25) < 1e-12 * abs(c["gamma_hat"])


def pin_two_scatterers_need_l1(pc, seed=0):
    rng, geom, A, xi, s = _setup(seed)
    rho = synth.rayleigh_resolution(geom)
    for _ in range(4):
        c0 = rng.uniform(-50, 50)
        g = np.exp(-2j * np.pi * xi * (c0 - 0.6 * rho)) + np.exp(-2j * np.pi * xi * (c0 + 0.6 * rho) + 1j)
        lam = synth.default_lambda(25, 200)
        assert pc.classify(A, xi, s, g, lam)["cls"] == 2


def pin_phase_and_scale(pc, seed=0):
    rng, geom, A, xi, s = _setup(seed)
    lam = synth.default_lambda(25, 200)
    g = (np.exp(-2j * np.pi * xi * rng.uniform(-80, 80))
         + 0.05 * (rng.standard_normal(25) + 1j * rng.standard_normal(25)))
    c = pc.classify(A, xi, s, g, lam)
    assert c["cls"] == 1
    ph = np.exp(0.7j)
    c2 = pc.classify(A, xi, s, ph * g, lam)
    # the search resolves the flat peak to ~1e-7 m (a relative change of |a^H g|^2 near 1e-16)
    assert c2["cls"] == 1 and abs(c2["s_hat"] - c["s_hat"]) < 2e-6
    assert abs(c2["gamma_hat"] - ph * c["gamma_hat"]) < 1e-6 * abs(c["gamma_hat"])
    c3 = pc.classify(A, xi, s, 3.0 * g, 3.0 * lam)
    assert c3["cls"] == 1 and abs(c3["gamma_hat"] - 3.0 * c["gamma_hat"]) < 3e-6 * abs(c["gamma_hat"])


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
@pytest.mark.parametrize("seed", [0, 1])
def test_preclass_pins(pin, seed):
    pin(opc, seed)


MUTANTS = {
    "steering_sign": ("return np.exp(-2j * np.pi * xi * s)", "return np.exp(2j * np.pi * xi * s)"),
    "zero_factor": ("umax = 2.0 * np.max(np.abs(u)) / lam", "umax = np.max(np.abs(u)) / lam"),
    "gamma_norm": ("gamma = np.vdot(a, g) / N", "gamma = np.vdot(a, g)"),
    "residual_sign": ("r = g - gamma * a", "r = g + gamma * a"),
    "bracket_one_side": ("hi = s_grid[min(l_hat + 1, L - 1)]", "hi = s_grid[l_hat]"),
    "golden_keeps_wrong_half": ("if fc >= fd:", "if fc < fd:"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_preclass_mutant_caught(name):
    old, new = MUTANTS[name]
    src = open(opc.__file__).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"preclass_{name}")
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    caught = []
    for pin in PINS:
        for seed in range(2):
            try:
                pin(mod, seed)
            except (AssertionError, ValueError, IndexError):
                caught.append(pin.__name__)
                break
        if caught:
            break
    assert caught, f"no pin catches the planted mistake {name}"
