"""Planted mistakes in the oracle (CPU only): each plausible slip in the C source --
a flipped sign, a dropped factor, a shifted index, a missing conjugate -- must make
at least one of the oracle's pins fail.  The mutant is compiled from a patched copy
of the C file into a temporary library; the oracle under test is left untouched."""
import ctypes
import os
import subprocess

import pytest

import oracle
import tests.test_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bpdn_oracle.c")

MUTANTS = {
    "operator_sign": ("cexp(-2.0 * ORC_PI * I * xi[n] * s[l])", "cexp(2.0 * ORC_PI * I * xi[n] * s[l])"),
    "grid_spacing": ("(double)l * (s_max - s_min) / (double)(L - 1)", "(double)l * (s_max - s_min) / (double)L"),
    "xi_factor": ("xi[n] = 2.0 * b[n] / (wavelength * range);", "xi[n] = b[n] / (wavelength * range);"),
    "soft_half": ("return v * (1.0 - tau / a);", "return v * (1.0 - 0.5 * tau / a);"),
    "grad_factor": ("grad[l] *= 2.0;", "grad[l] *= 1.0;"),
    "adjoint_no_conj": ("acc += conj(A[(size_t)n * L + l]) * r[n];", "acc += A[(size_t)n * L + l] * r[n];"),
    "momentum_index": ("k <= max_iter; ++k) {\n        double beta = (double)(k - 2) / (double)(k + 1);",
                       "k <= max_iter; ++k) {\n        double beta = (double)(k - 1) / (double)(k + 2);"),
    "accept_reversed": ("margin = fmin(margin, am);\n\n        int accepted = (Fb <= Fx);",
                        "margin = fmin(margin, am);\n\n        int accepted = (Fb >= Fx);"),
    "linesearch_factor": ("double rhs = dd / (2.0 * alpha);", "double rhs = dd / alpha;"),
    "cd_threshold": ("cplx nw = orc_soft(vv, 0.5 * lam) / Gll;", "cplx nw = orc_soft(vv, lam) / Gll;"),
    "repair_cd_threshold": ("cplx nw = orc_soft(q[i] + Gii * old, 0.5 * lam) / Gii;",
                            "cplx nw = orc_soft(q[i] + Gii * old, lam) / Gii;"),
    "repair_stale_residual": ("q[j] -= G[(size_t)j * m + i] * dlt;", "q[j] -= G[(size_t)i * m + j] * dlt;"),
    "newton_residual_sign": ("phi[i] = 2.0 * acc + lam * z[i] / cabs(z[i]);", "phi[i] = 2.0 * acc - lam * z[i] / cabs(z[i]);"),
    "kkt_factor": ("cplx zl = 2.0 * z[l];", "cplx zl = z[l];"),
    "adjoint_curvature_sign": ("Jm[(size_t)(2 * i) * n2 + 2 * i] += curv * (1.0 - u0 * u0);",
                               "Jm[(size_t)(2 * i) * n2 + 2 * i] -= curv * (1.0 - u0 * u0);"),
    "adjoint_gram_transposed": ("Gij += conj(A[(size_t)n * L + S[i]]) * A[(size_t)n * L + S[j]];",
                                "Gij += A[(size_t)n * L + S[i]] * conj(A[(size_t)n * L + S[j]]);"),
    "adjoint_dg_factor": ("dLdg[n] = 2.0 * acc;", "dLdg[n] = acc;"),
    "adjoint_lambda_sign": ("*dLdlam = -dl;", "*dLdlam = dl;"),
    "bf16_truncation": ("b += 0x7FFFu + ((b >> 16) & 1u);", "b += 0u;"),
    "bf16_residual_unrounded": ("                r[n] = bf16_c(r[n], &dn);", "                (void)bf16_c(r[n], &dn);"),
    "splitmix_shift": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;"),
    "block_extrapolate_everywhere": ("y[l] = (l >= lo && l < hi) ? x[l] + beta * (x[l] - xp[l]) : x[l];",
                                     "y[l] = x[l] + beta * (x[l] - xp[l]);"),
    "block_stop_first_small": ("? (done_mask | (1u << i)) : 0u;", "? all_mask : 0u;"),
    "block_alpha_wrong_block": ("alpha[i] *= c_alpha;", "alpha[0] *= c_alpha;"),
    "block_bounds_gap": ("const int lo = (int)(((int64_t)i * L) / J)", "const int lo = (int)(((int64_t)i * L + J - 1) / J)"),
    "block_draw_uniform": ("if (u < cum[j])", "if (u < (double)(j + 1) / J)"),
    "block_momentum_index": ("trace[k - 1] = i;\n        double beta = (double)(k - 2) / (double)(k + 1);",
                             "trace[k - 1] = i;\n        double beta = (double)(k - 1) / (double)(k + 2);"),
    "block_accept_reversed": ("l1(xb, L);\n        int accepted = (Fb <= Fx);", "l1(xb, L);\n        int accepted = (Fb >= Fx);"),
}

# the stored-answer test compares the oracle with its own earlier output: a regression
# guard, not a pin, so it does not count as catching a planted mistake; tests that take
# other arguments than a seed (such as the numpy operator's own mutant test) are not pins
def _is_pin(fn) -> bool:
    import inspect
    return set(inspect.signature(fn).parameters) <= {"seed"}


PINS = [getattr(pins, n) for n in dir(pins)
        if n.startswith("test_") and "stored" not in n and "mutant" not in n and _is_pin(getattr(pins, n))]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so),
                    str(path), "-lm"], check=True)
    return oracle._configure(ctypes.CDLL(str(so)))


def _run_pin(fn):
    import inspect
    params = inspect.signature(fn).parameters
    if "seed" in params:
        for seed in range(6):
            fn(seed)
    else:
        fn()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    lib = _build(tmp_path, name, old, new)
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fn in PINS:
        try:
            _run_pin(fn)
        except Exception:  # noqa: BLE001 - any failure of a pin counts
            caught.append(fn.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
