"""FP64 CPU oracle for batched complex BPDN (Eq. 6) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may
import this package.  It shares no code with the CUDA implementation in
``paper_1805_01759_gb300``: the C file ``bpdn_oracle.c`` is compiled on its own
(gcc, FP64, OpenMP over pixels) and loaded with ctypes.

Functions and what they follow:
  grid, xi, operator      Eq. 5 and the definitions after Eq. 2
  operator_md             Eq. 4's multi-component operator (elevation x motion grids)
  gram_toeplitz, aah      A^H A and A A^H of the Eq. 5 operator
  lipschitz               the step constant of Eq. 14's remark, read as 2*lambda_max(A^H A)
  soft                    Eq. 10 read for complex values (complex soft threshold)
  rbpg / rbpg_batch       Algorithm 1 with Eqs. 11-15 (the readings are listed in the C file);
                          optionally with the gradient's operands rounded to bfloat16
  bf16_round              rounding to bfloat16 (binary32 first, ties to even), from its definition
  rbpg_block(_batch)      Algorithm 1 with randomized blocks of one pixel's grid (Eqs. 13-14);
  block_probabilities     Eq. 14's P_j from the block Lipschitz constants;
  splitmix64              the counter-based generator of the block draws
  minimise(_batch)        the exact minimiser of Eq. 6 (coordinate descent + Newton + certificate;
                          a working-set loop from 0 for grids beyond 4096 points: minimise_ws)
  newton_polish           Newton on the smooth optimality system of Eq. 6 on a given support
  kkt, objective          optimality certificate and F of Eq. 6
  select (module)         SL1MMER steps (2)-(3) of Sec. III-A: scatterer candidates from the
                          minimiser's runs, BIC model order, least-squares elevations and
                          amplitudes, and the detection rule of the detection-rate experiment
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpdn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NOT_CONVERGED = 1
STATUS_BT_LIMIT = 2
STATUS_NONFINITE = 4
STATUS_ZERO_SOLUTION = 32


def build(force: bool = False) -> str:
    """Compile bpdn_oracle.c into oracle/_build/liboracle.so (gcc -O3, ISO C11: no FP contraction,
    the same results on x86-64 and aarch64; OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
        return _lib


def _configure(lib):
    """Declare the C signatures on a loaded liboracle."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lp = ctypes.POINTER(ctypes.c_long)
    c_int, c_double, c_long, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_int64
    lib.orc_grid.argtypes = [c_double, c_double, c_int, dp]
    lib.orc_xi.argtypes = [dp, c_int, c_double, c_double, dp]
    lib.orc_operator.argtypes = [dp, c_int, c_double, c_double, c_double, c_double, c_int, dp]
    lib.orc_gram_toeplitz.argtypes = [dp, c_int, c_double, c_int, dp]
    lib.orc_aah.argtypes = [dp, c_int, c_int, dp]
    lib.orc_soft_vec.argtypes = [dp, c_int, c_double, dp]
    lib.orc_objective.argtypes = [dp, c_int, c_int, dp, c_double, dp]
    lib.orc_objective.restype = c_double
    lib.orc_rbpg.argtypes = [dp, c_int, c_int, dp, c_double, c_double, c_double, c_double,
                             c_int, c_int, c_int, dp, ip, dp, ip, ip, dp, dp, dp]
    lib.orc_bf16_round.argtypes = [c_double, dp]
    lib.orc_bf16_round.restype = c_double
    lib.orc_rbpg.restype = c_int
    lib.orc_cd.argtypes = [dp, c_int, c_int, dp, c_double, c_double, c_long, dp, lp]
    lib.orc_cd.restype = c_int
    lib.orc_newton_polish.argtypes = [dp, c_int, c_int, dp, c_double, c_int, ip, dp, c_int,
                                      c_double, dp]
    lib.orc_newton_polish.restype = c_int
    lib.orc_kkt.argtypes = [dp, c_int, c_int, dp, c_double, dp, dp, dp, dp, ip]
    lib.orc_min.argtypes = [dp, c_int, c_int, dp, c_double, c_double, c_long, dp, dp, dp, dp,
                            ip, lp]
    lib.orc_min.restype = c_int
    lib.orc_rbpg_batch.argtypes = [dp, c_int, c_int, dp, c_i64, dp, c_double, c_double,
                                   c_double, c_int, c_int, dp, ip, ip]
    lib.orc_min_ws.argtypes = [dp, c_int, c_int, dp, c_double, dp, dp, dp, dp, ip]
    lib.orc_min_ws.restype = c_int
    lib.orc_min_batch.argtypes = [dp, c_int, c_int, dp, c_i64, dp, c_double, c_long, dp, dp,
                                  dp, dp, ip, lp, ip]
    lib.orc_adjoint.argtypes = [dp, c_int, c_int, c_double, dp, dp, dp, dp]
    lib.orc_adjoint.restype = c_int
    lib.orc_adjoint_batch.argtypes = [dp, c_int, c_int, dp, c_i64, dp, dp, dp, dp, ip]
    lib.orc_num_threads.restype = c_int
    u64, u64p = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)
    lib.orc_splitmix64.argtypes = [u64, c_int, u64p]
    lib.orc_rbpg_block.argtypes = [dp, c_int, c_int, dp, c_double, c_double, c_double, c_double,
                                   c_int, c_int, c_int, dp, u64, c_i64, dp, ip, ip]
    lib.orc_rbpg_block.restype = c_int
    lib.orc_rbpg_block_batch.argtypes = [dp, c_int, c_int, dp, c_i64, dp, c_double, c_double,
                                         c_double, c_int, c_int, c_int, dp, u64, dp, ip, ip]
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ------------------------------------------------------------------ operator

def grid(s_min: float, s_max: float, L: int) -> np.ndarray:
    s = np.empty(L, np.float64)
    _load().orc_grid(float(s_min), float(s_max), int(L), _dp(s))
    return s


def xi(baselines_m, wavelength_m: float, range_m: float) -> np.ndarray:
    b = np.ascontiguousarray(baselines_m, np.float64)
    out = np.empty_like(b)
    _load().orc_xi(_dp(b), b.size, float(wavelength_m), float(range_m), _dp(out))
    return out


def operator(geom) -> np.ndarray:
    """A (complex128, N x L): A_nl = exp(-j 2 pi xi_n s_l) (Eq. 5)."""
    b = np.ascontiguousarray(geom.baselines_m, np.float64)
    A = np.empty((b.size, geom.L), np.complex128)
    _load().orc_operator(_dp(b), b.size, float(geom.wavelength_m), float(geom.range_m),
                         float(geom.s_min_m), float(geom.s_max_m), int(geom.L), _dp(A))
    return A


def operator_md(geom) -> np.ndarray:
    """The multi-component operator of Eq. 4 (elevation x motion grids, elevation index
    fastest): A_nl = exp(-j 2 pi (xi_n s_{l_s} + sum_m eta_{m,n} p_{m,l_m})), in numpy FP64."""
    N = geom.baselines_m.size
    x = xi(geom.baselines_m, geom.wavelength_m, geom.range_m)
    cols = [np.outer(x, grid(geom.s_min_m, geom.s_max_m, geom.L))]  # [N, L_s]
    phase = cols[0]
    for m in range(np.asarray(geom.eta).shape[0]):
        pm = np.linspace(geom.p_min[m], geom.p_max[m], int(geom.L_p[m])) if geom.L_p[m] > 1 else np.array([geom.p_min[m]])
        part = np.outer(np.asarray(geom.eta, np.float64)[m], pm)  # [N, L_m]
        phase = (phase[:, None, :] + part[:, :, None]).reshape(N, -1)
    return np.exp(-2j * np.pi * phase)


def gram_toeplitz(geom) -> np.ndarray:
    """h[d + L - 1] = sum_n exp(j 2 pi xi_n d ds), so (A^H A)_{lm} = h(l - m)."""
    x = xi(geom.baselines_m, geom.wavelength_m, geom.range_m)
    L = geom.L
    ds = (geom.s_max_m - geom.s_min_m) / (L - 1) if L > 1 else 0.0
    h = np.empty(2 * L - 1, np.complex128)
    _load().orc_gram_toeplitz(_dp(x), x.size, float(ds), int(L), _dp(h))
    return h


def aah(A: np.ndarray) -> np.ndarray:
    A = _c128(A)
    N, L = A.shape
    M = np.empty((N, N), np.complex128)
    _load().orc_aah(_dp(A), N, L, _dp(M))
    return M


def lipschitz(A: np.ndarray) -> float:
    """L_f = 2 lambda_max(A^H A) = 2 lambda_max(A A^H), via LAPACK's Hermitian eigensolver."""
    return 2.0 * float(np.linalg.eigvalsh(aah(A)).max())


# ---------------------------------------------------------------- primitives

def soft(v, tau: float) -> np.ndarray:
    v = _c128(np.atleast_1d(v))
    out = np.empty_like(v)
    _load().orc_soft_vec(_dp(v), v.size, float(tau), _dp(out))
    return out


def objective(A, g, lam: float, x) -> float:
    A, g, x = _c128(A), _c128(g), _c128(x)
    N, L = A.shape
    return float(_load().orc_objective(_dp(A), N, L, _dp(g), float(lam), _dp(x)))


def default_alpha0(A: np.ndarray) -> float:
    """alpha_0 = 1 / (2 max_l ||a_l||^2): the largest step Eq. 15 can accept for any A
    with these column norms (equals 1/L_f when the columns are orthogonal)."""
    return 1.0 / (2.0 * float(np.max(np.sum(np.abs(A) ** 2, axis=0))))


def rbpg(A, g, lam: float, *, alpha0: float | None = None, c_alpha: float = 0.5,
         tol: float = 1e-6, max_iter: int = 500, max_bt: int = 64, trace: bool = False,
         bf16_operands: bool = False):
    """Algorithm 1 for one pixel in FP64.  Returns dict(x, iters, status[, trace arrays]).
    bf16_operands: the gradient's operands A and A y - g rounded to bfloat16 first."""
    A, g = _c128(A), _c128(g)
    N, L = A.shape
    a0 = default_alpha0(A) if alpha0 is None else float(alpha0)
    x = np.empty(L, np.complex128)
    it = np.zeros(1, np.int32)
    T = max(int(max_iter), 1)
    ta, tacc, tn, tF, tm, ts = (np.zeros(T), np.zeros(T, np.int32), np.zeros(T, np.int32),
                                np.zeros(T), np.zeros(T), np.zeros(T))
    st = _load().orc_rbpg(_dp(A), N, L, _dp(g), float(lam), a0, float(c_alpha), float(tol),
                          int(max_iter), int(max_bt), 1 if bf16_operands else 0, _dp(x), _ip(it), _dp(ta), _ip(tacc),
                          _ip(tn), _dp(tF), _dp(tm), _dp(ts))
    out = {"x": x, "iters": int(it[0]), "status": int(st)}
    if trace:
        k = int(it[0])
        out.update(alpha=ta[:k].copy(), accepted=tacc[:k].astype(bool), n_bt=tn[:k].copy(),
                   F=tF[:k].copy(), margin=tm[:k].copy(), step=ts[:k].copy())
    return out


def bf16_round(v: float) -> tuple[float, float]:
    """v rounded to bfloat16 (through binary32, ties to even) and its distance from the
    nearest rounding boundary in bfloat16 steps."""
    d = np.zeros(1)
    r = _load().orc_bf16_round(float(v), _dp(d))
    return float(r), float(d[0])


def rbpg_batch(A, G, lam, *, alpha0: float | None = None, c_alpha: float = 0.5,
               tol: float = 1e-6, max_iter: int = 500, max_bt: int = 64):
    """Algorithm 1 for every row of G (P x N).  lam: scalar or [P]."""
    A, G = _c128(A), _c128(G)
    N, L = A.shape
    P = G.shape[0]
    lam_v = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (P,)))
    a0 = default_alpha0(A) if alpha0 is None else float(alpha0)
    x = np.empty((P, L), np.complex128)
    iters = np.zeros(P, np.int32)
    status = np.zeros(P, np.int32)
    _load().orc_rbpg_batch(_dp(A), N, L, _dp(G), P, _dp(lam_v), a0, float(c_alpha), float(tol),
                           int(max_iter), int(max_bt), _dp(x), _ip(iters), _ip(status))
    return {"x": x, "iters": iters, "status": status}


# ------------------------------------------------- randomized blocks (Eqs. 13-14)

def splitmix64(state: int, n: int) -> np.ndarray:
    """n outputs of SplitMix64 from the given state (the generator the block draws use)."""
    out = np.zeros(n, np.uint64)
    _load().orc_splitmix64(ctypes.c_uint64(state & 0xFFFFFFFFFFFFFFFF), int(n),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def block_bounds(L: int, J: int):
    """[lo_j, hi_j) of the J contiguous blocks of an L-point grid."""
    lo = np.array([(j * L) // J for j in range(J)])
    hi = np.array([((j + 1) * L) // J for j in range(J)])
    return lo, hi


def block_probabilities(A, J: int):
    """Eq. 14: P_j = L_j / sum L_j with L_j = 2 lambda_max(A_j^H A_j), the Lipschitz constant of
    the block gradient (lambda_max taken from the N x N matrix A_j A_j^H).  Returns (P, cum)
    with the last cumulative entry exactly 1."""
    A = _c128(A)
    lo, hi = block_bounds(A.shape[1], J)
    Lj = np.array([2.0 * np.linalg.eigvalsh(A[:, a:b] @ A[:, a:b].conj().T)[-1] for a, b in zip(lo, hi)])
    P = Lj / Lj.sum()
    cum = np.cumsum(P)
    cum[-1] = 1.0
    return P, cum


def rbpg_block(A, g, lam: float, J: int, seed: int, pixel: int = 0, *, alpha0: float | None = None,
               c_alpha: float = 0.5, tol: float = 1e-6, max_iter: int = 500, max_bt: int = 64):
    """Algorithm 1 with J randomized blocks of the grid (orc_rbpg_block).  Returns
    (x, block iterations, status, drawn blocks)."""
    A, g = _c128(A), _c128(g)
    N, L = A.shape
    _, cum = block_probabilities(A, J)
    a0 = default_alpha0(A) if alpha0 is None else float(alpha0)
    x = np.zeros(L, np.complex128)
    it = np.zeros(1, np.int32)
    trace = np.full(max_iter * J, -1, np.int32)
    st = _load().orc_rbpg_block(_dp(A), N, L, _dp(g), float(lam), a0, float(c_alpha), float(tol),
                                int(max_iter), int(max_bt), int(J), _dp(np.ascontiguousarray(cum)),
                                ctypes.c_uint64(seed), int(pixel), _dp(x), _ip(it), _ip(trace))
    return x, int(it[0]), int(st), trace[:int(it[0])]


def rbpg_block_batch(A, G, lam, J: int, seed: int, *, alpha0: float | None = None, c_alpha: float = 0.5,
                     tol: float = 1e-6, max_iter: int = 500, max_bt: int = 64):
    """rbpg_block for every row of G; row p draws from the stream of pixel p."""
    A, G = _c128(A), _c128(G)
    N, L = A.shape
    P = G.shape[0]
    _, cum = block_probabilities(A, J)
    lam_v = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (P,)))
    a0 = default_alpha0(A) if alpha0 is None else float(alpha0)
    x = np.empty((P, L), np.complex128)
    iters = np.zeros(P, np.int32)
    status = np.zeros(P, np.int32)
    _load().orc_rbpg_block_batch(_dp(A), N, L, _dp(G), P, _dp(lam_v), a0, float(c_alpha), float(tol),
                                 int(max_iter), int(max_bt), int(J), _dp(np.ascontiguousarray(cum)),
                                 ctypes.c_uint64(seed), _dp(x), _ip(iters), _ip(status))
    return {"x": x, "iters": iters, "status": status}


# ---------------------------------------------------------- exact minimiser

def cd(A, g, lam: float, *, tol: float = 1e-14, max_sweeps: int = 200000):
    A, g = _c128(A), _c128(g)
    N, L = A.shape
    x = np.empty(L, np.complex128)
    sw = np.zeros(1, np.int64)
    rc = _load().orc_cd(_dp(A), N, L, _dp(g), float(lam), float(tol), int(max_sweeps), _dp(x),
                        _lp(sw))
    return x, int(sw[0]), int(rc)


def newton_polish(A, g, lam: float, support, z0, *, max_it: int = 50, ftol: float = 1e-13):
    """Newton on Phi(z) = 2 A_S^H (A_S z - g) + lambda z/|z| = 0 over the index set S."""
    A, g = _c128(A), _c128(g)
    N, L = A.shape
    S = np.ascontiguousarray(support, np.int32)
    z = _c128(np.array(z0, copy=True))
    res = np.zeros(1)
    rc = _load().orc_newton_polish(_dp(A), N, L, _dp(g), float(lam), S.size, _ip(S), _dp(z),
                                   int(max_it), float(ftol), _dp(res))
    return z, int(rc), float(res[0])


def kkt(A, g, lam: float, x):
    """(on_res, off_max, min_abs_on, nS) of the optimality certificate of Eq. 6."""
    A, g, x = _c128(A), _c128(g), _c128(x)
    N, L = A.shape
    on, off, mn = np.zeros(1), np.zeros(1), np.zeros(1)
    nS = np.zeros(1, np.int32)
    _load().orc_kkt(_dp(A), N, L, _dp(g), float(lam), _dp(x), _dp(on), _dp(off), _dp(mn), _ip(nS))
    return float(on[0]), float(off[0]), float(mn[0]), int(nS[0])


def minimise(A, g, lam: float, *, cd_tol: float = 1e-14, max_sweeps: int = 200000):
    r = minimise_batch(A, np.asarray(g)[None, :], lam, cd_tol=cd_tol, max_sweeps=max_sweeps)
    return {k: v[0] for k, v in r.items()}


def minimise_ws(A, g, lam: float):
    """The exact minimiser of Eq. 6 by the working-set loop from x = 0 (no full-grid
    coordinate descent; minimise_batch takes this path by itself for grids beyond 4096
    points).  Returns dict(x, on_res, off_max, min_abs_on, nS, flags)."""
    A, g = _c128(A), _c128(g)
    N, L = A.shape
    x = np.empty(L, np.complex128)
    on, off, mn = np.zeros(1), np.zeros(1), np.zeros(1)
    nS = np.zeros(1, np.int32)
    fl = _load().orc_min_ws(_dp(A), N, L, _dp(g), float(lam), _dp(x), _dp(on), _dp(off), _dp(mn), _ip(nS))
    return {"x": x, "on_res": float(on[0]), "off_max": float(off[0]), "min_abs_on": float(mn[0]),
            "nS": int(nS[0]), "flags": int(fl)}


def minimise_batch(A, G, lam, *, cd_tol: float = 1e-14, max_sweeps: int = 200000):
    """Exact minimiser x* of Eq. 6 for every row of G with its certificate.

    Returns dict of arrays: x [P, L], on_res, off_max (max |2 a_l^H r|/lambda off the
    support), margin = 1 - off_max, min_abs_on, nS, sweeps, flags.
    """
    A, G = _c128(A), _c128(G)
    N, L = A.shape
    P = G.shape[0]
    lam_v = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (P,)))
    x = np.empty((P, L), np.complex128)
    on, off, mn = np.zeros(P), np.zeros(P), np.zeros(P)
    nS = np.zeros(P, np.int32)
    sw = np.zeros(P, np.int64)
    fl = np.zeros(P, np.int32)
    _load().orc_min_batch(_dp(A), N, L, _dp(G), P, _dp(lam_v), float(cd_tol), int(max_sweeps),
                          _dp(x), _dp(on), _dp(off), _dp(mn), _ip(nS), _lp(sw), _ip(fl))
    return {"x": x, "on_res": on, "off_max": off, "margin": 1.0 - off, "min_abs_on": mn,
            "nS": nS, "sweeps": sw, "flags": fl}


# ---------------------------------------------------------------- adjoint

def adjoint(A, lam: float, x, dLdx):
    """Derivatives of the minimiser x of Eq. 6 in (g, lambda) for an upstream gradient
    dL/dx = dL/dRe x + j dL/dIm x (one pixel), by implicit differentiation of the
    optimality system on supp(x).  Returns (dL/dg [N] complex, dL/dlambda, flag)."""
    A, x, dLdx = _c128(A), _c128(x), _c128(dLdx)
    N, L = A.shape
    dg = np.zeros(N, np.complex128)
    dl = np.zeros(1)
    rc = _load().orc_adjoint(_dp(A), N, L, float(lam), _dp(x), _dp(dLdx), _dp(dg), _dp(dl))
    return dg, float(dl[0]), int(rc)


def adjoint_batch(A, lam, X, dLdX):
    """adjoint() for every row of X / dLdX (P x L); lam scalar or [P]."""
    A, X, dLdX = _c128(A), _c128(X), _c128(dLdX)
    N, L = A.shape
    P = X.shape[0]
    lam_v = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (P,)))
    dg = np.zeros((P, N), np.complex128)
    dl = np.zeros(P)
    fl = np.zeros(P, np.int32)
    _load().orc_adjoint_batch(_dp(A), N, L, _dp(lam_v), P, _dp(X), _dp(dLdX), _dp(dg), _dp(dl),
                              _ip(fl))
    return {"dLdg": dg, "dLdlam": dl, "flags": fl}
