"""Seeded synthetic TomoSAR pixel stacks (inputs only).

This module simulates measurements; it holds none of the solver's arithmetic.
Both the FP64 CPU oracle and the CUDA path take their inputs from here.

Physical model (Sec. II, Eq. 2 with the motion term d = 0, and Eq. 5): a pixel
observed at N baselines b_n returns

    g_n = sum_k gamma_k * exp(-j*2*pi*xi_n*s_k) + eps_n,   xi_n = 2*b_n/(wavelength*range)

for K point scatterers at continuous (off-grid) elevations s_k.  The sign of
the exponent follows the steering-matrix convention A_nl = exp(-j2*pi*xi_n*s_l)
so that a scatterer at s appears at +s on the elevation grid.

Scatterers have unit amplitude and a uniform phase; eps is circular complex
Gaussian noise of total variance sigma^2 = 10^(-SNR/10) per acquisition.
The Rayleigh resolution rho_s = wavelength*range/Delta_b is Eq. 16 and the
normalised separation kappa = s/rho_s is Eq. 17.

The regularisation weight is not given in the paper (it only says lambda is
fixed).  The workloads use lambda = 2*sigma_ref*sqrt(N*ln L) with a 10 dB
reference SNR: the level at which a noise-only pixel returns x = 0 with high
probability.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "StackGeometry",
    "Stack",
    "default_lambda",
    "rayleigh_resolution",
    "make_geometry",
    "make_stack",
    "workload_small",
    "workload_patch",
    "workload_diff",
    "workload_ragged",
    "dft_geometry",
    "elevation_resolution",
    "DetectionSet",
    "workload_detection",
    "MotionGeometry",
    "make_stack_md",
    "workload_motion",
    "workload_motion4d",
]


@dataclasses.dataclass
class StackGeometry:
    """Acquisition geometry of one stack (what bpdn_make_operator takes)."""

    baselines_m: np.ndarray  # float64 [N]
    wavelength_m: float
    range_m: float
    s_min_m: float
    s_max_m: float
    L: int

    @property
    def N(self) -> int:
        return int(self.baselines_m.shape[0])


@dataclasses.dataclass
class Stack:
    """One stack of P pixels sharing a geometry."""

    geom: StackGeometry
    g: np.ndarray  # complex64 [P, N], pixel-major
    lam: float  # regularisation weight lambda (Eq. 6)
    gamma_true: np.ndarray | None = None  # complex64 [P, L], scatterers at their nearest bin
    n_scat: np.ndarray | None = None  # int8 [P]
    snr_db: np.ndarray | None = None  # float32 [P]
    s_true: np.ndarray | None = None  # float64 [P, 2] (nan where absent)
    seed: int = 0


def rayleigh_resolution(geom: StackGeometry) -> float:
    """rho_s = wavelength * range / Delta_b (Eq. 16), Delta_b = aperture extent."""
    b = geom.baselines_m
    return geom.wavelength_m * geom.range_m / float(b.max() - b.min())


def default_lambda(N: int, L: int, snr_ref_db: float = 10.0) -> float:
    """lambda = 2*sigma_ref*sqrt(N ln L) at a reference SNR (the paper fixes no value)."""
    sigma = math.sqrt(10.0 ** (-snr_ref_db / 10.0))
    return 2.0 * sigma * math.sqrt(N * math.log(L))


def make_geometry(rng: np.random.Generator, N: int, L: int, half_aperture_m: float = 250.0,
                  half_height_m: float = 100.0, wavelength_m: float = 0.031,
                  range_m: float = 7.0e5) -> StackGeometry:
    b = rng.uniform(-half_aperture_m, half_aperture_m, N)
    return StackGeometry(np.asarray(b, np.float64), wavelength_m, range_m,
                         -half_height_m, half_height_m, L)


def _phasors(geom: StackGeometry, s: np.ndarray) -> np.ndarray:
    """exp(-j 2 pi xi_n s) for an array of elevations s[...] -> [..., N] (simulation only)."""
    xi = 2.0 * geom.baselines_m / (geom.wavelength_m * geom.range_m)
    return np.exp(-2j * np.pi * s[..., None] * xi)


def make_stack(geom: StackGeometry, P: int, rng: np.random.Generator, *, lam: float,
               snr_db_range: tuple[float, float] = (10.0, 10.0),
               k_probs: tuple[float, float, float] = (0.3, 0.5, 0.2),
               second_at_kappa: tuple[float, float] | None = None,
               seed: int = 0) -> Stack:
    """Simulate P pixels.

    K in {0,1,2} scatterers per pixel with probabilities k_probs.  The first
    scatterer is uniform over the elevation extent.  The second is either
    independent and uniform (second_at_kappa=None) or placed at s1 +/- kappa*rho_s with
    kappa ~ U[second_at_kappa], redrawn until it falls inside the extent.
    """
    N, L = geom.N, geom.L
    lo, hi = geom.s_min_m, geom.s_max_m
    K = rng.choice(3, size=P, p=np.asarray(k_probs))
    snr = rng.uniform(snr_db_range[0], snr_db_range[1], P)
    s1 = rng.uniform(lo, hi, P)
    ph1 = rng.uniform(0.0, 2.0 * np.pi, P)
    ph2 = rng.uniform(0.0, 2.0 * np.pi, P)
    if second_at_kappa is None:
        s2 = rng.uniform(lo, hi, P)
    else:
        rho = rayleigh_resolution(geom)
        s2 = np.full(P, np.nan)
        todo = np.arange(P)
        while todo.size:
            kap = rng.uniform(second_at_kappa[0], second_at_kappa[1], todo.size)
            sign = np.where(rng.uniform(0.0, 1.0, todo.size) < 0.5, -1.0, 1.0)
            cand = s1[todo] + sign * kap * rho
            ok = (cand >= lo) & (cand <= hi)
            s2[todo[ok]] = cand[ok]
            todo = todo[~ok]
    sigma2 = 10.0 ** (-snr / 10.0)
    noise = (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N))) * np.sqrt(sigma2 / 2.0)[:, None]

    g = noise.astype(np.complex128)
    a1 = np.exp(1j * ph1)
    a2 = np.exp(1j * ph2)
    m1 = K >= 1
    m2 = K >= 2
    g[m1] += a1[m1, None] * _phasors(geom, s1[m1])
    g[m2] += a2[m2, None] * _phasors(geom, s2[m2])

    ds = (hi - lo) / (L - 1) if L > 1 else 1.0
    gamma = np.zeros((P, L), np.complex64)
    idx1 = np.clip(np.rint((s1 - lo) / ds), 0, L - 1).astype(np.int64)
    idx2 = np.clip(np.rint((np.nan_to_num(s2) - lo) / ds), 0, L - 1).astype(np.int64)
    rows = np.arange(P)
    gamma[rows[m1], idx1[m1]] += a1[m1].astype(np.complex64)
    gamma[rows[m2], idx2[m2]] += a2[m2].astype(np.complex64)
    s_true = np.stack([np.where(m1, s1, np.nan), np.where(m2, s2, np.nan)], axis=1)
    # lambda is handed to the solver as float32: keep it exactly representable so
    # every consumer (oracle included) sees the same value
    return Stack(geom, np.ascontiguousarray(g.astype(np.complex64)), float(np.float32(lam)), gamma,
                 K.astype(np.int8), snr.astype(np.float32), s_true, seed)


def workload_small(P: int = 256, seed: int = 1) -> Stack:
    """One stack: N=25, b~U[-250,250] m, 0.031 m, 700 km, L=200 on [-100,100] m, 10 dB."""
    rng = np.random.default_rng(seed)
    geom = make_geometry(rng, 25, 200, 250.0, 100.0)
    return make_stack(geom, P, rng, lam=default_lambda(25, 200), snr_db_range=(10.0, 10.0), seed=seed)


def workload_patch(P: int = 1 << 20, seed: int = 2, part: int = 0) -> Stack:
    """Full patch: N=25, L=400 on [-200,200] m, second scatterer at kappa*rho_s with
    kappa~U[0.5,2], per-pixel SNR~U[0,20] dB.  `part` > 0 draws another set of pixels
    of the same stack (same geometry), e.g. one per GPU."""
    rng = np.random.default_rng(seed)
    geom = make_geometry(rng, 25, 400, 250.0, 200.0)
    if part:
        rng = np.random.default_rng([seed, part])
    return make_stack(geom, P, rng, lam=default_lambda(25, 400), snr_db_range=(0.0, 20.0),
                      second_at_kappa=(0.5, 2.0), seed=seed)


def workload_diff(P: int = 1 << 18, seed: int = 5) -> Stack:
    """Differentiation workload: N=25, L=400 on [-200,200] m, same scatterer law as the patch."""
    rng = np.random.default_rng(seed)
    geom = make_geometry(rng, 25, 400, 250.0, 200.0)
    return make_stack(geom, P, rng, lam=default_lambda(25, 400), snr_db_range=(0.0, 20.0),
                      second_at_kappa=(0.5, 2.0), seed=seed)


def workload_ragged(n_stacks: int = 64, seed: int = 3, p_log2: tuple[int, int] = (12, 16),
                    scale_pixels: float = 1.0) -> list[Stack]:
    """Ragged batch: per stack N~U{10..60}, L~U{100..600}, aperture B~U[200,600] m,
    elevation half-width h~U[50,300] m, P=2^U{12..16} (times scale_pixels)."""
    out = []
    for s in range(n_stacks):
        rng = np.random.default_rng(1000 * seed + s)
        N = int(rng.integers(10, 61))
        L = int(rng.integers(100, 601))
        B = float(rng.uniform(200.0, 600.0))
        h = float(rng.uniform(50.0, 300.0))
        P = max(1, int(round((1 << int(rng.integers(p_log2[0], p_log2[1] + 1))) * scale_pixels)))
        geom = make_geometry(rng, N, L, B / 2.0, h)
        out.append(make_stack(geom, P, rng, lam=default_lambda(N, L), snr_db_range=(0.0, 20.0),
                              second_at_kappa=(0.5, 2.0), seed=1000 * seed + s))
    return out


def dft_geometry(N: int, ds: float = 1.0, wavelength_m: float = 0.031,
                 range_m: float = 7.0e5) -> StackGeometry:
    """Geometry whose steering matrix is the N-point DFT (orthogonal columns).

    Grid s_l = l*ds (l = 0..N-1) and xi_n = n/(N*ds), i.e. b_n = xi_n*wavelength*range/2.
    """
    xi = np.arange(N, dtype=np.float64) / (N * ds)
    b = xi * wavelength_m * range_m / 2.0
    return StackGeometry(b, wavelength_m, range_m, 0.0, (N - 1) * ds, N)


def elevation_resolution(geom: StackGeometry) -> float:
    """Inherent elevation resolution 1 / (xi_max - xi_min) = wavelength*range/(2*Delta_b).

    Eq. 16 prints wavelength*range/Delta_b; the paper's own figures (a 269.5 m aperture
    giving 40.5 m at X band) and the two-way phase xi = 2b/(wavelength*range) of Eq. 5
    give half of that, which is what the detection experiment measures kappa against."""
    b = geom.baselines_m
    return geom.wavelength_m * geom.range_m / (2.0 * float(b.max() - b.min()))


@dataclasses.dataclass
class DetectionSet:
    """Two-scatterer pixels of the detection-rate experiment (Sec. IV-A, last figure)."""

    geom: StackGeometry
    g: np.ndarray        # complex64 [P, N]
    lam: np.ndarray      # float32 [P], per pixel (it follows the pixel's noise level)
    kappa: np.ndarray    # float64 [P] normalised separation (Eq. 17, against elevation_resolution)
    snr_db: np.ndarray   # float64 [P] per scatterer
    s_true: np.ndarray   # float64 [P, 2] ascending
    seed: int = 0


def workload_detection(kappas=tuple(np.round(np.arange(0.1, 1.51, 0.1), 2)), snrs_db=(2.0, 7.0),
                       n_per: int = 5000, seed: int = 6, N: int = 29, L: int = 201,
                       aperture_m: float = 269.5, half_height_m: float = 100.0) -> DetectionSet:
    """The detection-rate Monte Carlo: N = 29 acquisitions over a 269.5 m aperture (the
    paper's Las Vegas stack), two unit scatterers with equal phase (Delta phi = 0, the
    worst case) at c -/+ kappa*rho_s/2 with c ~ U[-0.5, 0.5] m (off the 1 m grid), per
    scatterer SNR in snrs_db, n_per realisations per (kappa, SNR).  Grid: L points on
    [-half_height, half_height].  lambda = 2*sigma*sqrt(N ln L) with the pixel's own
    noise sigma (the level of the other workloads, taken at the simulated SNR)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, N)
    b = (u - u.min()) / (u.max() - u.min()) * aperture_m - aperture_m / 2.0
    geom = StackGeometry(np.asarray(b, np.float64), 0.031, 7.0e5, -half_height_m, half_height_m, L)
    rho = elevation_resolution(geom)
    kap = np.repeat(np.tile(np.asarray(kappas, np.float64), len(snrs_db)), n_per)
    snr = np.repeat(np.asarray(snrs_db, np.float64), len(kappas) * n_per)
    P = kap.size
    c = rng.uniform(-0.5, 0.5, P)
    s_true = np.stack([c - 0.5 * kap * rho, c + 0.5 * kap * rho], axis=1)
    ph = rng.uniform(0.0, 2.0 * np.pi, P)
    sigma2 = 10.0 ** (-snr / 10.0)
    noise = (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N))) * np.sqrt(sigma2 / 2.0)[:, None]
    a = np.exp(1j * ph)[:, None]
    g = noise + a * (_phasors(geom, s_true[:, 0]) + _phasors(geom, s_true[:, 1]))
    lam = (2.0 * np.sqrt(sigma2) * math.sqrt(N * math.log(L))).astype(np.float32)
    return DetectionSet(geom, np.ascontiguousarray(g.astype(np.complex64)), lam, kap, snr, s_true, seed)


@dataclasses.dataclass
class MotionGeometry(StackGeometry):
    """A stack observed over time (Eqs. 2-4): besides the elevation grid, M motion
    coefficients p_m on grids of L_p[m] points, with temporal frequencies eta[m, n]
    (for linear motion p = velocity and eta = 2 t_n / wavelength).  L counts elevation
    points; the whole grid has L * prod(L_p) points, elevation index fastest."""

    eta: np.ndarray | None = None    # float64 [M, N]
    p_min: np.ndarray | None = None  # float64 [M]
    p_max: np.ndarray | None = None  # float64 [M]
    L_p: np.ndarray | None = None    # int [M]

    @property
    def L_total(self) -> int:
        return int(self.L * np.prod(self.L_p))

    def motion(self):
        return (self.eta, self.p_min, self.p_max, self.L_p)


def make_stack_md(geom: MotionGeometry, P: int, rng: np.random.Generator, *, lam: float,
                  snr_db_range=(5.0, 20.0), k_probs=(0.3, 0.5, 0.2)) -> Stack:
    """P pixels of K in {0,1,2} unit scatterers, each at an elevation uniform over the grid's
    extent and motion coefficients uniform over the inner 80 % of each motion grid:
    g_n = sum_k gamma_k exp(-j 2 pi (xi_n s_k + sum_m eta[m, n] p_{m,k})) + noise (Eq. 4)."""
    N, M = geom.N, geom.eta.shape[0]
    xi = 2.0 * geom.baselines_m / (geom.wavelength_m * geom.range_m)
    K = rng.choice(3, size=P, p=np.asarray(k_probs))
    snr = rng.uniform(snr_db_range[0], snr_db_range[1], P)
    g = np.zeros((P, N), np.complex128)
    gamma = np.zeros((P, geom.L_total), np.complex64)
    ds = (geom.s_max_m - geom.s_min_m) / (geom.L - 1) if geom.L > 1 else 1.0
    for k in range(2):
        on = K > k
        s = rng.uniform(geom.s_min_m, geom.s_max_m, P)
        ph = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, P))
        phase = np.outer(s, xi)
        idx = np.clip(np.rint((s - geom.s_min_m) / ds), 0, geom.L - 1).astype(np.int64)
        stride = geom.L
        for m in range(M):
            span = geom.p_max[m] - geom.p_min[m]
            pm = rng.uniform(geom.p_min[m] + 0.1 * span, geom.p_max[m] - 0.1 * span, P)
            phase += np.outer(pm, geom.eta[m])
            dp = span / (geom.L_p[m] - 1) if geom.L_p[m] > 1 else 1.0
            im = np.clip(np.rint((pm - geom.p_min[m]) / dp), 0, geom.L_p[m] - 1).astype(np.int64)
            idx = idx + stride * im
            stride *= int(geom.L_p[m])
        g[on] += ph[on, None] * np.exp(-2j * np.pi * phase[on])
        rows = np.flatnonzero(on)
        gamma[rows, idx[on]] += ph[on].astype(np.complex64)
    sigma2 = 10.0 ** (-snr / 10.0)
    g += (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N))) * np.sqrt(sigma2 / 2.0)[:, None]
    return Stack(geom, np.ascontiguousarray(g.astype(np.complex64)), float(np.float32(lam)), gamma,
                 K.astype(np.int8), snr.astype(np.float32), None, 0)


def workload_motion(P: int = 1 << 18, seed: int = 7, L_s: int = 32, L_v: int = 16) -> Stack:
    """Differential tomography with linear deformation: N = 25 acquisitions, baselines
    U[-250, 250] m, times U[0, 4] years (eta = 2 t_n / wavelength per m/yr of velocity),
    elevation grid L_s on [-100, 100] m, velocity grid L_v on [-0.02, 0.02] m/yr, SNR
    U[5, 20] dB; lambda by the rule of the other workloads with the whole grid's size."""
    rng = np.random.default_rng(seed)
    N = 25
    b = rng.uniform(-250.0, 250.0, N)
    t = rng.uniform(0.0, 4.0, N)
    geom = MotionGeometry(np.asarray(b, np.float64), 0.031, 7.0e5, -100.0, 100.0, L_s,
                          eta=(2.0 * t / 0.031)[None, :], p_min=np.array([-0.02]), p_max=np.array([0.02]),
                          L_p=np.array([L_v]))
    return make_stack_md(geom, P, rng, lam=default_lambda(N, geom.L_total))



def workload_motion4d(P: int = 1 << 12, seed: int = 8, L_s: int = 64, L_v: int = 16, L_a: int = 16) -> Stack:
    """The 4-D reading of Eqs. 3-4 (elevation, linear velocity and the amplitude of a
    seasonal motion): N = 25 acquisitions, baselines U[-250, 250] m, times U[0, 4] years,
    elevation grid L_s on [-100, 100] m, velocity grid L_v on [-0.02, 0.02] m/yr, seasonal
    amplitude grid L_a on [-0.01, 0.01] m with the base function sin(2 pi t) (t in years):
    eta_1 = 2 t_n / wavelength, eta_2 = 2 sin(2 pi t_n) / wavelength.  The default grid has
    64 x 16 x 16 = 16,384 points.  SNR U[5, 20] dB; lambda by the rule of the other
    workloads with the whole grid's size."""
    rng = np.random.default_rng(seed)
    N = 25
    b = rng.uniform(-250.0, 250.0, N)
    t = rng.uniform(0.0, 4.0, N)
    eta = np.stack([2.0 * t / 0.031, 2.0 * np.sin(2.0 * np.pi * t) / 0.031])
    geom = MotionGeometry(np.asarray(b, np.float64), 0.031, 7.0e5, -100.0, 100.0, L_s, eta=eta,
                          p_min=np.array([-0.02, -0.01]), p_max=np.array([0.02, 0.01]),
                          L_p=np.array([L_v, L_a]))
    return make_stack_md(geom, P, rng, lam=default_lambda(N, geom.L_total))
