#!/usr/bin/env python3
"""Throughput of the batched BPDN hot path on GB300 (pixels/s at 1e-4 vs the FP64 oracle).

Workload: one stack, N=25 acquisitions (baselines U[-250,250] m), wavelength 0.031 m,
range 700 km, elevation grid L=400 on [-200,200] m, P=2^20 pixels per GPU, K in
{0,1,2} scatterers (second at kappa*rho_s, kappa~U[0.5,2]), SNR~U[0,20] dB, seeded
synthetic data.  One step = the whole hot path over the batch: Algorithm 1 on every
pixel (iteration kernel) followed by the FP64 refit and certificate (refit kernel).
Both paths of the metric are timed -- the plain FP32 contraction and the BF16
tensor-core contraction, each followed by the FP64 refit -- and the BF16 path is
the headline value; pixels count only when certified and the oracle sample agrees.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload ragged       # the 64-stack ragged batch (its own line)
    python bench.py --workload detection    # detection-rate Monte Carlo, solve + model selection
    python bench.py --workload blocks       # randomized-block reading of Eqs. 13-14 vs the default
    python bench.py --workload motion       # elevation x velocity grids (Eq. 4)

Prints one JSON line (rank 0).  Under torchrun each rank solves its own 2^20 pixels
of the same stack (weak scaling, no collective on the data path; a barrier and a
max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pixels/s to 1e-4 rel err vs FP64 oracle: plain FP32 vs BF16+FP64-refit"
UNIT = "pixels/s"
N_ACQ, L_GRID = 25, 400
FP32_LANES_PER_SM = 128


# ------------------------------------------------------------ distributed helpers

def dist_env() -> tuple[int, int, int]:
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_part(rank: int) -> int:
    """Pixel set of a rank: rank 0 takes the base draw, rank r the r-th extra draw."""
    return rank


def reduce_max(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(device=None) -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        sm = [r[0] for r in rows]
        load = [r for r in rows if r[2] > 200.0] or rows
        out["sm_mhz"] = statistics.median(r[0] for r in load)
        out["sm_max_mhz"] = max(r[1] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    seen.add(n)
        out["reasons"] = sorted(seen)
        out["samples"] = len(sm)
        out["power_w_max"] = max(r[2] for r in rows)
        return out


# ---------------------------------------------------------------- reference arm

def run_reference(args) -> None:
    """The FP64 CPU oracle (Algorithm 1 as the paper states it) on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1805_01759_gb300 import synth
    sample = args.ref_sample
    st = synth.workload_patch(P=sample, seed=2)
    A = oracle.operator(st.geom)
    oracle.rbpg_batch(A, st.g[:32], st.lam)  # load + warm the library
    times = []
    for _ in range(max(1, args.warmup)):
        oracle.rbpg_batch(A, st.g[:64], st.lam)
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        oracle.rbpg_batch(A, st.g, st.lam, tol=1e-6, max_iter=500)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    value = sample / t
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"one stack N={N_ACQ}, L={L_GRID} on [-200,200] m; "
                               f"bounded sample of {sample} pixels of the 2^20-pixel patch",
                   "P_sample": sample, "N": N_ACQ, "L": L_GRID},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} pixels of the patch, Algorithm 1 in FP64, "
                                   f"tol 1e-6, max 500 iterations, OpenMP over pixels"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def _kernel_hash(name: str) -> str:
    src = os.path.join(ROOT, "paper_1805_01759_gb300", "csrc", name)
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def _traffic_per_launch(pixels: int, path_name: str) -> float | None:
    """DRAM bytes of one iteration-kernel launch from the committed ncu counters
    (profiles/counters_<path>.txt, taken on a smaller patch), scaled by the pixels the
    launch processes -- the traffic is the per-pixel read of g and write of x -- and
    only while the kernel source is the one the counters were taken on."""
    src = "rbpg.cu"
    path = os.path.join(ROOT, "profiles", f"counters_{path_name}.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            rec[parts[0]] = parts[1]
    if rec.get("kernel_sha256_16") != _kernel_hash(src) or "dram_bytes_per_pixel" not in rec:
        return None
    return float(rec["dram_bytes_per_pixel"]) * pixels


PEAK_KINDS = {0: ("ffma", "TFLOP/s"), 1: ("ffma2", "TFLOP/s"), 2: ("dfma", "TFLOP/s"), 3: ("mufu_rsqrt", "Top/s")}


def measure_peaks(dev, kinds=(0, 1, 2, 3), seconds: float = 0.15, repeats: int = 5) -> dict:
    """Pipe rates of this GPU from the library's microbenchmark loops (bpdn_bench_peak):
    every SM full of threads running independent FMA (or rsqrt) chains, timed with CUDA
    events on the launching stream; the best of `repeats` launches of about `seconds` each."""
    import torch
    from paper_1805_01759_gb300 import _lib
    lib = _lib.load()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * n_sm, 256
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ops = ctypes.c_double()
    out = {}
    for kind in kinds:
        name, unit = PEAK_KINDS[kind]
        iters = 1 << 10
        while True:  # grow the loop until one launch takes about `seconds`
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.check(lib.bpdn_bench_peak(kind, blocks, threads, iters, sink.data_ptr(), ctypes.byref(ops),
                                           stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            if ms >= 1e3 * seconds or iters >= (1 << 30):
                break
            iters *= 2 if ms < 1e3 * seconds / 8 else max(2, int(1e3 * seconds / max(ms, 1e-3)))
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.check(lib.bpdn_bench_peak(kind, blocks, threads, iters, sink.data_ptr(), ctypes.byref(ops),
                                           stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        rate = blocks * threads * float(iters) * ops.value / (best / 1e3) / 1e12
        out[name] = {"value": rate, "unit": unit, "ms": best, "iters": iters, "blocks": blocks, "threads": threads}
    return out


def run_peaks(args) -> None:
    """The arithmetic-pipe peaks of this GPU (FFMA, FFMA2, DFMA, MUFU), with the SM clock
    sampled while they run and the unit-count figures beside them."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    with ClockSampler(dev.index) as clk:
        pk = measure_peaks(dev, seconds=0.3)
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    nominal = {"ffma": n_sm * 128 * 2 * mhz * 1e6 / 1e12, "ffma2": n_sm * 128 * 2 * mhz * 1e6 / 1e12}
    if rank == 0:
        print(json.dumps({"metric": "arithmetic pipe peaks", "value": pk["ffma2"]["value"], "unit": "TFLOP/s",
                          "n_gpus": 1, "workload": "peaks", "peaks": pk,
                          "unit_count_at_sampled_clock": nominal,
                          "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                                     "reasons": clocks.get("reasons"), "power_w_max": clocks.get("power_w_max")}}),
              flush=True)


def cpu_baseline_leg(sample: int) -> dict:
    import oracle
    from paper_1805_01759_gb300 import synth
    st = synth.workload_patch(P=sample, seed=2)
    A = oracle.operator(st.geom)
    oracle.rbpg_batch(A, st.g[:32], st.lam)
    t0 = time.perf_counter()
    oracle.rbpg_batch(A, st.g, st.lam, tol=1e-6, max_iter=500)
    t = time.perf_counter() - t0
    return {"value": sample / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{sample} pixels of the patch: Algorithm 1 in FP64 (tol 1e-6, max 500 "
                      f"iterations), OpenMP over pixels, {t:.1f} s"}


def alu_flops_per_sweep(path: str, N: int, L: int) -> float:
    """Algorithmic FP32 flops of one sweep of Algorithm 1 for one pixel on the CUDA cores
    (an FMA counts 2): per grid point the extrapolation y = x + beta (x - x_prev) (6),
    v = y - 2 alpha grad (4), |v|^2 (3), the prox scale and xbar (4), |xbar| - tau (2),
    ||xbar - y||^2 (5), ||xbar - x||^2 (5), ||xbar||^2 (3) and the four sums over the
    grid (4): 36 L.  The plain FP32 path adds the gradient contraction, 8 N L (one
    complex multiply-add, four real FMAs, per (n, l)).  A xbar over the nonzeros of
    xbar (8 N per nonzero) is left out."""
    flops = 36.0 * L
    if path.startswith("fp32"):
        flops += 8.0 * N * L
    return flops


class OracleSample:
    """The exact minimiser (FP64 oracle) on a seeded sample of a stack's pixels."""

    def __init__(self, st, n_sample: int, seed: int = 20):
        import oracle
        rng = np.random.default_rng(seed)
        P = st.g.shape[0]
        self.idx = np.arange(P) if n_sample >= P else np.sort(rng.choice(P, size=n_sample, replace=False))
        A = oracle.operator(st.geom)
        self.ref = oracle.minimise_batch(A, st.g[self.idx], st.lam)
        ref = self.ref
        # pixels where the oracle's own certificate failed have no reference answer
        self.resolved = ref["flags"] == 0
        self.degen = (ref["margin"] < 1e-6) | ((ref["nS"] > 0) & (ref["min_abs_on"] < 1e-6 * np.abs(ref["x"]).max(1)))

    def errors(self, x) -> tuple[np.ndarray, np.ndarray]:
        """Relative l2 error and support equality of x[idx] against the minimiser."""
        xs = x[self.idx].astype(np.complex128)
        ref = self.ref["x"]
        nr = np.linalg.norm(ref, axis=1)
        err = np.linalg.norm(xs - ref, axis=1) / np.where(nr > 0, nr, 1.0)
        supp = np.all((xs != 0) == (ref != 0), axis=1) | self.degen
        return err, supp

    def gate(self, x, status) -> dict:
        """The accuracy gate: certified pixels with error <= 1e-4 and the oracle's support."""
        err, supp = self.errors(x)
        cert = ((status[self.idx] & 64) != 0) & self.resolved
        ok = cert & (err <= 1e-4) & supp
        return {"n": int(self.idx.size), "oracle_unresolved": int((~self.resolved).sum()),
                "certified": int(cert.sum()), "ok": int(ok.sum()), "cert_and_wrong": int((cert & ~ok).sum()),
                "max_err_certified": float(err[cert].max()) if cert.any() else None,
                "degenerate": int(self.degen.sum())}

    def summary(self, x, tol: float) -> dict:
        err, supp = self.errors(x)
        e = err[self.resolved]
        return {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)), "max": float(e.max()),
                f"frac_le_{tol:g}": float((e <= tol).mean()), "support_equal_frac": float(supp[self.resolved].mean())}


def precision_report(api, oracle_patch: "OracleSample", st_patch, op_patch, g_patch, lam_patch,
                     paths: dict) -> dict:
    """Error against the FP64 oracle before and after the refit, per path, on the small
    stack (all 256 pixels) and on the oracle sample of the patch."""
    from paper_1805_01759_gb300 import synth
    import torch
    small = synth.workload_small(P=256, seed=1)
    o_small = OracleSample(small, 256)
    op_small = api.Operator.from_geometry(small.geom)
    g_small = torch.from_numpy(small.g).cuda()
    out = {}
    for cname, (o, op, g, lam) in {"small_N25_L200_P256": (o_small, op_small, g_small, small.lam),
                                   "patch_sample": (oracle_patch, op_patch, g_patch, lam_patch)}.items():
        rows = {}
        for name, (prec, tol, tile) in paths.items():
            it = api.solve(op, g, lam, precision=prec, tol=tol, refit=0, tile_pixels=tile)
            x_it = it.x.cpu().numpy()
            x_rf, _, _, st_rf = api.refit(op, g, lam, it.x, status=it.status)
            torch.cuda.synchronize()
            before = o.summary(x_it, 1e-3)
            before["frac_le_0.0001"] = o.summary(x_it, 1e-4)["frac_le_0.0001"]
            rows[name] = {"before_refit": before, "after_refit": o.summary(x_rf.cpu().numpy(), 1e-4),
                          "certified_frac": float(((st_rf.cpu().numpy() & 64) != 0).mean())}
        out[cname] = rows
    return out


class PathRunner:
    """One configuration of the hot path (iteration kernel + refit) on resident inputs."""

    def __init__(self, lib, _lib, op, g_dev, lam_t, P, precision, tol, stream, tile=0):
        import torch
        self.lib, self._lib, self.op, self.g_dev, self.lam_t, self.P = lib, _lib, op, g_dev, lam_t, P
        dev = g_dev.device
        self.opt_solve = _lib.default_options(refit=0, precision=precision, tol=tol, tile_pixels=tile)
        self.opt_refit = _lib.default_options()
        L = op.L
        self.x = torch.empty((P, L), dtype=torch.complex64, device=dev)
        self.status = torch.empty(P, dtype=torch.int32, device=dev)
        self.iters = torch.empty(P, dtype=torch.int32, device=dev)
        self.nbt = torch.empty(P, dtype=torch.int32, device=dev)
        self.nsupp = torch.empty(P, dtype=torch.int32, device=dev)
        self.support = torch.empty((P, self.opt_refit.s_max), dtype=torch.int32, device=dev)
        self.ws_bytes = lib.bpdn_solve_workspace_bytes(op.handle, P, ctypes.byref(self.opt_solve))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.rws_bytes = lib.bpdn_refit_workspace_bytes(op.handle, P)
        self.rws = torch.empty(max(self.rws_bytes, 1), dtype=torch.uint8, device=dev)
        self.stream = stream
        self.precision, self.tol = precision, tol

    def step(self):
        """bpdn_solve (Algorithm 1) then bpdn_refit; returns the event between the two."""
        import torch
        lib, _lib, s = self.lib, self._lib, self.stream.cuda_stream
        _lib.check(lib.bpdn_solve(self.op.handle, self.g_dev.data_ptr(), self.P, self.lam_t.data_ptr(), 0,
                                  ctypes.byref(self.opt_solve), self.x.data_ptr(), None,
                                  self.nsupp.data_ptr(), self.status.data_ptr(), self.iters.data_ptr(),
                                  self.nbt.data_ptr(), self.ws.data_ptr(), self.ws_bytes, s))
        ev_mid = torch.cuda.Event(enable_timing=True)
        ev_mid.record(self.stream)
        _lib.check(lib.bpdn_refit(self.op.handle, self.g_dev.data_ptr(), self.P, self.lam_t.data_ptr(), 0,
                                  ctypes.byref(self.opt_refit), self.x.data_ptr(), self.x.data_ptr(),
                                  self.support.data_ptr(), self.nsupp.data_ptr(), self.status.data_ptr(),
                                  self.rws.data_ptr(), self.rws_bytes, s))
        return ev_mid

    def timed(self, steps: int, warmup: int, dev):
        import torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        barrier(dev)
        torch.cuda.synchronize()
        evs = []
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(self.stream)
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            em = self.step()
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(self.stream)
            evs.append((e0, em, e1))
        t1.record(self.stream)
        torch.cuda.synchronize()
        barrier(dev)
        return {"total_ms": t0.elapsed_time(t1),
                "rbpg_ms": [a.elapsed_time(b) for a, b, _ in evs],
                "refit_ms": [b.elapsed_time(c) for _, b, c in evs]}


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1805_01759_gb300 import _lib, api, synth
    lib = _lib.load()

    P = args.pixels
    st = synth.workload_patch(P=P, seed=2, part=shard_part(rank))
    op = api.Operator.from_geometry(st.geom)
    N, L = op.N, op.L
    stream = torch.cuda.current_stream(dev)
    g_dev = torch.from_numpy(st.g).to(dev)
    lam_t = torch.tensor([st.lam], dtype=torch.float32, device=dev)

    # plain FP32 at its own tolerance, FP32 at the BF16 path's tolerance (the same stopping
    # rule, so that the two precisions are compared at equal work per pixel), and BF16
    # (precision, tol, tile_pixels): bf16 is the grid-point-per-thread BF16 kernel (the default);
    # bf16_pixel_per_thread the alternative layout (tile_pixels 128) on the same solve
    paths = {"fp32": (0, args.tol_fp32, 0), "fp32_tol_bf16": (0, args.tol_bf16, 0), "bf16": (1, args.tol_bf16, 0),
             "bf16_pixel_per_thread": (1, args.tol_bf16, 128)}
    if args.precision == "fp32":
        paths = {"fp32": paths["fp32"], "fp32_tol_bf16": paths["fp32_tol_bf16"]}
    elif args.precision == "bf16":
        paths = {"bf16": paths["bf16"]}
    # the oracle's answers for the accuracy gate, computed on the host before timing
    oracle_patch = OracleSample(st, args.sample) if rank == 0 else None
    results = {}
    launches = 0
    with ClockSampler(dev.index) as clk:
        for name, (prec, tol, tile) in paths.items():
            runner = PathRunner(lib, _lib, op, g_dev, lam_t, P, prec, tol, stream, tile)
            tm = runner.timed(args.steps, args.warmup, dev)
            launches += 2 * args.steps
            results[name] = (runner, tm)

    # headline path: BF16 + FP64 refit when timed, else the one that ran
    head = "bf16" if "bf16" in results else next(iter(results))
    out_paths = {}
    acc_head = None
    good_head = None
    ms_head = None
    for name, (runner, tm) in results.items():
        ms_step = reduce_max(tm["total_ms"] / args.steps, dev)
        it_np = runner.iters.cpu().numpy()
        st_np = runner.status.cpu().numpy()
        nbt_np = runner.nbt.cpu().numpy()
        x_np = runner.x.cpu().numpy()
        certified = int(((st_np & 64) != 0).sum())
        acc = oracle_patch.gate(x_np, st_np) if rank == 0 else None
        good = (certified / P) * (acc["ok"] / max(acc["certified"], 1) if acc else 1.0)
        pixel_iters = float(it_np.astype(np.int64).sum())
        sweeps = pixel_iters + float(nbt_np.astype(np.int64).sum())  # a step cut is one more sweep
        rbpg_avg_s = statistics.mean(tm["rbpg_ms"]) / 1e3
        out_paths[name] = {
            "value": P * world * good / (ms_step / 1e3), "ms_per_step": ms_step,
            "kernels_ms": {"iteration": statistics.mean(tm["rbpg_ms"]), "refit_fp64": statistics.mean(tm["refit_ms"])},
            "tol": runner.tol, "certified_frac": certified / P, "good_frac": good, "sample": acc,
            "mean_iters": float(it_np.mean()), "frac_max_iter": float((it_np >= 500).mean()),
            "mean_step_cuts": float(nbt_np.mean()),
            "pixel_sweeps": sweeps,
            # time of one sweep over every pixel of the batch (iteration kernel time / mean sweeps)
            "ms_per_sweep": statistics.mean(tm["rbpg_ms"]) / (sweeps / P),
            "alu_tflops": sweeps * alu_flops_per_sweep(name, N, L) / rbpg_avg_s / 1e12,
        }
        if name.startswith("bf16"):
            out_paths[name]["tensor_tflops"] = sweeps * 8.0 * N * L / rbpg_avg_s / 1e12
        out_paths[name]["alu_flops_per_sweep"] = alu_flops_per_sweep(name, N, L)
        if name == head:
            acc_head, good_head, ms_head = acc, good, ms_step
            head_runner, head_tm, head_sweeps = runner, tm, sweeps

    # end to end through the public API with host buffers (copies inside the timed region):
    # the batch in chunks on two streams, each chunk's copies overlapping its neighbours' solves
    runner = head_runner
    g_host = torch.from_numpy(st.g).pin_memory()
    x_host = torch.empty((P, L), dtype=torch.complex64).pin_memory()
    st_host = torch.empty(P, dtype=torch.int32).pin_memory()
    h2d = g_host.numel() * g_host.element_size()
    d2h = x_host.numel() * x_host.element_size() + st_host.numel() * 4
    hs = api.HostSolver(op, P, chunks=args.e2e_chunks, precision=paths[head][0], tol=paths[head][1])
    hs.run(g_host, st.lam, x_host, st_host)  # warm-up (buffers, streams)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    barrier(dev)
    e_a = torch.cuda.Event(enable_timing=True)
    e_b = torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    for _ in range(e2e_steps):
        hs.run(g_host, st.lam, x_host, st_host)
        launches += 2 * hs.chunks
    e_b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e_a.elapsed_time(e_b) / e2e_steps, dev)
    e2e_cert = float(((st_host.numpy() & 64) != 0).mean())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.cpu_sample)
    prec_report = None
    if rank == 0 and not args.no_precision_report:
        prec_report = precision_report(api, oracle_patch, st, op, g_dev, st.lam, paths)
        # the same paths without the refit: Algorithm 1's own output against the 1e-4 gate
        # (the fraction of the oracle sample within 1e-4, over the iteration kernel's time)
        for name in out_paths:
            frac = prec_report["patch_sample"][name]["before_refit"]["frac_le_0.0001"]
            it_ms = out_paths[name]["kernels_ms"]["iteration"]
            out_paths[name]["without_refit"] = {"frac_within_1e-4": frac,
                                                "value": P * world * frac / (it_ms / 1e3)}
    pixels_total = P * world
    value = pixels_total * good_head / (ms_head / 1e3)
    # the e2e result's own certified fraction, times the sample's agreement rate
    e2e_value = pixels_total * e2e_cert * (acc_head["ok"] / max(acc_head["certified"], 1) if acc_head else 1.0) / (e2e_ms / 1e3)

    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    unit_count_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # the FP32 pipe's peak measured on this GPU (the faster of the FFMA and packed FFMA2 loops)
    pk = measure_peaks(dev, kinds=(0, 1))
    peak_tflops = max(pk["ffma"]["value"], pk["ffma2"]["value"])
    # the dominant kernel of the headline path is its iteration kernel (its share of a step
    # is reported under kernels); the pipe that bounds it is the FP32 one (alu_flops_per_sweep)
    rbpg_avg_s = statistics.mean(head_tm["rbpg_ms"]) / 1e3
    achieved = head_sweeps * alu_flops_per_sweep(head, N, L) / rbpg_avg_s / 1e12
    traffic = _traffic_per_launch(P, head)
    # a second count for the same kernel: per pixel sweep 16 N L flops of contraction on the
    # tensor cores (BF16; the FP32 path's contraction runs on the FP32 pipe) and 20 L of FP32
    # elementwise work; roofline time = the slowest of the pipes and HBM (3.4 kB per pixel)
    peaks_file = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mp = json.load(open(peaks_file)) if os.path.exists(peaks_file) else {}
    bf16_peak = float(mp.get("bf16_tflops", 1900.0))
    hbm_gbs = float(mp.get("hbm_gbs", 6800.0))
    if head.startswith("bf16"):
        t_pipe = max(head_sweeps * 16.0 * N * L / (bf16_peak * 1e12), head_sweeps * 20.0 * L / (peak_tflops * 1e12))
    else:
        t_pipe = head_sweeps * (16.0 * N * L + 20.0 * L) / (peak_tflops * 1e12)
    t_hbm = P * (8.0 * N + 8.0 * L + 16.0) / (hbm_gbs * 1e9)
    frac_16nl = max(t_pipe, t_hbm) / rbpg_avg_s

    if rank != 0:
        return
    kname = "k_rbpg<BF16>" if head == "bf16" else "k_rbpg<FP32>"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_head, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if head == "bf16" else "f32", "data": "synthetic",
        "config": {
            "workload": f"one stack N={N}, L={L} on [-200,200] m, P=2^{int(np.log2(P))} pixels per GPU, "
                        "K in {0,1,2} (second at kappa*rho_s, kappa~U[0.5,2]), SNR~U[0,20] dB",
            "path": ("BF16 tensor-core contraction (FP32 accumulate, FP32 iterate) + FP64 refit/certificate"
                     if head == "bf16" else "plain FP32 Algorithm 1 + FP64 refit/certificate"),
            "P_per_gpu": P, "N": N, "L": L, "lambda": st.lam, "max_iter": 500,
            "l2": "inputs larger than L2 (g 210 MB, x 3.4 GB per GPU); no flush",
            "parallelism": f"pixels sharded over {world} GPU(s), no collective",
        },
        "paths": out_paths,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic, "kernel": kname,
                     "frac_count_16NL_20L": frac_16nl,
                     "count_16NL_20L": "16 N L tensor (BF16 peak %s) + 20 L FP32 per sweep, HBM 3.4 kB per pixel" % (
                         "measured" if mp else "fallback 1.9 PFLOP/s"),
                     "peak_source": "measured: FFMA/FFMA2 loops of bpdn_bench_peak on this GPU",
                     "peak_unit_count": unit_count_tflops, "peaks_measured": pk,
                     "note": "the fused iteration (Algorithm 1); see kernels for the refit's share. "
                             "peak = the FP32 FMA rate measured on this GPU (the faster of the FFMA and "
                             f"FFMA2 loops; the unit count {n_sm} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz "
                             "is peak_unit_count); achieved = the algorithmic FP32 work of "
                             "Algorithm 1 per pixel sweep (36 L elementwise flops"
                             + ("" if head == "bf16" else " + 8 N L for the contraction") +
                             "; a step cut is one more sweep) over the iteration kernel's event-timed "
                             "duration" + ("; the BF16 contraction (8 N L per sweep) runs on the tensor "
                                           "cores, see paths.bf16.tensor_tflops" if head == "bf16" else "")},
        "kernels": {
            "iteration": {"name": kname, "ms": statistics.mean(head_tm["rbpg_ms"]),
                          "share": statistics.mean(head_tm["rbpg_ms"]) / ms_head,
                          "bound": "FP32 pipe (roofline above)"},
            "refit": {"name": "k_refit_t<1> + k_refit_t<2> + k_refit_t<3>",
                      "ms": statistics.mean(head_tm["refit_ms"]),
                      "share": statistics.mean(head_tm["refit_ms"]) / ms_head,
                      "bound": "latency (one warp per pixel): the FP32 support search issues at ~55 %, "
                               "the FP64 finish keeps the FP64 pipe ~60 % busy, the further rounds are "
                               "few but long; no throughput roofline applies"},
        },
        "precision_report": prec_report,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "chunks": hs.chunks, "note": "api.HostSolver: pinned host g in, x and status out, copies "
                                             "overlapped with the solves of neighbouring chunks"},
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                   "reasons": clocks.get("reasons"), "power_w_max": clocks.get("power_w_max")},
    }
    print(json.dumps(line), flush=True)


def run_ragged(args) -> None:
    """The ragged batch (64 stacks: N 10..60, L 100..600, 2^12..2^16 pixels each) through
    one bpdn_solve_ragged call replayed as a CUDA graph, with the library's kernel choice and
    with each stack's kernel and tile picked by timing (api.autotune_stack), next to the same
    stacks solved one after another on one stream."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1805_01759_gb300 import api, synth
    sts = synth.workload_ragged(n_stacks=64, seed=3)
    # with several ranks each takes the stacks dealt to it by estimated cost P * N * L
    owner = api.deal_stacks([st.g.shape[0] * st.geom.N * st.geom.L for st in sts], world)
    sts = [st for st, r in zip(sts, owner) if r == rank]
    items = [(api.Operator.from_geometry(st.geom), torch.from_numpy(st.g).cuda(), st.lam) for st in sts]
    P_total = sum(st.g.shape[0] for st in sts)
    prec = 1 if args.precision == "bf16" else 0
    tol = args.tol_bf16 if prec else args.tol_fp32
    # BF16 where the grid-point tensor-core kernel takes the stack (2N <= 128, L <= 512); the
    # other stacks run in FP32 in either mode (in the BF16 mode at the same tolerance as the
    # BF16 stacks; the refit certifies both), which is faster there than the tensor-core
    # split-grid kernel
    def opts(op):
        ok = prec == 1 and 2 * op.N <= 128 and op.L <= 512
        return dict(precision=1 if ok else 0, tol=tol)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        barrier(dev)
        return reduce_max(e0.elapsed_time(e1) / steps, dev)

    out = {}
    # per-stack precision differs, so the stacks are grouped into one solver per option set
    for mode in ("graph", "graph_autotuned"):
        solvers = []
        for key in sorted({tuple(sorted(opts(op).items())) for op, _, _ in items}):
            sub = [it for it in items if tuple(sorted(opts(it[0]).items())) == key]
            solvers.append(api.RaggedSolver(sub, autotune=(mode == "graph_autotuned"), **dict(key)))
        for sv in solvers:
            sv.capture()
        ms = timed(lambda: [sv.replay() for sv in solvers], args.steps, args.warmup)
        cert = sum(int(((r.status & 64) != 0).sum().item()) for sv in solvers for r in sv.results)
        out[mode] = {"ms": ms, "pixels_per_s_certified": cert / (ms / 1e3), "certified_frac": cert / P_total,
                     "kernel_tile": [[k, t] for sv in solvers for k, t in zip(sv.kernels, sv.tiles)]}
    ms = timed(lambda: [api.solve(op, g, lam, **opts(op)) for op, g, lam in items], args.steps, args.warmup)
    out["sequential_one_stream"] = {"ms": ms}
    best = min(("graph", "graph_autotuned"), key=lambda k: out[k]["ms"])
    # whole job: certified pixels of every rank over the slowest rank's time
    cert_all = reduce_sum(out[best]["pixels_per_s_certified"] * out[best]["ms"] / 1e3, dev)
    P_all = int(reduce_sum(float(P_total), dev))
    if rank != 0:
        return
    print(json.dumps({"metric": "ragged batch: certified pixels/s", "workload":
                      "64 stacks, N~U{10..60}, L~U{100..600}, 2^U{12..16} pixels each, seed 3"
                      + (f", dealt to {world} ranks by P*N*L" if world > 1 else ""),
                      "value": cert_all / (out[best]["ms"] / 1e3), "unit": "pixels/s", "best": best,
                      "n_gpus": world, "pixels": P_all, "precision": args.precision, "runs": out}), flush=True)


def _detected(khat, s_hat, s_true):
    """Detection rule of the detection-rate experiment: K_hat = 2 and each sorted estimate
    within half the true separation of its sorted true elevation (vectorised)."""
    st = np.sort(s_true, axis=1)
    se = np.sort(np.where(np.isnan(s_hat[:, :2]), np.inf, s_hat[:, :2]), axis=1)
    half = 0.5 * (st[:, 1] - st[:, 0])
    return (khat == 2) & np.all(np.abs(se - st) < half[:, None], axis=1)


def run_detection(args) -> None:
    """The detection-rate Monte Carlo (N = 29, two equal-phase scatterers, SNR 2 and 7 dB,
    kappa 0.1..1.5, args.det_per realisations each) through the whole SL1MMER chain on the
    GPU: bpdn_solve (BF16 + FP64 refit) and bpdn_select.  Prints one JSON line with the
    chain's pixels/s, the kernel split, P_D per (SNR, kappa), and the oracle chain timed on
    a bounded sample of the same pixels with its model orders compared."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1805_01759_gb300 import api, synth
    d = synth.workload_detection(n_per=args.det_per)
    P = d.g.shape[0]
    op = api.Operator.from_geometry(d.geom)
    g = torch.from_numpy(d.g).cuda()
    lam = torch.from_numpy(d.lam).cuda()
    kw = dict(precision=1, tol=args.tol_bf16)

    def step():
        res = api.solve(op, g, lam, **kw)
        return res, api.select(op, g, res)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_chain, t_sel = [], []
    for _ in range(args.steps):
        ev[0].record()
        res = api.solve(op, g, lam, **kw)
        ev[1].record()
        sel = api.select(op, g, res)
        ev[2].record()
        torch.cuda.synchronize()
        t_chain.append(ev[0].elapsed_time(ev[2]))
        t_sel.append(ev[1].elapsed_time(ev[2]))
    ms = statistics.mean(t_chain)
    kh = sel.khat.cpu().numpy()
    sh = sel.s_hat.cpu().numpy()
    cert = (res.status.cpu().numpy() & 64) != 0
    det = _detected(kh, sh, d.s_true)
    pd = {}
    for snr in sorted(set(d.snr_db.tolist())):
        row = {}
        for k in sorted(set(d.kappa.tolist())):
            m = (d.snr_db == snr) & (d.kappa == k)
            row[f"{k:.1f}"] = round(float(det[m].mean()), 4)
        pd[f"{snr:g} dB"] = row
    line = {
        "metric": "SL1MMER chain pixels/s (BF16 solve + FP64 refit + model selection)",
        "value": P / (ms / 1e3), "unit": "pixels/s", "higher_is_better": True, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "pixels": P, "data": "synthetic",
        "workload": f"detection-rate Monte Carlo: N=29 over 269.5 m, L=201 on [-100,100] m, two unit "
                    f"scatterers with equal phase at c -/+ kappa*rho/2, SNR 2 and 7 dB, kappa 0.1..1.5, "
                    f"{args.det_per} realisations each, seed 6",
        "kernels_ms": {"solve_and_refit": ms - statistics.mean(t_sel), "select": statistics.mean(t_sel)},
        "certified_frac": float(cert.mean()),
        "khat_hist": np.bincount(kh + 1, minlength=6).tolist(),
        "detection_rate": pd,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _detection_cpu_leg(d, kh, sh, cert, args.cpu_det_sample)
    print(json.dumps(line), flush=True)


def _detection_cpu_leg(d, kh, sh, cert, n):
    """The oracle chain (FP64 minimiser + model selection) on a seeded sample of the
    detection pixels: its rate, and its model orders against the GPU's."""
    import oracle
    from oracle import select as osel
    rng = np.random.default_rng(61)
    idx = np.sort(rng.choice(d.g.shape[0], size=min(n, d.g.shape[0]), replace=False))
    A = oracle.operator(d.geom)
    xi = oracle.xi(d.geom.baselines_m, d.geom.wavelength_m, d.geom.range_m)
    s = oracle.grid(d.geom.s_min_m, d.geom.s_max_m, d.geom.L)
    t0 = time.perf_counter()
    ref = oracle.minimise_batch(A, d.g[idx], d.lam[idx].astype(np.float64))
    okh, osh, _ = osel.select_batch(d.g[idx], ref["x"], xi, s)
    t = time.perf_counter() - t0
    both = cert[idx] & (ref["flags"] == 0)
    agree = int(np.sum(okh[both] == kh[idx][both]))
    elev = np.abs(np.nan_to_num(osh[both] - sh[idx][both], nan=0.0)).max() if both.any() else 0.0
    return {"value": len(idx) / t, "unit": "pixels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(idx)} seeded pixels of the same set: FP64 coordinate-descent minimiser + "
                      f"model selection, {t:.1f} s",
            "khat_agree": agree, "khat_compared": int(both.sum()), "max_elevation_diff_m": float(elev)}


def run_hybrid(args) -> None:
    """The pre-classified chain on the patch (classify, then solve + refit + select only for
    the pixels the linear pass leaves to L1, merged back) against the plain chain (solve +
    refit + select on every pixel), both BF16 with the FP64 refit.  Reports both rates, the
    class fractions, and on an oracle sample the model orders and elevations of both chains
    against the oracle's chain (exact minimiser + model selection)."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1805_01759_gb300 import api, synth
    P = args.pixels
    st = synth.workload_patch(P=P, seed=2)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    kw = dict(precision=1, tol=args.tol_bf16)

    def plain():
        res = api.solve(op, g, st.lam, **kw)
        return api.select(op, g, res)

    def hybrid():
        return api.hybrid(op, g, st.lam, **kw)

    out = {}
    for name, fn in (("plain", plain), ("hybrid", hybrid)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = (statistics.mean(times), r)
    ms_plain, sel_plain = out["plain"]
    ms_hyb, (cls_out, sel_hyb, _) = out["hybrid"]
    cls = cls_out.cls.cpu().numpy()
    # the oracle's chain on a seeded sample
    import oracle
    from oracle import select as osel
    rng = np.random.default_rng(62)
    idx = np.sort(rng.choice(P, size=min(args.sample, P), replace=False))
    A = oracle.operator(st.geom)
    xi = oracle.xi(st.geom.baselines_m, st.geom.wavelength_m, st.geom.range_m)
    sg = oracle.grid(st.geom.s_min_m, st.geom.s_max_m, st.geom.L)
    ref = oracle.minimise_batch(A, st.g[idx], st.lam)
    okh, osh, _ = osel.select_batch(st.g[idx], ref["x"], xi, sg)

    def agree(sel):
        kh = sel.khat.cpu().numpy()[idx]
        sh = sel.s_hat.cpu().numpy()[idx]
        both = ref["flags"] == 0
        same = both & (kh == okh)
        per_cls = {str(c): {"n": int(np.sum(both & (cls[idx] == c))),
                            "khat_agree": int(np.sum(same & (cls[idx] == c)))} for c in (0, 1, 2)}
        d = np.abs(np.nan_to_num(sh[same] - osh[same], nan=0.0))
        return {"khat_agree": int(same.sum()), "compared": int(both.sum()), "by_class": per_cls,
                "max_elevation_diff_m": float(d.max()) if d.size else 0.0,
                "median_elevation_diff_m": float(np.median(d[d > 0])) if np.any(d > 0) else 0.0}

    line = {
        "metric": "pixels/s of the SL1MMER chain, pre-classified (linear pass + L1 on the rest) vs L1 on every pixel",
        "value": P / (ms_hyb / 1e3), "unit": "pixels/s", "higher_is_better": True, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_hyb, "data": "synthetic", "workload": "hybrid",
        "config": {"workload": f"the 2^{int(np.log2(P))}-pixel patch (N=25, L=400), BF16 + FP64 refit + selection"},
        "plain": {"value": P / (ms_plain / 1e3), "ms_per_step": ms_plain, "vs_oracle": agree(sel_plain)},
        "hybrid": {"value": P / (ms_hyb / 1e3), "ms_per_step": ms_hyb, "vs_oracle": agree(sel_hyb),
                   "class_frac": (np.bincount(cls, minlength=3) / P).tolist(),
                   "skipped_frac": float(np.mean(cls < 2))},
        "speedup": ms_plain / ms_hyb,
    }
    print(json.dumps(line), flush=True)


def run_blocks(args) -> None:
    """The randomized-block reading of Eqs. 13-14 (options.blocks = J) against the default
    reading (a block is a whole pixel) on the same pixels of the patch: both FP32 with the
    FP64 refit, certified pixels/s, iterations, and a seeded oracle sample of each."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1805_01759_gb300 import api, synth
    st = synth.workload_patch(P=args.block_pixels, seed=2)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    P = st.g.shape[0]
    out = {}
    for name, kw in (("default_reading", dict(tol=args.tol_fp32)),
                     (f"blocks_{args.blocks}", dict(tol=args.tol_fp32, blocks=args.blocks, seed=1))):
        for _ in range(args.warmup):
            api.solve(op, g, st.lam, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            res = api.solve(op, g, st.lam, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        cert = (res.status & 64) != 0
        it = res.iters.double()
        out[name] = {"ms_per_step": ms, "certified_frac": float(cert.float().mean()),
                     "certified_pixels_per_s": float(cert.sum()) / (ms / 1e3),
                     "mean_iterations": float(it.mean()),
                     "frac_max_iter": float(((res.status & 1) != 0).float().mean())}
        if not args.no_cpu_baseline:
            out[name]["oracle_sample"] = _block_sample(st, res, 64)
    print(json.dumps({"metric": "certified pixels/s, randomized-block reading vs default reading (FP32 + refit)",
                      "value": out[f"blocks_{args.blocks}"]["certified_pixels_per_s"], "unit": "pixels/s",
                      "workload": f"patch N=25, L=400, {P} pixels, seed 2; blocks={args.blocks} (iterations "
                                  f"counted in block steps, max 500*blocks)", "runs": out}), flush=True)


def _block_sample(st, res, n):
    """Certified pixels of a seeded sample against the exact minimiser (oracle)."""
    import oracle
    rng = np.random.default_rng(62)
    idx = np.sort(rng.choice(st.g.shape[0], size=n, replace=False))
    A = oracle.operator(st.geom)
    ref = oracle.minimise_batch(A, st.g[idx], st.lam)
    import torch
    x = res.x[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    cert = (res.status.cpu().numpy()[idx] & 64) != 0
    ok = 0
    for j in range(n):
        if not cert[j] or ref["flags"][j] != 0:
            continue
        nr = np.linalg.norm(ref["x"][j])
        err = np.linalg.norm(x[j] - ref["x"][j]) / nr if nr > 0 else np.linalg.norm(x[j])
        ok += int(err <= 1e-4 and np.array_equal(x[j] != 0, ref["x"][j] != 0))
    return {"n": n, "certified": int(cert.sum()), "certified_and_ok": ok}


def run_motion(args) -> None:
    """Differential tomography (Eq. 4): a stack observed over four years with linear
    deformation, on an elevation x velocity grid (32 x 16 = 512 points, BF16 + refit, and
    64 x 16 = 1024 points, FP32 + refit).  Certified pixels/s per path, and a seeded oracle
    sample of each (exact minimiser on the same multi-component operator)."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1805_01759_gb300 import api, synth
    out = {}
    for name, L_s, kw in (("bf16_32x16", 32, dict(precision=1, tol=args.tol_bf16)),
                          ("fp32_64x16", 64, dict(precision=0, tol=args.tol_fp32)),
                          ("bf16_64x16", 64, dict(precision=1, tol=args.tol_bf16))):
        st = synth.workload_motion(P=args.motion_pixels, seed=7, L_s=L_s, L_v=16)
        op = api.Operator.from_geometry(st.geom)
        g = torch.from_numpy(st.g).cuda()
        for _ in range(args.warmup):
            api.solve(op, g, st.lam, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            res = api.solve(op, g, st.lam, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        cert = (res.status & 64) != 0
        out[name] = {"L": op.L, "ms_per_step": ms, "certified_frac": float(cert.float().mean()),
                     "certified_pixels_per_s": float(cert.sum()) / (ms / 1e3),
                     "mean_iterations": float(res.iters.double().mean())}
        if not args.no_cpu_baseline:
            out[name]["oracle_sample"] = _motion_sample(st, res, 32)
    if args.motion4d_pixels > 0:
        out["fp32_4d_64x16x16"] = _motion4d(args, 0)
        out["bf16_4d_64x16x16"] = _motion4d(args, 1)
    print(json.dumps({"metric": "certified pixels/s, multi-component operator (elevation x velocity)",
                      "value": out["bf16_32x16"]["certified_pixels_per_s"], "unit": "pixels/s",
                      "workload": f"N=25, times U[0,4] yr, linear velocity grid 16 points on [-0.02,0.02] m/yr, "
                                  f"elevation on [-100,100] m, {args.motion_pixels} pixels, seed 7",
                      "runs": out}), flush=True)


def run_motion4d(args) -> None:
    """The 4-D grid runs of the motion leg on their own (one JSON line)."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    runs = {"fp32": _motion4d(args, 0), "bf16": _motion4d(args, 1)}
    print(json.dumps({"metric": "certified pixels/s, 4-D grid (elevation x velocity x seasonal amplitude)",
                      "value": max(r["certified_pixels_per_s"] for r in runs.values()), "unit": "pixels/s",
                      "workload": "N=25, 64 x 16 x 16 = 16,384 grid points, seed 8", "runs": runs}), flush=True)


def _motion4d(args, precision: int = 0) -> dict:
    """The 4-D grid (elevation x velocity x seasonal amplitude, 64 x 16 x 16 = 16,384 points)
    through the split-grid kernel (FP32 CUDA cores at tol 1e-6, or BF16 tensor cores at
    tol 1e-3) and the refit: the whole solve, the iterations alone, and the contraction's rate
    (8 N L flops per sweep of a pixel) over the iteration time."""
    import torch
    from paper_1805_01759_gb300 import api, synth
    st = synth.workload_motion4d(P=args.motion4d_pixels, seed=8)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    row = {"L": op.L, "N": op.N, "pixels": int(g.shape[0]), "precision": "bf16" if precision else "fp32"}
    tol = args.tol_bf16 if precision else args.tol_fp32
    for key, kw in (("solve", dict(precision=precision, tol=tol)),
                    ("iterations_only", dict(precision=precision, tol=tol, refit=0))):
        for _ in range(max(1, min(args.warmup, 2))):
            api.solve(op, g, st.lam, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(1, min(args.steps, 3))
        e0.record()
        for _ in range(steps):
            res = api.solve(op, g, st.lam, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if key == "solve":
            cert = (res.status & 64) != 0
            row.update(ms_per_step=ms, certified_frac=float(cert.float().mean()),
                       certified_pixels_per_s=float(cert.sum()) / (ms / 1e3),
                       mean_iterations=float(res.iters.double().mean()))
            keep = res
        else:
            sweeps = float((res.iters.double() + res.nbt.double()).sum())
            row.update(ms_iterations=ms, sweeps=sweeps,
                       gradient_tflops=sweeps * 8.0 * op.N * op.L / (ms / 1e3) / 1e12)
    if not args.no_cpu_baseline:
        row["oracle_sample"] = _motion_sample(st, keep, 16)
    return row


def _motion_sample(st, res, n):
    import oracle
    import torch
    rng = np.random.default_rng(63)
    idx = np.sort(rng.choice(st.g.shape[0], size=n, replace=False))
    A = oracle.operator_md(st.geom)
    ref = oracle.minimise_batch(A, st.g[idx], st.lam)
    x = res.x[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    cert = (res.status.cpu().numpy()[idx] & 64) != 0
    ok = 0
    for j in range(n):
        if not cert[j] or ref["flags"][j] != 0:
            continue
        nr = np.linalg.norm(ref["x"][j])
        err = np.linalg.norm(x[j] - ref["x"][j]) / nr if nr > 0 else np.linalg.norm(x[j])
        ok += int(err <= 1e-4 and np.array_equal(x[j] != 0, ref["x"][j] != 0))
    return {"n": n, "certified": int(cert.sum()), "certified_and_ok": ok}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--pixels", type=int, default=1 << 20, help="pixels per GPU (workload: 2^20)")
    ap.add_argument("--sample", type=int, default=256, help="pixels checked against the oracle")
    ap.add_argument("--cpu-sample", type=int, default=2048, help="pixels of the CPU baseline leg")
    ap.add_argument("--ref-sample", type=int, default=1024, help="pixels per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--motion4d-pixels", type=int, default=1 << 14,
                    help="pixels of the 4-D grid run of the motion leg (0: skip)")
    ap.add_argument("--no-precision-report", action="store_true",
                    help="skip the error-before/after-refit report (small stack and patch sample)")
    ap.add_argument("--precision", choices=["fp32", "bf16", "both"], default="both")
    ap.add_argument("--tol-fp32", type=float, default=1e-6)
    ap.add_argument("--tol-bf16", type=float, default=1e-3,
                    help="stopping tolerance of the BF16 path: BF16 operands carry 2^-9 relative error, "
                         "so smaller steps are not resolved")
    ap.add_argument("--e2e-chunks", type=int, default=2, help="chunks of the end-to-end leg")
    ap.add_argument("--workload", choices=["patch", "ragged", "detection", "blocks", "motion", "motion4d", "peaks", "hybrid"], default="patch",
                    help="patch: the headline line; ragged: the 64-stack ragged batch; detection: the "
                         "detection-rate Monte Carlo through solve + model selection (separate lines)")
    ap.add_argument("--det-per", type=int, default=5000, help="realisations per (SNR, kappa)")
    ap.add_argument("--blocks", type=int, default=4, help="blocks of the randomized-block reading")
    ap.add_argument("--block-pixels", type=int, default=1 << 16, help="pixels of the block comparison")
    ap.add_argument("--motion-pixels", type=int, default=1 << 18, help="pixels of the motion workload")
    ap.add_argument("--cpu-det-sample", type=int, default=256, help="oracle pixels of the detection leg")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ragged":
        run_ragged(args)
    elif args.workload == "detection":
        run_detection(args)
    elif args.workload == "blocks":
        run_blocks(args)
    elif args.workload == "motion":
        run_motion(args)
    elif args.workload == "motion4d":
        run_motion4d(args)
    elif args.workload == "peaks":
        run_peaks(args)
    elif args.workload == "hybrid":
        run_hybrid(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
