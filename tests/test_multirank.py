"""Multi-rank logic of bench.py on CPU: two gloo ranks (one process each).

The weak-scaling run shards the patch by rank (each rank draws its own pixel set of
the same stack), synchronises with a barrier and reports the maximum step time over
ranks.  These are exercised here without a GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        import bench
        from paper_1805_01759_gb300 import synth

        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        # the slowest rank's time is the job's time
        t = bench.reduce_max(10.0 + 3.0 * rank)
        bench.barrier()
        # each rank draws a different pixel set of the same stack
        st = synth.workload_patch(P=64, seed=2, part=bench.shard_part(rank))
        gsum = torch.tensor([float(np.abs(st.g).sum())], dtype=torch.float64)
        bsum = torch.tensor([float(st.geom.baselines_m.sum()), st.lam], dtype=torch.float64)
        gs = [torch.zeros_like(gsum) for _ in range(world)]
        bs = [torch.zeros_like(bsum) for _ in range(world)]
        dist.all_gather(gs, gsum)
        dist.all_gather(bs, bsum)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([t] + [float(x) for x in gs] + [float(x) for b in bs for x in b]))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    for r in res:
        assert r[0] == 13.0  # max over ranks of 10 + 3 rank
        g0, g1 = r[1], r[2]
        assert g0 != g1  # different pixel sets
        b0, lam0, b1, lam1 = r[3], r[4], r[5], r[6]
        assert b0 == b1 and lam0 == lam1  # same stack geometry and lambda
    assert np.array_equal(res[0], res[1])


def test_single_process_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    assert bench.reduce_max(4.5) == 4.5
    bench.barrier()
    assert bench.shard_part(0) == 0


def _tune_rank(rank: int, world: int, port: int, out_dir: str) -> None:
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        from paper_1805_01759_gb300 import api
        # rank r holds a shard with error numerator n_r, normaliser d_r and derivative q_r
        n, d, q = [3.0, 5.0][rank], [10.0, 30.0][rank], [-0.2, 0.6][rank]
        err, grad = api.global_error_and_grad(n, d, q)
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([err, grad]))
    finally:
        dist.destroy_process_group()


def test_two_rank_lambda_tuning_reduction(tmp_path):
    """The collective of lambda tuning with sharded pixels: every rank gets the error and
    derivative of the whole batch, (n_0 + n_1) / (d_0 + d_1) and (q_0 + q_1) / (d_0 + d_1)."""
    world = 2
    mp.spawn(_tune_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        err, grad = np.load(tmp_path / f"t{r}.npy")
        assert abs(err - 8.0 / 40.0) < 1e-15 and abs(grad - 0.4 / 40.0) < 1e-15


def test_lambda_tuning_reduction_without_process_group():
    sys.path.insert(0, ROOT)
    from paper_1805_01759_gb300 import api
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    err, grad = api.global_error_and_grad(3.0, 12.0, -0.6)
    assert err == 0.25 and abs(grad + 0.05) < 1e-16


def test_deal_stacks_by_cost():
    """Stacks go to ranks by estimated cost, largest first, each to the least-loaded rank:
    every stack exactly once, the dealing deterministic, and the heaviest rank's load within
    the largest single cost of the average (the greedy bound)."""
    sys.path.insert(0, ROOT)
    from paper_1805_01759_gb300 import api, synth
    sts = synth.workload_ragged(n_stacks=64, seed=3, scale_pixels=0.01)
    costs = [st.g.shape[0] * st.geom.N * st.geom.L for st in sts]
    for world in (1, 2, 3, 8):
        owner = api.deal_stacks(costs, world)
        assert owner == api.deal_stacks(costs, world) and len(owner) == len(costs)
        assert set(owner) <= set(range(world))
        loads = [sum(c for c, r in zip(costs, owner) if r == k) for k in range(world)]
        assert max(loads) <= sum(costs) / world + max(costs)
    assert api.deal_stacks(costs, 1) == [0] * len(costs)
    assert api.deal_stacks([5, 1, 4, 2], 2) == [0, 0, 1, 1]  # 5 | 4, then 2 -> rank 1, 1 -> rank 0



class _ClosedFormSolve:
    """A CPU stand-in for BPDNFunction on an operator with orthogonal columns (A^H A = N I):
    the minimiser of Eq. 6 is x = S_{lambda/2}(A^H g) / N (the complex soft threshold of the
    matched filter), differentiable in lambda through torch's autograd."""

    @staticmethod
    def apply(g, lam, op, options=None):
        A = op
        c = g @ A.conj()  # (A^H g)_l for every pixel
        mag = c.abs()
        scale = torch.clamp(1.0 - lam.to(torch.float64) / (2.0 * mag.clamp_min(1e-300)), min=0.0)
        return c * scale / A.shape[0], None


def _dft_shards(world: int, per: int):
    """Pixels with up to two on-grid scatterers and noise over the DFT geometry (N = L = 16),
    split into `world` shards, with their on-grid ground truth."""
    rng = np.random.default_rng(11)
    N = 16
    n = np.arange(N)
    A = np.exp(-2j * np.pi * np.outer(n, n) / N)
    P = world * per
    gam = np.zeros((P, N), np.complex128)
    for p in range(P):
        for _ in range(int(rng.integers(0, 3))):
            gam[p, rng.integers(0, N)] = np.exp(2j * np.pi * rng.uniform())
    G = gam @ A.T + 0.4 * (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N)))
    lam_default = 2.0 * 0.4 * np.sqrt(N * np.log(N))
    return A, G, gam, lam_default


def _tune_full_rank(rank: int, world: int, port: int, out_dir: str) -> None:
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        from paper_1805_01759_gb300 import api
        api.BPDNFunction = _ClosedFormSolve
        A, G, gam, lam_d = _dft_shards(world, 32)
        sl = slice(32 * rank, 32 * (rank + 1))
        lam, hist = api.tune_lambda(torch.from_numpy(A), torch.from_numpy(G[sl]), torch.from_numpy(gam[sl]),
                                    0.5 * lam_d, steps=12, lr=0.5)
        np.save(os.path.join(out_dir, f"h{rank}.npy"), np.array([[l, e] for l, e in hist] + [[lam, 0.0]]))
    finally:
        dist.destroy_process_group()


def test_two_rank_lambda_tuning_end_to_end(tmp_path):
    """tune_lambda with the pixels sharded over two gloo ranks: both ranks take identical
    steps, the same steps as one process over all the pixels, and from half the default
    lambda the line search lowers the error at every accepted step."""
    world = 2
    mp.spawn(_tune_full_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    h = [np.load(tmp_path / f"h{r}.npy") for r in range(world)]
    assert np.array_equal(h[0], h[1])
    sys.path.insert(0, ROOT)
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    from paper_1805_01759_gb300 import api
    saved = api.BPDNFunction
    try:
        api.BPDNFunction = _ClosedFormSolve
        A, G, gam, lam_d = _dft_shards(world, 32)
        lam, hist = api.tune_lambda(torch.from_numpy(A), torch.from_numpy(G), torch.from_numpy(gam),
                                    0.5 * lam_d, steps=12, lr=0.5)
    finally:
        api.BPDNFunction = saved
    one = np.array([[l, e] for l, e in hist] + [[lam, 0.0]])
    np.testing.assert_allclose(h[0], one, rtol=1e-9, atol=0)
    errs = one[:-1, 1]
    assert np.all(np.diff(errs) <= 1e-12) and errs[-1] < errs[0], errs
