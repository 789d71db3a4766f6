"""bpdn_solve_ragged through the C ABI: many stacks with their own operators.

Each stack's results must equal a plain bpdn_solve of that stack bit for bit (the
kernels are deterministic); a sample of pixels is checked against the FP64 oracle;
a CUDA-graph capture of the call must reproduce the eager results on replay.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_01759_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1805_01759_gb300 import api as _api
    from paper_1805_01759_gb300 import _lib
    _lib.load()
    return _api


@pytest.fixture(scope="module")
def stacks(api):
    """Six stacks of the ragged law (N 10..60, L 100..600), 64..256 pixels each."""
    sts = synth.workload_ragged(n_stacks=6, seed=3, p_log2=(6, 8))
    items = []
    for st in sts:
        op = api.Operator.from_geometry(st.geom)
        items.append((op, torch.from_numpy(st.g).cuda(), st.lam))
    return sts, items


def _same(a, b):
    return all(torch.equal(getattr(a, f), getattr(b, f)) for f in ("x", "status", "iters", "nbt", "nsupp", "support"))


def test_ragged_equals_single_stack_solves(api, stacks):
    sts, items = stacks
    out = api.solve_ragged(items)
    singles = [api.solve(op, g, lam) for op, g, lam in items]
    torch.cuda.synchronize()
    for i, (r, s) in enumerate(zip(out, singles)):
        assert _same(r, s), i
    # the sizes span the kernels' shapes: N above and below 32, L above and below 512 (the
    # FP32 stacks beyond 512 points run the split-grid kernel in both calls)
    Ns = [st.geom.N for st in sts]
    Ls = [st.geom.L for st in sts]
    assert max(Ns) > 32 and min(Ns) <= 32 and max(Ls) > 512 and min(Ls) <= 512


def test_ragged_against_oracle(api, stacks):
    sts, items = stacks
    out = api.solve_ragged(items)
    torch.cuda.synchronize()
    checked = 0
    for st, r in zip(sts[:3], out[:3]):
        A = oracle.operator(st.geom)
        idx = np.arange(0, st.g.shape[0], max(1, st.g.shape[0] // 12))
        ref = oracle.minimise_batch(A, st.g[idx], st.lam)
        x = r.x.cpu().numpy()[idx].astype(np.complex128)
        status = r.status.cpu().numpy()[idx]
        for j in range(idx.size):
            if not (status[j] & 64) or ref["margin"][j] < 1e-6:
                continue
            if ref["nS"][j] and ref["min_abs_on"][j] < 1e-6 * np.abs(ref["x"][j]).max():
                continue
            assert np.array_equal(x[j] != 0, ref["x"][j] != 0)
            nr = np.linalg.norm(ref["x"][j])
            assert np.linalg.norm(x[j] - ref["x"][j]) <= 1e-4 * max(nr, 1e-30) or (nr == 0 and np.all(x[j] == 0))
            checked += 1
    assert checked >= 20


def test_ragged_graph_replay(api, stacks):
    sts, items = stacks
    # private copies of g, so the replay can be fed new data in place
    own = [(op, g.clone(), lam) for op, g, lam in items]
    solver = api.RaggedSolver(own)
    solver.capture()
    eager = [api.solve(op, g, lam) for op, g, lam in own]
    for r in solver.results:
        r.x.zero_()
        r.status.fill_(-1)
    solver.replay()
    torch.cuda.synchronize()
    for r, e in zip(solver.results, eager):
        assert _same(r, e)
    # new inputs written into the captured tensors are picked up by the next replay
    for op, g, lam in own:
        g.copy_(torch.flip(g, dims=[0]))
    solver.replay()
    fresh = [api.solve(op, g, lam) for op, g, lam in own]
    torch.cuda.synchronize()
    for r, e in zip(solver.results, fresh):
        assert _same(r, e)


def test_ragged_rejects_bad_stack_before_launch(api, stacks):
    from paper_1805_01759_gb300 import _lib
    sts, items = stacks
    solver = api.RaggedSolver(items[:3])
    for r in solver.results:
        r.status.fill_(-7)
    solver._arr[2].d_g = None  # third stack has no g
    with pytest.raises(_lib.BPDNError) as ei:
        solver.run()
    assert "stack 2" in str(ei.value)
    torch.cuda.synchronize()
    for r in solver.results:
        assert torch.all(r.status == -7)  # nothing ran


def test_tile_pixels_do_not_change_results(api, stacks):
    """8 or 16 pixels in flight per SM: every pixel's arithmetic is the same (sums in a
    fixed order, the same reduction tree for every slot), so results are bitwise equal."""
    from paper_1805_01759_gb300 import _lib
    sts, items = stacks
    compared = 0
    for op, g, lam in items:
        a = api.solve(op, g, lam, tile_pixels=8)
        try:
            b = api.solve(op, g, lam, tile_pixels=16)
        except _lib.BPDNError as e:  # two groups exceed 1024 threads at this L
            assert e.code == _lib.BPDN_ESIZE
            continue
        torch.cuda.synchronize()
        assert _same(a, b)
        compared += 1
    assert compared >= 2
    op, g, lam = items[0]
    with pytest.raises(_lib.BPDNError) as ei:
        api.solve(op, g, lam, tile_pixels=12)
    assert ei.value.code == _lib.BPDN_EINVAL


def test_per_stack_tiles_equal_default(api, stacks):
    """A stack's own tile_pixels (here 8: one group of slots per CTA, which fits wherever the
    default does; for FP32 stacks beyond 512 points it also selects the grid-point kernel
    over the split-grid one) gives exactly what bpdn_solve gives with that tile_pixels."""
    sts, items = stacks
    tiles = [8 if i % 2 else 0 for i in range(len(items))]
    out = api.RaggedSolver(items, tiles=tiles).run()
    ref = [api.solve(op, g, lam, tile_pixels=t) for (op, g, lam), t in zip(items, tiles)]
    torch.cuda.synchronize()
    for r, e in zip(out, ref):
        assert _same(r, e)


def test_autotuned_ragged_equals_per_stack_solves(api, stacks):
    """The autotuner's per-stack (kernel, tile_pixels) choice: the batch gives exactly what
    bpdn_solve gives each stack with those options, and every choice is a valid one."""
    sts, items = stacks
    tuned = api.RaggedSolver(items, autotune=True)
    assert all((k, t) in ((1, 0), (1, 16), (1, 8), (2, 0), (0, 0)) for k, t in zip(tuned.kernels, tuned.tiles))
    out = tuned.run()
    ref = [api.solve(op, g, lam, kernel=k, tile_pixels=t)
           for (op, g, lam), k, t in zip(items, tuned.kernels, tuned.tiles)]
    torch.cuda.synchronize()
    for r, e in zip(out, ref):
        assert _same(r, e)


def test_kernel_option(api, stacks):
    """kernel 1 (grid-point) and 2 (split-grid) on the same FP32 stack both reach the exact
    minimiser; kernel 2 is refused with a tile or randomized blocks."""
    from paper_1805_01759_gb300 import _lib
    sts, items = stacks
    st, (op, g, lam) = sts[0], items[0]
    A = oracle.operator(st.geom)
    ref = oracle.minimise_batch(A, st.g, st.lam)
    for kern in (1, 2):
        res = api.solve(op, g, lam, kernel=kern)
        x = res.x.cpu().numpy().astype(np.complex128)
        cert = (res.status.cpu().numpy() & 64) != 0
        sel = cert & (ref["flags"] == 0) & (ref["margin"] > 1e-6)
        assert cert.mean() >= 0.99 and sel.sum() >= 0.9 * len(sel), (kern, cert.mean(), sel.sum())
        assert np.array_equal(x[sel] != 0, ref["x"][sel] != 0), kern
        nr = np.linalg.norm(ref["x"][sel], axis=1)
        err = np.linalg.norm(x[sel] - ref["x"][sel], axis=1) / np.where(nr > 0, nr, 1.0)
        assert err.max() <= 1e-4, (kern, err.max())
    for bad in (dict(kernel=2, tile_pixels=8), dict(kernel=2, blocks=2), dict(kernel=3)):
        with pytest.raises(_lib.BPDNError) as e:
            api.solve(op, g, lam, **bad)
        assert e.value.code == _lib.BPDN_EINVAL, bad


def test_host_solver_equals_device_solve(api):
    """Chunked solve from pinned host memory (copies overlapped on two streams) returns
    the device solve's results bit for bit, with lambda shared or per pixel."""
    st = synth.workload_small(P=256, seed=1)
    op = api.Operator.from_geometry(st.geom)
    g_host = torch.from_numpy(st.g).pin_memory()
    ref = api.solve(op, g_host.cuda(), st.lam)
    for lam in (st.lam, torch.full((256,), st.lam, dtype=torch.float32)):
        x_host = torch.empty((256, st.geom.L), dtype=torch.complex64).pin_memory()
        s_host = torch.empty(256, dtype=torch.int32).pin_memory()
        api.solve_host(op, g_host, lam, x_host, s_host, chunks=5)
        torch.cuda.synchronize()
        assert torch.equal(x_host, ref.x.cpu()) and torch.equal(s_host, ref.status.cpu())
