"""Grids of more than 1024 points (the split-grid FP32 kernel): the 4-D grid of Eqs. 3-4
(elevation x linear velocity x seasonal amplitude, 64 x 16 x 16 = 16,384 points) and a
wide elevation-only grid, against the FP64 oracle on the same operator.

Bars as for the one-CTA grids: the first iterations of Algorithm 1 within 2e-4 relative
of the oracle's FP64 iterates on pixels with no decision within 1e-5 of its boundary (on
16,384 points some prox decision almost always lies within 1e-3 of the threshold, so the
one-CTA grids' 1e-3 would leave no pixel; the FP32 error of |v| and of the sums of
Eq. 15 over the few nonzero terms is ~1e-6 relative, well inside 1e-5);
the certified solution equal to the exact minimiser (identical support, relative l2
error <= 1e-4) on every certified, non-degenerate pixel; the edges (ragged P, a
non-finite pixel, max_iter 0, options the kernel does not take, the ragged batch).
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
def grid4d():
    return synth.workload_motion4d(P=64, seed=8)


def _rel(a, b):
    nb = np.linalg.norm(b, axis=-1)
    return np.linalg.norm(a - b, axis=-1) / np.where(nb > 0, nb, 1.0)


def _wide_elevation(L):
    """The small workload's pixels on an elevation grid of L points with the small
    workload's spacing (the grid widened about its centre)."""
    st = synth.workload_small(P=64, seed=4)
    ds = (st.geom.s_max_m - st.geom.s_min_m) / (st.geom.L - 1)
    mid = 0.5 * (st.geom.s_max_m + st.geom.s_min_m)
    half = 0.5 * ds * (L - 1)
    geom = synth.StackGeometry(st.geom.baselines_m, st.geom.wavelength_m, st.geom.range_m, mid - half, mid + half, L)
    return synth.Stack(geom, st.g, st.lam)


def _exact(A, G, lam):
    """The oracle's exact minimiser of every row by its working-set loop (no full-grid
    coordinate descent, which is slow on grids this large)."""
    rs = [oracle.minimise_ws(A, g, lam) for g in G]
    ref = {k: np.array([r[k] for r in rs]) for k in ("on_res", "off_max", "min_abs_on", "nS", "flags")}
    ref["x"] = np.stack([r["x"] for r in rs])
    ref["margin"] = 1.0 - ref["off_max"]
    return ref


def _check_minimiser(res, ref, min_sel):
    x = res.x.cpu().numpy().astype(np.complex128)
    cert = (res.status.cpu().numpy() & 64) != 0
    degenerate = (ref["margin"] < 1e-6) | ((ref["nS"] > 0) & (ref["min_abs_on"] < 1e-6 * np.abs(ref["x"]).max(1)))
    sel = cert & ~degenerate & (ref["flags"] == 0)
    assert sel.sum() >= min_sel, (sel.sum(), cert.mean())
    assert np.array_equal(x[sel] != 0, ref["x"][sel] != 0)
    assert _rel(x[sel], ref["x"][sel]).max() <= 1e-4
    return cert


def test_split_grid_operator_tables(api, grid4d):
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    assert op.L == 16384 == A.shape[1]
    np.testing.assert_allclose(op.export("A64").cpu().numpy(), A, rtol=0, atol=1e-12)
    np.testing.assert_allclose(op.export("A").cpu().numpy(), A, rtol=0, atol=2e-7)


@pytest.mark.parametrize("k", [1, 2, 3, 10])
def test_split_grid_first_iterations(api, grid4d, k):
    """x after k iterations of Algorithm 1 on the 16,384-point grid (refit off, no early stop)."""
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    g = torch.from_numpy(grid4d.g).cuda()
    res = api.solve(op, g, grid4d.lam, max_iter=k, tol=0.0, refit=0)
    x = res.x.cpu().numpy()
    iters = res.iters.cpu().numpy()
    nbt = res.nbt.cpu().numpy()
    checked = 0
    for p in range(grid4d.g.shape[0]):
        r = oracle.rbpg(A, grid4d.g[p], grid4d.lam, max_iter=k, tol=0.0, trace=True)
        if np.min(r["margin"]) < 1e-5:
            continue
        assert iters[p] == r["iters"], p
        assert nbt[p] == int(r["n_bt"].sum()), p
        ref = r["x"]
        err = np.linalg.norm(x[p] - ref)
        assert err <= 2e-4 * max(np.linalg.norm(ref), 1e-6), (p, err)
        assert np.array_equal(x[p] != 0, ref != 0), p
        checked += 1
    assert checked >= (28 if k <= 3 else 22), checked


def test_split_grid_solve_refit_4d(api, grid4d):
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    res = api.solve(op, torch.from_numpy(grid4d.g).cuda(), grid4d.lam)
    ref = _exact(A, grid4d.g, grid4d.lam)
    cert = _check_minimiser(res, ref, 48)
    assert cert.mean() >= 0.9, cert.mean()


@pytest.mark.parametrize("L", [1025, 4096])
def test_split_grid_solve_refit_elevation(api, L):
    """Elevation-only grids past 1024 points: the refit's Toeplitz Gram path with the
    split-grid iterations."""
    st = _wide_elevation(L)
    A = oracle.operator(st.geom)
    op = api.Operator.from_geometry(st.geom)
    res = api.solve(op, torch.from_numpy(st.g).cuda(), st.lam)
    ref = _exact(A, st.g, st.lam)
    cert = _check_minimiser(res, ref, 40)
    assert cert.mean() >= 0.9, cert.mean()


def test_split_grid_deterministic(api, grid4d):
    op = api.Operator.from_geometry(grid4d.geom)
    g = torch.from_numpy(np.concatenate([grid4d.g] * 8)).cuda()  # 512 pixels: slots refill
    r1 = api.solve(op, g, grid4d.lam, max_iter=80)
    r2 = api.solve(op, g, grid4d.lam, max_iter=80)
    torch.cuda.synchronize()
    assert torch.equal(r1.status, r2.status) and torch.equal(r1.iters, r2.iters)
    assert torch.equal(torch.view_as_real(r1.x), torch.view_as_real(r2.x))
    # the eight copies of a pixel got the same bits whichever slot and CTA ran them
    x = torch.view_as_real(r1.x).reshape(8, 64, -1)
    assert all(torch.equal(x[0], x[i]) for i in range(1, 8))


def test_split_grid_edges(api, grid4d):
    from paper_1805_01759_gb300 import _lib
    op = api.Operator.from_geometry(grid4d.geom)
    G = grid4d.g[:7].copy()  # not a multiple of the CTA's four slots
    G[2, 5] = np.nan
    lam = np.full(7, grid4d.lam, np.float32)
    lam[4] = 1e5  # zero solution at the first iteration
    g = torch.from_numpy(G).cuda()
    res = api.solve(op, g, torch.from_numpy(lam).cuda(), max_iter=50, refit=0)
    x = res.x.cpu().numpy()
    st = res.status.cpu().numpy()
    it = res.iters.cpu().numpy()
    assert st[2] == 4 and it[2] == 0 and np.all(x[2] == 0)
    assert np.all(x[4] == 0) and it[4] == 1 and (st[4] & 32)
    ok = np.ones(7, bool)
    ok[2] = False
    assert np.all(np.isfinite(x[ok])) and np.all(it[ok] >= 1)
    # no pixels; no iterations
    assert api.solve(op, g[:0], grid4d.lam).x.shape == (0, 16384)
    r0 = api.solve(op, g[3:6], grid4d.lam, max_iter=0, refit=0)
    assert torch.all(r0.x == 0) and torch.all(r0.iters == 0) and torch.all(r0.status == 33)
    # options the split-grid kernel does not take are refused before any launch
    for bad in (dict(precision=1, tile_pixels=16), dict(tile_pixels=16), dict(blocks=2), dict(kernel=1)):
        with pytest.raises(_lib.BPDNError) as e:
            api.solve(op, g, grid4d.lam, **bad)
        assert e.value.code == _lib.BPDN_ESIZE, bad
    # the ragged batch runs such a stack in its own launch: bpdn_solve's results bit for bit,
    # next to a stack of the batch launch
    small = synth.workload_small(P=40, seed=5)
    op_s = api.Operator.from_geometry(small.geom)
    g_s = torch.from_numpy(small.g).cuda()
    gg = torch.from_numpy(grid4d.g[:9]).cuda()
    out = api.solve_ragged([(op_s, g_s, small.lam), (op, gg, grid4d.lam)])
    refs = [api.solve(op_s, g_s, small.lam), api.solve(op, gg, grid4d.lam)]
    torch.cuda.synchronize()
    for r, e in zip(out, refs):
        assert torch.equal(torch.view_as_real(r.x), torch.view_as_real(e.x))
        assert torch.equal(r.status, e.status) and torch.equal(r.iters, e.iters)


def _max_stack():
    """The library's largest sizes: N = 80 acquisitions on the 4-D grid 64 x 32 x 32 =
    65,536 points (BPDN_MAX_N, BPDN_MAX_L), 12 pixels."""
    rng = np.random.default_rng(11)
    N = 80
    b = rng.uniform(-250.0, 250.0, N)
    t = rng.uniform(0.0, 4.0, N)
    eta = np.stack([2.0 * t / 0.031, 2.0 * np.sin(2.0 * np.pi * t) / 0.031])
    geom = synth.MotionGeometry(b, 0.031, 7.0e5, -100.0, 100.0, 64, eta=eta, p_min=np.array([-0.02, -0.01]),
                                p_max=np.array([0.02, 0.01]), L_p=np.array([32, 32]))
    return synth.make_stack_md(geom, 12, rng, lam=synth.default_lambda(N, geom.L_total))


def test_split_grid_maximum_sizes(api):
    from paper_1805_01759_gb300 import _lib
    st = _max_stack()
    A = oracle.operator_md(st.geom)
    op = api.Operator.from_geometry(st.geom)
    assert (op.N, op.L) == (_lib.MAX_N, _lib.MAX_L) == A.shape
    g = torch.from_numpy(st.g).cuda()
    for k, need in ((1, 5), (3, 3)):
        res = api.solve(op, g, st.lam, max_iter=k, tol=0.0, refit=0)
        x = res.x.cpu().numpy()
        checked = 0
        for p in range(12):
            r = oracle.rbpg(A, st.g[p], st.lam, max_iter=k, tol=0.0, trace=True)
            if np.min(r["margin"]) < 1e-5:
                continue
            assert int(res.iters[p]) == r["iters"], (k, p)
            assert np.linalg.norm(x[p] - r["x"]) <= 2e-4 * max(np.linalg.norm(r["x"]), 1e-6), (k, p)
            assert np.array_equal(x[p] != 0, r["x"] != 0), (k, p)
            checked += 1
        assert checked >= need, (k, checked)
    res = api.solve(op, g, st.lam)
    ref = _exact(A, st.g, st.lam)
    cert = _check_minimiser(res, ref, 10)
    assert cert.sum() >= 11, cert


def test_split_grid_adjoint(api, grid4d):
    """dL/dg and dL/dlambda through the adjoint on the 16,384-point grid, against the
    oracle's adjoint of its own minimiser (pixels with a slack dual margin and the oracle's
    support), to 1e-3 relative."""
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    P = 32
    g = torch.from_numpy(grid4d.g[:P]).cuda()
    res = api.solve(op, g, grid4d.lam)
    rng = np.random.default_rng(21)
    c = rng.standard_normal((P, op.L)) + 1j * rng.standard_normal((P, op.L))
    lam = torch.full((P,), grid4d.lam, dtype=torch.float32, device="cuda")
    dg, dl = api.backward(op, res.x, res.support, res.nsupp, torch.from_numpy(c.astype(np.complex64)).cuda(), lam,
                          status=res.status)
    torch.cuda.synchronize()
    ref = _exact(A, grid4d.g[:P], grid4d.lam)
    r = oracle.adjoint_batch(A, np.full(P, grid4d.lam), ref["x"], c)
    x = res.x.cpu().numpy()
    cert = (res.status.cpu().numpy() & 64) != 0
    dg, dl = dg.cpu().numpy(), dl.cpu().numpy()
    checked = 0
    for p in range(P):
        if not cert[p] or ref["flags"][p] != 0 or ref["margin"][p] < 1e-3 or r["flags"][p] != 0:
            continue
        if not np.array_equal(x[p] != 0, ref["x"][p] != 0):
            continue
        scale = max(np.linalg.norm(r["dLdg"][p]), 1e-12)
        assert np.linalg.norm(dg[p] - r["dLdg"][p]) <= 1e-3 * scale, p
        assert abs(dl[p] - r["dLdlam"][p]) <= 1e-3 * max(abs(r["dLdlam"][p]), 1e-9 * scale), p
        checked += 1
    assert checked >= 16, checked


@pytest.mark.parametrize("k", [1, 3])
def test_split_grid_bf16_first_iterations(api, grid4d, k):
    """The tensor-core split-grid kernel on the 16,384-point grid against the oracle's
    Algorithm 1 with the same BF16 operands, element by element (2e-4), on pixels with no
    decision (including the bfloat16 rounding of a residual entry) within 1e-5 of its
    boundary."""
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    g = torch.from_numpy(grid4d.g).cuda()
    res = api.solve(op, g, grid4d.lam, max_iter=k, tol=0.0, refit=0, precision=1)
    x = res.x.cpu().numpy()
    iters = res.iters.cpu().numpy()
    checked = 0
    for p in range(grid4d.g.shape[0]):
        r = oracle.rbpg(A, grid4d.g[p], grid4d.lam, max_iter=k, tol=0.0, trace=True, bf16_operands=True)
        if np.min(r["margin"]) < 1e-5:
            continue
        assert iters[p] == r["iters"], p
        ref = r["x"]
        assert np.linalg.norm(x[p] - ref) <= 2e-4 * max(np.linalg.norm(ref), 1e-6), p
        assert np.array_equal(x[p] != 0, ref != 0), p
        checked += 1
    assert checked >= 12, checked


def test_split_grid_bf16_solve_refit_4d(api, grid4d):
    """BF16 (tol 1e-3) on the tensor-core split-grid kernel, then the FP64 refit: the exact
    minimiser on every certified, non-degenerate pixel."""
    A = oracle.operator_md(grid4d.geom)
    op = api.Operator.from_geometry(grid4d.geom)
    res = api.solve(op, torch.from_numpy(grid4d.g).cuda(), grid4d.lam, precision=1, tol=1e-3)
    ref = _exact(A, grid4d.g, grid4d.lam)
    cert = _check_minimiser(res, ref, 48)
    assert cert.mean() >= 0.9, cert.mean()
