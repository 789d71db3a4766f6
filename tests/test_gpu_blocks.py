"""Algorithm 1 with randomized blocks of a pixel's grid (options.blocks >= 2, Eqs. 13-14),
through the C ABI, against the FP64 oracle of the same reading.

Both sides draw the blocks from SplitMix64 started at seed + pixel * 2^40 with Eq. 14's
probabilities (the GPU computes them from its FP64 operator, the oracle with LAPACK; they
agree to ~1e-13, so the draws coincide), so the trajectories are comparable iterate by
iterate.  FP32 against FP64 after a few block iterations: pixels whose discrete decisions
(accept, Eq. 15, the small-step test) all agree end with the same iteration count; on those
the relative error must stay within 2e-4 (the bar of the FP32 trajectory test of the
default reading).  The whole path (blocks + refit) must produce the exact minimiser on
every certified pixel.
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
def small(api):
    st = synth.workload_small(P=256, seed=1)
    op = api.Operator.from_geometry(st.geom)
    return st, op, torch.from_numpy(st.g).cuda(), oracle.operator(st.geom)


def _rel(a, b):
    nb = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)


@pytest.mark.parametrize("epochs", [1, 2, 5])
def test_block_trajectory_matches_oracle(api, small, epochs):
    st, op, g, A = small
    J, seed = 4, 3
    res = api.solve(op, g, st.lam, blocks=J, seed=seed, refit=0, max_iter=epochs, tol=1e-6)
    torch.cuda.synchronize()
    ref = oracle.rbpg_block_batch(A, st.g, st.lam, J, seed, tol=1e-6, max_iter=epochs)
    it = res.iters.cpu().numpy()
    same = it == ref["iters"]
    assert same.mean() >= 0.9, same.mean()
    err = _rel(res.x.cpu().numpy().astype(np.complex128)[same], ref["x"][same])
    assert np.median(err) <= 1e-5, np.median(err)
    assert (err <= 2e-4).mean() >= 0.95, np.sort(err)[-10:]


def test_block_solve_with_refit_is_exact_where_certified(api, small):
    st, op, g, A = small
    res = api.solve(op, g, st.lam, blocks=4, seed=3, tol=1e-6)
    torch.cuda.synchronize()
    ref = oracle.minimise_batch(A, st.g, st.lam)
    x = res.x.cpu().numpy().astype(np.complex128)
    cert = (res.status.cpu().numpy() & 64) != 0
    degenerate = (ref["margin"] < 1e-6) | ((ref["nS"] > 0) & (ref["min_abs_on"] < 1e-6 * np.abs(ref["x"]).max(1)))
    sel = cert & ~degenerate & (ref["flags"] == 0)
    assert cert.mean() >= 0.5, cert.mean()
    assert np.array_equal(x[sel] != 0, ref["x"][sel] != 0)
    assert _rel(x[sel], ref["x"][sel]).max() <= 1e-4


def test_block_solve_is_deterministic(api, small):
    st, op, g, A = small
    a = api.solve(op, g, st.lam, blocks=3, seed=11, tol=1e-6)
    b = api.solve(op, g, st.lam, blocks=3, seed=11, tol=1e-6)
    c = api.solve(op, g, st.lam, blocks=3, seed=12, tol=1e-6, refit=0)
    torch.cuda.synchronize()
    assert torch.equal(a.x, b.x) and torch.equal(a.iters, b.iters) and torch.equal(a.status, b.status)
    assert not torch.equal(a.iters, c.iters)  # another seed draws other blocks


def test_block_option_checks(api, small):
    from paper_1805_01759_gb300 import _lib
    st, op, g, A = small
    with pytest.raises(_lib.BPDNError) as e:
        api.solve(op, g, st.lam, blocks=4, precision=1)
    assert e.value.code == _lib.BPDN_EINVAL
    with pytest.raises(_lib.BPDNError) as e:
        api.solve(op, g, st.lam, blocks=9)
    assert e.value.code == _lib.BPDN_EINVAL
    with pytest.raises(_lib.BPDNError) as e:
        api.solve_ragged([(op, g, st.lam)], blocks=4)
    assert e.value.code == _lib.BPDN_EINVAL
    tiny = api.Operator.from_geometry(synth.make_geometry(np.random.default_rng(0), 8, 3, 100.0, 10.0))
    with pytest.raises(_lib.BPDNError) as e:
        api.solve(tiny, torch.zeros((4, 8), dtype=torch.complex64, device="cuda"), 1.0, blocks=4)
    assert e.value.code == _lib.BPDN_ESIZE
    # the no-allocation entry has 256 bytes of scratch: block draws need more
    lib = _lib.load()
    opt = _lib.default_options(blocks=4)
    P = 4
    x = torch.empty((P, op.L), dtype=torch.complex64, device="cuda")
    ints = [torch.empty(P, dtype=torch.int32, device="cuda") for _ in range(4)]
    lam = torch.tensor([st.lam], dtype=torch.float32, device="cuda")
    import ctypes
    rc = lib.bpdn_solve_noalloc(op.handle, g.data_ptr(), P, lam.data_ptr(), 0, ctypes.byref(opt), x.data_ptr(),
                                None, ints[0].data_ptr(), ints[1].data_ptr(), ints[2].data_ptr(),
                                ints[3].data_ptr(), None)
    assert rc == _lib.BPDN_ESIZE
