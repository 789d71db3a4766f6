"""The multi-component operator of Eq. 4 (bpdn_make_operator_md: elevation x linear-velocity
grid) through the whole path, against the FP64 oracle on the same operator.

A^H A is not Toeplitz in one index on such a grid, so the refit and the adjoint form Gram
entries from the FP64 operator; these tests cover exactly that path.  Same bars as the
elevation-only tests: operator tables to FP64/FP32 rounding, the certified solution equal
to the exact minimiser (identical support, relative error <= 1e-4), the adjoint equal to
the oracle's adjoint on pixels with a slack dual margin.
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


def _rel(a, b):
    nb = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)


@pytest.mark.parametrize("L_s,L_v,precision", [(64, 16, 0), (32, 16, 1)])
def test_motion_operator_solve_refit(api, L_s, L_v, precision):
    st = synth.workload_motion(P=96, seed=7, L_s=L_s, L_v=L_v)
    A = oracle.operator_md(st.geom)
    op = api.Operator.from_geometry(st.geom)
    assert op.L == L_s * L_v == A.shape[1]
    np.testing.assert_allclose(op.export("A64").cpu().numpy(), A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.export("A").cpu().numpy(), A, rtol=0, atol=2e-7)
    ref = oracle.minimise_batch(A, st.g, st.lam)
    res = api.solve(op, torch.from_numpy(st.g).cuda(), st.lam, precision=precision,
                    tol=1e-3 if precision else 1e-6)
    x = res.x.cpu().numpy().astype(np.complex128)
    cert = (res.status.cpu().numpy() & 64) != 0
    assert cert.mean() >= 0.9, cert.mean()
    degenerate = (ref["margin"] < 1e-6) | ((ref["nS"] > 0) & (ref["min_abs_on"] < 1e-6 * np.abs(ref["x"]).max(1)))
    sel = cert & ~degenerate & (ref["flags"] == 0)
    assert sel.sum() >= 60, sel.sum()
    assert np.array_equal(x[sel] != 0, ref["x"][sel] != 0)
    assert _rel(x[sel], ref["x"][sel]).max() <= 1e-4


def test_motion_operator_backward(api):
    st = synth.workload_motion(P=64, seed=8, L_s=32, L_v=16)
    A = oracle.operator_md(st.geom)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    res = api.solve(op, g, st.lam)
    rng = np.random.default_rng(9)
    c = rng.standard_normal((64, op.L)) + 1j * rng.standard_normal((64, op.L))
    lam = torch.full((64,), st.lam, dtype=torch.float32, device="cuda")
    dg, dl = api.backward(op, res.x, res.support, res.nsupp, torch.from_numpy(c.astype(np.complex64)).cuda(), lam,
                          status=res.status)
    torch.cuda.synchronize()
    ref = oracle.minimise_batch(A, st.g, st.lam)
    r = oracle.adjoint_batch(A, np.full(64, st.lam), ref["x"], c)
    rdg, rdl, flags = r["dLdg"], r["dLdlam"], r["flags"]
    x = res.x.cpu().numpy()
    cert = (res.status.cpu().numpy() & 64) != 0
    dg, dl = dg.cpu().numpy(), dl.cpu().numpy()
    checked = 0
    for p in range(64):
        if not cert[p] or ref["flags"][p] != 0 or ref["margin"][p] < 1e-3 or flags[p] != 0:
            continue
        if not np.array_equal(x[p] != 0, ref["x"][p] != 0):
            continue
        scale = max(np.linalg.norm(rdg[p]), 1e-12)
        assert np.linalg.norm(dg[p] - rdg[p]) <= 1e-3 * scale, p
        assert abs(dl[p] - rdl[p]) <= 1e-3 * max(abs(rdl[p]), 1e-9 * scale), p
        checked += 1
    assert checked >= 32, checked


def test_motion_operator_refusals(api):
    from paper_1805_01759_gb300 import _lib
    st = synth.workload_motion(P=8, seed=7, L_s=16, L_v=4)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    res = api.solve(op, g, st.lam)
    with pytest.raises(_lib.BPDNError) as e:
        api.select(op, g, res)
    assert e.value.code == _lib.BPDN_EINVAL
    with pytest.raises(_lib.BPDNError):
        op.export("h")
    # a grid larger than the library's maximum is refused before any launch
    big = synth.MotionGeometry(st.geom.baselines_m, 0.031, 7e5, -100.0, 100.0, 1024, eta=st.geom.eta,
                               p_min=st.geom.p_min, p_max=st.geom.p_max, L_p=np.array([65]))
    with pytest.raises(_lib.BPDNError) as e:
        api.Operator.from_geometry(big)
    assert e.value.code == _lib.BPDN_ESIZE
