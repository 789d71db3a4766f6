"""Adjoint of the minimiser (bpdn_backward, through the C ABI) against the FP64 oracle.

The oracle differentiates its own exact minimiser; the GPU differentiates its own
certified solution.  Both see the same seeded g, lambda and upstream gradient c.
Compared on certified pixels whose support equals the oracle's and whose dual margin
is at least 1e-3 (the support is then locally constant, the premise of the adjoint).

Tolerance: the GPU builds J from x stored in complex64 (relative rounding 6e-8 per
entry) and returns FP32 derivatives; a relative perturbation e of J changes
v = J^{-1} c by at most about cond(J) e.  The test computes cond(J) from the oracle's
minimiser and requires ||d_gpu - d_oracle|| <= (1e-6 cond(J) + 1e-5) ||d_oracle||.
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
def case(api):
    st = synth.workload_small(P=256, seed=1)
    A = oracle.operator(st.geom)
    ref = oracle.minimise_batch(A, st.g, st.lam)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    res = api.solve(op, g, st.lam)
    torch.cuda.synchronize()
    rng = np.random.default_rng(55)
    c = (rng.standard_normal((st.g.shape[0], st.geom.L)) + 1j * rng.standard_normal((st.g.shape[0], st.geom.L)))
    return st, A, ref, op, g, res, c


def _cond_J(A, lam, x):
    """Condition number of the real Jacobian of the optimality system on supp(x)."""
    S = np.nonzero(x)[0]
    if S.size == 0:
        return 1.0
    G = A[:, S].conj().T @ A[:, S]
    m = S.size
    J = np.zeros((2 * m, 2 * m))
    J[0::2, 0::2] = 2 * G.real
    J[0::2, 1::2] = -2 * G.imag
    J[1::2, 0::2] = 2 * G.imag
    J[1::2, 1::2] = 2 * G.real
    for i, l in enumerate(S):
        u = np.array([x[l].real, x[l].imag]) / abs(x[l])
        J[2 * i:2 * i + 2, 2 * i:2 * i + 2] += lam / abs(x[l]) * (np.eye(2) - np.outer(u, u))
    return float(np.linalg.cond(J))


def test_backward_matches_oracle(api, case):
    st, A, ref, op, g, res, c = case
    P = st.g.shape[0]
    lam_pp = torch.full((P,), st.lam, dtype=torch.float32, device="cuda")
    dg, dl = api.backward(op, res.x, res.support, res.nsupp, torch.from_numpy(c.astype(np.complex64)).cuda(), lam_pp)
    torch.cuda.synchronize()
    dg, dl = dg.cpu().numpy(), dl.cpu().numpy()
    x = res.x.cpu().numpy()
    status = res.status.cpu().numpy()
    oref = oracle.adjoint_batch(A, st.lam, ref["x"], c.astype(np.complex64).astype(np.complex128))
    checked = 0
    for p in range(P):
        if not (status[p] & 64) or ref["margin"][p] < 1e-3:
            continue
        if not np.array_equal(x[p] != 0, ref["x"][p] != 0) or oref["flags"][p]:
            continue
        if ref["nS"][p] > 0 and ref["min_abs_on"][p] < 1e-3 * np.abs(ref["x"][p]).max():
            continue
        kappa = _cond_J(A, st.lam, ref["x"][p])
        tol = 1e-6 * kappa + 1e-5
        dref = oref["dLdg"][p]
        scale = max(np.linalg.norm(dref), 1e-30)
        assert np.linalg.norm(dg[p] - dref) <= tol * scale, (p, kappa)
        lref = oref["dLdlam"][p]
        assert abs(dl[p] - lref) <= tol * max(abs(lref), scale * np.abs(ref["x"][p]).max() / st.lam), (p, kappa)
        if ref["nS"][p] == 0:
            assert np.all(dg[p] == 0) and dl[p] == 0
        checked += 1
    assert checked >= 150


def test_backward_shared_lambda_is_fixed_order_sum(api, case):
    st, A, ref, op, g, res, c = case
    P = st.g.shape[0]
    ct = torch.from_numpy(c.astype(np.complex64)).cuda()
    lam1 = torch.tensor([st.lam], dtype=torch.float32, device="cuda")
    lam_pp = lam1.expand(P).contiguous()
    dg1, dl1 = api.backward(op, res.x, res.support, res.nsupp, ct, lam1)
    dg2, dl2 = api.backward(op, res.x, res.support, res.nsupp, ct, lam_pp)
    dg3, dl3 = api.backward(op, res.x, res.support, res.nsupp, ct, lam1)
    torch.cuda.synchronize()
    assert dl1.shape == (1,) and dl2.shape == (P,)
    assert torch.equal(dg1, dg2) and torch.equal(dg1, dg3) and torch.equal(dl1, dl3)
    per = dl2.double().cpu().numpy()
    assert abs(float(dl1.item()) - per.sum()) <= 1e-6 * np.abs(per).sum() + 1e-30


def test_backward_edges(api, case):
    st, A, ref, op, g, res, c = case
    from paper_1805_01759_gb300 import _lib
    lam1 = torch.tensor([st.lam], dtype=torch.float32, device="cuda")
    # no pixels
    x0 = torch.empty((0, st.geom.L), dtype=torch.complex64, device="cuda")
    s0 = torch.empty((0, 16), dtype=torch.int32, device="cuda")
    n0 = torch.empty(0, dtype=torch.int32, device="cuda")
    dg, dl = api.backward(op, x0, s0, n0, x0, lam1)
    torch.cuda.synchronize()
    assert dg.shape == (0, st.geom.N) and float(dl.item()) == 0.0
    # uncertified pixels get zero derivatives when the status is passed
    ct = torch.from_numpy(c.astype(np.complex64)).cuda()
    st_unc = res.status & ~64
    dgu, dlu = api.backward(op, res.x, res.support, res.nsupp, ct, lam1, status=st_unc)
    torch.cuda.synchronize()
    assert torch.all(dgu == 0) and float(dlu.item()) == 0.0
    # empty supports and supports naming zero entries give zero derivatives
    P = 8
    x = torch.zeros((P, st.geom.L), dtype=torch.complex64, device="cuda")
    sup = torch.full((P, 16), -1, dtype=torch.int32, device="cuda")
    sup[:, 0] = 5
    nsupp = torch.tensor([0, 1, 1, 1, 20, -3, 1, 1], dtype=torch.int32, device="cuda")
    dg, dl = api.backward(op, x, sup, nsupp, torch.ones_like(x), lam1.expand(P).contiguous())
    torch.cuda.synchronize()
    assert torch.all(dg == 0) and torch.all(dl == 0)
    # bad s_max is refused on the host
    lib = _lib.load()
    rc = lib.bpdn_backward(op.handle, P, lam1.data_ptr(), 0, x.data_ptr(), sup.data_ptr(), nsupp.data_ptr(), None, 33,
                           x.data_ptr(), dg.data_ptr(), dl.data_ptr(), None, 0, None)
    assert rc == _lib.BPDN_EINVAL


def test_autograd_function_and_lambda_tuning(api):
    st = synth.workload_diff(P=4096, seed=5)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda().requires_grad_(True)
    lam = torch.tensor([st.lam], dtype=torch.float32, device="cuda", requires_grad=True)
    x, status = api.BPDNFunction.apply(g, lam, op, None)
    gt = torch.from_numpy(st.gamma_true).cuda()
    loss = (x - gt).abs().pow(2).mean()
    loss.backward()
    # the same derivatives straight from the C ABI
    res = api.solve(op, g.detach(), lam.detach())
    gx = 2 * (res.x - gt) / (x.shape[0] * x.shape[1])
    dg, dl = api.backward(op, res.x, res.support, res.nsupp, gx, lam.detach(), status=res.status)
    torch.cuda.synchronize()
    assert torch.allclose(g.grad, dg, rtol=1e-5, atol=1e-12) and torch.allclose(lam.grad, dl, rtol=1e-5)
    # d(error)/d(lambda) of the whole batch against a central difference of the forward map,
    # at 1.5 times the default weight (supports small and strict on nearly every pixel).
    # The sum runs over the pixels certified at all three weights: elsewhere x is the last
    # iterate of Algorithm 1, whose changes with lambda the adjoint does not describe.
    gd = g.detach()
    lam0 = 1.5 * st.lam
    eps = 1e-3
    rp = api.solve(op, gd, lam0 * (1 + eps))
    rm = api.solve(op, gd, lam0 * (1 - eps))
    r0 = api.solve(op, gd, lam0)
    keep = (((rp.status & rm.status & r0.status) & 64) != 0).unsqueeze(1).to(torch.float32)
    den = gt.abs().pow(2).sum()

    def masked_err(xx):
        return ((xx - gt).abs().pow(2) * keep).sum() / den

    lt = torch.tensor([lam0], dtype=torch.float32, device="cuda", requires_grad=True)
    xt, _ = api.BPDNFunction.apply(gd, lt, op, None)
    (d,) = torch.autograd.grad(masked_err(xt), lt)
    fd = (masked_err(rp.x).item() - masked_err(rm.x).item()) / (2 * eps * lam0)
    assert keep.mean().item() > 0.9
    assert abs(d.item() - fd) <= 0.05 * abs(fd), (d.item(), fd)
    # gradient descent on log lambda (first step 0.1 in log lambda) lowers the error
    lr = 0.1 / abs(d.item() * lam0)
    lam_end, hist = api.tune_lambda(op, gd, gt, lam0, steps=5, lr=lr)
    assert min(h[1] for h in hist[1:]) < hist[0][1], hist
    # from half the default weight (supports larger than the truth's, where the implicit
    # gradient misses the support jumps) the line search still descends
    lam_end, hist = api.tune_lambda(op, gd, gt, 0.5 * st.lam, steps=5, lr=lr)
    errs = np.array([h[1] for h in hist])
    assert np.all(np.diff(errs) <= 1e-7 * errs[:-1]) and errs[-1] < errs[0], hist


@pytest.mark.parametrize("N,k", [(32, 16), (64, 32)])
def test_backward_full_support(api, N, k):
    """k nonzeros: 16 (the fast refit's and the fast adjoint's capacity) and 32 (the largest
    support the library handles: the refit's wide pass and the adjoint's wide kernel, each
    unknown pair of lanes then holding two of the 64 real unknowns).  Orthogonal columns (DFT
    geometry), lambda between the k-th and (k+1)-th largest |2 a_l^H g|."""
    rng = np.random.default_rng(77 + k)
    geom = synth.dft_geometry(N)
    A = oracle.operator(geom)
    P = 16
    G = (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N))).astype(np.complex64)
    lam_v = np.empty(P, np.float32)
    for p in range(P):
        w = np.sort(np.abs(2 * A.conj().T @ G[p].astype(np.complex128)))[::-1]
        lam_v[p] = np.float32(0.5 * (w[k - 1] + w[k]))
    op = api.Operator.from_geometry(geom)
    lam_t = torch.from_numpy(lam_v).cuda()
    res = api.solve(op, torch.from_numpy(G).cuda(), lam_t)
    c = (rng.standard_normal((P, N)) + 1j * rng.standard_normal((P, N)))
    dg, dl = api.backward(op, res.x, res.support, res.nsupp, torch.from_numpy(c.astype(np.complex64)).cuda(),
                          lam_t, status=res.status)
    torch.cuda.synchronize()
    assert torch.all(res.nsupp == k) and torch.all((res.status & 64) != 0)
    dg, dl = dg.cpu().numpy(), dl.cpu().numpy()
    for p in range(P):
        xs = oracle.minimise(A, G[p].astype(np.complex128), float(lam_v[p]))["x"]
        rg, rl, rc = oracle.adjoint(A, float(lam_v[p]), xs, c[p].astype(np.complex64).astype(np.complex128))
        assert rc == 0
        assert np.linalg.norm(dg[p] - rg) <= 1e-4 * np.linalg.norm(rg)
        assert abs(dl[p] - rl) <= 1e-4 * max(abs(rl), 1e-6)
