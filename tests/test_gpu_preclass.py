"""Pre-classification (bpdn_classify, bpdn_classify_merge) against the oracle's classifier
(oracle/preclass.py, FP64) and against the full L1 chain.

Tolerances: the classes must be equal wherever neither decision ratio 2 max|A^H g|/lambda,
2 max|A^H r|/lambda lies within 1e-9 of 1 (both sides decide in FP64); for class 1 the
elevation within 2e-6 m (the oracle's derivative-free search resolves the flat beam peak
to ~1e-7 m, the kernel's Newton iteration to ~1e-12 m) and the amplitude within 1e-5
relative (its sensitivity to the elevation is 2 pi max|xi| ~ 0.15 per metre)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import preclass as opc
from paper_1805_01759_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1805_01759_gb300 import api as _api
    return _api


def _oracle_classes(st, idx=None):
    A = oracle.operator(st.geom)
    xi = oracle.xi(st.geom.baselines_m, st.geom.wavelength_m, st.geom.range_m)
    s = oracle.grid(st.geom.s_min_m, st.geom.s_max_m, st.geom.L)
    G = st.g if idx is None else st.g[idx]
    return A, opc.classify_batch(A, xi, s, G.astype(np.complex128), st.lam)


def _compare(c, ref, idx):
    cls = c.cls.cpu().numpy()[idx]
    sh = c.sel.s_hat.cpu().numpy()[idx, 0]
    gh = c.sel.gamma_hat.cpu().numpy()[idx, 0]
    kh = c.sel.khat.cpu().numpy()[idx]
    tie = (np.abs(ref["umax"] - 1.0) < 1e-9) | (np.abs(np.nan_to_num(ref["rmax"], nan=0.0) - 1.0) < 1e-9)
    ok = ~tie
    assert np.array_equal(cls[ok], ref["cls"][ok])
    assert np.array_equal(kh[ok], np.where(ref["cls"][ok] == 2, -1, ref["cls"][ok]))
    one = ok & (ref["cls"] == 1)
    assert np.all(np.abs(sh[one] - ref["s_hat"][one]) < 2e-6), np.abs(sh[one] - ref["s_hat"][one]).max()
    assert np.all(np.abs(gh[one] - ref["gamma_hat"][one]) <= 1e-5 * np.abs(ref["gamma_hat"][one]))
    assert np.all(np.isnan(sh[ok & (ref["cls"] != 1)]))
    return cls


def test_classes_match_the_oracle_small(api):
    st = synth.workload_small(P=256, seed=1)
    op = api.Operator.from_geometry(st.geom)
    c = api.classify(op, torch.from_numpy(st.g).cuda(), st.lam)
    torch.cuda.synchronize()
    A, ref = _oracle_classes(st)
    cls = _compare(c, ref, np.arange(256))
    # all three classes occur on this workload (K = 0, 1, 2 at 10 dB)
    assert np.all(np.bincount(cls, minlength=3) >= 10), np.bincount(cls, minlength=3)


def test_classes_match_the_oracle_patch_sample(api):
    P = 1 << 16
    st = synth.workload_patch(P=P, seed=2)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    c = api.classify(op, g, st.lam)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(7).choice(P, 512, replace=False))
    A, ref = _oracle_classes(st, idx)
    _compare(c, ref, idx)
    # the compaction lists exactly the class-2 pixels, with their measurements
    n = int(c.count.item())
    cls = c.cls.cpu().numpy()
    lst = c.idx[:n].cpu().numpy()
    assert n == int((cls == 2).sum()) and np.array_equal(np.sort(lst), np.flatnonzero(cls == 2))
    assert torch.equal(c.g_compact[:n], g[c.idx[:n]])


def test_class_zero_is_the_zero_solution(api):
    """Every class-0 pixel's L1 solution is exactly zero, and every pixel whose L1 solution is
    the certified zero vector is class 0 (the screen is exact for Eq. 6)."""
    st = synth.workload_small(P=256, seed=3)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    c = api.classify(op, g, st.lam)
    res = api.solve(op, g, st.lam)
    torch.cuda.synchronize()
    cls = c.cls.cpu().numpy()
    st_ = res.status.cpu().numpy()
    zero = np.all(res.x.cpu().numpy() == 0, axis=1)
    assert np.all(zero[cls == 0])
    cert_zero = zero & ((st_ & 64) != 0)
    assert np.all(cls[cert_zero] == 0)


def test_hybrid_chain_equals_the_l1_chain_on_class_two(api):
    """The merged selection: classes 0 and 1 from the classifier, class 2 exactly what the
    full L1 chain (solve with refit + select on every pixel) gives those pixels."""
    st = synth.workload_small(P=256, seed=1)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    c, sel, res_c = api.hybrid(op, g, st.lam, precision=0)
    full = api.solve(op, g, st.lam, precision=0)
    fsel = api.select(op, g, full)
    torch.cuda.synchronize()
    cls = c.cls.cpu().numpy()
    two = cls == 2
    assert torch.equal(sel.khat[torch.from_numpy(two).cuda()], fsel.khat[torch.from_numpy(two).cuda()])
    s_h, fs_h = sel.s_hat.cpu().numpy(), fsel.s_hat.cpu().numpy()
    assert np.array_equal(np.nan_to_num(s_h[two], nan=-1e9), np.nan_to_num(fs_h[two], nan=-1e9))
    assert np.array_equal(sel.khat.cpu().numpy()[~two], cls[~two])
    # the compact solve's rows are the full solve's rows of the same pixels
    n = int(c.count.item())
    assert torch.equal(res_c.x, full.x[c.idx[:n]])


def test_edges(api):
    st = synth.workload_small(P=40, seed=1)
    op = api.Operator.from_geometry(st.geom)
    G = st.g.copy()
    G[3, 2] = np.nan
    g = torch.from_numpy(G).cuda()
    lam = np.full(40, st.lam, np.float32)
    lam[5] = 1e6
    c = api.classify(op, g, torch.from_numpy(lam).cuda(), kmax=1)
    torch.cuda.synchronize()
    cls = c.cls.cpu().numpy()
    assert cls[3] == 2 and cls[5] == 0
    # no pixels
    c0 = api.classify(op, g[:0], st.lam)
    assert int(c0.count.item()) == 0
    from paper_1805_01759_gb300 import _lib
    with pytest.raises(_lib.BPDNError):
        api.classify(op, g, st.lam, kmax=5)
    geom = synth.workload_motion(P=4, L_s=16, L_v=4).geom
    op_md = api.Operator.from_geometry(geom)
    with pytest.raises(_lib.BPDNError):
        api.classify(op_md, torch.zeros((4, op_md.N), dtype=torch.complex64, device="cuda"), 1.0)
