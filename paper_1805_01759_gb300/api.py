"""Python API over libbpdn: torch tensors supply device memory and streams.

    op = Operator(baselines_m, wavelength_m, range_m, s_min_m, s_max_m, L)
    res = solve(op, g, lam)            # g: complex64 [P, N] on the GPU
    res.x, res.status, res.iters, ...

Only argument marshalling happens here; every step of the solve runs in the CUDA
library.
"""
from __future__ import annotations

import contextlib
import ctypes
import math
import dataclasses
from typing import NamedTuple

import numpy as np
import torch

from . import _lib


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream: torch.cuda.Stream | None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


@contextlib.contextmanager
def _launch_on(stream: torch.cuda.Stream | None, *inputs):
    """Make `stream` the current stream for one call's allocations and launches.

    When `stream` is not the caller's current stream, it first waits for the work queued
    on the current stream (which produced the inputs), the input tensors are recorded as
    used on `stream` (so the caching allocator does not hand their memory to new work
    before the launch has read them), and every temporary (workspace, lambda, contiguous
    copies) is allocated while `stream` is current, so that it is only reused after the
    kernels that read it."""
    if stream is None:
        yield
        return
    cur = torch.cuda.current_stream(stream.device)
    if stream == cur:
        yield
        return
    stream.wait_stream(cur)
    for t in inputs:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            t.record_stream(stream)
    with torch.cuda.stream(stream):
        yield


class Operator:
    """The steering operator of one stack (Eq. 5), resident on the current GPU."""

    def __init__(self, baselines_m, wavelength_m: float, range_m: float, s_min_m: float,
                 s_max_m: float, L: int, *, motion=None, device: torch.device | str | None = None,
                 stream: torch.cuda.Stream | None = None):
        """motion: None (elevation only, Eq. 5) or (eta [M, N], p_min [M], p_max [M], L_p [M]) for
        the multi-component grid of Eq. 4 (bpdn_make_operator_md); L is then the number of
        elevation points and self.L the size of the whole grid."""
        lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        b = np.ascontiguousarray(baselines_m, dtype=np.float64)
        self.N, self.Ls = int(b.size), int(L)
        self.L = self.Ls
        if motion is not None:
            eta = np.ascontiguousarray(motion[0], dtype=np.float64).reshape(-1, self.N)
            pmin = np.ascontiguousarray(motion[1], dtype=np.float64).reshape(-1)
            pmax = np.ascontiguousarray(motion[2], dtype=np.float64).reshape(-1)
            Lp = np.ascontiguousarray(motion[3], dtype=np.int32).reshape(-1)
            self.L = self.Ls * int(np.prod(Lp))
        nbytes = lib.bpdn_op_workspace_bytes(self.N, self.L)
        if nbytes == 0:
            raise _lib.BPDNError(-3, f"N = {self.N}, L = {self.L} outside the supported range")
        dp = ctypes.POINTER(ctypes.c_double)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            if motion is None:
                _lib.check(lib.bpdn_make_operator(
                    b.ctypes.data_as(dp), self.N, float(wavelength_m), float(range_m), float(s_min_m),
                    float(s_max_m), self.L, self.workspace.data_ptr(), nbytes, _stream(stream), ctypes.byref(h)))
            else:
                _lib.check(lib.bpdn_make_operator_md(
                    b.ctypes.data_as(dp), self.N, float(wavelength_m), float(range_m), float(s_min_m),
                    float(s_max_m), self.Ls, int(eta.shape[0]), eta.ctypes.data_as(dp), pmin.ctypes.data_as(dp),
                    pmax.ctypes.data_as(dp), Lp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    self.workspace.data_ptr(), nbytes, _stream(stream), ctypes.byref(h)))
        self._h = h
        self.baselines_m = b
        self.wavelength_m, self.range_m = float(wavelength_m), float(range_m)
        self.s_min_m, self.s_max_m = float(s_min_m), float(s_max_m)
        N, Lc, ds, lip = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
        _lib.check(lib.bpdn_op_info(self._h, ctypes.byref(N), ctypes.byref(Lc), ctypes.byref(ds),
                                    ctypes.byref(lip)))
        self.ds_m, self.lipschitz = ds.value, lip.value

    @classmethod
    def from_geometry(cls, geom, **kw) -> "Operator":
        motion = getattr(geom, "motion", None)
        return cls(geom.baselines_m, geom.wavelength_m, geom.range_m, geom.s_min_m, geom.s_max_m,
                   geom.L, motion=motion() if callable(motion) else motion, **kw)

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def export(self, what: str) -> torch.Tensor:
        """Device tables: 'A' (complex64 N x L), 'A64', 'h' (complex128 2L-1), 'AAH'."""
        code, shape, dt = {"A": (0, (self.N, self.L), torch.complex64),
                           "A64": (1, (self.N, self.L), torch.complex128),
                           "h": (2, (2 * self.L - 1,), torch.complex128),
                           "AAH": (3, (self.N, self.N), torch.complex128)}[what]
        out = torch.empty(shape, dtype=dt, device=self.device)
        _lib.check(_lib.load().bpdn_op_export(self._h, code, out.data_ptr(),
                                              out.numel() * out.element_size(), _stream(None)))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib.load().bpdn_destroy_operator(h)
            except Exception:  # pragma: no cover - interpreter shutdown
                pass
            self._h = ctypes.c_void_p()


@dataclasses.dataclass
class SolveResult:
    x: torch.Tensor          # complex64 [P, L]
    status: torch.Tensor     # int32 [P]
    iters: torch.Tensor      # int32 [P]
    nbt: torch.Tensor        # int32 [P]
    nsupp: torch.Tensor      # int32 [P]
    support: torch.Tensor | None  # int32 [P, s_max]


def _lambda_tensor(lam, P: int, device) -> tuple[torch.Tensor, int]:
    if isinstance(lam, torch.Tensor):
        t = lam.to(device=device, dtype=torch.float32).contiguous()
        if t.numel() == 1:
            return t.reshape(1), 0
        if t.numel() != P:
            raise ValueError("lambda must have 1 or P entries")
        return t.reshape(P), 1
    return torch.tensor([float(lam)], dtype=torch.float32, device=device), 0


def _check_g(op: Operator, g: torch.Tensor) -> torch.Tensor:
    if g.dtype != torch.complex64 or g.device.type != "cuda":
        raise TypeError("g must be a complex64 CUDA tensor")
    if g.dim() != 2 or g.shape[1] != op.N:
        raise ValueError(f"g must be [P, {op.N}]")
    return g.contiguous()


def solve(op: Operator, g: torch.Tensor, lam, *, out: SolveResult | None = None,
          stream: torch.cuda.Stream | None = None, **options) -> SolveResult:
    """Algorithm 1 (+ the FP64 refit unless refit=0) for every row of g."""
    with _launch_on(stream, g, lam):
        return _solve(op, g, lam, out, stream, **options)


def _solve(op, g, lam, out, stream, **options) -> SolveResult:
    lib = _lib.load()
    g = _check_g(op, g)
    P = g.shape[0]
    opt = _lib.default_options(**options)
    lam_t, pp = _lambda_tensor(lam, P, g.device)
    dev = g.device
    if out is None:
        out = SolveResult(
            x=torch.empty((P, op.L), dtype=torch.complex64, device=dev),
            status=torch.empty(P, dtype=torch.int32, device=dev),
            iters=torch.empty(P, dtype=torch.int32, device=dev),
            nbt=torch.empty(P, dtype=torch.int32, device=dev),
            nsupp=torch.empty(P, dtype=torch.int32, device=dev),
            support=(torch.empty((P, opt.s_max), dtype=torch.int32, device=dev) if opt.refit else None),
        )
    ws_bytes = lib.bpdn_solve_workspace_bytes(op.handle, P, ctypes.byref(opt))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    _lib.check(lib.bpdn_solve(op.handle, g.data_ptr(), P, lam_t.data_ptr(), pp, ctypes.byref(opt),
                              out.x.data_ptr(), _ptr(out.support), _ptr(out.nsupp),
                              out.status.data_ptr(), out.iters.data_ptr(), _ptr(out.nbt),
                              ws.data_ptr(), ws_bytes, _stream(stream)))
    out._keepalive = (ws, lam_t, g)  # type: ignore[attr-defined]
    return out


def refit(op: Operator, g: torch.Tensor, lam, x_in: torch.Tensor, *, status: torch.Tensor | None = None,
          stream: torch.cuda.Stream | None = None, **options):
    """Support extraction + FP64 refit of x_in on its own.  Returns (x, support, nsupp, status)."""
    with _launch_on(stream, g, lam, x_in, status):
        return _refit(op, g, lam, x_in, status, stream, **options)


def _refit(op, g, lam, x_in, status, stream, **options):
    lib = _lib.load()
    g = _check_g(op, g)
    P = g.shape[0]
    opt = _lib.default_options(**options)
    lam_t, pp = _lambda_tensor(lam, P, g.device)
    x_in = x_in.contiguous()
    x = torch.empty_like(x_in)
    support = torch.empty((P, opt.s_max), dtype=torch.int32, device=g.device)
    nsupp = torch.empty(P, dtype=torch.int32, device=g.device)
    st = torch.zeros(P, dtype=torch.int32, device=g.device) if status is None else status.clone()
    ws_bytes = lib.bpdn_refit_workspace_bytes(op.handle, P)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=g.device)
    _lib.check(lib.bpdn_refit(op.handle, g.data_ptr(), P, lam_t.data_ptr(), pp, ctypes.byref(opt),
                              x_in.data_ptr(), x.data_ptr(), support.data_ptr(), nsupp.data_ptr(),
                              st.data_ptr(), ws.data_ptr() if ws_bytes else None, ws_bytes, _stream(stream)))
    return x, support, nsupp, st


def backward(op: Operator, x: torch.Tensor, support: torch.Tensor, nsupp: torch.Tensor,
             dLdx: torch.Tensor, lam, *, status: torch.Tensor | None = None,
             stream: torch.cuda.Stream | None = None):
    """Adjoint of the minimiser (bpdn_backward): (dL/dg [P, N] complex64, dL/dlambda).

    dL/dlambda has P entries when lam has P entries, else one (the sum over pixels).
    With status given, pixels the solve did not certify get zero derivatives."""
    with _launch_on(stream, x, support, nsupp, dLdx, lam, status):
        return _backward(op, x, support, nsupp, dLdx, lam, status, stream)


def _backward(op, x, support, nsupp, dLdx, lam, status, stream):
    lib = _lib.load()
    if x.dtype != torch.complex64 or x.device.type != "cuda" or x.dim() != 2 or x.shape[1] != op.L:
        raise TypeError(f"x must be a complex64 CUDA tensor [P, {op.L}]")
    P = x.shape[0]
    dev = x.device
    x = x.contiguous()
    dLdx = dLdx.to(dtype=torch.complex64).contiguous()
    support = support.to(dtype=torch.int32).contiguous()
    nsupp = nsupp.to(dtype=torch.int32).contiguous()
    if dLdx.shape != x.shape or support.dim() != 2 or support.shape[0] != P or nsupp.shape != (P,):
        raise ValueError("dL/dx, support and nsupp must match x")
    lam_t, pp = _lambda_tensor(lam, P, dev)
    if status is not None:
        status = status.to(dtype=torch.int32).contiguous()
        if status.shape != (P,):
            raise ValueError("status must have P entries")
    dLdg = torch.empty((P, op.N), dtype=torch.complex64, device=dev)
    dLdlam = torch.empty(P if pp else 1, dtype=torch.float32, device=dev)
    ws_bytes = 0 if pp else lib.bpdn_backward_workspace_bytes(op.handle, P)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    _lib.check(lib.bpdn_backward(op.handle, P, lam_t.data_ptr(), pp, x.data_ptr(), support.data_ptr(),
                                 nsupp.data_ptr(), _ptr(status), support.shape[1], dLdx.data_ptr(), dLdg.data_ptr(),
                                 dLdlam.data_ptr(), ws.data_ptr() if ws_bytes else None, ws_bytes,
                                 _stream(stream)))
    return dLdg, dLdlam


class Selection(NamedTuple):
    """Output of select(): khat [P] int32 (-1: not selected), s_hat [P, kmax] float64
    (NaN past khat), gamma_hat [P, kmax] complex128 (0 past khat)."""
    khat: torch.Tensor
    s_hat: torch.Tensor
    gamma_hat: torch.Tensor


def select(op: Operator, g: torch.Tensor, res: "SolveResult", *, kmax: int = _lib.MAX_KSEL,
           penalty: float = 0.0, stream: torch.cuda.Stream | None = None) -> Selection:
    """SL1MMER model selection and parameter estimation (bpdn_select) on a solve's result
    (which must come from a solve with the refit, so that its support is written)."""
    with _launch_on(stream, g, res.x, res.support, res.nsupp, res.status):
        return _select(op, g, res, kmax, penalty, stream)


def _select(op, g, res, kmax, penalty, stream) -> Selection:
    lib = _lib.load()
    g = _check_g(op, g)
    P = g.shape[0]
    if res.support is None:
        raise ValueError("select needs the support of a solve with refit")
    if res.x.shape != (P, op.L) or res.support.shape[0] != P:
        raise ValueError("the solve result does not match g")
    dev = g.device
    out = Selection(torch.empty(P, dtype=torch.int32, device=dev),
                    torch.empty((P, kmax), dtype=torch.float64, device=dev),
                    torch.empty((P, kmax), dtype=torch.complex128, device=dev))
    _lib.check(lib.bpdn_select(op.handle, g.data_ptr(), P, res.x.data_ptr(), res.support.data_ptr(),
                               res.nsupp.data_ptr(), _ptr(res.status), res.support.shape[1], kmax,
                               float(penalty), out.khat.data_ptr(), out.s_hat.data_ptr(),
                               out.gamma_hat.data_ptr(), _stream(stream)))
    return out


class Classes(NamedTuple):
    """Output of classify(): cls [P] int32 (0 no scatterer, 1 one scatterer by the linear
    estimator, 2 left to L1), the estimates of classes 0 and 1 in the layout of select()
    (khat -1 for class 2), and the class-2 pixels: idx [P] int64 of which the first `count`
    are valid, g_compact [P, N] their measurements in the same order."""
    cls: torch.Tensor
    sel: "Selection"
    idx: torch.Tensor
    count: torch.Tensor
    g_compact: torch.Tensor


def classify(op: Operator, g: torch.Tensor, lam, *, kmax: int = _lib.MAX_KSEL,
             stream: torch.cuda.Stream | None = None) -> Classes:
    """Pre-classification before the L1 solve (bpdn_classify)."""
    with _launch_on(stream, g, lam):
        lib = _lib.load()
        g = _check_g(op, g)
        P = g.shape[0]
        dev = g.device
        lam_t, pp = _lambda_tensor(lam, P, dev)
        out = Classes(torch.empty(P, dtype=torch.int32, device=dev),
                      Selection(torch.empty(P, dtype=torch.int32, device=dev),
                                torch.empty((P, kmax), dtype=torch.float64, device=dev),
                                torch.empty((P, kmax), dtype=torch.complex128, device=dev)),
                      torch.empty(P, dtype=torch.int64, device=dev),
                      torch.empty(1, dtype=torch.int64, device=dev),
                      torch.empty((P, op.N), dtype=torch.complex64, device=dev))
        _lib.check(lib.bpdn_classify(op.handle, g.data_ptr(), P, lam_t.data_ptr(), pp, kmax, out.cls.data_ptr(),
                                     out.sel.khat.data_ptr(), out.sel.s_hat.data_ptr(), out.sel.gamma_hat.data_ptr(),
                                     out.idx.data_ptr(), out.count.data_ptr(), out.g_compact.data_ptr(),
                                     _stream(stream)))
        return out


def hybrid(op: Operator, g: torch.Tensor, lam, *, kmax: int = _lib.MAX_KSEL, penalty: float = 0.0,
           **options):
    """The pre-classified chain: bpdn_classify, then for the class-2 pixels only bpdn_solve
    (with the refit) and bpdn_select, merged back by bpdn_classify_merge.  Reads the class-2
    count back to the host once (to size the L1 batch).  Returns (Classes, Selection over all
    pixels, SolveResult of the class-2 pixels in Classes.idx order)."""
    lib = _lib.load()
    c = classify(op, g, lam, kmax=kmax)
    n = int(c.count.item())
    sel = Selection(c.sel.khat.clone(), c.sel.s_hat.clone(), c.sel.gamma_hat.clone())
    if n == 0:
        return c, sel, None
    P = g.shape[0]
    if isinstance(lam, torch.Tensor) and lam.numel() == P:
        lam_c = lam.to(device=g.device, dtype=torch.float32).reshape(P)[c.idx[:n]]
    else:
        lam_c = lam
    gc = c.g_compact[:n]
    res = solve(op, gc, lam_c, refit=1, **options)
    sc = select(op, gc, res, kmax=kmax, penalty=penalty)
    _lib.check(lib.bpdn_classify_merge(n, c.idx.data_ptr(), kmax, sc.khat.data_ptr(), sc.s_hat.data_ptr(),
                                       sc.gamma_hat.data_ptr(), sel.khat.data_ptr(), sel.s_hat.data_ptr(),
                                       sel.gamma_hat.data_ptr(), _stream(None)))
    return c, sel, res


class BPDNFunction(torch.autograd.Function):
    """x = argmin ||A x - g||^2 + lambda ||x||_1 (Eq. 6) per pixel as a differentiable map of
    (g, lambda): forward = bpdn_solve with the refit, backward = bpdn_backward (zero
    derivatives on pixels the refit did not certify).

    Usage: x = BPDNFunction.apply(g, lam, op, options) with g complex64 [P, N] and lam a
    float32 tensor of 1 or P entries; options is a dict of solve options (or None)."""

    @staticmethod
    def forward(ctx, g, lam, op, options=None):
        opts = dict(options or {})
        opts["refit"] = 1
        lam_d = lam.detach()
        res = solve(op, g.detach(), lam_d, **opts)
        ctx.op = op
        ctx.lam_shape = lam.shape
        ctx.save_for_backward(res.x, res.support, res.nsupp, res.status, lam_d)
        ctx.mark_non_differentiable(res.status)
        return res.x, res.status

    @staticmethod
    def backward(ctx, grad_x, grad_status):
        x, support, nsupp, status, lam_d = ctx.saved_tensors
        if grad_x is None:
            return None, None, None, None
        dLdg, dLdlam = backward(ctx.op, x, support, nsupp, grad_x, lam_d, status=status)
        return dLdg, dLdlam.reshape(ctx.lam_shape), None, None


def global_error_and_grad(num: float, den: float, dnum: float, group=None):
    """Sum (error numerator, its normaliser, d numerator / d log lambda) over the ranks of the
    default (or given) process group, when one is initialised, and return the batch's
    relative squared error and its derivative in log lambda.  This is the one collective of
    lambda tuning with pixels sharded over GPUs: two sums and a derivative, reduced in FP64."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
            else torch.device("cpu")
        v = torch.tensor([num, den, dnum], dtype=torch.float64, device=dev)
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
        num, den, dnum = (float(t) for t in v.cpu())
    den = max(den, 1e-30)
    return num / den, dnum / den


def tune_lambda(op: Operator, g: torch.Tensor, gamma_true: torch.Tensor, lam0: float, *,
                steps: int = 50, lr: float = 0.1, options: dict | None = None, group=None,
                line_search: bool = True):
    """Learn one lambda by gradient descent on log lambda, minimising the relative squared
    error sum |x(lambda) - gamma_true|^2 / sum |gamma_true|^2 over pixels and grid points.

    The direction is the implicit gradient (bpdn_backward), which covers the error's smooth
    part on fixed supports; the changes of support as lambda moves are jumps it does not see.
    With line_search (the default) a step is taken only where the error, evaluated by a
    forward solve, decreases: lr times the gradient, then half and a quarter of it; if none
    of these lowers the error, the implicit gradient is misled by support jumps and the step
    of the same length in the opposite direction is tried; if that fails too, lambda stays
    and lr is halved.  Every accepted step is thus a descent of the error itself.  Without
    line_search every step is lr times the gradient.

    Under torch.distributed (pixels sharded over ranks) every sum runs over every rank's
    pixels (global_error_and_grad), so all ranks take the same decisions and steps.
    Returns (lambda, [(lambda, error) per step])."""
    import torch.distributed as dist
    sharded = dist.is_available() and dist.is_initialized()
    den_local = gamma_true.abs().pow(2).sum()

    def error_and_grad(log_lam):
        lam = log_lam.exp()
        x, _ = BPDNFunction.apply(g, lam, op, options)
        num = (x - gamma_true).abs().pow(2).sum()
        (dnum,) = torch.autograd.grad(num, log_lam)
        return global_error_and_grad(float(num.item()), float(den_local.item()), float(dnum.item()),
                                     group if sharded else None)

    def error_at(v: float) -> float:
        with torch.no_grad():
            lam = torch.tensor([math.exp(v)], dtype=torch.float32, device=g.device)
            x, _ = BPDNFunction.apply(g, lam, op, options)
            num = (x - gamma_true).abs().pow(2).sum()
        return global_error_and_grad(float(num.item()), float(den_local.item()), 0.0,
                                     group if sharded else None)[0]

    log_lam = torch.tensor([math.log(lam0)], dtype=torch.float32, device=g.device, requires_grad=True)
    history = []
    for _ in range(steps):
        err, grad = error_and_grad(log_lam)
        cur = float(log_lam.item())
        history.append((math.exp(cur), err))
        step = -lr * grad
        if not line_search:
            nxt = cur + step
        else:
            nxt = None
            for cand in (cur + step, cur + 0.5 * step, cur + 0.25 * step, cur - step):
                if cand != cur and error_at(cand) < err:
                    nxt = cand
                    break
            if nxt is None:
                nxt = cur
                lr *= 0.5
        with torch.no_grad():
            log_lam.fill_(nxt)
    return float(log_lam.exp().item()), history


_TUNE_CACHE: dict = {}


def autotune_stack(op: Operator, g: torch.Tensor, lam, *, repeats: int = 2, **options):
    """Pick the iteration kernel and tile for this operator and batch by timing bpdn_solve
    on g itself: (kernel, tile_pixels) among the grid-point kernel with the library's number
    of slot groups, with 16 or with 8 pixels per CTA, and the split-grid kernel (CUDA cores in
    FP32, tensor cores with BF16).
    Cached by (N, L, precision, P);
    candidates the library refuses at these sizes are skipped.  Returns (0, 0), the
    library's own choice, when nothing could be timed."""
    P = g.shape[0]
    prec = int(options.get("precision", 0))
    key = (op.N, op.L, prec, P, int(options.get("blocks", 0)))
    if key in _TUNE_CACHE:
        return _TUNE_CACHE[key]
    cands = [(1, 0), (1, 16), (1, 8), (2, 0)]
    opts = {k: v for k, v in options.items() if k not in ("kernel", "tile_pixels")}
    best, best_ms = (0, 0), float("inf")
    for kern, tile in cands:
        try:
            solve(op, g, lam, kernel=kern, tile_pixels=tile, **opts)  # warm-up, and checks that it runs
        except _lib.BPDNError:
            continue
        ms = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            solve(op, g, lam, kernel=kern, tile_pixels=tile, **opts)
            e1.record()
            torch.cuda.synchronize()
            ms = min(ms, e0.elapsed_time(e1))
        if ms < best_ms:
            best, best_ms = (kern, tile), ms
    _TUNE_CACHE[key] = best
    return best


class RaggedSolver:
    """Many stacks, each with its own operator and pixel count, through bpdn_solve_ragged.

    items: list of (Operator, g [P_s, N_s] complex64 CUDA tensor, lambda); tiles and kernels
    (optional): each stack's tile_pixels and kernel options (0 = the options' value); with
    autotune=True each stack's (kernel, tile_pixels) is chosen by autotune_stack first.
    Outputs are allocated once (`results`, one SolveResult per stack).  run() launches on the
    current (or given) stream; capture() records one call into a CUDA graph and replay()
    relaunches it: the graph reads the same g tensors, so new data is copied into them."""

    def __init__(self, items, *, tiles=None, kernels=None, autotune: bool = False, **options):
        lib = _lib.load()
        self.opt = _lib.default_options(**options)
        if autotune:
            picks = [autotune_stack(op, _check_g(op, g), lam, **options) for op, g, lam in items]
            kernels = [k for k, _ in picks]
            tiles = [t for _, t in picks]
        self.tiles = [0] * len(items) if tiles is None else [int(t) for t in tiles]
        self.kernels = [0] * len(items) if kernels is None else [int(k) for k in kernels]
        if len(self.tiles) != len(items) or len(self.kernels) != len(items):
            raise ValueError("tiles and kernels must name one value per stack")
        self.items = []
        self.results = []
        self._keep = []
        arr = (_lib.Stack * len(items))()
        for i, (op, g, lam) in enumerate(items):
            g = _check_g(op, g)
            P = g.shape[0]
            dev = g.device
            lam_t, pp = _lambda_tensor(lam, P, dev)
            res = SolveResult(
                x=torch.empty((P, op.L), dtype=torch.complex64, device=dev),
                status=torch.empty(P, dtype=torch.int32, device=dev),
                iters=torch.empty(P, dtype=torch.int32, device=dev),
                nbt=torch.empty(P, dtype=torch.int32, device=dev),
                nsupp=torch.empty(P, dtype=torch.int32, device=dev),
                support=(torch.empty((P, self.opt.s_max), dtype=torch.int32, device=dev)
                         if self.opt.refit else None),
            )
            arr[i] = _lib.Stack(op.handle.value, g.data_ptr(), P, lam_t.data_ptr(), pp, res.x.data_ptr(),
                                _ptr(res.support), res.nsupp.data_ptr(), res.status.data_ptr(),
                                res.iters.data_ptr(), res.nbt.data_ptr(), self.tiles[i], self.kernels[i])
            self.items.append((op, g, lam_t))
            self.results.append(res)
        self._arr = arr
        # room for every stack's refit to run in three launches
        self.ws_bytes = lib.bpdn_solve_ragged_workspace_bytes_for(arr, len(items), ctypes.byref(self.opt))
        dev = self.items[0][1].device if self.items else torch.device("cuda")
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.graph = None

    def run(self, stream: torch.cuda.Stream | None = None) -> list:
        lib = _lib.load()
        _lib.check(lib.bpdn_solve_ragged(self._arr, len(self.items), ctypes.byref(self.opt),
                                         self.ws.data_ptr(), self.ws_bytes, _stream(stream)))
        return self.results

    def capture(self) -> "torch.cuda.CUDAGraph":
        self.run()  # the first call creates the library's streams outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run()
        self.graph = graph
        return graph

    def replay(self) -> list:
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()
        return self.results


def deal_stacks(costs, world: int) -> list:
    """Deal stacks to `world` ranks by estimated cost (e.g. P * N * L per stack): largest first,
    each to the rank with the least cost so far (ties: the lower rank).  Deterministic, so every
    rank computes the same dealing without communicating.  Returns the rank of each stack."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    rank_of = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        rank_of[i] = r
        load[r] += float(costs[i])
    return rank_of


def solve_ragged(items, *, stream: torch.cuda.Stream | None = None, **options) -> list:
    """Solve every (Operator, g, lambda) stack of `items` in one bpdn_solve_ragged call."""
    return RaggedSolver(items, **options).run(stream)


class HostSolver:
    """Solve pixels that live in (pinned) host memory, with the copies overlapped.

    The batch is cut into `chunks` pieces on two streams with two sets of device buffers:
    while one piece is solved, the next one's g is copied in and the previous one's x
    is copied out, so the transfers hide behind the solves.  Results go straight into
    the host tensors passed to run().  Two chunks are the default: the copies run at about
    200 GB/s, so one chunk's x (1.7 GB for half of 2^20 pixels at L = 400) hides behind the
    other's solve, while every further chunk adds the tails of its own launches (2^20
    pixels, N = 25, L = 400, BF16: 869 ms per step with 2 chunks, 913 with 8, 991 with 16,
    against 860 for the device-resident solve)."""

    def __init__(self, op: Operator, P: int, *, chunks: int = 2, device=None, **options):
        self.op = op
        self.P = P
        self.chunks = max(1, min(chunks, P)) if P else 1
        self.C = (P + self.chunks - 1) // self.chunks if P else 0
        self.options = options
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        opt = _lib.default_options(**options)
        C = max(self.C, 1)
        self.g = [torch.empty((C, op.N), dtype=torch.complex64, device=dev) for _ in range(2)]
        self.res = [SolveResult(
            x=torch.empty((C, op.L), dtype=torch.complex64, device=dev),
            status=torch.empty(C, dtype=torch.int32, device=dev),
            iters=torch.empty(C, dtype=torch.int32, device=dev),
            nbt=torch.empty(C, dtype=torch.int32, device=dev),
            nsupp=torch.empty(C, dtype=torch.int32, device=dev),
            support=(torch.empty((C, opt.s_max), dtype=torch.int32, device=dev) if opt.refit else None))
            for _ in range(2)]
        self.device = dev

    def run(self, g_host: torch.Tensor, lam, x_host: torch.Tensor, status_host: torch.Tensor) -> None:
        """g_host complex64 [P, N], x_host complex64 [P, L], status_host int32 [P] (pinned host
        tensors for overlap); lam a float or a [P] tensor.  Returns when every copy is queued;
        the caller synchronises the current stream before reading x_host."""
        if g_host.shape != (self.P, self.op.N) or x_host.shape != (self.P, self.op.L):
            raise ValueError("host tensors do not match the solver's P, N, L")
        cur = torch.cuda.current_stream(self.device)
        lam_pp = isinstance(lam, torch.Tensor) and lam.numel() == self.P
        lam_d = (lam.to(self.device, dtype=torch.float32, non_blocking=True).reshape(-1) if lam_pp
                 else _lambda_tensor(lam, self.P, self.device)[0])
        start = torch.cuda.Event()
        start.record(cur)
        for i in range(self.chunks):
            a, b = i * self.C, min(self.P, (i + 1) * self.C)
            if a >= b:
                break
            n = b - a
            k = i & 1
            s = self.streams[k]
            s.wait_event(start)
            with torch.cuda.stream(s):
                g = self.g[k][:n]
                g.copy_(g_host[a:b], non_blocking=True)
                r = self.res[k]
                out = SolveResult(x=r.x[:n], status=r.status[:n], iters=r.iters[:n], nbt=r.nbt[:n],
                                  nsupp=r.nsupp[:n], support=None if r.support is None else r.support[:n])
                solve(self.op, g, lam_d[a:b] if lam_pp else lam_d, out=out, stream=s, **self.options)
                x_host[a:b].copy_(out.x, non_blocking=True)
                status_host[a:b].copy_(out.status, non_blocking=True)
        for s in self.streams:
            ev = torch.cuda.Event()
            ev.record(s)
            cur.wait_event(ev)


def solve_host(op: Operator, g_host: torch.Tensor, lam, x_host: torch.Tensor, status_host: torch.Tensor,
               *, chunks: int = 2, **options) -> None:
    """One-shot HostSolver: solve the pixels of g_host into x_host / status_host."""
    HostSolver(op, g_host.shape[0], chunks=chunks, **options).run(g_host, lam, x_host, status_host)
