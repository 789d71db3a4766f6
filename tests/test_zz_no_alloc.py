"""bpdn_solve_noalloc: the solve for callers that may not allocate device memory.

Such callers (for example a module inside a processing chain whose host
application owns every GPU buffer) pass only the inputs and outputs they already
hold; the solver's scratch lives in a fixed device array inside the library.
This test calls the entry point through the C ABI twice in a row and checks each
result against bpdn_solve with a caller-provided workspace: same status and
iteration counts, and x within the relative tolerance the parity tests use (1e-4).
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_01759_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_workspace_solve_twice():
    lib = _lib.load()
    st = synth.workload_small(P=256, seed=1)
    op = api.Operator.from_geometry(st.geom)
    g = torch.from_numpy(st.g).cuda()
    lam = torch.tensor([st.lam], dtype=torch.float32, device="cuda")
    ref = api.solve(op, g, lam)
    torch.cuda.synchronize()
    x_ref = ref.x.cpu().numpy()
    opt = _lib.default_options()
    P, L = st.g.shape[0], op.L
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.full((P, L), float("nan"), dtype=torch.complex64, device="cuda")
        status = torch.zeros(P, dtype=torch.int32, device="cuda")
        iters = torch.empty(P, dtype=torch.int32, device="cuda")
        nbt = torch.empty(P, dtype=torch.int32, device="cuda")
        nsupp = torch.empty(P, dtype=torch.int32, device="cuda")
        support = torch.empty((P, opt.s_max), dtype=torch.int32, device="cuda")
        rc = lib.bpdn_solve_noalloc(op.handle, g.data_ptr(), P, lam.data_ptr(), 0, ctypes.byref(opt),
                                    x.data_ptr(), support.data_ptr(), nsupp.data_ptr(),
                                    status.data_ptr(), iters.data_ptr(), nbt.data_ptr(), stream)
        assert rc == 0, lib.bpdn_last_error()
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        assert np.all(np.isfinite(xs)), call
        assert np.array_equal(status.cpu().numpy(), ref.status.cpu().numpy()), call
        assert np.array_equal(iters.cpu().numpy(), ref.iters.cpu().numpy()), call
        nr = np.linalg.norm(x_ref, axis=1)
        err = np.linalg.norm(xs - x_ref, axis=1) / np.where(nr > 0, nr, 1.0)
        assert err.max() <= 1e-4, (call, err.max())
        assert np.array_equal(xs != 0, x_ref != 0), call
