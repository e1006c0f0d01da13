"""fmm_eval_static: the evaluation for callers that cannot allocate device
memory when they evaluate (inside another framework's stream capture, in
real-time loops that forbid allocation, or with all device memory owned by a
pool).  Its scratch is a 32 MiB static device array instead of a caller
workspace; its results must match fmm_eval's on the same inputs, call after
call, since every call reuses (and must re-clear) the same array.

Collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_13080_gb300 import FMM, inputs  # noqa: E402
from paper_2212_13080_gb300 import _binding as B  # noqa: E402

TOL_FP32 = 1e-6


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_eval_static_matches_eval_on_two_calls():
    pos, q, box = inputs.uniform_cont(20000, 77)
    n = len(q)
    plan = FMM(box, 4, 4, continuous=True, split_ratio=1 / 32, max_n=n)
    assert plan.workspace_size(n) <= B.FMM_STATIC_WORKSPACE_BYTES
    P = torch.from_numpy(pos).cuda()
    Q = torch.from_numpy(q).cuda()
    ref = plan.eval(P, Q)
    ref = {k: v.clone() for k, v in ref.items()}
    L = B.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        phi = torch.full((n,), float("nan"), device="cuda")
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        F = torch.full((n, 3), float("nan"), device="cuda")
        rc = L.fmm_eval_static(plan._h, n, _p(P), _p(Q), _p(phi), _p(E), _p(F), stream)
        assert rc == B.FMM_OK, B.fmm_strerror(rc)
        torch.cuda.synchronize()
        assert _rel(phi, ref["potential"]) < TOL_FP32, call
        assert _rel(F, ref["forces"]) < TOL_FP32, call
        assert abs(E.item() - ref["energy"].item()) <= TOL_FP32 * abs(ref["energy"].item()), call
    plan.close()


def test_eval_static_rejects_too_large():
    pos, q, box = inputs.uniform_cont(1000, 78)
    plan = FMM(box, 6, 4, max_n=1 << 16)  # depth-6 grid charges alone exceed 32 MiB
    assert plan.workspace_size(1000) > B.FMM_STATIC_WORKSPACE_BYTES
    P = torch.from_numpy(pos).cuda()
    Q = torch.from_numpy(q).cuda()
    phi = torch.empty(1000, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = B.lib().fmm_eval_static(plan._h, 1000, _p(P), _p(Q), _p(phi), None, None, stream)
    assert rc == B.FMM_ERR_WORKSPACE
    plan.close()
