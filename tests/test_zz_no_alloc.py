"""fmm_eval_static: the evaluation for callers that cannot allocate device
memory when they evaluate (a plugin whose host application owns all device
memory through its own allocator or pool, real-time loops that must not
allocate inside the time step).  Its scratch is a 32 MiB static device array
instead of a caller workspace; its results must match fmm_eval's on the same
inputs, call after call, since every call reuses (and must re-clear) the same
array, and the calls must leave the device's free memory unchanged.

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
    # on the host: a device-side conversion would allocate device memory
    a = a.cpu().double().numpy()
    b = b.cpu().double().numpy()
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
    outs = [(torch.full((n,), float("nan"), device="cuda"),
             torch.full((1,), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((n, 3), float("nan"), device="cuda")) for _ in range(3)]
    torch.cuda.synchronize()
    free0 = None
    for call, (phi, E, F) in enumerate(outs):
        if call == 1:  # after the first call's one-time set-up
            free0 = torch.cuda.mem_get_info()[0]
        rc = L.fmm_eval_static(plan._h, n, _p(P), _p(Q), _p(phi), _p(E), _p(F), stream)
        assert rc == B.FMM_OK, B.fmm_strerror(rc)
        torch.cuda.synchronize()
        assert _rel(phi, ref["potential"]) < TOL_FP32, call
        assert _rel(F, ref["forces"]) < TOL_FP32, call
        assert abs(E.item() - ref["energy"].item()) <= TOL_FP32 * abs(ref["energy"].item()), call
    assert torch.cuda.mem_get_info()[0] == free0  # the calls allocated no device memory
    plan.close()


def test_eval_static_status_without_waiting():
    """With opts.sync = 0 the call returns after queueing; the status of the
    scratch array is read afterwards through fmm_status with no workspace."""
    pos, q, box = inputs.uniform_cont(5000, 79)
    n = len(q)
    plan = FMM(box, 4, 4, continuous=True, split_ratio=1 / 32, max_n=n, sync=False)
    ref = {k: v.clone() for k, v in plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()).items()}
    P = torch.from_numpy(pos).cuda()
    Q = torch.from_numpy(q).cuda()
    phi = torch.empty(n, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = B.lib()
    assert L.fmm_eval_static(plan._h, n, _p(P), _p(Q), _p(phi), None, None, stream) == B.FMM_OK
    assert L.fmm_status(plan._h, None, stream) == B.FMM_OK
    assert _rel(phi, ref["potential"]) < TOL_FP32
    # a position outside the open box: the device status says so, read later
    P[0, 0] = 2.0
    assert L.fmm_eval_static(plan._h, n, _p(P), _p(Q), _p(phi), None, None, stream) == B.FMM_OK
    assert L.fmm_status(plan._h, None, stream) == B.FMM_ERR_OUT_OF_BOX
    plan.close()


def test_eval_static_rejects_another_devices_plan():
    """The plan's tables live on the device it was created on; a call with
    another device current is refused before any device work."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no other device to make current")
    pos, q, box = inputs.uniform_cont(1000, 80)
    plan = FMM(box, 3, 4, max_n=1000)
    with torch.cuda.device(1):
        P = torch.from_numpy(pos).cuda()
        Q = torch.from_numpy(q).cuda()
        phi = torch.empty(1000, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = B.lib().fmm_eval_static(plan._h, 1000, _p(P), _p(Q), _p(phi), None, None, stream)
        assert rc == B.FMM_ERR_ARG
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
