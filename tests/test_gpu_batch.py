"""Batched evaluation of many independent systems (own box, depth, count):
every system must equal its own single-system evaluation (same kernels, same
inputs), and the single-system path is pinned to the oracle elsewhere; a few
systems are also checked against the oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2212_13080_gb300 import FMM, FMMBatch, inputs  # noqa: E402


def _depths(counts):
    return np.clip(np.rint(np.log(counts / 32.0) / np.log(8.0)), 3, 5).astype(int)


@pytest.mark.parametrize("precision,schedule", [("fp32", -1), ("tf32x3", 0), ("tf32x3", 1), ("fp32", 1),
                                                 ("fp64", -1)])
def test_batch_matches_single_system(precision, schedule):
    """Single-precision plans run every launch site once for all systems
    (merged form; depths 3, 4 and 5 mixed, so that the systems' level loops
    and their scan and launch-order variants differ), in the schedule the
    autotuner picks (-1) or a fixed one: one stream (0), or the near field on
    a second stream (1), where each system's near field must still wait for
    its own sort although the merged order interleaves the systems' sort
    variants with the near-field launches; FP64 plans run as per-system
    pipelines on stream lanes."""
    pos, q, offs, boxes, counts = inputs.batch_systems(12, 7, lo=1024, hi=20000)
    boxes[3] = (0.25, -1.0, 2.0, 1.5)  # one system in another box
    pos[offs[3]:offs[4]] = (pos[offs[3]:offs[4]] * np.float32(1.5) +
                            np.array([0.25, -1.0, 2.0], np.float32)).astype(np.float32)
    depths = _depths(counts)
    depths[int(np.argmax(counts))] = 5  # sparse finest cells, 32,768 of them
    bt = FMMBatch(boxes, depths, 4, periodic=True, continuous=True, precision=precision,
                  max_n=counts)
    if schedule >= 0:
        bt.set_schedule(schedule)
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    for call in range(2):  # first call tunes and captures, second replays the graph
        r = bt.eval(P, Q, offs)
        torch.cuda.synchronize()
        st = bt.stats()
        if precision == "fp64":
            assert not st["merged"] and st["lanes"] in (2, 4, 8, 12, 16, 32) and st["launches"] > 12
        else:
            # one launch per call site (levels and variants included) plus the status kernel
            assert st["merged"] and st["lanes"] == 0 and st["schedule"] in ((0, 1) if schedule < 0 else (schedule,))
            assert 12 < st["launches"] < 80
        for i in range(len(counts)):
            a, b = offs[i], offs[i + 1]
            plan = FMM(boxes[i], int(depths[i]), 4, periodic=True, continuous=True,
                       precision=precision, max_n=int(counts[i]))
            s = plan.eval(P[a:b].contiguous(), Q[a:b].contiguous())
            assert torch.equal(r["potential"][a:b], s["potential"]), (call, i)
            assert torch.equal(r["forces"][a:b], s["forces"]), (call, i)
            assert r["energy"][i].item() == s["energy"].item(), (call, i)
            plan.close()
    bt.close()


def test_batch_against_oracle():
    pos, q, offs, boxes, counts = inputs.batch_systems(6, 11, lo=1024, hi=8000)
    depths = _depths(counts)
    bt = FMMBatch(boxes, depths, 4, periodic=True, continuous=True, precision="fp64", max_n=counts)
    r = bt.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda(), offs)
    for i in (0, 5):
        a, b = offs[i], offs[i + 1]
        ref = oracle.fmm(pos[a:b], q[a:b], boxes[i], depth=int(depths[i]), n=4, periodic=True,
                         continuous=True)
        phi = r["potential"][a:b].cpu().numpy()
        assert np.linalg.norm(phi - ref["phi"]) < 1e-11 * np.linalg.norm(ref["phi"])
        assert abs(r["energy"][i].item() - ref["E"]) < 1e-11 * abs(ref["E"])
    bt.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("periodic,kernel,force_mode", [(True, "coulomb", "kernel"),
                                                         (False, "inverse_square", "adjoint")])
def test_batch_other_kernels_match_single_system(periodic, kernel, force_mode, precision):
    """Force-kernel forces (§4.1) and the 1/r^2 kernel through the batched
    path: each system equals its own single-system evaluation bit for bit
    (the batched systems share their depth's tables, four kernel components
    for force-kernel plans; with the tensor cores, the small levels of all
    systems in shared cross-system tiles, from level 1 periodic or 2 open)."""
    pos, q, offs, boxes, counts = inputs.batch_systems(6, 17, lo=1024, hi=12000)
    depths = _depths(counts)
    bt = FMMBatch(boxes, depths, 4, periodic=periodic, continuous=True, precision=precision,
                  max_n=counts, kernel=kernel, force_mode=force_mode)
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    r = bt.eval(P, Q, offs)
    torch.cuda.synchronize()
    for i in range(len(counts)):
        a, b = offs[i], offs[i + 1]
        plan = FMM(boxes[i], int(depths[i]), 4, periodic=periodic, continuous=True, precision=precision,
                   max_n=int(counts[i]), kernel=kernel, force_mode=force_mode)
        s = plan.eval(P[a:b].contiguous(), Q[a:b].contiguous())
        assert torch.equal(r["potential"][a:b], s["potential"]), i
        assert torch.equal(r["forces"][a:b], s["forces"]), i
        assert r["energy"][i].item() == s["energy"].item(), i
        plan.close()
    bt.close()
