"""App. A.2 (bilinear forms without shifts) on the GPU against the oracle.

The plan precomputes the forms BB_{C~,o} = shift_{S->C~}^T K_o shift_{S->C}
on the device from the closed form of shift_{S->C} (stored as their right
parts K_o shift_{S->C}, the common left factor applied once per target); the
oracle applies the three factors one pair after the other, with shift_{S->C}
obtained by inverting shift_{C->S}.  Both run in FP64 and round differently
inside factors whose entries grow like 2^{l(p-1)}: the outputs agree to that
conditioning (measured 1e-12 at depth 3, order 4; 1e-9 at order 5), not to
the 1e-11 of the shifted FP64 plans.  The integer work and the box-basis
grid charges (sums of box weights, no extrapolation) keep the FP64
tolerance.  The box-basis functionals L^S are not compared: most of their
directions are nearly invisible inside the cell they serve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2212_13080_gb300 import FMM, FmmError, fmm_energy, inputs  # noqa: E402
from paper_2212_13080_gb300 import _binding as B  # noqa: E402

TOL_FP64 = 1e-11
# outputs of the shift-free form (FP64 on both sides, forms of conditioning
# ~2^{2l(p-1)}), relative L2 / relative energy
TOL_SF = {(2, 3): 1e-12, (4, 3): 1e-10, (3, 4): 2e-11, (3, 5): 2e-8}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    # name, generator, depth, p, periodic, continuous, dt
    ("uniform4k-open-plain-d3-p4", lambda: inputs.uniform_pm1(4096, 1), 3, 4, False, False, None),
    ("uniform20k-open-cont-d3-p4", lambda: inputs.uniform_cont(20000, 5), 3, 4, False, True, 1 / 32),
    ("water3k-periodic-cont-d3-p5", lambda: inputs.water(1001, 3), 3, 5, True, True, 1 / 16),
    ("uniform5k-periodic-plain-d2-p3", lambda: inputs.uniform_pm1(5000, 9), 2, 3, True, False, None),
    ("uniform30k-open-plain-d4-p3", lambda: inputs.uniform_pm1(30000, 13), 4, 3, False, False, None),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_shift_free(case):
    name, gen, depth, p, periodic, cont, dt = case
    pos, q, box = gen()
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, dt=dt,
                     shift_free=True)
    std = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, dt=dt,
                     keep=False)
    plan = FMM(box, depth, p, periodic=periodic, continuous=cont, split_ratio=dt, precision="fp64",
               max_n=len(q), shift_free=True)
    r = plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in r.items()}
    # integer work as in every plan
    assert int(plan.dump("counts")[1]) == ref["n_points"]
    np.testing.assert_array_equal(plan.dump("perm"), ref["perm"])
    np.testing.assert_array_equal(plan.dump("start"), ref["start"])
    # box-basis grid charges of every level: sums of box weights
    Phi = plan.dump("phi").reshape(-1)
    for l in range(0 if periodic else 2, depth + 1):
        a, b = oracle.level_offset(p, l), oracle.level_offset(p, l + 1)
        assert _rel(Phi[a:b], ref["Phi"][a:b]) < 10 * TOL_FP64, ("Phi^S", l)
    tol = TOL_SF[(depth, p)]
    e = dict(phi=_rel(out["potential"], ref["phi"]), F=_rel(out["forces"], ref["F"]),
             E=abs(out["energy"][0] - ref["E"]) / abs(ref["E"]),
             phi_std=_rel(out["potential"], std["phi"]), F_std=_rel(out["forces"], std["F"]))
    assert max(e.values()) < tol, e
    plan.close()


def test_shift_free_backward_and_repeat():
    """fmm_backward of a shift-free plan (far force from the box weights'
    derivatives) matches the oracle's adjoint forces and potentials; a second
    evaluation on the same plan reproduces the first bit for bit."""
    pos, q, box = inputs.water(800, 17)
    ref = oracle.fmm(pos, q, box, depth=3, n=4, periodic=True, continuous=True, dt=1 / 16,
                     shift_free=True)
    plan = FMM(box, 3, 4, periodic=True, continuous=True, split_ratio=1 / 16, precision="fp64",
               max_n=len(q), shift_free=True)
    P = torch.from_numpy(pos).cuda().requires_grad_(True)
    Q = torch.from_numpy(q).cuda().requires_grad_(True)
    E = fmm_energy(plan, P, Q)
    (2.0 * E).backward()
    tol = 5 * TOL_SF[(3, 4)]  # periodic: lists from level 1 on
    assert abs(E.item() - ref["E"]) < tol * abs(ref["E"])
    tol = max(tol, 2e-7)  # gradients come back in the inputs' float32
    assert _rel(P.grad.cpu().numpy().astype(np.float64), -2.0 * ref["F"]) < tol
    assert _rel(Q.grad.cpu().numpy().astype(np.float64), 2.0 * ref["phi"]) < tol
    a = plan.eval(P.detach(), Q.detach())["potential"].clone()
    b = plan.eval(P.detach(), Q.detach())["potential"]
    assert torch.equal(a, b)
    plan.close()


def test_shift_free_rejections():
    box = (0, 0, 0, 1)
    for kw in (dict(precision="fp32"), dict(precision="tf32x3")):
        with pytest.raises(FmmError) as e:
            FMM(box, 3, 4, shift_free=True, max_n=100, **kw)
        assert e.value.code == B.FMM_ERR_UNSUPPORTED
    with pytest.raises(FmmError) as e:
        FMM(box, 2, 6, shift_free=True, precision="fp64", max_n=100)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED
