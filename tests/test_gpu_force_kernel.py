"""Far forces from the force kernels r/|r|^3 (§4.1, other kernels) on the GPU
against the oracle's same construction: three more functionals per cell
through the same interaction lists (periodic: the gradient of the lattice
term), read with the plain weights; a particle's force is the sum of its
charges' forces.  Potentials and energy are those of the default plans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2212_13080_gb300 import FMM, fmm_energy, inputs  # noqa: E402

TOL = {"fp64": 1e-11, "fp32": 1e-6, "tf32x3": 1e-5, "bf16x3": 1e-5}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # name, generator, depth, p, periodic, continuous, dt
    ("uniform4k-open-plain-d3-p4", lambda: inputs.uniform_pm1(4096, 1), 3, 4, False, False, None),
    ("uniform20k-open-cont-d4-p4", lambda: inputs.uniform_cont(20000, 5), 4, 4, False, True, 1 / 32),
    ("water3k-periodic-cont-d3-p5", lambda: inputs.water(1001, 3), 3, 5, True, True, 1 / 16),
    ("uniform30k-open-plain-d4-p6", lambda: inputs.uniform_pm1(30000, 34), 4, 6, False, False, None),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_force_kernel(case, precision):
    name, gen, depth, p, periodic, cont, dt = case
    if precision == "fp64" and p == 6:
        pytest.skip("covered by the smaller FP64 cases")
    pos, q, box = gen()
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, dt=dt,
                     force_kernel=True, keep=False)
    plan = FMM(box, depth, p, periodic=periodic, continuous=cont, split_ratio=dt,
               precision=precision, max_n=len(q), force_mode="kernel")
    r = plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    phi = r["potential"].cpu().numpy().astype(np.float64)
    F = r["forces"].cpu().numpy().astype(np.float64)
    E = r["energy"].item()
    tol = TOL[precision]
    assert _rel(phi, ref["phi"]) < tol
    assert _rel(F, ref["F"]) < tol, _rel(F, ref["F"])
    assert abs(E - ref["E"]) < tol * abs(ref["E"])
    # total momentum: zero up to the rounding of the forces themselves
    net = np.abs(F.sum(axis=0)).max() / np.abs(F).sum()
    assert net < (1e-13 if precision == "fp64" else 1e-6), net
    plan.close()


def test_force_kernel_backward_is_the_adjoint():
    """The backward pass of a force-kernel plan is still the gradient of the
    energy: -dE/dx from the weights' derivatives, not the kernel forces."""
    pos, q, box = inputs.water(800, 17)
    ref = oracle.fmm(pos, q, box, depth=3, n=5, periodic=True, continuous=True, dt=1 / 16)
    plan = FMM(box, 3, 5, periodic=True, continuous=True, split_ratio=1 / 16, precision="fp64",
               max_n=len(q), force_mode="kernel")
    P = torch.from_numpy(pos).cuda().requires_grad_(True)
    Q = torch.from_numpy(q).cuda().requires_grad_(True)
    E = fmm_energy(plan, P, Q)
    E.backward()
    assert abs(E.item() - ref["E"]) < 1e-11 * abs(ref["E"])
    assert _rel(P.grad.cpu().numpy().astype(np.float64), -ref["F"]) < 2e-7
    assert _rel(Q.grad.cpu().numpy().astype(np.float64), ref["phi"]) < 2e-7
    plan.close()


# --- the 1/r^2 kernel (§4.1, other functions) -------------------------------------

R2_CASES = [
    ("uniform4k-open-plain-d3-p4", lambda: inputs.uniform_pm1(4096, 1), 3, 4, False, None),
    ("uniform20k-open-cont-d4-p5", lambda: inputs.uniform_cont(20000, 5), 4, 5, True, 1 / 32),
]


@pytest.mark.parametrize("force_mode", ["adjoint", "kernel"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("case", R2_CASES, ids=[c[0] for c in R2_CASES])
def test_parity_inverse_square(case, precision, force_mode):
    """F(P, P~) = 1/|P - P~|^2 for the far forms and the near field: the GPU
    path (tables, level scales 4^l / 8^l, near-field pair function 1/r^2 with
    force 2 r/r^4, output scaling L^-2 / L^-3) against the oracle's."""
    name, gen, depth, p, cont, dt = case
    pos, q, box = gen()
    box = (0.0, 0.0, 0.0, 2.5)  # a box edge != 1 checks the output scaling
    pos = (pos.astype(np.float64) * 2.5).astype(np.float32)
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, continuous=cont, dt=dt, power=2,
                     force_kernel=force_mode == "kernel", keep=False)
    plan = FMM(box, depth, p, continuous=cont, split_ratio=dt, precision=precision,
               max_n=len(q), force_mode=force_mode, kernel="inverse_square")
    r = plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    tol = TOL[precision]
    assert _rel(r["potential"].cpu().numpy().astype(np.float64), ref["phi"]) < TOL[precision]
    assert _rel(r["forces"].cpu().numpy().astype(np.float64), ref["F"]) < tol
    assert abs(r["energy"].item() - ref["E"]) < TOL[precision] * abs(ref["E"])
    plan.close()
