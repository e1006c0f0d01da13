"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs.

Integer work (Morton keys, split charges and their particles, the sort
permutation, finest-cell ranges) must be bit-exact.  Floating point:
  FP64 plans: relative error <= 1e-11 (rounding order only);
  FP32 plans: relative L2 error <= 1e-6 on potentials and forces and
              relative energy error <= 1e-6, on top of the method's own error
              (the oracle runs the same method in FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2212_13080_gb300 import FMM, FmmError, inputs  # noqa: E402
from paper_2212_13080_gb300 import _binding as B  # noqa: E402

TOL_FP32 = 1e-6
TOL_FP64 = 1e-11
# Intermediate grid charges / functionals of coarse cells sum many charges of
# both signs: their FP32 rounding relative to their own (cancelled) size is
# larger than that of the outputs.
TOL_LEVELS_FP32 = 3e-5


def _gpu(pos, q, box, depth, p, periodic=False, continuous=False, dt=None, precision="fp32",
         forces=True, force_mode="adjoint"):
    plan = FMM(box, depth, p, periodic=periodic, continuous=continuous, split_ratio=dt,
               precision=precision, max_n=max(len(q), 1), force_mode=force_mode)
    r = plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda(), forces=forces)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy().astype(np.float64) if v is not None else None) for k, v in r.items()}
    return plan, out


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _check_integer_work(plan, ref):
    cnt = plan.dump("counts")
    n_eff = int(cnt[1])
    assert n_eff == ref["n_points"]
    np.testing.assert_array_equal(plan.dump("keys"), ref["pt_key"])
    np.testing.assert_array_equal(plan.dump("perm"), ref["perm"])
    np.testing.assert_array_equal(plan.dump("start"), ref["start"])
    np.testing.assert_array_equal(plan.dump("origin"), ref["pt_origin"][ref["perm"]])


def occupied_cells(start, depth, l):
    """Cells of level l (natural order (cz S + cy) S + cx) whose finest cells
    hold charges, from the finest-cell ranges (Morton order)."""
    S = 1 << l
    c = np.arange(S ** 3, dtype=np.int64)
    cx, cy, cz = c % S, (c // S) % S, c // (S * S)
    k = np.zeros_like(c)
    for bit in range(l):
        k |= (((cx >> bit) & 1) << (3 * bit)) | (((cy >> bit) & 1) << (3 * bit + 1)) | \
            (((cz >> bit) & 1) << (3 * bit + 2))
    sh = 3 * (depth - l)
    start = np.asarray(start, np.int64)
    return start[(k + 1) << sh] > start[k << sh]


def _check_levels(plan, ref, p, depth, periodic, tol):
    """Grid charges of every level; functionals of the cells that hold charges
    (the only ones the method reads; the library reports the others as zero)."""
    Phi = plan.dump("phi").reshape(-1).astype(np.float64)
    Lv = plan.dump("local").reshape(-1).astype(np.float64)
    lmin_phi = 0 if periodic else 2
    n3 = p ** 3
    for l in range(lmin_phi, depth + 1):
        a, b = oracle.level_offset(p, l), oracle.level_offset(p, l + 1)
        e = _rel_l2(Phi[a:b], ref["Phi"][a:b])
        assert e < tol, ("Phi", l, e)
        occ = np.repeat(occupied_cells(ref["start"], depth, l), n3)
        np.testing.assert_array_equal(Lv[a:b][~occ], 0.0)
        e = _rel_l2(Lv[a:b][occ], ref["L"][a:b][occ])
        assert e < tol, ("L", l, e)


CASES = [
    # name, generator, depth, p, periodic, continuous, dt
    ("uniform4k-open-plain", lambda: inputs.uniform_pm1(4096, 1), 3, 4, False, False, None),
    ("uniform20k-open-cont", lambda: inputs.uniform_cont(20000, 5), 4, 4, False, True, 1 / 32),
    ("uniform9k-open-cont-p5", lambda: inputs.uniform_cont(9001, 6), 3, 5, False, True, 1 / 16),
    ("water3k-periodic-cont-p5", lambda: inputs.water(1001, 3), 3, 5, True, True, 1 / 16),
    ("uniform5k-periodic-plain-p3", lambda: inputs.uniform_pm1(5000, 9), 3, 3, True, False, None),
    ("uniform3k-open-cont-p6-d2", lambda: inputs.uniform_cont(3001, 8), 2, 6, False, True, 1 / 8),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_small(case, precision):
    name, gen, depth, p, periodic, cont, dt = case
    pos, q, box = gen()
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, dt=dt)
    plan, out = _gpu(pos, q, box, depth, p, periodic, cont, dt, precision)
    _check_integer_work(plan, ref)
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32
    # sorted charges: unsplit charges carry the exact binned coordinate
    pts = plan.dump("points").astype(np.float64)
    st = ref["pt_t"][ref["perm"]]
    sq = ref["pt_q"][ref["perm"]]
    unsplit = ref["count"][ref["pt_origin"][ref["perm"]]] == 1
    np.testing.assert_array_equal(pts[unsplit, :3], st[unsplit])
    assert np.max(np.abs(pts[:, :3] - st)) < (1e-15 if precision == "fp64" else 1e-7)
    # split weights: products of three p-point Lagrange evaluations
    assert _rel_l2(pts[:, 3], sq) < (1e-15 if precision == "fp64" else 5e-7)
    _check_levels(plan, ref, p, depth, periodic, tol * 10 if precision == "fp64" else TOL_LEVELS_FP32)
    e_phi = _rel_l2(out["potential"], ref["phi"])
    e_F = _rel_l2(out["forces"], ref["F"])
    e_E = abs(out["energy"][0] - ref["E"]) / abs(ref["E"])
    assert e_phi < tol and e_F < tol and e_E < tol, (e_phi, e_F, e_E)
    plan.close()


TOL_TF32X3 = 1e-5  # reduced-precision far field (3-pass split TF32 on tensor cores)


TF32_CASES = [
    # name, generator, depth, p, periodic, continuous
    ("uniform40k-d4-p4-cont", lambda: inputs.uniform_cont(40000, 31), 4, 4, False, True),
    ("uniform300k-d5-p4-cont", lambda: inputs.uniform_cont(300000, 32), 5, 4, False, True),
    ("water45k-d4-p5-periodic-cont", lambda: inputs.water(15000, 33), 4, 5, True, True),
    ("uniform60k-d4-p6-open", lambda: inputs.uniform_pm1(60000, 34), 4, 6, False, False),
    ("uniform30k-d4-p3-open", lambda: inputs.uniform_pm1(30000, 35), 4, 3, False, False),
    ("uniform200k-d5-p3-periodic", lambda: inputs.uniform_pm1(200000, 36), 5, 3, True, False),
    # sparse (Plummer) inputs: segments below the box threshold take gathered
    # tiles, for every tile width (N = 64, 128, 224), with and without split
    ("plummer20k-d5-p4-open", lambda: inputs.plummer(20000, 37), 5, 4, False, False),
    ("plummer60k-d5-p5-open-cont", lambda: inputs.plummer(60000, 38), 5, 5, False, True),
    ("plummer100k-d5-p6-open", lambda: inputs.plummer(100000, 39), 5, 6, False, False),
    ("plummer30k-d4-p5-periodic", lambda: inputs.plummer(30000, 40), 4, 5, True, False),
]


@pytest.mark.parametrize("case", TF32_CASES, ids=[c[0] for c in TF32_CASES])
def test_parity_tf32x3(case):
    """Far-field contraction of every level on the tcgen05 tensor cores (3-pass
    split TF32, per-offset accumulators, p^3 padded to a multiple of 32; box
    and gathered tiles); potentials and forces within the reduced-precision
    tolerance of the FP64 oracle (sampled outputs), functionals of every level
    at the cells that hold charges."""
    name, gen, depth, p, periodic, cont = case
    pos, q, box = gen()
    n = len(q)
    s = np.arange(0, n, max(1, n // 1500))
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, sample=s)
    plan, out = _gpu(pos, q, box, depth, p, periodic, cont, None, "tf32x3")
    _check_integer_work(plan, ref)
    full = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont) if n <= 100000 else None
    if full is not None:
        _check_levels(plan, full, p, depth, periodic, TOL_LEVELS_FP32)
    assert _rel_l2(out["potential"][s], ref["phi"]) < TOL_TF32X3
    assert _rel_l2(out["forces"][s], ref["F"]) < TOL_TF32X3
    plan.close()


# Other tensor-core forms.  The split BF16 form keeps 16 significant bits of
# each operand (8 + 8); the dropped lo*lo product and the residual of the lo
# parts bound each product's relative error by about 3 * 2^-17.  The 1-pass
# TF32 form keeps 11 significant bits (round to nearest): about 2 * 2^-12 per
# product, so it states its error rather than meeting the 1e-5 bar.
TOL_TC_MODE = {"bf16x3": 1e-5, "tf32x1": 1e-3}


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x1"])
@pytest.mark.parametrize("case", TF32_CASES, ids=[c[0] for c in TF32_CASES])
def test_parity_tc_modes(case, precision):
    """Far-field contraction on the tensor cores in split BF16 (kind::f16) and
    1-pass TF32 forms against the FP64 oracle (sampled outputs)."""
    name, gen, depth, p, periodic, cont = case
    pos, q, box = gen()
    n = len(q)
    s = np.arange(0, n, max(1, n // 1500))
    ref = oracle.fmm(pos, q, box, depth=depth, n=p, periodic=periodic, continuous=cont, sample=s)
    plan, out = _gpu(pos, q, box, depth, p, periodic, cont, None, precision)
    _check_integer_work(plan, ref)
    tol = TOL_TC_MODE[precision]
    assert _rel_l2(out["potential"][s], ref["phi"]) < tol
    assert _rel_l2(out["forces"][s], ref["F"]) < tol
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_force_mode(precision):
    """The paper's force for split particles (sum of the forces their split
    charges feel, §2.3) is well conditioned: FP32 meets the 1e-6 bar."""
    pos, q, box = inputs.uniform_cont(20000, 12)
    ref = oracle.fmm(pos, q, box, depth=4, n=4, continuous=True, dt=1 / 32)
    plan, out = _gpu(pos, q, box, 4, 4, False, True, 1 / 32, precision, force_mode="paper")
    assert _rel_l2(out["forces"], ref["F_paper"]) < (TOL_FP64 if precision == "fp64" else TOL_FP32)
    assert _rel_l2(out["potential"], ref["phi"]) < (TOL_FP64 if precision == "fp64" else TOL_FP32)
    plan.close()


def test_energy_only_and_potential_only():
    pos, q, box = inputs.uniform_pm1(3000, 13)
    ref = oracle.fmm(pos, q, box, depth=3, n=4)
    plan, out = _gpu(pos, q, box, 3, 4, precision="fp64", forces=False)
    assert out["forces"] is None
    assert _rel_l2(out["potential"], ref["phi"]) < TOL_FP64
    assert abs(out["energy"][0] - ref["E"]) < TOL_FP64 * abs(ref["E"])
    plan.close()


def test_deterministic():
    pos, q, box = inputs.uniform_cont(30000, 14)
    plan = FMM(box, 4, 4, continuous=True, max_n=len(q))
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    a = plan.eval(P, Q)
    a = {k: v.clone() for k, v in a.items()}
    b = plan.eval(P, Q)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    plan.close()


def test_edge_cases():
    box = (0.0, 0.0, 0.0, 1.0)
    # n = 0
    plan = FMM(box, 3, 4, max_n=16)
    r = plan.eval(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"))
    assert r["energy"].item() == 0.0
    # one particle: no interaction at all
    r = plan.eval(torch.tensor([[0.3, 0.6, 0.1]], device="cuda"), torch.tensor([1.0], device="cuda"))
    assert r["energy"].item() == 0.0 and r["potential"].item() == 0.0
    # all particles in one finest cell; particles exactly on planes
    pos = np.array([[0.5, 0.5, 0.5], [0.55, 0.52, 0.51], [0.25, 0.5, 0.75], [0.125, 0.0, 0.999],
                    [0.0, 0.0, 0.0], [0.5, 0.125, 0.625]], np.float32)
    q = np.array([1, -1, 1, -1, 1, -1], np.float32)
    for cont in (False, True):
        ref = oracle.fmm(pos, q, box, depth=3, n=4, continuous=cont, dt=1 / 8)
        plan2 = FMM(box, 3, 4, continuous=cont, split_ratio=1 / 8, precision="fp64", max_n=6,
                    split_capacity=64)
        r = plan2.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
        out = {k: v.cpu().numpy() for k, v in r.items()}
        _check_integer_work(plan2, ref)
        assert _rel_l2(out["potential"], ref["phi"]) < TOL_FP64
        plan2.close()
    # open form: a position outside the box is an error, not a wrong answer
    with pytest.raises(FmmError) as e:
        plan.eval(torch.tensor([[1.5, 0.5, 0.5]], device="cuda"), torch.tensor([1.0], device="cuda"))
    assert e.value.code == 3
    with pytest.raises(FmmError) as e:
        plan.eval(torch.tensor([[float("nan"), 0.5, 0.5]], device="cuda"),
                  torch.tensor([1.0], device="cuda"))
    assert e.value.code == 4
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_coincident_split_charges_across_cells(precision):
    """Odd p, continuous form: the middle split charges of a particle sit on the
    cell plane (local coordinate 1 in the lower cell, 0 in the upper one), so two
    particles on either side of a plane with the same transverse coordinates
    have coincident charges in different cells.  Those pairs are skipped like
    every coincident pair (the oracle's rule); nothing may become infinite."""
    rng = np.random.default_rng(23)
    pos = rng.random((3000, 3)).astype(np.float32)
    extra = np.array([[0.5 - 0.001, 0.3, 0.7], [0.5 + 0.002, 0.3, 0.7],
                      [0.25 + 0.003, 0.61, 0.33], [0.25 - 0.001, 0.61, 0.33],
                      [0.9, 0.375 - 0.002, 0.1], [0.9, 0.375 + 0.001, 0.1]], np.float32)
    pos = np.concatenate([pos, extra])
    q = rng.uniform(-1, 1, len(pos)).astype(np.float32)
    box = (0.0, 0.0, 0.0, 1.0)
    ref = oracle.fmm(pos, q, box, depth=3, n=5, continuous=True, dt=1 / 8)
    plan, out = _gpu(pos, q, box, 3, 5, False, True, 1 / 8, precision)
    _check_integer_work(plan, ref)
    assert np.isfinite(out["potential"]).all() and np.isfinite(out["forces"]).all()
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32
    assert _rel_l2(out["potential"], ref["phi"]) < tol
    assert _rel_l2(out["forces"], ref["F"]) < tol
    plan.close()


def test_wait_timeout_is_reported_and_context_survives():
    """Failure detection without a fault: the tensor-core contraction's producer
    arms one stage's barrier without issuing its copies (a flag nothing sets);
    the consumer's bounded wait expires, the kernel records where, frees its
    tensor memory and returns; the call reports FMM_ERR_TIMEOUT and the next
    evaluation on the same context is correct."""
    pos, q, box = inputs.uniform_cont(20000, 41)
    n = len(q)
    plan = FMM(box, 4, 4, continuous=True, precision="tf32x3", max_n=n)
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    plan.inject("tc_stall")
    with pytest.raises(FmmError) as e:
        plan.eval(P, Q)
    assert e.value.code == B.FMM_ERR_TIMEOUT
    site, block, level, it = [int(v) for v in plan.dump("wait")]
    assert site in (1, 2, 3, 4) and 2 <= level <= 4 and block >= 0
    r = plan.eval(P, Q)  # the hook disarmed itself; same context, same plan
    ref = oracle.fmm(pos, q, box, depth=4, n=4, continuous=True, keep=False)
    assert _rel_l2(r["potential"].cpu().numpy().astype(np.float64), ref["phi"]) < TOL_TF32X3
    assert int(plan.dump("wait")[0]) == 0
    plan.close()
    # plans without the tensor-core contraction have nothing to stall
    plan32 = FMM(box, 4, 4, precision="fp32", max_n=n)
    with pytest.raises(FmmError) as e:
        plan32.inject("tc_stall")
    assert e.value.code == B.FMM_ERR_UNSUPPORTED
    plan32.close()


def test_split_overflow_is_reported():
    # every particle near a corner: 64 charges each, capacity 2 per particle
    rng = np.random.default_rng(3)
    c = rng.integers(1, 7, size=(500, 3))
    pos = ((c + rng.uniform(-1, 1, size=(500, 3)) * 0.01) / 8).astype(np.float32)
    q = np.ones(500, np.float32)
    plan = FMM((0, 0, 0, 1), 3, 4, continuous=True, split_ratio=1 / 16, max_n=500)
    with pytest.raises(FmmError) as e:
        plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    assert e.value.code == 5
    # with room for the split it evaluates and matches the oracle
    plan2 = FMM((0, 0, 0, 1), 3, 4, continuous=True, split_ratio=1 / 16, max_n=500,
                split_capacity=70, precision="fp64")
    r = plan2.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    ref = oracle.fmm(pos, q, (0, 0, 0, 1), depth=3, n=4, continuous=True, dt=1 / 16)
    assert _rel_l2(r["potential"].cpu().numpy(), ref["phi"]) < TOL_FP64
    plan.close()
    plan2.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_matches_forces_and_potential(precision):
    pos, q, box = inputs.water(800, 17)
    ref = oracle.fmm(pos, q, box, depth=3, n=5, periodic=True, continuous=True, dt=1 / 16)
    plan = FMM(box, 3, 5, periodic=True, continuous=True, split_ratio=1 / 16, precision=precision,
               max_n=len(q))
    from paper_2212_13080_gb300 import fmm_energy
    P = torch.from_numpy(pos).cuda().requires_grad_(True)
    Q = torch.from_numpy(q).cuda().requires_grad_(True)
    E = fmm_energy(plan, P, Q)
    (2.0 * E).backward()
    tol = TOL_FP64 if precision == "fp64" else TOL_FP32
    assert abs(E.item() - ref["E"]) < tol * abs(ref["E"])
    # autograd returns gradients in the inputs' dtype (float32)
    tol = max(tol, 2e-7)
    assert _rel_l2(P.grad.cpu().numpy().astype(np.float64), -2.0 * ref["F"]) < tol
    assert _rel_l2(Q.grad.cpu().numpy().astype(np.float64), 2.0 * ref["phi"]) < tol
    plan.close()


def test_backward_rejects_a_workspace_another_plan_wrote():
    """fmm_backward reuses the state the last evaluation left in the workspace;
    once another plan has evaluated into the same workspace it fails with
    FMM_ERR_STATE instead of returning gradients of the other system."""
    pos, q, box = inputs.uniform_cont(3000, 41)
    pos2, q2, _ = inputs.uniform_cont(3000, 42)
    a = FMM(box, 3, 4, continuous=True, split_ratio=1 / 16, max_n=len(q))
    b = FMM(box, 3, 4, continuous=True, split_ratio=1 / 16, max_n=len(q))
    ws = a.workspace(len(q))
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    a.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda(), workspace=ws)
    gpos, gq = a.backward(gE)
    ref = oracle.fmm(pos, q, box, depth=3, n=4, continuous=True, dt=1 / 16)
    assert _rel_l2(gq.cpu().numpy().astype(np.float64), ref["phi"]) < TOL_FP32
    b.eval(torch.from_numpy(pos2).cuda(), torch.from_numpy(q2).cuda(), workspace=ws)
    with pytest.raises(FmmError) as e:
        a.backward(gE)
    assert e.value.code == B.FMM_ERR_STATE
    # a new evaluation of the first plan makes the workspace its own again
    a.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda(), workspace=ws)
    gpos, gq = a.backward(gE)
    assert _rel_l2(gq.cpu().numpy().astype(np.float64), ref["phi"]) < TOL_FP32
    a.close()
    b.close()


def test_forces_central_differences_fp64():
    """Forces are -dE/dx of the GPU's own energy (central differences, h = 2^-14,
    particles away from the split-band edges)."""
    pos, q, box = inputs.uniform_pm1(700, 19)
    pos = (pos * np.float32(0.5) + np.float32(0.25)).astype(np.float32)
    dt = 1 / 8
    plan = FMM(box, 3, 4, continuous=True, split_ratio=dt, precision="fp64", max_n=len(q))
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    F = plan.eval(P, Q)["forces"].cpu().numpy()
    h = np.float32(2.0 ** -14)
    ref = oracle.fmm(pos, q, box, depth=3, n=4, continuous=True, dt=dt)
    t = ref["t"]
    edge = np.minimum(np.abs(t - dt), np.abs(1 - t - dt)).min(axis=1) * 8
    idx = np.where(edge > 4 * h)[0][:12]
    for i in idx:
        for a in range(3):
            Es = []
            for s in (1, -1):
                pp = pos.copy()
                pp[i, a] += s * h
                Es.append(plan.eval(torch.from_numpy(pp).cuda(), Q)["energy"].item())
            fd = -(Es[0] - Es[1]) / (2 * float(h))
            assert abs(fd - F[i, a]) < 2e-4 * max(1.0, np.abs(F[i]).max()), (i, a, fd, F[i, a])
    plan.close()


@pytest.mark.parametrize("name,sample,precision", [("uniform1m", None, "fp32"), ("water2m", 2048, "fp32"),
                                                    ("uniform1m", None, "tf32x3"),
                                                    ("water2m", 2048, "tf32x3"),
                                                    ("water2m", 2048, "bf16x3"),
                                                    ("plummer8m", 2048, "fp32"),
                                                    ("plummer8m", 2048, "tf32x3"),
                                                    ("plummer8m", 2048, "bf16x3")])
def test_parity_full_size_sampled(name, sample, precision):
    """Full-size workloads in the benchmark's launch configuration: integer work
    on every charge; outputs on every particle (uniform1m: the oracle runs the
    whole workload in about a second) or on sampled particles (the oracle
    computes those one by one from its full upward pass).  Adjoint forces of
    split particles are a difference of potentials across 2d (§2.3), formed in
    difference form; the whole-workload comparison is the stronger check."""
    w = inputs.workload(name)
    pos, q, box = w["pos"], w["q"], w["box"]
    rng = np.random.default_rng(0)
    s = np.arange(len(q)) if sample is None else np.sort(rng.choice(len(q), sample, replace=False))
    ref = oracle.fmm(pos, q, box, depth=w["depth"], n=w["p"], periodic=w["periodic"],
                     continuous=w["continuous"], sample=None if sample is None else s)
    plan, out = _gpu(pos, q, box, w["depth"], w["p"], w["periodic"], w["continuous"], None, precision)
    _check_integer_work(plan, ref)
    tol = {"fp32": TOL_FP32, "tf32x3": TOL_TF32X3}.get(precision) or TOL_TC_MODE[precision]
    assert _rel_l2(out["potential"][s], ref["phi"]) < tol
    assert _rel_l2(out["forces"][s], ref["F"]) < tol
    if sample is None:
        assert abs(out["energy"][0] - ref["E"]) / abs(ref["E"]) < tol
    # energy: the sum is a property at any size; E = 1/2 sum q phi of the GPU's own phi
    E_from_phi = 0.5 * np.dot(q.astype(np.float64), out["potential"])
    assert abs(out["energy"][0] - E_from_phi) < 1e-9 * np.sum(np.abs(q * out["potential"]))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3"])
def test_table1_error_trend_on_gpu(precision):
    """§3.1 Table 1 reproduced by the GPU path: Error1 / Error2 (mean relative
    errors of potentials and forces against the direct sum) for 23040 random +-1
    charges in 8^3 finest cells, orders 3-7 (3-6 on the tensor cores); median of
    5 seeded configurations within a factor 2.5 of the printed values, as for the
    oracle.  The method's error dominates every precision's rounding here."""
    from conftest import read_golden
    rows = [r for r in read_golden("table1_errors.txt") if precision != "tf32x3" or int(r[0]) <= 6]
    e1 = {int(r[0]): [] for r in rows}
    e2 = {int(r[0]): [] for r in rows}
    for seed in range(11, 16):
        pos, q, box = inputs.uniform_pm1(23040, seed)
        pd, Fd = oracle.direct(pos, q, box)
        P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
        for r in rows:
            n = int(r[0])
            plan = FMM(box, 3, n, precision=precision, max_n=len(q))
            o = plan.eval(P, Q)
            phi = o["potential"].cpu().numpy().astype(np.float64)
            F = o["forces"].cpu().numpy().astype(np.float64)
            e1[n].append(np.mean(np.abs((phi - pd) / pd)))
            e2[n].append(np.mean(np.abs((F - Fd) / Fd)))
            plan.close()
    for r in rows:
        n = int(r[0])
        m1, m2 = np.median(e1[n]), np.median(e2[n])
        print("order %d  Error1 %.3e (paper %.2e)  Error2 %.3e (paper %.2e)" % (n, m1, r[1], m2, r[2]))
        assert r[1] / 2.5 < m1 < r[1] * 2.5, (n, m1, r[1])
        assert r[2] / 2.5 < m2 < r[2] * 2.5, (n, m2, r[2])


def test_drag_continuity_at_planes_fp64():
    """§3.2 / Fig. 6 on the GPU: a particle moved from just below a plane of the
    finest cells onto it changes the continuous-form energy by about |F| dx,
    while the plain form jumps (same protocol as the oracle's pin); at the edges
    of the split band (distance d from the plane) the continuous-form energy is
    continuous too (the split weights put the whole charge on the particle's own
    position there)."""
    pos, q, box = inputs.uniform_pm1(1500, 71)
    P0 = torch.from_numpy(pos).cuda()
    Q = torch.from_numpy(q).cuda()
    d = (1.0 / 8) / 256  # split half-width at depth 3, d = w/256
    plans = {cont: FMM(box, 3, 4, continuous=cont, precision="fp64", max_n=len(q))
             for cont in (False, True)}

    def energy_force(plan, x):
        p = P0.clone()
        p[0, 0] = float(x)
        o = plan.eval(p, Q)
        return o["energy"].item(), abs(o["forces"][0, 0].item())

    for plane in (np.float32(0.5), np.float32(0.25)):
        below = np.nextafter(plane, np.float32(-1))
        jumps, slope = {}, {}
        for cont in (False, True):
            (E0, F0), (E1, F1) = energy_force(plans[cont], below), energy_force(plans[cont], plane)
            jumps[cont] = abs(E1 - E0)
            slope[cont] = max(F0, F1) * (float(plane) - float(below))
        assert jumps[True] < 3 * slope[True] + 1e-12 * abs(E0), (plane, jumps, slope)
        assert jumps[False] > 20 * slope[False], (plane, jumps, slope)
        # band edges: just outside and just inside distance d
        for side in (-1.0, 1.0):
            xo = np.float32(float(plane) + side * d * 1.001)
            xi = np.float32(float(plane) + side * d * 0.999)
            (Eo, Fo), (Ei, Fi) = energy_force(plans[True], xo), energy_force(plans[True], xi)
            dx = abs(float(xo) - float(xi))
            assert abs(Eo - Ei) < 3 * max(Fo, Fi) * dx + 1e-12 * abs(Eo), (plane, side, Eo - Ei, dx)
    for plan in plans.values():
        plan.close()


def test_drag_energy_curve_fig6():
    """Fig. 6 protocol (§3.2): one particle dragged along x = k/1000,
    k = 1..999, through the other 23039 charges, order 4, continuous form with
    2d = 1/1024 (d = w/256 at 8^3 cells).  The FP32 plan's energy curve follows
    the FP64 plan's (oracle-pinned) within FP32 accuracy at every point, through
    every cell plane and split band."""
    pos, q, box = inputs.uniform_pm1(23040, 12)
    P0 = torch.from_numpy(pos).cuda()
    Q = torch.from_numpy(q).cuda()
    xs = np.arange(1, 1000) / 1000.0
    curves = {}
    for prec in ("fp64", "fp32"):
        plan = FMM(box, 3, 4, continuous=True, split_ratio=1 / 256, precision=prec, max_n=len(q))
        E = []
        for x in xs:
            p = P0.clone()
            p[0, 0] = float(np.float32(x))
            o = plan.eval(p, Q)
            E.append(o["energy"].item())
            if prec == "fp64" and x == 0.5:
                terms = q.astype(np.float64) * o["potential"].cpu().numpy()
        plan.close()
        curves[prec] = np.array(E)
    # E = 1/2 sum q phi of +-1 charges cancels heavily (|E| ~ 1e-3 sum |q phi|):
    # the FP32 rounding of the potentials adds up like a random walk, so the
    # scale of the energy's FP32 error is the L2 norm of its terms
    scale = 0.5 * np.linalg.norm(terms)
    assert np.max(np.abs(curves["fp32"] - curves["fp64"])) < 1e-6 * scale


def _lebesgue(p, s):
    """max over [0,1] of sum_i |g_i(t)| for the points 1/2 + s (i/(p-1) - 1/2)."""
    tau = 0.5 + s * (np.arange(p) / (p - 1) - 0.5)
    t = np.linspace(0.0, 1.0, 4001)
    total = np.zeros_like(t)
    for i in range(p):
        g = np.ones_like(t)
        for k in range(p):
            if k != i:
                g *= (t - tau[k]) / (tau[i] - tau[k])
        total += np.abs(g)
    return total.max()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("periodic,p", [(False, 4), (True, 5)])
def test_parity_reduced_arrangement(precision, periodic, p):
    """§4.1's reduced arrangement of the p-division points (spacing x 1/1.2
    about the cell centre), plain form: the GPU path with its tables built on
    the moved points matches the oracle on the same points."""
    pos, q, box = inputs.uniform_pm1(30000, 57)
    s = 1 / 1.2
    ref = oracle.fmm(pos, q, box, depth=4, n=p, periodic=periodic, grid_scale=s)
    plan = FMM(box, 4, p, periodic=periodic, precision=precision, max_n=len(q), grid_scale=s)
    r = plan.eval(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    tol = {"fp64": TOL_FP64, "fp32": TOL_FP32, "tf32x3": TOL_TF32X3}[precision]
    if precision != "fp64":
        # near the faces the moved points extrapolate: rounding in replacement and
        # evaluation grows with the tensor-product Lebesgue constant (1-D cubed)
        tol *= (_lebesgue(p, s) / _lebesgue(p, 1.0)) ** 3
    assert _rel_l2(r["potential"].cpu().numpy().astype(np.float64), ref["phi"]) < tol
    assert _rel_l2(r["forces"].cpu().numpy().astype(np.float64), ref["F"]) < tol
    plan.close()
    with pytest.raises(FmmError) as e:
        FMM(box, 4, p, continuous=True, max_n=len(q), grid_scale=s)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED


def test_water_autograd_forces_central_differences():
    """The periodic continuous water-like configuration (p = 5): forces from the
    adjoint pass (autograd through fmm_energy) against central differences of
    the GPU's own FP64 energy, h = 1e-4 (as represented in float32), on 64
    seeded particles away from the split-band edges.  A reduced system (10,000
    triples, depth 3): at full size the FP64 energy takes seconds per
    evaluation and FP32 energy differences are below the rounding."""
    pos, q, box = inputs.water(10000, 3)
    plan = FMM(box, 3, 5, periodic=True, continuous=True, precision="fp64", max_n=len(q))
    P = torch.from_numpy(pos).cuda().requires_grad_(True)
    Q = torch.from_numpy(q).cuda()
    from paper_2212_13080_gb300 import fmm_energy
    E = fmm_energy(plan, P, Q)
    E.backward()
    F = -P.grad.double().cpu().numpy()
    L, S = box[3], 8
    ref = oracle.fmm(pos, q, box, depth=3, n=5, periodic=True, continuous=True, keep=True)
    t, dt = ref["t"].astype(np.float64), 1.0 / 256
    h = 1e-4
    edge = np.minimum(np.abs(t - dt), np.abs(1 - t - dt)).min(axis=1) * (L / S)  # physical units
    rng = np.random.default_rng(3)
    idx = rng.choice(np.where(edge > 4 * h)[0], 64, replace=False)
    Fmax = np.abs(F).max()
    for i in idx:
        for a in range(3):
            Es, xs = [], []
            for s in (1, -1):
                pp = pos.copy()
                pp[i, a] = np.float32(pos[i, a] + s * h)
                xs.append(float(pp[i, a]))
                Es.append(plan.eval(torch.from_numpy(pp).cuda(), Q, forces=False)["energy"].item())
            fd = -(Es[0] - Es[1]) / (xs[0] - xs[1])
            assert abs(fd - F[i, a]) < 1e-4 * Fmax, (i, a, fd, F[i, a])
    plan.close()


def test_continuity_through_the_periodic_wall_fp64():
    """§4.2: a particle moved from just below the wall x = 1 of the periodic box
    to x = 0 (the same physical place) changes the continuous periodic form's
    energy by about |F| dx and its force by nearly nothing; the plain periodic
    form jumps (its near-field partition changes at the wall)."""
    pos, q, box = inputs.uniform_pm1(1500, 71)
    Q = torch.from_numpy(q).cuda()
    below = np.nextafter(np.float32(1.0), np.float32(0))
    dx = 1.0 - float(below)
    for cont in (True, False):
        plan = FMM(box, 3, 4, periodic=True, continuous=cont, precision="fp64", max_n=len(q))
        out = []
        for x in (below, np.float32(0.0)):
            p = pos.copy()
            p[0, 0] = x
            r = plan.eval(torch.from_numpy(p).cuda(), Q)
            out.append((r["energy"].item(), r["forces"][0].cpu().numpy()))
        (E0, F0), (E1, F1) = out
        Fm = np.abs(F0).max()
        if cont:
            assert abs(E1 - E0) < 3 * Fm * dx + 1e-12 * abs(E0), (E1 - E0, Fm * dx)
            assert np.abs(F1 - F0).max() < 1e-4 * Fm, (F0, F1)
        else:
            assert abs(E1 - E0) > 20 * Fm * dx, (E1 - E0, Fm * dx)
        plan.close()


def test_sync_plan_refuses_a_stream_being_captured():
    """Through the C ABI: a plan that waits for the device at the end of the
    call (opts.sync = 1) returns FMM_ERR_ARG, before any work, when its stream
    is being captured into a CUDA graph (the wait would end the capture); the
    capture stays valid, and the same call outside a capture evaluates."""
    import ctypes
    from paper_2212_13080_gb300 import _ptr
    pos, q, box = inputs.uniform_cont(3000, 21)
    n = len(q)
    P, Q = torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda()
    o = B.fmm_opts_default()
    o.continuous = 1
    o.sync = 1
    h = B.fmm_plan_create(box, 3, 4, False, o, n)
    nb = B.fmm_workspace_size(h, n)
    ws = FMM._aligned(torch.empty(nb + 256, dtype=torch.uint8, device="cuda"))
    phi = torch.zeros(n, device="cuda")
    g = torch.cuda.CUDAGraph()
    with pytest.raises(FmmError) as e:
        with torch.cuda.graph(g):
            st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            B.fmm_eval(h, n, _ptr(P), _ptr(Q), _ptr(phi), None, None, _ptr(ws), nb, st)
    assert e.value.code == B.FMM_ERR_ARG
    torch.cuda.synchronize()
    assert not torch.any(phi != 0)  # nothing ran
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    B.fmm_eval(h, n, _ptr(P), _ptr(Q), _ptr(phi), None, None, _ptr(ws), nb, st)
    torch.cuda.synchronize()
    plan = FMM(box, 3, 4, continuous=True, max_n=n)  # the same plan, its status read by the binding
    assert torch.equal(phi, plan.eval(P, Q, energy=False, forces=False)["potential"])
    plan.close()
    B.fmm_plan_destroy(h)
