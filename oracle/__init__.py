"""FP64 CPU oracle of the replacement-based FMM (Kajima, arXiv:2212.13080).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the product package.  It shares no
code with the CUDA library; the seeded input generators that both sides use
hold none of the method's arithmetic.

`fmm()` runs the steps of §2.2 in the paper's order on top of the C routines of
fmm_oracle.c:

  1. divide the box (canonical single-precision map to the unit cube),
  +  split near the planes of the finest cells (continuous form, §2.3; box
     walls too in the periodic form, §4.2),
  2. upward pass: replacement at the leaves (eq. ex66), shifts to the parents
     (eq. threethree),
  3. downward pass: Psi_child = Psi_parent o shift, plus the bilinear forms of
     the interaction list (eq. bilinear); periodic form: lattice term at level 0,
  4. far-field potential and force at every charge (end of §2.2),
  5. near field over the 27 neighbouring cells,
  +  combination of the split charges back into their particles.

`fmm(..., shift_free=True)` takes App. A.2 instead of steps 2-4: every
cell's grid charges and functional are taken with respect to the box, the
upward pass sums children, the interaction lists apply the shift-free
bilinear forms BB_{C~,C} (target and source shifted from the box,
shift_{S->C} the inverse of shift_{C->S}), and the downward pass is the
identity.

`fmm(..., force_kernel=True)` takes the far forces from the force kernels
(x - x~)/|P - P~|^3 (§4.1's remark on other kernels): three more functionals
per cell from the same interaction lists (the periodic lattice term from the
gradient of the Ewald lattice potential), read with the plain weights; a
particle's force is the sum of the forces on its charges.

The energy is E = 1/2 sum_i q_i phi_i, phi_i the potential at particle i from
every other particle (steps 4 and 5 each count every pair from both sides).

Forces: "adjoint" is -dE/dx of this energy.  For an axis along which a particle
is split, its split charges do not move with it, only their weights change, so
the component is -q sum_k (dW_k/dx) phi(s_k).  "paper" sums the forces that
the split charges feel (§2.3); the two agree on every axis that is not split.

Parity unpinned: none (every routine is exercised by tests/test_oracle_pins.py).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, f, i32, i64, u8 = (ctypes.c_double, ctypes.c_float, ctypes.c_int, ctypes.c_int64,
                              ctypes.c_void_p)
        P = ctypes.c_void_p
        L.orc_lagrange.argtypes = [i32, d, P]
        L.orc_set_grid_scale.argtypes = [d]
        L.orc_lagrange_deriv.argtypes = [i32, d, P]
        L.orc_shift_matrix.argtypes = [i32, i32, P]
        L.orc_m2l_kernel.argtypes = [i32, i32, i32, i32, P]
        L.orc_lattice_psi.argtypes = [d, d, d]
        L.orc_lattice_psi.restype = d
        L.orc_lattice_kernel.argtypes = [i32, P]
        L.orc_ewald_direct.argtypes = [i64, P, P, i64, P, P, P]
        L.orc_direct_open.argtypes = [i64, P, P, i64, P, P, P]
        L.orc_bin.argtypes = [i64, P, P, i32, i32, P, P, P, P]
        L.orc_bin.restype = i32
        L.orc_morton.argtypes = [i32, i32, i32, i32]
        L.orc_morton.restype = ctypes.c_uint32
        L.orc_split_count.argtypes = [i64, P, P, i32, i32, i32, i32, f, P, P]
        L.orc_split_emit.argtypes = [i64, P, P, P, i32, i32, i32, i32, f, P, P, P, P, P, P, P, P]
        L.orc_sort.argtypes = [i64, P, i32, P, P]
        L.orc_level_offset.argtypes = [i32, i32]
        L.orc_level_offset.restype = i64
        L.orc_p2m.argtypes = [i32, i32, P, P, P, P]
        L.orc_m2m.argtypes = [i32, i32, i32, P]
        L.orc_downward.argtypes = [i32, i32, i32, P, P, P, P]
        L.orc_evaluate.argtypes = [i32, i32, i32, i64, P, P, P, P, P, P, P, P, P, P]
        L.orc_sf_shift_to_box.argtypes = [i32, i32, i32, P]
        L.orc_sf_shift_from_box.argtypes = [i32, i32, i32, P]
        L.orc_sf_shift_from_box.restype = i32
        L.orc_sf_p2m.argtypes = [i32, i32, P, P, P, P, P]
        L.orc_sf_upward.argtypes = [i32, i32, i32, P]
        L.orc_sf_bilinear.argtypes = [i32, i32, P, P, P, P]
        L.orc_sf_bilinear.restype = i32
        L.orc_sf_downward.argtypes = [i32, i32, i32, P, P, P, P]
        L.orc_sf_downward.restype = i32
        L.orc_sf_evaluate.argtypes = [i32, i32, i32, i64, P, P, P, P, P, P, P, P, P, P]
        L.orc_set_kernel.argtypes = [i32]
        L.orc_set_power.argtypes = [i32]
        L.orc_lattice_grad.argtypes = [d, d, d, P]
        L.orc_evaluate_kernel.argtypes = [i32, i32, i32, i64, P, P, P, P, P, P, P, P, P, P, P, P,
                                          P]
        L.orc_interaction_list.argtypes = [i32, i32, i32, i32, i32, P, P]
        L.orc_interaction_list.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# Elementary definitions (§2.1)
# ---------------------------------------------------------------------------

def nodes(n):
    """§2.1.2: n-division points of the unit segment, end points included."""
    return np.arange(n, dtype=np.float64) / (n - 1)


def lagrange(n, x):
    """§2.1.1 eq. (Lag1): g_i(x) for each x (array) -> shape (len(x), n)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty((x.size, n))
    buf = np.empty(n)
    for k, xv in enumerate(x):
        lib().orc_lagrange(n, float(xv), _p(buf))
        out[k] = buf
    return out


def lagrange_deriv(n, x):
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty((x.size, n))
    buf = np.empty(n)
    for k, xv in enumerate(x):
        lib().orc_lagrange_deriv(n, float(xv), _p(buf))
        out[k] = buf
    return out


def shift_matrix(n, h):
    """§2.1.6 eq. (trans): child half h -> parent segment, G[J, i]."""
    G = np.empty((n, n))
    lib().orc_shift_matrix(n, h, _p(G))
    return G


def m2l_kernel(n, o, comp=0):
    """§2.1.7 eq. (bilinear): K[a, b] = 1/|a - (o + b)| for unit cells; comp
    1..3 the x, y, z component of the force kernel r/|r|^3 at r = a - (o + b)."""
    n3 = n ** 3
    K = np.empty((n3, n3))
    L = lib()
    L.orc_set_kernel(int(comp))
    try:
        L.orc_m2l_kernel(n, int(o[0]), int(o[1]), int(o[2]), _p(K))
    finally:
        L.orc_set_kernel(0)
    return K


def lattice_kernel(n, comp=0):
    """Level-0 lattice kernel psi(a - b) (§4.2); comp 1..3: -d psi/d r_c."""
    n3 = n ** 3
    K = np.empty((n3, n3))
    L = lib()
    L.orc_set_kernel(int(comp))
    try:
        L.orc_lattice_kernel(n, _p(K))
    finally:
        L.orc_set_kernel(0)
    return K


def lattice_psi(r):
    return lib().orc_lattice_psi(float(r[0]), float(r[1]), float(r[2]))


def lattice_grad(r):
    g = np.empty(3)
    lib().orc_lattice_grad(float(r[0]), float(r[1]), float(r[2]), _p(g))
    return g


def sf_shift_to_box(n, l, c):
    """App. A.2: shift_{C->S} along one axis for the level-l cell at
    coordinate c, G[b, i] = g_b((c + a_i) / 2^l)."""
    G = np.empty((n, n))
    lib().orc_sf_shift_to_box(n, l, c, _p(G))
    return G


def sf_shift_from_box(n, l, c):
    """App. A.2: shift_{S->C} along one axis (the inverse of sf_shift_to_box,
    by elimination), H[i, b]."""
    H = np.empty((n, n))
    if lib().orc_sf_shift_from_box(n, l, c, _p(H)):
        raise ArithmeticError("singular shift")
    return H


def sf_bilinear(n, l, ct, cs, o):
    """App. A.2: the matrix of BB_{C~,C} (target cell ct, source cell cs,
    offset o before wrapping, level l, unit-box units), box-node indices
    [target, source]."""
    n3 = n ** 3
    B = np.empty((n3, n3))
    a = lambda v: np.ascontiguousarray(v, dtype=np.int32)
    ct, cs, o = a(ct), a(cs), a(o)
    if lib().orc_sf_bilinear(n, l, _p(ct), _p(cs), _p(o), _p(B)):
        raise ArithmeticError("singular shift")
    return B


def replace(n, t, q):
    """Replacement (eq. ex66) of charges q at cell-local positions t (m x 3)
    with respect to the unit cell: the n^3 vector, index (k*n + j)*n + i."""
    t = np.asarray(t, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    gx, gy, gz = lagrange(n, t[:, 0]), lagrange(n, t[:, 1]), lagrange(n, t[:, 2])
    v = np.einsum("p,pk,pj,pi->kji", q, gz, gy, gx)
    return v.reshape(-1)


# ---------------------------------------------------------------------------
# Truth references
# ---------------------------------------------------------------------------

def unit_coords(pos, box, periodic):
    """The canonical single-precision unit-cube coordinates, widened to FP64."""
    pos = _c(pos, np.float32).reshape(-1, 3)
    N = pos.shape[0]
    box = _c(box, np.float64)
    u = np.empty((N, 3), np.float32)
    t = np.empty((N, 3), np.float32)
    cell = np.empty((N, 3), np.int32)
    key = np.empty(N, np.uint32)
    err = lib().orc_bin(N, _p(pos), _p(box), 2, int(periodic), _p(u), _p(t), _p(cell), _p(key))
    return u.astype(np.float64), err


def direct(pos, q, box, periodic=False, targets=None, power=1):
    """O(N^2) Coulomb sum (open) or Ewald sum with tin-foil boundary
    (periodic) on the canonical coordinates.  Returns (phi, F) at targets,
    physical units.  power=2: the 1/r^2 sum (open only)."""
    if power != 1:
        if periodic:
            raise ValueError("the lattice sum of 1/r^2 diverges")
        L_ = lib()
        L_.orc_set_power(int(power))
        try:
            phi, F = direct(pos, q, box, False, targets)
        finally:
            L_.orc_set_power(1)
        Lb = float(np.asarray(box, np.float64)[3])
        return phi * Lb / Lb ** power, F * Lb ** 2 / Lb ** (power + 1)
    u, err = unit_coords(pos, box, periodic)
    if err:
        raise ValueError("oracle: input outside the box or not finite (flags %d)" % err)
    q64 = _c(q, np.float64)
    N = u.shape[0]
    tg = np.arange(N, dtype=np.int64) if targets is None else _c(targets, np.int64)
    phi = np.empty(tg.size)
    F = np.empty((tg.size, 3))
    x = _c(u, np.float64)
    fn = lib().orc_ewald_direct if periodic else lib().orc_direct_open
    fn(N, _p(x), _p(q64), tg.size, _p(tg), _p(phi), _p(F))
    Lb = float(box[3])
    return phi / Lb, F / (Lb * Lb)


def ewald_unit(x, q, targets=None):
    """Ewald sum on unit-cube coordinates x (FP64), no canonicalisation."""
    x = _c(x, np.float64).reshape(-1, 3)
    q = _c(q, np.float64)
    tg = np.arange(x.shape[0], dtype=np.int64) if targets is None else _c(targets, np.int64)
    phi = np.empty(tg.size)
    F = np.empty((tg.size, 3))
    lib().orc_ewald_direct(x.shape[0], _p(x), _p(q), tg.size, _p(tg), _p(phi), _p(F))
    return phi, F


# ---------------------------------------------------------------------------
# The FMM of §2.2 (+ §2.3, §4.2)
# ---------------------------------------------------------------------------

DEFAULT_SPLIT_RATIO = 1.0 / 256.0  # d / (leaf width), i.e. 2d = w/128


def interaction_list(l, periodic, cx, cy, cz):
    """§2.2 step 3: the interaction list of cell (cx, cy, cz) of level l, the list
    the downward pass iterates over: (source cells in natural order (z S + y) S +
    x, offset indices ((oz + 3) 7 + oy + 3) 7 + ox + 3), in (z, y, x) order of
    the source; open form: sources inside the box only; periodic: wrapped."""
    src = np.zeros(189, np.int64)
    oi = np.zeros(189, np.int32)
    m = lib().orc_interaction_list(int(l), int(periodic), int(cx), int(cy), int(cz), _p(src), _p(oi))
    return src[:m].copy(), oi[:m].copy()


def level_offset(n, l):
    return int(lib().orc_level_offset(n, l))


def fmm(pos, q, box, depth, n, periodic=False, continuous=False, dt=None, sample=None,
        keep=True, grid_scale=1.0, shift_free=False, force_kernel=False, power=1):
    """Runs the oracle FMM; grid_scale < 1 takes the reduced arrangement of the
    n-division points (§4.1: spacing times grid_scale about the cell centre);
    shift_free takes the bilinear forms without shifts of App. A.2 (grid
    charges and functionals of every cell with respect to the box).  See _fmm
    for the other arguments.  force_kernel takes the far forces from the force
    kernels (x - x~)/|P - P~|^3 (§4.1) instead of the derivative of the weights;
    "F" is then the sum of the forces on a particle's charges.  power=2 takes
    F(P, P~) = 1/|P - P~|^2 (the other function §4.1 names) for the far forms
    and the near field alike (open boundary: its lattice sum diverges)."""
    if continuous and grid_scale != 1.0:
        raise ValueError("the reduced arrangement is defined for the plain form")
    if shift_free and force_kernel:
        raise ValueError("the shift-free forms are built for the potential kernel")
    if power != 1 and (periodic or shift_free):
        raise ValueError("1/r^2: open boundary, shifted forms only")
    L_ = lib()
    L_.orc_set_grid_scale(float(grid_scale))
    L_.orc_set_power(int(power))
    try:
        out = _fmm(pos, q, box, depth, n, periodic, continuous, dt, sample, keep, shift_free,
                   force_kernel)
    finally:
        L_.orc_set_grid_scale(1.0)
        L_.orc_set_kernel(0)
        L_.orc_set_power(1)
    if power != 1:  # unit-box results scale as L^-power (potential), L^-(power+1) (forces)
        Lb = float(np.asarray(box, np.float64)[3])
        f_phi, f_F = Lb / Lb ** power, Lb ** 2 / Lb ** (power + 1)
        for k in ("phi", "E"):
            if out.get(k) is not None:
                out[k] = out[k] * f_phi
        for k in ("F", "F_paper"):
            out[k] = out[k] * f_F
    return out


def _fmm(pos, q, box, depth, n, periodic=False, continuous=False, dt=None, sample=None,
         keep=True, shift_free=False, force_kernel=False):
    """Runs the oracle FMM.

    pos: (N,3) float32 positions, q: (N,) float32 charges, box = (x0,y0,z0,L).
    dt: split half-width d in units of the finest-cell width (float32);
        default 1/256.
    sample: optional particle indices; then only the outputs of those
        particles are computed (upward pass in full, downward pass and
        evaluation only where those particles need them) and E is None.

    shift_free: App. A.2; Phi and L of the result are then the box-basis
        vectors Phi^S and L^S of every cell.

    Returns a dict with phi (potential per unit charge), F (adjoint force),
    F_paper, E (physical units), and the intermediates when keep=True.
    """
    L_ = lib()
    pos = _c(pos, np.float32).reshape(-1, 3)
    qf = _c(q, np.float32).reshape(-1)
    N = pos.shape[0]
    box = _c(box, np.float64)
    if depth < 2:
        raise ValueError("depth must be >= 2 (§2.2 step 1)")
    dtf = np.float32(DEFAULT_SPLIT_RATIO if dt is None else dt)
    S = 1 << depth
    n3 = n ** 3

    # step 1: divide the box
    u = np.empty((N, 3), np.float32)
    t = np.empty((N, 3), np.float32)
    cell = np.empty((N, 3), np.int32)
    key = np.empty(N, np.uint32)
    err = L_.orc_bin(N, _p(pos), _p(box), depth, int(periodic), _p(u), _p(t), _p(cell), _p(key))
    if err:
        raise ValueError("oracle: input outside the box or not finite (flags %d)" % err)

    # §2.3 split (one charge per particle when not continuous)
    count = np.empty(N, np.int32)
    axes = np.empty((N, 3), np.int8)
    L_.orc_split_count(N, _p(t), _p(cell), n, depth, int(periodic), int(continuous), dtf,
                       _p(count), _p(axes))
    offset = np.zeros(N + 1, np.int64)
    np.cumsum(count, out=offset[1:])
    npts = int(offset[-1])
    pt_t = np.empty((npts, 3))
    pt_cell = np.empty((npts, 3), np.int32)
    pt_key = np.empty(npts, np.uint32)
    pt_q = np.empty(npts)
    pt_w = np.empty(npts)
    pt_dw = np.empty((npts, 3))
    pt_origin = np.empty(npts, np.int64)
    L_.orc_split_emit(N, _p(t), _p(cell), _p(qf), n, depth, int(periodic), int(continuous), dtf,
                      _p(offset), _p(pt_t), _p(pt_cell), _p(pt_key), _p(pt_q), _p(pt_w),
                      _p(pt_dw), _p(pt_origin))

    # finest-cell ranges
    perm = np.empty(npts, np.int64)
    start = np.empty(S ** 3 + 1, np.int64)
    L_.orc_sort(npts, _p(pt_key), depth, _p(perm), _p(start))
    st = _c(pt_t[perm], np.float64)
    scell = _c(pt_cell[perm], np.int32)
    sq = _c(pt_q[perm], np.float64)
    sorigin = _c(pt_origin[perm], np.int64)

    # step 2: upward pass
    Phi = np.zeros(level_offset(n, depth + 1))
    lmin = 0 if periodic else 2
    if shift_free:
        L_.orc_sf_p2m(n, depth, _p(st), _p(scell), _p(sq), _p(start), _p(Phi))
        L_.orc_sf_upward(n, depth, lmin, _p(Phi))
    else:
        L_.orc_p2m(n, depth, _p(st), _p(sq), _p(start), _p(Phi))
        L_.orc_m2m(n, depth, lmin, _p(Phi))

    # step 3: downward pass
    Klat = lattice_kernel(n) if periodic else None
    need_arrays = None
    need_ptrs = None
    mask = None
    if sample is not None:
        sample = _c(sample, np.int64)
        want = np.zeros(N, bool)
        want[sample] = True
        mask = want[sorigin].astype(np.uint8)
        need_arrays = [np.zeros(8 ** l, np.uint8) for l in range(depth + 1)]
        c = scell[mask.astype(bool)]
        for l in range(depth, -1, -1):
            cl = c >> (depth - l)
            sl = 1 << l
            need_arrays[l][(cl[:, 2] * sl + cl[:, 1]) * sl + cl[:, 0]] = 1
        ptr_t = ctypes.c_void_p * (depth + 1)
        need_ptrs = ptr_t(*[a.ctypes.data for a in need_arrays])
    Lv = np.zeros_like(Phi)
    need_arg = ctypes.cast(need_ptrs, ctypes.c_void_p) if need_ptrs is not None else None
    if shift_free:
        if L_.orc_sf_downward(n, depth, int(periodic), _p(Phi), _p(Lv), need_arg,
                              _p(Klat) if Klat is not None else None):
            raise ArithmeticError("singular shift")
    else:
        L_.orc_downward(n, depth, int(periodic), _p(Phi), _p(Lv), need_arg,
                        _p(Klat) if Klat is not None else None)

    LF = []
    if force_kernel:  # the functionals of the three force kernels, same lists
        for c in (1, 2, 3):
            L_.orc_set_kernel(c)
            Kc = lattice_kernel(n, c) if periodic else None
            L_.orc_set_kernel(c)
            LF.append(np.zeros_like(Phi))
            L_.orc_downward(n, depth, int(periodic), _p(Phi), _p(LF[-1]), need_arg,
                            _p(Kc) if Kc is not None else None)
        L_.orc_set_kernel(0)

    # steps 4-5 at every charge
    phi_pt = np.zeros(npts)
    F_pt = np.zeros((npts, 3))
    ncoinc = ctypes.c_int64(0)
    if force_kernel:
        L_.orc_evaluate_kernel(n, depth, int(periodic), npts, _p(st), _p(scell), _p(sq),
                               _p(sorigin), _p(start), _p(Lv), _p(LF[0]), _p(LF[1]), _p(LF[2]),
                               _p(mask), _p(phi_pt), _p(F_pt), ctypes.byref(ncoinc))
    else:
        evaluate = L_.orc_sf_evaluate if shift_free else L_.orc_evaluate
        evaluate(n, depth, int(periodic), npts, _p(st), _p(scell), _p(sq), _p(sorigin),
                 _p(start), _p(Lv), _p(mask), _p(phi_pt), _p(F_pt), ctypes.byref(ncoinc))

    # split charges back into their particles
    inv = np.empty(npts, np.int64)
    inv[perm] = np.arange(npts, dtype=np.int64)
    phi_e = phi_pt[inv]
    F_e = F_pt[inv]
    phi_u = np.bincount(pt_origin, weights=pt_w * phi_e, minlength=N)
    F_paper = np.stack([np.bincount(pt_origin, weights=F_e[:, a], minlength=N)
                        for a in range(3)], axis=1)
    F_norm = np.stack([-qf.astype(np.float64) *
                       np.bincount(pt_origin, weights=pt_dw[:, a] * phi_e, minlength=N)
                       for a in range(3)], axis=1)
    F_adj = F_paper if force_kernel else np.where(axes.astype(bool), F_norm, F_paper)

    Lb = float(box[3])
    out = {
        "phi": phi_u / Lb,
        "F": F_adj / (Lb * Lb),
        "F_paper": F_paper / (Lb * Lb),
        "E": None if sample is not None else 0.5 * float(np.dot(qf.astype(np.float64), phi_u)) / Lb,
        "n_coincident": int(ncoinc.value),
        "n_points": npts,
    }
    if sample is not None:
        out["phi"] = out["phi"][sample]
        out["F"] = out["F"][sample]
        out["F_paper"] = out["F_paper"][sample]
    if keep:
        out.update(dict(u=u, t=t, cell=cell, key=key, count=count, axes=axes, offset=offset,
                        pt_t=pt_t, pt_cell=pt_cell, pt_key=pt_key, pt_q=pt_q, pt_w=pt_w,
                        pt_dw=pt_dw, pt_origin=pt_origin, perm=perm, start=start, Phi=Phi,
                        L=Lv, LF=LF, phi_pt=phi_pt, F_pt=F_pt))
    return out


def level_view(arr, n, l):
    """Level l of a Phi/L array as (8^l, n^3), natural cell order."""
    a, b = level_offset(n, l), level_offset(n, l + 1)
    return arr[a:b].reshape(8 ** l, n ** 3)
