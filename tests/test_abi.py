"""The C-ABI library builds, loads, and exports every symbol the header declares
(no compute: this runs without a GPU)."""
import os
import re
import subprocess

from conftest import ROOT


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_header_symbols():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2212_13080_gb300 import _binding
    lib = _binding.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fmm_[a-z_0-9]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert sorted(declared) == sorted(_binding.EXPORTED)


def test_host_only_entry_points():
    from paper_2212_13080_gb300 import _binding as B
    assert B.fmm_version() >= 100
    assert B.fmm_strerror(B.FMM_ERR_OUT_OF_BOX) == "position outside the box (open form)"
    assert B.fmm_strerror(12345) == "unknown status"
    o = B.fmm_opts_default()
    assert o.continuous == 0 and abs(o.split_ratio - 1 / 256) < 1e-15 and o.sync == 1


def test_plan_argument_checks():
    """Invalid arguments are rejected before any device call."""
    import ctypes
    from paper_2212_13080_gb300 import _binding as B
    L = B.lib()
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 4)(0, 0, 0, 1)
    for depth, p, max_n in [(1, 4, 10), (9, 4, 10), (3, 1, 10), (3, 9, 10), (3, 4, -1)]:
        assert L.fmm_plan_create(ctypes.byref(h), box, depth, p, 0, None, max_n) == B.FMM_ERR_ARG
    bad = (ctypes.c_double * 4)(0, 0, 0, 0)
    assert L.fmm_plan_create(ctypes.byref(h), bad, 3, 4, 0, None, 10) == B.FMM_ERR_ARG
    o = B.fmm_opts_default()
    o.continuous = 1
    o.split_ratio = 0.6
    assert L.fmm_plan_create(ctypes.byref(h), box, 3, 4, 0, ctypes.byref(o), 10) == B.FMM_ERR_ARG
    assert L.fmm_eval(None, 1, None, None, None, None, None, None, 0, None) == B.FMM_ERR_ARG
    assert L.fmm_batch_set_schedule(None, 0) == B.FMM_ERR_ARG


def test_shift_free_options_rejected_before_any_device_call():
    """App. A.2 plans: FP64 only (the forms extrapolate over 2^l cells), p <= 5,
    the standard arrangement, tables of at most 32 GiB, single systems; the
    checks come before the plan touches the device."""
    import pytest
    from paper_2212_13080_gb300 import _binding as B
    box = (0.0, 0.0, 0.0, 1.0)

    def opts(**kw):
        o = B.fmm_opts_default()
        o.precision = B.FMM_PREC_FP64
        o.shift_free = 1
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    for depth, p, o in [(3, 4, opts(precision=B.FMM_PREC_FP32)),
                        (3, 4, opts(precision=B.FMM_PREC_TF32X3)),
                        (2, 6, opts()),
                        (3, 4, opts(grid_scale=1 / 1.2)),
                        (4, 5, opts())]:  # 110 GB of forms
        with pytest.raises(B.FmmError) as e:
            B.fmm_plan_create(box, depth, p, False, o, 1000)
        assert e.value.code == B.FMM_ERR_UNSUPPORTED, (depth, p)


def test_force_mode_validated_before_any_device_call():
    import pytest
    from paper_2212_13080_gb300 import _binding as B
    box = (0.0, 0.0, 0.0, 1.0)
    o = B.fmm_opts_default()
    o.force_mode = 7
    with pytest.raises(B.FmmError) as e:
        B.fmm_plan_create(box, 3, 4, False, o, 1000)
    assert e.value.code == B.FMM_ERR_ARG
    o = B.fmm_opts_default()
    o.force_mode = B.FMM_FORCE_KERNEL
    o.precision = B.FMM_PREC_FP64
    o.shift_free = 1
    with pytest.raises(B.FmmError) as e:
        B.fmm_plan_create(box, 3, 4, False, o, 1000)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED


def test_inverse_square_kernel_options():
    """1/r^2: open boundary only (its lattice sum diverges), not shift-free."""
    import pytest
    from paper_2212_13080_gb300 import _binding as B
    box = (0.0, 0.0, 0.0, 1.0)
    o = B.fmm_opts_default()
    assert o.kernel == B.FMM_KERNEL_COULOMB
    o.kernel = B.FMM_KERNEL_INV_SQUARE
    with pytest.raises(B.FmmError) as e:
        B.fmm_plan_create(box, 3, 4, True, o, 1000)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED
    o.precision = B.FMM_PREC_FP64
    o.shift_free = 1
    with pytest.raises(B.FmmError) as e:
        B.fmm_plan_create(box, 3, 4, False, o, 1000)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED
    o = B.fmm_opts_default()
    o.kernel = 5
    with pytest.raises(B.FmmError) as e:
        B.fmm_plan_create(box, 3, 4, False, o, 1000)
    assert e.value.code == B.FMM_ERR_ARG
