"""ctypes binding of libfmm_gb300.so: argument marshalling only.

Every function here has the name of the C entry point it forwards to and does
no arithmetic of the method: all of it runs in the library's CUDA kernels.
The library must have been built (build.py); a missing library raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfmm_gb300.so")

FMM_OK = 0
FMM_ERR_ARG = 1
FMM_ERR_OOM = 2
FMM_ERR_OUT_OF_BOX = 3
FMM_ERR_NONFINITE = 4
FMM_ERR_SPLIT_OVERFLOW = 5
FMM_ERR_TIMEOUT = 6
FMM_ERR_CUDA = 7
FMM_ERR_STATE = 8
FMM_ERR_WORKSPACE = 9
FMM_ERR_UNSUPPORTED = 10

FMM_PREC_FP32 = 0
FMM_PREC_FP64 = 1
FMM_PREC_TF32X3 = 2
FMM_PREC_TF32X1 = 3
FMM_PREC_BF16X3 = 4

FMM_FORCE_ADJOINT = 0
FMM_FORCE_PAPER = 1
FMM_FORCE_KERNEL = 2
FMM_KERNEL_COULOMB = 0
FMM_KERNEL_INV_SQUARE = 1

FMM_DUMP_COUNTS = 0
FMM_DUMP_KEYS = 1
FMM_DUMP_ORIGIN = 2
FMM_DUMP_PERM = 3
FMM_DUMP_START = 4
FMM_DUMP_POINTS = 5
FMM_DUMP_PHI = 6
FMM_DUMP_LOCAL = 7
FMM_DUMP_OUT = 8
FMM_DUMP_WAIT = 9
FMM_INJECT_NONE = 0
FMM_INJECT_TC_STALL = 1

# every symbol include/fmm_gb300.h declares
EXPORTED = ["fmm_opts_default", "fmm_plan_create", "fmm_plan_destroy", "fmm_workspace_size",
            "fmm_eval", "fmm_backward", "fmm_status", "fmm_debug_dump", "fmm_debug_size",
            "fmm_set_timing", "fmm_get_stats", "fmm_strerror", "fmm_version",
            "fmm_eval_static", "fmm_batch_create", "fmm_batch_destroy",
            "fmm_batch_workspace_size", "fmm_batch_eval", "fmm_batch_get_stats",
            "fmm_batch_set_schedule", "fmm_debug_inject"]

FMM_STATIC_WORKSPACE_BYTES = 32 << 20

STAGES = ["bin", "sort", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "unsplit"]


class fmm_opts_t(ctypes.Structure):
    _fields_ = [("continuous", ctypes.c_int), ("split_ratio", ctypes.c_double),
                ("split_capacity", ctypes.c_double), ("precision", ctypes.c_int),
                ("force_mode", ctypes.c_int), ("sync", ctypes.c_int),
                ("grid_scale", ctypes.c_double), ("shift_free", ctypes.c_int),
                ("kernel", ctypes.c_int)]


class fmm_stats_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int), ("timed", ctypes.c_int),
                ("stage_ms", ctypes.c_double * 9)]


class fmm_batch_stats_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int), ("lanes", ctypes.c_int), ("graph", ctypes.c_int),
                ("tune_ms", ctypes.c_double * 8), ("merged", ctypes.c_int), ("schedule", ctypes.c_int)]


class FmmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, fmm_strerror(code), code))


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfmm_gb300.so is not built (%s): run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        L.fmm_opts_default.argtypes = [ctypes.POINTER(fmm_opts_t)]
        L.fmm_opts_default.restype = None
        L.fmm_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ctypes.c_double), i32, i32,
                                      i32, ctypes.POINTER(fmm_opts_t), i64]
        L.fmm_plan_destroy.argtypes = [P]
        L.fmm_plan_destroy.restype = None
        L.fmm_workspace_size.argtypes = [P, i64, ctypes.POINTER(sz)]
        L.fmm_eval.argtypes = [P, i64, P, P, P, P, P, P, sz, P]
        L.fmm_backward.argtypes = [P, i64, P, P, P, P, P, P, sz, P]
        L.fmm_status.argtypes = [P, P, P]
        L.fmm_debug_dump.argtypes = [P, i32, P, P, sz, P]
        L.fmm_debug_size.argtypes = [P, i32, P, ctypes.POINTER(sz), P]
        L.fmm_set_timing.argtypes = [P, i32]
        L.fmm_debug_inject.argtypes = [P, i32]
        L.fmm_get_stats.argtypes = [P, ctypes.POINTER(fmm_stats_t)]
        L.fmm_strerror.argtypes = [i32]
        L.fmm_strerror.restype = ctypes.c_char_p
        L.fmm_version.argtypes = []
        L.fmm_eval_static.argtypes = [P, i64, P, P, P, P, P, P]
        L.fmm_batch_create.argtypes = [ctypes.POINTER(P), i32, P, P, i32, i32,
                                       ctypes.POINTER(fmm_opts_t), P]
        L.fmm_batch_destroy.argtypes = [P]
        L.fmm_batch_destroy.restype = None
        L.fmm_batch_workspace_size.argtypes = [P, P, ctypes.POINTER(sz)]
        L.fmm_batch_eval.argtypes = [P, P, P, P, P, P, P, P, sz, P]
        L.fmm_batch_get_stats.argtypes = [P, ctypes.POINTER(fmm_batch_stats_t)]
        L.fmm_batch_set_schedule.argtypes = [P, i32]
        _lib = L
    return _lib


def fmm_strerror(code):
    return lib().fmm_strerror(int(code)).decode()


def fmm_version():
    return lib().fmm_version()


def fmm_opts_default():
    o = fmm_opts_t()
    lib().fmm_opts_default(ctypes.byref(o))
    return o


def _check(rc, where):
    if rc != FMM_OK:
        raise FmmError(rc, where)


def fmm_plan_create(box, depth, p, periodic, opts, max_n):
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 4)(*[float(x) for x in box])
    _check(lib().fmm_plan_create(ctypes.byref(h), b, int(depth), int(p), int(bool(periodic)),
                                 ctypes.byref(opts) if opts is not None else None, int(max_n)),
           "fmm_plan_create")
    return h


def fmm_plan_destroy(h):
    if h:
        lib().fmm_plan_destroy(h)


def fmm_workspace_size(h, n):
    s = ctypes.c_size_t()
    _check(lib().fmm_workspace_size(h, int(n), ctypes.byref(s)), "fmm_workspace_size")
    return s.value


def fmm_eval(h, n, pos, q, potential, energy, forces, workspace, ws_bytes, stream):
    _check(lib().fmm_eval(h, int(n), pos, q, potential, energy, forces, workspace, ws_bytes,
                          stream), "fmm_eval")


def fmm_backward(h, n, pos, q, grad_energy, grad_pos, grad_q, workspace, ws_bytes, stream):
    _check(lib().fmm_backward(h, int(n), pos, q, grad_energy, grad_pos, grad_q, workspace,
                              ws_bytes, stream), "fmm_backward")


def fmm_status(h, workspace, stream):
    return lib().fmm_status(h, workspace, stream)


def fmm_debug_size(h, what, workspace, stream):
    s = ctypes.c_size_t()
    _check(lib().fmm_debug_size(h, int(what), workspace, ctypes.byref(s), stream),
           "fmm_debug_size")
    return s.value


def fmm_debug_dump(h, what, workspace, dst, nbytes, stream):
    _check(lib().fmm_debug_dump(h, int(what), workspace, dst, nbytes, stream), "fmm_debug_dump")


def fmm_set_timing(h, on):
    _check(lib().fmm_set_timing(h, int(on)), "fmm_set_timing")


def fmm_debug_inject(h, what):
    _check(lib().fmm_debug_inject(h, int(what)), "fmm_debug_inject")


def fmm_get_stats(h):
    st = fmm_stats_t()
    _check(lib().fmm_get_stats(h, ctypes.byref(st)), "fmm_get_stats")
    return {"launches": st.launches, "timed": bool(st.timed),
            "stage_ms": dict(zip(STAGES, list(st.stage_ms)))}


def fmm_batch_create(boxes, depths, p, periodic, opts, max_n):
    import numpy as np
    h = ctypes.c_void_p()
    b = np.ascontiguousarray(boxes, dtype=np.float64)
    d = np.ascontiguousarray(depths, dtype=np.int32)
    m = np.ascontiguousarray(max_n, dtype=np.int64)
    _check(lib().fmm_batch_create(ctypes.byref(h), len(d), b.ctypes.data_as(ctypes.c_void_p),
                                  d.ctypes.data_as(ctypes.c_void_p), int(p), int(bool(periodic)),
                                  ctypes.byref(opts) if opts is not None else None,
                                  m.ctypes.data_as(ctypes.c_void_p)), "fmm_batch_create")
    return h


def fmm_batch_destroy(h):
    if h:
        lib().fmm_batch_destroy(h)


def fmm_batch_workspace_size(h, n):
    import numpy as np
    a = np.ascontiguousarray(n, dtype=np.int64)
    s = ctypes.c_size_t()
    _check(lib().fmm_batch_workspace_size(h, a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(s)),
           "fmm_batch_workspace_size")
    return s.value


def fmm_batch_eval(h, offsets, pos, q, potential, energy, forces, workspace, ws_bytes, stream):
    import numpy as np
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(lib().fmm_batch_eval(h, o.ctypes.data_as(ctypes.c_void_p), pos, q, potential, energy,
                                forces, workspace, ws_bytes, stream), "fmm_batch_eval")


def fmm_batch_set_schedule(h, schedule):
    _check(lib().fmm_batch_set_schedule(h, int(schedule)), "fmm_batch_set_schedule")


def fmm_batch_get_stats(h):
    st = fmm_batch_stats_t()
    _check(lib().fmm_batch_get_stats(h, ctypes.byref(st)), "fmm_batch_get_stats")
    tm = list(st.tune_ms)
    return {"launches": st.launches, "lanes": st.lanes, "graph": bool(st.graph), "merged": bool(st.merged),
            "schedule": st.schedule,
            "tune_ms": ({"one_stream": tm[5], "near_stream": tm[6]} if st.merged
                        else dict(zip([2, 4, 8, 16, 32], tm[:5])))}
