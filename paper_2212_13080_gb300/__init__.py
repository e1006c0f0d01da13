"""GB300-native replacement-based fast multipole method.

Y. Kajima, "Notes on the Fast Multipole Method" (arXiv:2212.13080): charges
of every octree cell are replaced by charges on the cell's p-division points
(§2.1), far interactions are dense p^3 x p^3 bilinear forms between grid
charges (§2.1.7), near interactions a direct sum over 27 cells (§2.2); the
continuous form splits charges near cell planes (§2.3) and the periodic form
also at the box walls (§4.2).

All computation runs in libfmm_gb300.so (hand-written sm_103a kernels behind a
C ABI, include/fmm_gb300.h); this package only marshals torch tensors to it.
PyTorch supplies device memory and streams.
"""
import ctypes

import torch

from . import _binding as B
from ._binding import FmmError  # noqa: F401

__all__ = ["FMM", "FMMBatch", "FmmError", "fmm_energy"]

_PREC = {"fp32": B.FMM_PREC_FP32, "fp64": B.FMM_PREC_FP64, "tf32x3": B.FMM_PREC_TF32X3,
         "tf32x1": B.FMM_PREC_TF32X1, "bf16x3": B.FMM_PREC_BF16X3}
_FORCE = {"adjoint": B.FMM_FORCE_ADJOINT, "paper": B.FMM_FORCE_PAPER, "kernel": B.FMM_FORCE_KERNEL}
_KERNEL = {"coulomb": B.FMM_KERNEL_COULOMB, "inverse_square": B.FMM_KERNEL_INV_SQUARE}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class FMM:
    """One plan of the method: box (x0, y0, z0, L), octree depth, order p.

    eval(pos, q) -> dict(potential, energy, forces) for device tensors
    (float32 positions (n,3), charges (n,)); outputs are float32, or float64
    for precision="fp64".  Host tensors are copied to the device and the
    results back (the end-to-end path); host results are views of pinned
    buffers the plan keeps and overwrites on its next host call (clone to keep).
    precision: "fp32" (SIMT contraction), "fp64", "tf32x3" / "tf32x1" /
    "bf16x3" (bilinear forms of every level on the tcgen05 tensor cores).
    grid_scale < 1: the reduced arrangement of the p-division points (§4.1).
    shift_free: App. A.2, precomputed bilinear forms on box-basis grid charges
    (precision "fp64", p <= 5).
    force_mode: "adjoint" (-dE/dx), "paper" (split charges' forces summed) or
    "kernel" (far forces from the force kernels, §4.1).
    kernel: "coulomb" (1/r) or "inverse_square" (1/r^2, open boundary).
    """

    def __init__(self, box, depth, p, periodic=False, continuous=False, split_ratio=None,
                 precision="fp32", force_mode="adjoint", max_n=1 << 20, split_capacity=None,
                 sync=True, device=None, grid_scale=1.0, shift_free=False, kernel="coulomb"):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.box = tuple(float(x) for x in box)
        self.depth, self.p, self.periodic, self.continuous = int(depth), int(p), bool(periodic), bool(continuous)
        self.precision = precision
        self.max_n = int(max_n)
        o = B.fmm_opts_default()
        o.continuous = int(self.continuous)
        if split_ratio is not None:
            o.split_ratio = float(split_ratio)
        if split_capacity is not None:
            o.split_capacity = float(split_capacity)
        o.precision = _PREC[precision]
        o.force_mode = _FORCE[force_mode]
        # the library call never waits here: with sync=True the status is read
        # after the call (device inputs) or after the output copies (host inputs),
        # one wait per call either way
        self.sync = bool(sync)
        o.sync = 0
        o.grid_scale = float(grid_scale)
        o.shift_free = int(bool(shift_free))
        o.kernel = _KERNEL[kernel]
        self.shift_free = bool(shift_free)
        with torch.cuda.device(self.device):
            self._h = B.fmm_plan_create(self.box, self.depth, self.p, self.periodic, o, self.max_n)
        self.out_dtype = torch.float64 if precision == "fp64" else torch.float32
        self._ws = None
        self._last = None

    def close(self):
        if getattr(self, "_h", None):
            B.fmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self, n):
        return B.fmm_workspace_size(self._h, n)

    def workspace(self, n):
        """A device workspace for n particles (kept by the plan and reused)."""
        need = self.workspace_size(n)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        return self._ws

    @staticmethod
    def _aligned(ws):
        off = (-ws.data_ptr()) % 256
        return ws[off:]

    def eval(self, pos, q, potential=True, energy=True, forces=True, workspace=None, stream=None,
             out=None):
        host = pos.device.type == "cpu"
        if host:
            pos_d = pos.to(self.device, non_blocking=True)
            q_d = q.to(self.device, non_blocking=True)
        else:
            pos_d, q_d = pos, q
        if pos_d.dtype != torch.float32 or q_d.dtype != torch.float32:
            raise TypeError("positions and charges must be float32")
        pos_d = pos_d.contiguous()
        q_d = q_d.contiguous()
        n = q_d.numel()
        if pos_d.numel() != 3 * n:
            raise ValueError("pos must be (n, 3) with n = q.numel()")
        ws = self._aligned(self.workspace(n) if workspace is None else workspace)
        o = out if out is not None else {}
        phi = o.get("potential")
        if potential and phi is None:
            phi = torch.empty(n, dtype=self.out_dtype, device=self.device)
        E = o.get("energy")
        if energy and E is None:
            E = torch.empty(1, dtype=torch.float64, device=self.device)
        F = o.get("forces")
        if forces and F is None:
            F = torch.empty((n, 3), dtype=self.out_dtype, device=self.device)
        if self.sync and torch.cuda.is_current_stream_capturing():
            # the status wait after the call would end the capture (as the library's
            # own opts.sync = 1 refuses it): plans for captured streams take sync=False
            raise FmmError(B.FMM_ERR_ARG, "fmm_eval (sync plan on a stream being captured)")
        # recorded first: a failed call's workspace still holds its status and wait site
        self._last = (ws, n, pos_d, q_d)
        B.fmm_eval(self._h, n, _ptr(pos_d), _ptr(q_d), _ptr(phi) if potential else None,
                   _ptr(E) if energy else None, _ptr(F) if forces else None, _ptr(ws),
                   ws.numel(), _stream(stream))
        res = {"potential": phi if potential else None, "energy": E if energy else None,
               "forces": F if forces else None}
        if self.sync and not host:
            self._check_status(ws, stream)
        if host:
            # results into pinned host buffers (kept by the plan), one wait at the end
            hb = self._host_out(n)
            stream_t = torch.cuda.current_stream() if stream is None else stream
            out_h = {}
            for k, v in res.items():
                if v is None:
                    out_h[k] = None
                    continue
                h = hb[k][: v.numel()].view(v.shape)
                h.copy_(v, non_blocking=True)
                out_h[k] = h
            # the device status word travels with the outputs; only a nonzero
            # word needs the library's decoding (a second, short read)
            hb["status"].copy_(ws[:4].view(torch.int32), non_blocking=True)
            stream_t.synchronize()
            if int(hb["status"][0]) != 0:
                self._check_status(ws, stream)
            res = out_h
        return res

    def _check_status(self, ws, stream, where="fmm_eval"):
        rc = B.fmm_status(self._h, _ptr(ws), _stream(stream))
        if rc:
            raise FmmError(rc, where)

    def _host_out(self, n):
        hb = getattr(self, "_hbuf", None)
        if hb is None or hb["n"] < n:
            hb = {"n": n,
                  "potential": torch.empty(n, dtype=self.out_dtype).pin_memory(),
                  "energy": torch.empty(1, dtype=torch.float64).pin_memory(),
                  "forces": torch.empty(3 * n, dtype=self.out_dtype).pin_memory(),
                  "status": torch.zeros(1, dtype=torch.int32).pin_memory()}
            self._hbuf = hb
        return hb

    def backward(self, grad_energy, stream=None):
        """dLoss/dpos = -F * gE and dLoss/dq = phi * gE from the last eval's state."""
        if self._last is None:
            raise FmmError(B.FMM_ERR_STATE, "fmm_backward")
        ws, n, pos_d, q_d = self._last
        gE = grad_energy.to(device=self.device, dtype=torch.float64).reshape(1).contiguous()
        gpos = torch.empty((n, 3), dtype=self.out_dtype, device=self.device)
        gq = torch.empty(n, dtype=self.out_dtype, device=self.device)
        B.fmm_backward(self._h, n, _ptr(pos_d), _ptr(q_d), _ptr(gE), _ptr(gpos), _ptr(gq),
                       _ptr(ws), ws.numel(), _stream(stream))
        if self.sync:  # the device-side checks, among them the workspace's evaluation tag
            self._check_status(ws, stream, "fmm_backward")
        return gpos, gq

    def inject(self, what="tc_stall"):
        """Failure-detection test hook: the next evaluation's tensor-core
        contraction withholds one stage's copies, its bounded wait expires and
        the call raises FMM_ERR_TIMEOUT ("none" disarms)."""
        B.fmm_debug_inject(self._h, {"none": B.FMM_INJECT_NONE, "tc_stall": B.FMM_INJECT_TC_STALL}[what])

    def set_timing(self, on=True, serial=False):
        """Bracket every stage of later calls with CUDA events (see stats()).

        serial=True runs every stage on the call's stream (no near/far overlap), so
        that each stage time is its kernels' own duration."""
        B.fmm_set_timing(self._h, (2 if serial else 1) if on else 0)

    def stats(self):
        """Launch count and per-stage device time (ms) of the last call."""
        return B.fmm_get_stats(self._h)

    def dump(self, what, stream=None):
        """An intermediate of the last evaluation (debug / parity), as a torch CPU tensor."""
        import numpy as np
        if self._last is None:
            raise FmmError(B.FMM_ERR_STATE, "fmm_debug_dump")
        ws = self._last[0]
        code = getattr(B, "FMM_DUMP_" + what.upper())
        nb = B.fmm_debug_size(self._h, code, _ptr(ws), _stream(stream))
        buf = np.empty(max(nb, 1), dtype=np.uint8)
        B.fmm_debug_dump(self._h, code, _ptr(ws), buf.ctypes.data_as(ctypes.c_void_p), nb,
                         _stream(stream))
        buf = buf[:nb]
        real = np.float64 if self.precision == "fp64" else np.float32
        if what in ("counts", "origin", "perm", "start", "wait"):
            return buf.view(np.int32)
        if what == "keys":
            return buf.view(np.uint32)
        if what in ("points", "out"):
            return buf.view(real).reshape(-1, 4)
        return buf.view(real).reshape(-1, self.p ** 3)


class FMMBatch:
    """Many independent systems (own box, depth, particle count; one p, form
    and precision) evaluated together: one CUDA-graph launch per call after
    the first (which also picks the number of stream lanes by timing).

    eval(pos, q, offsets) with pos (N,3) / q (N,) device tensors holding the
    systems' particles back to back and offsets (nsys+1) the CSR boundaries
    -> dict(potential (N,), energy (nsys,), forces (N,3)).
    """

    def __init__(self, boxes, depths, p, periodic=False, continuous=False, split_ratio=None,
                 precision="fp32", force_mode="adjoint", max_n=None, split_capacity=None,
                 sync=True, device=None, kernel="coulomb"):
        import numpy as np
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.nsys = len(depths)
        o = B.fmm_opts_default()
        o.continuous = int(bool(continuous))
        if split_ratio is not None:
            o.split_ratio = float(split_ratio)
        if split_capacity is not None:
            o.split_capacity = float(split_capacity)
        o.precision = _PREC[precision]
        o.force_mode = _FORCE[force_mode]
        o.kernel = _KERNEL[kernel]
        o.sync = int(bool(sync))
        self.out_dtype = torch.float64 if precision == "fp64" else torch.float32
        with torch.cuda.device(self.device):
            self._h = B.fmm_batch_create(np.asarray(boxes, np.float64).reshape(-1, 4),
                                         np.asarray(depths), p, periodic, o,
                                         np.asarray(max_n, np.int64))
        self._ws = None

    def close(self):
        if getattr(self, "_h", None):
            B.fmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, pos, q, offsets, potential=True, energy=True, forces=True, stream=None,
             out=None):
        import numpy as np
        offs = np.asarray(offsets, np.int64)
        counts = np.diff(offs)
        need = B.fmm_batch_workspace_size(self._h, counts)
        if self._ws is None or self._ws.numel() < need + 256:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        ws = FMM._aligned(self._ws)
        n = int(offs[-1])
        o = out if out is not None else {}
        phi = o.get("potential") if potential else None
        if potential and phi is None:
            phi = torch.empty(n, dtype=self.out_dtype, device=self.device)
        E = o.get("energy") if energy else None
        if energy and E is None:
            E = torch.empty(self.nsys, dtype=torch.float64, device=self.device)
        F = o.get("forces") if forces else None
        if forces and F is None:
            F = torch.empty((n, 3), dtype=self.out_dtype, device=self.device)
        B.fmm_batch_eval(self._h, offs, _ptr(pos.contiguous()), _ptr(q.contiguous()), _ptr(phi),
                         _ptr(E), _ptr(F), _ptr(ws), ws.numel(), _stream(stream))
        return {"potential": phi, "energy": E, "forces": F}

    def stats(self):
        return B.fmm_batch_get_stats(self._h)

    def set_schedule(self, schedule):
        """Fixes the merged launches' schedule (0: one stream, 1: the near
        field on a second stream) or returns to the autotuner (-1)."""
        B.fmm_batch_set_schedule(self._h, schedule)


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, q, plan):
        r = plan.eval(pos, q, potential=False, energy=True, forces=False)
        ctx.plan = plan
        return r["energy"][0]

    @staticmethod
    def backward(ctx, gE):
        gpos, gq = ctx.plan.backward(gE.detach())
        return gpos.to(torch.float32), gq.to(torch.float32), None


def fmm_energy(plan, pos, q):
    """Differentiable FMM energy: backward gives dE/dpos = -F and dE/dq = phi,
    computed by the library's adjoint pass from the evaluation's kept state."""
    return _Energy.apply(pos, q, plan)
