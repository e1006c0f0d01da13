#!/usr/bin/env python
"""Benchmark of the replacement-based FMM (energy + potentials + forces).

Workload (default "plummer8m"): 8,388,608 particles of a Plummer sphere (scale
radius 0.1 of the unit box, centred, redrawn outside the box) with +-1
charges summing to zero, open boundary, plain form, octree depth 7 (2,097,152
finest cells, 61% of them empty), p = 6 (216 grid charges per cell).
Default precision "tf32x3": every stage in FP32, the far-field contraction of
every level on the tcgen05 tensor cores in 3-pass split TF32 (its parity with
the FP64 oracle meets the FP32 tolerance).  The line also reports the plain
FP32 form (SIMT contraction), the force-kernel form, the shift-free forms, and
shorter lines for BF16x3 and for the uniform (1,048,576 particles, continuous
form, depth 5, p 4) and water-like (2,097,150 particles, periodic continuous
form, depth 6, p 5) workloads.

One step = one full evaluation: binning, split, sort, upward pass, downward
pass, far and near field, recombination, FP64 energy.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision P] [--no-extras] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the host cores, on the same workload (above 2M particles: the outputs
of 512 sampled particles per step, with the full upward pass).  Multi-GPU
(torchrun): every rank evaluates its own replica of the workload (weak
scaling, no collective on the data path); the value is the particles of all
ranks over the slowest rank.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM energy+forces Mparticles/s"
UNIT = "Mparticles/s"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
P2P_FLOPS_PER_PAIR = 20
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor), nominal
# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture of the current kernels (scaled to a full launch where the capture
# ran on a smaller case of the same distribution); reported as the
# rooflines' traffic
PROFILED_TRAFFIC = {("uniform1m", "tf32x3", "k_p2p"): 48267520 + 187352576,
                    ("plummer8m", "tf32x3", "k_m2l_tcg"): 339113666816 + 960174080,
                    ("plummer8m", "tf32x3", "k_p2p"): 353114368 + 1788425728}


def _peaks():
    """HBM GB/s and bf16 TF/s (burst, sustained) measured on this GPU model, else fallbacks."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return (d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0),
                d.get("bf16_tflops_sustained", 1700.0), "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def job_step_ms(t_ms, dist, device):
    """The slowest rank's mean step time: every rank runs the same replica and
    the job is as fast as its slowest rank."""
    if dist is None:
        return t_ms
    import torch
    tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(world, n_per_rank, t_ms):
    """Whole-job throughput in Mparticles/s: all ranks' particles over the
    slowest rank's step time (weak scaling, one replica per rank)."""
    return world * n_per_rank / (t_ms * 1e-3) / 1e6


def fence(dist, cuda=True):
    """Barrier across ranks and device synchronisation (both sides of a timed region)."""
    if dist is not None:
        dist.barrier()
    if cuda:
        import torch
        torch.cuda.synchronize()


def init_ranks(world, local):
    import torch
    torch.cuda.set_device(local)
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("nccl")
    return dist


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def m2l_cell_pairs(depth, periodic):
    """Cell pairs of the interaction lists over all levels (189 per interior cell)."""
    total = 0
    for l in range(1 if periodic else 2, depth + 1):
        S = 1 << l
        for par in range(8):
            b = [(par >> a) & 1 for a in range(3)]
            for oz in range(-2 - b[2], 4 - b[2]):
                for oy in range(-2 - b[1], 4 - b[1]):
                    for ox in range(-2 - b[0], 4 - b[0]):
                        if max(abs(ox), abs(oy), abs(oz)) <= 1:
                            continue
                        c = 1
                        for a, o in enumerate((ox, oy, oz)):
                            cs = range(b[a], S, 2)
                            c *= len(cs) if periodic else sum(1 for x in cs if 0 <= x + o < S)
                        total += c
    return total


def p2p_pairs(plan, depth, periodic):
    """Ordered charge pairs of the near field (27 cells, same-particle pairs excluded)."""
    import numpy as np
    start = plan.dump("start").astype(np.int64)
    origin = plan.dump("origin")
    S = 1 << depth
    cnt = np.diff(start)
    # Morton key -> (x, y, z)
    keys = np.arange(S ** 3, dtype=np.int64)
    xyz = np.zeros((S ** 3, 3), np.int64)
    for bit in range(depth):
        for a in range(3):
            xyz[:, a] |= ((keys >> (3 * bit + a)) & 1) << bit
    grid = np.zeros((S, S, S), np.int64)
    grid[xyz[:, 2], xyz[:, 1], xyz[:, 0]] = cnt
    nb = np.zeros_like(grid)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if periodic:
                    nb += np.roll(grid, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
                else:
                    g = np.zeros((S + 2, S + 2, S + 2), np.int64)
                    g[1:-1, 1:-1, 1:-1] = grid
                    nb += g[1 + dz:S + 1 + dz, 1 + dy:S + 1 + dy, 1 + dx:S + 1 + dx]
    m = np.bincount(origin)
    return int(np.sum(grid * nb) - np.sum(m.astype(np.int64) ** 2))


def run_reference(args, workload, world, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2212_13080_gb300 import inputs
    w = inputs.workload(workload)
    pos, q, box = w["pos"], w["q"], w["box"]
    n = len(q)
    idx = _oracle_targets(n)
    kw = dict(depth=w["depth"], n=w["p"], periodic=w["periodic"], continuous=w["continuous"],
              sample=idx, keep=False)
    for _ in range(args.warmup):
        oracle.fmm(pos, q, box, **kw)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fmm(pos, q, box, **kw)
        ts.append(time.perf_counter() - t0)
    t = statistics.mean(ts)
    cores = os.cpu_count()
    m = n if idx is None else len(idx)
    v = m / t / 1e6
    sample = ("whole workload (%d particles) per step, oracle.fmm FP64, OpenMP" % n
              if idx is None else
              "outputs of %d sampled particles of %d per step (full upward pass), oracle.fmm "
              "FP64, OpenMP" % (m, n))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload, "n": n, "depth": w["depth"],
                                        "p": w["p"], "periodic": w["periodic"],
                                        "continuous": w["continuous"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


WHOLE_ORACLE_MAX_N = 1 << 21   # above this the oracle runs on a bounded sample of targets
ORACLE_SAMPLE = 512


def _oracle_targets(n):
    import numpy as np
    if n <= WHOLE_ORACLE_MAX_N:
        return None
    return np.sort(np.random.default_rng(12345).choice(n, ORACLE_SAMPLE, replace=False))


def cpu_baseline(workload, gpu_outputs=None, kernel_outputs=None):
    """The FP64 oracle on the host cores (whole workload up to 2M particles, else the
    outputs of 512 sampled particles) and, from the same run, the relative L2 error of
    the GPU results against it; for the open form also the method's own error (the
    oracle against the direct O(N) sum at the sampled particles).  kernel_outputs:
    the GPU results of a force-kernel plan (§4.1), checked against the oracle's
    force-kernel run on the same particles (and against the direct sum)."""
    import numpy as np
    import oracle
    from paper_2212_13080_gb300 import inputs
    w = inputs.workload(workload)
    n = len(w["q"])
    idx = _oracle_targets(n)
    t0 = time.perf_counter()
    r = oracle.fmm(w["pos"], w["q"], w["box"], depth=w["depth"], n=w["p"],
                   periodic=w["periodic"], continuous=w["continuous"], sample=idx, keep=False)
    t = time.perf_counter() - t0
    m = n if idx is None else len(idx)
    base = {"value": m / t / 1e6, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": ("whole workload (%d particles), one oracle.fmm run (FP64, OpenMP), %.1f s"
                       % (n, t)) if idx is None else
                      ("outputs of %d sampled particles of %d (full upward pass, downward pass "
                       "where they need it), one oracle.fmm run (FP64, OpenMP), %.1f s"
                       % (m, n, t))}
    err = None
    if gpu_outputs:
        sel = np.arange(n) if idx is None else idx
        phi_o = np.asarray(r["phi"], np.float64)
        F_o = np.asarray(r["F"], np.float64).reshape(-1, 3)
        if idx is not None and phi_o.shape[0] == n:
            phi_o, F_o = phi_o[idx], F_o[idx]

        def rel(a, b):
            return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

        err = {"particles": int(len(sel)), "reference": "oracle (FP64, same method and p)"}
        for name, (phi_g, F_g, E_g) in gpu_outputs.items():
            e = {"potential_rel_l2": rel(phi_g[sel].astype(np.float64), phi_o),
                 "forces_rel_l2": rel(F_g[sel].astype(np.float64), F_o)}
            if idx is None and r.get("E") is not None:
                e["energy_rel"] = abs(E_g - r["E"]) / abs(r["E"])
            err[name] = e
        if not w["periodic"]:
            tg = idx if idx is not None else np.sort(
                np.random.default_rng(12345).choice(n, ORACLE_SAMPLE, replace=False))
            phi_d, F_d = oracle.direct(w["pos"], w["q"], w["box"], targets=tg)
            phi_m = np.asarray(r["phi"], np.float64)
            F_m = np.asarray(r["F"], np.float64).reshape(-1, 3)
            if phi_m.shape[0] == n:
                phi_m, F_m = phi_m[tg], F_m[tg]
            err["method_error_vs_direct"] = {"particles": int(len(tg)),
                                             "potential_rel_l2": rel(phi_m, phi_d),
                                             "forces_rel_l2": rel(F_m, F_d)}
        if kernel_outputs is not None:
            rk = oracle.fmm(w["pos"], w["q"], w["box"], depth=w["depth"], n=w["p"],
                            periodic=w["periodic"], continuous=w["continuous"], sample=idx,
                            keep=False, force_kernel=True)
            Fk = np.asarray(rk["F"], np.float64).reshape(-1, 3)
            if idx is not None and Fk.shape[0] == n:
                Fk = Fk[idx]
            _, F_g, _ = kernel_outputs
            ek = {"forces_rel_l2": rel(F_g[sel].astype(np.float64), Fk)}
            if not w["periodic"]:
                Fm = np.asarray(rk["F"], np.float64).reshape(-1, 3)
                if Fm.shape[0] == n:
                    Fm = Fm[tg]
                ek["oracle_forces_vs_direct_rel_l2"] = rel(Fm, F_d)
            err["force_kernel"] = ek
    return base, err


def run_batch(args, world, rank, local, dist=None):
    """512 independent periodic systems (continuous form, p = 4), N per system
    log-uniform in [1024, 65536], depth = clamp(round(log8(N/32)), 3, 5):
    one CUDA-graph launch per step."""
    import numpy as np
    import torch
    from paper_2212_13080_gb300 import FMMBatch, inputs
    pos_h, q_h, offs, boxes, counts = inputs.batch_systems(512, 5)
    depths = np.clip(np.rint(np.log(counts / 32.0) / np.log(8.0)), 3, 5).astype(int)
    dev = torch.device("cuda", local)
    pos = torch.from_numpy(pos_h).to(dev)
    q = torch.from_numpy(q_h).to(dev)
    bt = FMMBatch(boxes, depths, 4, periodic=True, continuous=True, precision=args.precision,
                  max_n=counts, sync=False)
    out = {"potential": torch.empty(len(q_h), device=dev),
           "energy": torch.empty(512, dtype=torch.float64, device=dev),
           "forces": torch.empty((len(q_h), 3), device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.eval(pos, q, offs, out=out)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    fence(dist)
    sampler.start()
    time.sleep(0.3)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.eval(pos, q, offs, out=out)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    fence(dist)
    clocks = sampler.stop()
    st = bt.stats()
    t = job_step_ms(statistics.mean(ms), dist, dev)
    n = int(offs[-1])
    outs = {args.precision: {k: v.cpu().numpy() for k, v in out.items()}}
    bt.close()

    # the plain FP32 batched form, same protocol, fewer steps
    plain = None
    if args.precision != "fp32":
        b32 = FMMBatch(boxes, depths, 4, periodic=True, continuous=True, precision="fp32",
                       max_n=counts, sync=False)
        for _ in range(2):
            b32.eval(pos, q, offs, out=out)
        t32 = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b32.eval(pos, q, offs, out=out)
            b.record(stream)
            b.synchronize()
            t32.append(a.elapsed_time(b))
        outs["fp32"] = {k: v.cpu().numpy() for k, v in out.items()}
        plain = {"precision": "fp32", "ms_per_step": statistics.mean(t32),
                 "value": world * n / (statistics.mean(t32) * 1e-3) / 1e6, "unit": UNIT,
                 "merged": b32.stats()["merged"], "schedule": b32.stats()["schedule"]}
        b32.close()
    res = None
    if rank == 0:
        res = {
            "metric": METRIC, "value": job_value(world, n, t), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "precision": args.precision, "data": "synthetic",
            "config": {"workload": "batch512", "systems": 512, "n_total": n,
                       "n_min": int(counts.min()), "n_max": int(counts.max()),
                       "depths": {str(d): int((depths == d).sum()) for d in sorted(set(depths))},
                       "p": 4, "periodic": True, "continuous": True,
                       "outputs": "potential+energy+forces per system",
                       "l2": "flushed (256 MB write) before every timed step"},
            "gpu_launches": st["launches"] * args.steps, "graph_launches_per_step": 1,
            "merged": st["merged"], "schedule": st["schedule"], "lanes": st["lanes"],
            "tune_ms": st["tune_ms"], "clocks": clocks,
            "plain_fp32": plain}
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"], res["error_vs_fp64_oracle"] = batch_cpu_baseline(
                pos_h, q_h, offs, boxes, counts, depths, outs)
        print(json.dumps(res), flush=True)


def batch_cpu_baseline(pos_h, q_h, offs, boxes, counts, depths, outs):
    """The oracle on 16 whole systems of the batch (the smallest, the largest and
    14 seeded picks): its throughput on that sample, and the relative L2 error
    of the GPU's batched outputs against it for those systems."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(55)
    pick = sorted(set([int(np.argmin(counts)), int(np.argmax(counts))] +
                      [int(v) for v in rng.choice(len(counts), 14, replace=False)]))
    t_tot, m_tot = 0.0, 0
    err = {name: {"potential_rel_l2": [], "forces_rel_l2": [], "energy_rel": []} for name in outs}

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    for i in pick:
        a, b = int(offs[i]), int(offs[i + 1])
        t0 = time.perf_counter()
        r = oracle.fmm(pos_h[a:b], q_h[a:b], boxes[i], depth=int(depths[i]), n=4, periodic=True,
                       continuous=True, keep=False)
        t_tot += time.perf_counter() - t0
        m_tot += b - a
        for name, o in outs.items():
            err[name]["potential_rel_l2"].append(rel(o["potential"][a:b].astype(np.float64), r["phi"]))
            err[name]["forces_rel_l2"].append(rel(o["forces"][a:b].astype(np.float64),
                                                  np.asarray(r["F"]).reshape(-1, 3)))
            err[name]["energy_rel"].append(abs(float(o["energy"][i]) - r["E"]) / abs(r["E"]))
    base = {"value": m_tot / t_tot / 1e6, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d whole systems of the batch (%d particles; the smallest, the largest and "
                      "seeded picks), oracle.fmm FP64, OpenMP, %.1f s" % (len(pick), m_tot, t_tot)}
    summary = {"systems": pick, "reference": "oracle (FP64, same method and p)"}
    for name, e in err.items():
        summary[name] = {k: {"max": max(v), "mean": float(np.mean(v))} for k, v in e.items()}
    return base, summary


def cell_occupancy(start, depth):
    """Per level l, a boolean grid [z][y][x] of the cells whose finest cells hold
    charges, from the finest-cell ranges (Morton order)."""
    import numpy as np
    start = np.asarray(start, np.int64)
    out = {}
    for l in range(depth + 1):
        S, sh = 1 << l, 3 * (depth - l)
        k = np.arange(S ** 3, dtype=np.int64)
        occ = start[(k + 1) << sh] > start[k << sh]
        xyz = np.zeros((S ** 3, 3), np.int64)
        for bit in range(l):
            for a in range(3):
                xyz[:, a] |= ((k >> (3 * bit + a)) & 1) << bit
        g = np.zeros((S, S, S), bool)
        g[xyz[:, 2], xyz[:, 1], xyz[:, 0]] = occ
        out[l] = g
    return out


def m2l_work(start, depth, periodic, p, precision):
    """Cell pairs of the interaction lists: every pair in range (dense), the pairs
    whose target and source both hold charges (the method's own work: a functional
    is read only where there are charges, an empty source adds nothing), and the
    tensor-core work the contraction executes (128-row tiles of the occupied
    targets, 189 offsets each, p^3 padded to the MMA shape, 3 passes for the
    split forms)."""
    import numpy as np
    occ = cell_occupancy(start, depth)
    dense = both = tiles = 0
    for l in range(1 if periodic else 2, depth + 1):
        g, H = occ[l], 1 << (l - 1)
        mode = "wrap" if periodic else "constant"
        for par in range(8):
            b = [(par >> a) & 1 for a in range(3)]  # x, y, z
            T = g[b[2]::2, b[1]::2, b[0]::2]
            nocc = int(T.sum())
            tiles += (1 if nocc else 0) if H < 8 else (nocc + 127) // 128
            for oz in range(-2 - b[2], 4 - b[2]):
                for oy in range(-2 - b[1], 4 - b[1]):
                    for ox in range(-2 - b[0], 4 - b[0]):
                        if max(abs(ox), abs(oy), abs(oz)) <= 1:
                            continue
                        s = [b[0] + ox, b[1] + oy, b[2] + oz]
                        src = np.pad(g[s[2] & 1::2, s[1] & 1::2, s[0] & 1::2], 1, mode=mode)
                        d = [v >> 1 for v in s]
                        src = src[1 + d[2]:1 + d[2] + H, 1 + d[1]:1 + d[1] + H, 1 + d[0]:1 + d[0] + H]
                        both += int(np.count_nonzero(T & src))
                        if periodic:
                            dense += H ** 3
                        else:
                            dense += int(np.prod([H - abs(v) for v in d]))
    p3 = p ** 3
    n_pad = (p3 + 31) // 32 * 32
    k_pad = (p3 + 63) // 64 * 64 if precision == "bf16x3" else n_pad
    passes = 1 if precision == "tf32x1" else 3
    return {"dense_pairs": dense, "occupied_pairs": both, "tiles": tiles,
            "algorithmic_flops": 2.0 * p3 * p3 * both, "dense_flops": 2.0 * p3 * p3 * dense,
            "executed_flops": 2.0 * tiles * 128 * 189 * n_pad * k_pad * passes}


def tc_peak(precision, long_step):
    """Dense tensor peak of the contraction's MMA kind (TF/s) and its source."""
    hbm, bf16_burst, bf16_sust, kind = _peaks()
    ref = bf16_sust if long_step else bf16_burst
    which = "sustained" if long_step else "burst"
    if precision == "bf16x3":  # kind::f16: the measured bf16 rate itself
        return ref, "%s bf16 %s %.1f TF/s" % (kind, which, ref)
    # kind::tf32: 1/2 of it (nominal 1.1 vs 2.25 PF/s)
    return ref / 2, "%s bf16 %s %.1f TF/s x 1/2 (nominal tf32:bf16 ratio)" % (kind, which, ref)


class Run:
    """One workload and precision: its plan, workspace, outputs and step."""

    def __init__(self, name, precision, dev, shift_free=False, force_mode="adjoint", w=None):
        import torch
        from paper_2212_13080_gb300 import FMM, inputs
        self.name, self.precision = name, precision
        self.w = w if w is not None else inputs.workload(name)
        w = self.w
        self.n = n = len(w["q"])
        self.pos = torch.from_numpy(w["pos"]).to(dev)
        self.q = torch.from_numpy(w["q"]).to(dev)
        self.mk = dict(periodic=w["periodic"], continuous=w["continuous"], precision=precision,
                       max_n=n, shift_free=shift_free, force_mode=force_mode)
        self.plan = FMM(w["box"], w["depth"], w["p"], sync=False, **self.mk)
        self.ws = self.plan.workspace(n)
        od = self.plan.out_dtype
        self.out = {"potential": torch.empty(n, dtype=od, device=dev),
                    "energy": torch.empty(1, dtype=torch.float64, device=dev),
                    "forces": torch.empty((n, 3), dtype=od, device=dev)}

    def step(self):
        self.plan.eval(self.pos, self.q, workspace=self.ws, out=self.out)

    def check(self):
        rc = plan_status(self.plan, self.ws)
        if rc:
            raise SystemExit("%s %s: evaluation failed: status %d" % (self.name, self.precision, rc))

    def time(self, steps, warmup, flush, stream, timing=True):
        """Mean device ms per step (CUDA events on the launching stream, L2
        flushed before every step), the library's stage times and launches."""
        import torch
        self.plan.set_timing(timing)
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        self.check()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        stage_tot, launches = {}, 0
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            self.step()
            evs[i][1].record(stream)
            st = self.plan.stats()
            launches += st["launches"]
            for k, v in st["stage_ms"].items():
                stage_tot[k] = stage_tot.get(k, 0.0) + v
        torch.cuda.synchronize()
        self.check()
        ms = [a.elapsed_time(b) for a, b in evs]
        return statistics.mean(ms), {k: v / steps for k, v in stage_tot.items()}, launches

    def isolated(self, steps, flush):
        """Each stage's own duration: the same steps with every stage on one stream."""
        import torch
        self.plan.set_timing(True, serial=True)
        tot = {}
        for _ in range(steps):
            flush.zero_()
            self.step()
            for k, v in self.plan.stats()["stage_ms"].items():
                tot[k] = tot.get(k, 0.0) + v / steps
        torch.cuda.synchronize()
        self.plan.set_timing(True)
        return tot

    def host_outputs(self):
        return (self.out["potential"].cpu().numpy(), self.out["forces"].cpu().numpy(),
                float(self.out["energy"].item()))

    def close(self):
        self.plan.close()


def rooflines(run, t_step, stage_ms, stage_iso):
    """The contraction's and the near field's rooflines (algorithmic flops over
    their stage time), and which of the two dominates by isolated time."""
    w = run.w
    start = run.plan.dump("start")
    pairs = p2p_pairs(run.plan, w["depth"], w["periodic"])
    mw = m2l_work(start, w["depth"], w["periodic"], w["p"], run.precision)
    long_step = t_step >= 100.0
    tc = run.precision in ("tf32x3", "tf32x1", "bf16x3")
    out = {}
    p2p_flops = float(P2P_FLOPS_PER_PAIR) * pairs
    ach = p2p_flops / (stage_ms["p2p"] * 1e-3) / 1e12
    ach_iso = p2p_flops / (stage_iso["p2p"] * 1e-3) / 1e12
    out["p2p"] = {"kernel": "k_p2p", "bound": "alu", "achieved": ach_iso, "peak": FP32_ALU_PEAK_TFLOPS,
                  "unit": "TFLOP/s", "frac": ach_iso / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                  "algorithmic": "%d ordered pairs x %d flop" % (pairs, P2P_FLOPS_PER_PAIR),
                  "duration": "isolated stage time (every stage on one stream)",
                  "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz",
                  "achieved_in_step": ach, "frac_in_step": ach / FP32_ALU_PEAK_TFLOPS,
                  "ordered_pairs": pairs}
    m_ms, m_iso = stage_ms["m2l"], stage_iso["m2l"]
    if tc:
        peak, src = tc_peak(run.precision, long_step)
        a = mw["algorithmic_flops"] / (m_ms * 1e-3) / 1e12
        out["m2l"] = {"kernel": "k_m2l_tcg", "bound": "tensor", "achieved": a, "peak": peak,
                      "unit": "TFLOP/s", "frac": a / peak, "traffic": None,
                      "algorithmic": "%d cell pairs whose cells both hold charges x 2 p^6 flop "
                                     "(all levels per step)" % mw["occupied_pairs"],
                      "duration": "in-step stage time (far-field stream; split, lists and "
                                  "contraction)",
                      "peak_source": src,
                      "dense_pairs": mw["dense_pairs"],
                      "achieved_on_dense_count": mw["dense_flops"] / (m_ms * 1e-3) / 1e12,
                      "executed_tflops": mw["executed_flops"] / (m_ms * 1e-3) / 1e12,
                      "executed_frac": mw["executed_flops"] / (m_ms * 1e-3) / 1e12 / peak,
                      "executed": "%d tiles x 128 rows x 189 offsets, p^3 padded, %d passes"
                                  % (mw["tiles"], 1 if run.precision == "tf32x1" else 3),
                      "achieved_isolated": mw["algorithmic_flops"] / (m_iso * 1e-3) / 1e12}
    else:
        a = mw["algorithmic_flops"] / (m_ms * 1e-3) / 1e12
        out["m2l"] = {"kernel": "k_m2l_simt", "bound": "alu", "achieved": a,
                      "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": a / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                      "algorithmic": "%d cell pairs whose cells both hold charges x 2 p^6 flop"
                                     % mw["occupied_pairs"],
                      "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz",
                      "dense_pairs": mw["dense_pairs"],
                      "achieved_on_dense_count": mw["dense_flops"] / (m_ms * 1e-3) / 1e12}
    dom = max(("m2l", "p2p"), key=lambda k: stage_iso.get(k, 0.0))
    for k, r in out.items():
        r["traffic"] = PROFILED_TRAFFIC.get((run.name, run.precision, r["kernel"]))
        if r["traffic"] is not None:
            r["traffic_unit"] = ("bytes per launch (ncu dram__bytes_read.sum + "
                                 "dram__bytes_write.sum)")
    return dom, out, pairs, mw


def extra_line(name, precision, dev, flush, stream, steps):
    """A shorter line for another workload or precision: throughput, stage
    times, the two rooflines (no CPU leg)."""
    r = Run(name, precision, dev)
    t, st, launches = r.time(steps, 3, flush, stream)
    iso = r.isolated(max(3, steps // 3), flush)
    dom, roofs, pairs, mw = rooflines(r, t, st, iso)
    w = r.w
    res = {"workload": name, "precision": precision, "n": r.n, "depth": w["depth"], "p": w["p"],
           "periodic": w["periodic"], "continuous": w["continuous"], "ms_per_step": t,
           "value": r.n / (t * 1e-3) / 1e6, "unit": UNIT, "gpu_launches_per_step": launches // steps,
           "stage_ms": st, "stage_ms_isolated": iso, "dominant": dom, "roofline_m2l": roofs["m2l"],
           "roofline_p2p": roofs["p2p"]}
    r.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plummer8m")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra lines (other workloads, BF16x3, plain FP32, force kernels, "
                         "shift-free forms)")
    ap.add_argument("--shift-free", action="store_true",
                    help="App. A.2 forms for the main plan (precision fp64, p <= 5)")
    ap.add_argument("--profile", action="store_true",
                    help="run only the warm-up and timed steps of the headline plan (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.workload == "batch512":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle reference arm covers the single-system workload"}))
            return
        run_reference(args, args.workload, world, rank)
        return
    import torch
    dist = init_ranks(world, local)
    if args.workload == "batch512":
        run_batch(args, world, rank, local, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    from paper_2212_13080_gb300 import FMM
    dev = torch.device("cuda", local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    run = Run(args.workload, args.precision, dev, shift_free=args.shift_free)
    w, n = run.w, run.n

    if args.profile:
        for _ in range(args.warmup + args.steps):
            run.step()
        torch.cuda.synchronize()
        print(json.dumps({"profile": True, "workload": args.workload, "steps": args.steps,
                          "precision": args.precision, "status": plan_status(run.plan, run.ws)}))
        return

    # the timed steps, with clocks sampled during them
    run.plan.set_timing(True)
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()
    run.check()
    sampler = ClockSampler(local)
    fence(dist)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stage_tot, launches = {}, 0
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        run.step()
        evs[i][1].record(stream)
        st = run.plan.stats()
        launches += st["launches"]
        for k, v in st["stage_ms"].items():
            stage_tot[k] = stage_tot.get(k, 0.0) + v
    fence(dist)
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    run.check()
    t_step = job_step_ms(statistics.mean(ms), dist, dev)
    value = job_value(world, n, t_step)
    stage_ms = {k: v / args.steps for k, v in stage_tot.items()}
    stage_ms_iso = run.isolated(max(3, args.steps // 4), flush)
    gpu_outputs = {args.precision: run.host_outputs()}
    dom, roofs, pairs, mw = rooflines(run, t_step, stage_ms, stage_ms_iso)
    roof = dict(roofs[dom])
    hbm, _, _, peak_kind = _peaks()
    roof["hbm_peak_gbs"] = hbm
    roof["hbm_peak_source"] = peak_kind

    extras = not args.no_extras and world == 1
    # the plain FP32 form (SIMT contraction), same timing protocol, fewer steps
    plain = None
    if extras and args.precision != "fp32" and not args.shift_free:
        r32 = Run(args.workload, "fp32", dev, w=w)
        k32 = 3 if n > (1 << 21) else max(3, args.steps // 4)
        t32, st32, _ = r32.time(k32, 1, flush, stream, timing=False)
        gpu_outputs["fp32"] = r32.host_outputs()
        plain = {"precision": "fp32", "ms_per_step": t32, "value": n / (t32 * 1e-3) / 1e6,
                 "unit": UNIT}
        r32.close()

    # far forces from the force kernels (§4.1), same workload and precision
    force_kernel, fk_host = None, None
    if extras and not args.shift_free:
        rk = Run(args.workload, args.precision, dev, force_mode="kernel", w=w)
        tk, _, _ = rk.time(max(5, args.steps // 2), 3, flush, stream, timing=False)
        fk_iso = rk.isolated(5, flush)
        fk_host = rk.host_outputs()
        force_kernel = {"force_mode": "kernel", "precision": args.precision, "ms_per_step": tk,
                        "value": world * n / (tk * 1e-3) / 1e6, "unit": UNIT,
                        "stage_ms_isolated": fk_iso,
                        "m2l_tflops_algorithmic": 4 * mw["algorithmic_flops"] / (fk_iso["m2l"] * 1e-3) / 1e12,
                        "note": "four contractions (1/r and the x, y, z force kernels), plain-weight "
                                "far-field evaluation"}
        rk.close()

    # end to end through the public API with host buffers (pinned)
    plan_e2e = FMM(w["box"], w["depth"], w["p"], sync=True, **dict(run.mk, force_mode="adjoint"))
    pos_p = torch.from_numpy(w["pos"]).pin_memory()
    q_p = torch.from_numpy(w["q"]).pin_memory()
    for _ in range(2):
        plan_e2e.eval(pos_p, q_p)
    torch.cuda.synchronize()
    te = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        r = plan_e2e.eval(pos_p, q_p)
        te.append(time.perf_counter() - t0)
    e2e_v = world * n / statistics.mean(te) / 1e6
    h2d = pos_p.numel() * 4 + q_p.numel() * 4
    d2h = r["potential"].numel() * r["potential"].element_size() + \
        r["forces"].numel() * r["forces"].element_size() + 8
    plan_e2e.close()

    cfg = {"workload": args.workload, "n": n, "depth": w["depth"], "p": w["p"],
           "periodic": w["periodic"], "continuous": w["continuous"],
           "outputs": "potential+energy+forces",
           "l2": "flushed (256 MB write) before every timed step",
           "parallelism": "replicas" if world > 1 else "single"}
    if w["continuous"]:
        cfg["split_2d_over_w"] = 1 / 128
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "precision": args.precision,
        "data": "synthetic",
        "config": cfg,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_m2l": roofs["m2l"], "roofline_p2p": roofs["p2p"],
        "stage_ms": stage_ms, "stage_ms_isolated": stage_ms_iso,
        "pairs_per_s": pairs / (t_step * 1e-3),
        "m2l_cell_pairs": {"dense": mw["dense_pairs"], "both_occupied": mw["occupied_pairs"],
                           "tiles": mw["tiles"]},
        "clocks": clocks,
        "plain_fp32": plain,
        "force_kernel": force_kernel,
    }
    run.close()
    if extras:
        res["shift_free"] = shift_free_line(args.steps, dev, flush, stream)
        res["extra"] = []
        if args.workload == "plummer8m" and args.precision == "tf32x3":
            res["extra"].append(extra_line("plummer8m", "bf16x3", dev, flush, stream, 5))
        for name in ("uniform1m", "water2m"):
            if name != args.workload:
                res["extra"].append(extra_line(name, "tf32x3", dev, flush, stream, 10))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"], res["error_vs_fp64_oracle"] = cpu_baseline(args.workload, gpu_outputs,
                                                                        fk_host)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def shift_free_line(steps, dev, flush, stream):
    """App. A.2 (bilinear forms without shifts) beside the shifted form, both
    FP64, on 23,040 uniform +-1 charges (open, plain, depth 3, p 4: the size
    of §3.1's runs and the depth the paper keeps the forms for).  The
    dominant kernel, k_sf_m2l, streams one p^6 FP64 right part per cell pair
    of the interaction lists: its roofline is that read against HBM, and its
    FP64 multiply-adds against the nominal FP64 rate."""
    import torch
    from paper_2212_13080_gb300 import FMM, inputs
    w = inputs.workload("uniform23k")
    n, p = len(w["q"]), w["p"]
    pos = torch.from_numpy(w["pos"]).to(dev)
    q = torch.from_numpy(w["q"]).to(dev)
    res, outs = {}, {}
    for sf in (True, False):
        t0 = time.perf_counter()
        plan = FMM(w["box"], w["depth"], p, precision="fp64", shift_free=sf, max_n=n, sync=False)
        torch.cuda.synchronize()
        create_ms = (time.perf_counter() - t0) * 1e3
        ws = plan.workspace(n)
        out = {"potential": torch.empty(n, dtype=torch.float64, device=dev),
               "energy": torch.empty(1, dtype=torch.float64, device=dev),
               "forces": torch.empty((n, 3), dtype=torch.float64, device=dev)}
        for _ in range(3):
            plan.eval(pos, q, workspace=ws, out=out)
        t = []
        for _ in range(max(5, steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.eval(pos, q, workspace=ws, out=out)
            b.record(stream)
            b.synchronize()
            t.append(a.elapsed_time(b))
        if plan_status(plan, ws):
            raise SystemExit("shift-free line: evaluation failed")
        plan.set_timing(True, serial=True)
        iso, k = {}, 5
        for _ in range(k):
            flush.zero_()
            plan.eval(pos, q, workspace=ws, out=out)
            for s_, v in plan.stats()["stage_ms"].items():
                iso[s_] = iso.get(s_, 0.0) + v / k
        torch.cuda.synchronize()
        outs[sf] = (out["potential"].cpu().numpy(), out["forces"].cpu().numpy())
        res["shift_free" if sf else "shifted"] = {
            "ms_per_step": statistics.mean(t), "value": n / (statistics.mean(t) * 1e-3) / 1e6,
            "unit": UNIT, "plan_create_ms": create_ms, "stage_ms_isolated": iso}
        plan.close()
    import numpy as np
    pairs = m2l_cell_pairs(w["depth"], False)
    tab_bytes = pairs * p ** 6 * 8
    m2l_ms = res["shift_free"]["stage_ms_isolated"]["m2l"]
    hbm, _, _, peak_kind = _peaks()
    gbs = tab_bytes / (m2l_ms * 1e-3) / 1e9
    fp64 = 2.0 * p ** 6 * pairs / (m2l_ms * 1e-3) / 1e12
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    res.update({
        "workload": "uniform23k: 23,040 uniform +-1, open, plain, depth 3, p 4, fp64",
        "kernel": "k_sf_m2l", "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
        "frac": gbs / hbm, "peak_source": peak_kind,
        "algorithmic": "%d cell pairs x p^6 FP64 right parts (%d bytes per step)" % (pairs, tab_bytes),
        "fp64_tflops": fp64, "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
        "fp64_frac_of_nominal": fp64 / FP64_NOMINAL_TFLOPS,
        "rel_diff_vs_shifted": {"potential": rel(outs[True][0], outs[False][0]),
                                "forces": rel(outs[True][1], outs[False][1])}})
    return res


def plan_status(plan, ws):
    from paper_2212_13080_gb300 import _binding as B
    import ctypes
    import torch
    ws_al = plan._aligned(ws)
    return B.fmm_status(plan._h, ctypes.c_void_p(ws_al.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


if __name__ == "__main__":
    main()
