"""Seeded synthetic workloads for the replacement-based FMM.

This module only draws random numbers: it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle take their inputs from
it.  Every generator uses numpy's PCG64 with the given seed and returns
float32 positions (N, 3), float32 charges (N,) and the box (x0, y0, z0, L).

The paper's own workload (23040 random +-1 charges in a unit cube drawn by the
sample program of Ogata et al., §3.1) is not available; these generators
stand in for it with the sizes and distributions named per workload.
"""
import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _pm1(rng, n):
    """n charges, half +1 and half -1 (n even), in random order."""
    q = np.ones(n, np.float32)
    q[n // 2:] = -1.0
    rng.shuffle(q)
    return q


def uniform_pm1(n, seed, L=1.0):
    """n particles uniform in [0, L)^3 with +-1 charges, zero net charge."""
    rng = _rng(seed)
    pos = rng.random((n, 3), dtype=np.float32)
    if L != 1.0:
        pos = (pos.astype(np.float64) * L).astype(np.float32)
        pos = np.minimum(pos, np.nextafter(np.float32(L), np.float32(0)))
    return pos, _pm1(rng, n), (0.0, 0.0, 0.0, float(L))


def uniform_cont(n, seed):
    """n particles uniform in [0,1)^3, charges uniform in [-1,1] shifted to
    zero mean (computed in float64, stored as float32)."""
    rng = _rng(seed)
    pos = rng.random((n, 3), dtype=np.float32)
    q = rng.uniform(-1.0, 1.0, n)
    q = (q - q.mean()).astype(np.float32)
    return pos, q, (0.0, 0.0, 0.0, 1.0)


def water(n_triples, seed, density=33.0, r_oh=0.1, angle_deg=104.52,
          q_o=-0.834, q_h=0.417):
    """Water-like rigid triples: O uniform in a cubic box of side
    (n_triples/density)^(1/3), two H at distance r_oh from O with the given
    H-O-H angle, uniformly random orientation.  Positions are returned
    wrapped into [0, L) (periodic box)."""
    rng = _rng(seed)
    L = (n_triples / density) ** (1.0 / 3.0)
    O = rng.random((n_triples, 3)) * L
    # uniformly random rotation from a random unit quaternion
    qv = rng.normal(size=(n_triples, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)
    half = math.radians(angle_deg) / 2.0
    h1 = np.array([r_oh * math.sin(half), 0.0, r_oh * math.cos(half)])
    h2 = np.array([-r_oh * math.sin(half), 0.0, r_oh * math.cos(half)])
    H1 = O + R @ h1
    H2 = O + R @ h2
    pos = np.stack([O, H1, H2], axis=1).reshape(-1, 3)
    pos = np.mod(pos, L)
    pos = pos.astype(np.float32)
    pos = np.where(pos >= np.float32(L), np.float32(0), pos)
    q = np.tile(np.array([q_o, q_h, q_h], np.float32), n_triples)
    return pos, q, (0.0, 0.0, 0.0, float(L))


def plummer(n, seed, a=0.1, centre=(0.5, 0.5, 0.5)):
    """n particles of a Plummer sphere of scale radius a about centre,
    truncated to [0,1)^3 by redrawing, with +-1 charges, zero net charge."""
    rng = _rng(seed)
    out = np.empty((0, 3))
    c = np.asarray(centre)
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.3) + 16
        U = rng.random(m)
        U = U[U > 0]
        r = a / np.sqrt(U ** (-2.0 / 3.0) - 1.0)
        d = rng.normal(size=(U.size, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = c + r[:, None] * d
        p32 = p.astype(np.float32)
        ok = np.all((p32 >= 0) & (p32 < 1), axis=1)
        out = np.concatenate([out, p[ok]], axis=0)
    pos = out[:n].astype(np.float32)
    return pos, _pm1(rng, n), (0.0, 0.0, 0.0, 1.0)


def batched_sizes(nsys, seed, lo=1024, hi=65536):
    """Per-system sizes, log-uniform in [lo, hi], rounded down to even."""
    rng = _rng(seed)
    n = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), nsys))).astype(np.int64)
    return n - (n % 2)


def batch_systems(nsys, seed, lo=1024, hi=65536):
    """nsys independent unit-box systems: N log-uniform in [lo, hi] (even),
    uniform positions, +-1 charges with zero net charge per system.  Returns
    (pos (sum N, 3) float32, q float32, offsets (nsys+1) int64, boxes (nsys,4),
    counts)."""
    counts = batched_sizes(nsys, seed, lo, hi)
    rng = _rng(seed + 1)
    pos = rng.random((int(counts.sum()), 3), dtype=np.float32)
    q = np.concatenate([_pm1(rng, int(c)) for c in counts])
    offsets = np.zeros(nsys + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    boxes = np.tile(np.array([0.0, 0.0, 0.0, 1.0]), (nsys, 1))
    return pos, q, offsets, boxes, counts


# ---- the named workloads -------------------------------------------------

def workload(name, seed=None, n=None):
    """Named workloads: returns dict(pos, q, box, depth, p, periodic, continuous)."""
    if name == "uniform4k":  # 4096 uniform +-1, open, plain, depth 3, p 4
        pos, q, box = uniform_pm1(4096 if n is None else n, 1 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=3, p=4, periodic=False, continuous=False)
    if name == "uniform23k":  # 23,040 uniform +-1 (the size of §3.1's runs), open, plain, depth 3, p 4
        pos, q, box = uniform_pm1(23040 if n is None else n, 7 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=3, p=4, periodic=False, continuous=False)
    if name == "uniform1m":  # 1,048,576 uniform, open, continuous, depth 5, p 4
        pos, q, box = uniform_cont(1 << 20 if n is None else n, 2 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=5, p=4, periodic=False, continuous=True)
    if name == "water2m":  # 699,050 triples, periodic continuous, depth 6, p 5
        pos, q, box = water(699050 if n is None else n // 3, 3 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=6, p=5, periodic=True, continuous=True)
    if name == "plummer8m":  # 8,388,608 Plummer, open, plain, depth 7, p 6
        pos, q, box = plummer(1 << 23 if n is None else n, 4 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=7, p=6, periodic=False, continuous=False)
    if name == "plummer1m":  # 1,048,576 Plummer, open, plain, depth 6, p 6 (a small case of plummer8m)
        pos, q, box = plummer(1 << 20 if n is None else n, 4 if seed is None else seed)
        return dict(pos=pos, q=q, box=box, depth=6, p=6, periodic=False, continuous=False)
    raise KeyError(name)
