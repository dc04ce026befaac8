"""Seeded synthetic inputs for the VRP-RPD evaluator, its searches and their tests.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no distances, no schedules, no capacities).  Both the CPU
oracle and the CUDA library consume what it produces, so it is the one piece
they share.

Workload shapes follow the paper's benchmark family (Section 5.1: TSPLIB-derived
instances of 17-1000 nodes with the processing-time variants base, 2x, 5x,
1R10 and 1R20).  TSPLIB itself is not available, so instances are synthetic:

* coordinates: integer points, uniform on [0,1000]^2, or Gaussian clusters
  (8 centres uniform on [0,1000]^2, sigma 60, rounded and clipped).
  Node 0 is the depot and is the first point drawn.
* processing times (int32):
    base  p = U_int[50,150]          2x  p = 2 * base        5x  p = 5 * base
    1R10  p = round(U_int[1,10] * mbar / 5)
    1R20  p = round(U_int[1,20] * mbar / 10)
  where mbar is the mean Euclidean (unrounded) depot-to-customer distance,
  a scale factor of the synthetic input only.
* candidates: route-major op arrays.  Op code o = 2c + isPickup for customer
  c in 1..n; ops has 2n entries, off has m+1 entries (off[0]=0, off[m]=2n).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Instance", "uniform_coords", "clustered_coords", "processing_times",
    "make_instance", "random_candidates", "precedence_candidates",
    "random_keys", "loguniform_sizes", "CONFIGS", "paper_fleet", "paper_processing_times",
    "make_paper_instance",
]


class Instance:
    """Plain container: coords ((n+1) x 2 int32), p (n int32), sizes."""

    def __init__(self, coords, p, m, R, Q, name=""):
        self.coords = np.ascontiguousarray(coords, dtype=np.int32)
        self.p = np.ascontiguousarray(p, dtype=np.int32)
        self.n = int(self.p.shape[0])
        assert self.coords.shape == (self.n + 1, 2)
        self.m, self.R, self.Q = int(m), int(R), int(Q)
        self.name = name

    def __repr__(self):
        return f"Instance({self.name!r}, n={self.n}, m={self.m}, R={self.R}, Q={self.Q})"


def _rng(seed, salt):
    return np.random.Generator(np.random.PCG64([int(seed), int(salt)]))


def uniform_coords(n, seed, lo=0, hi=1000):
    g = _rng(seed, 1)
    return g.integers(lo, hi + 1, size=(n + 1, 2), dtype=np.int64).astype(np.int32)


def clustered_coords(n, seed, k=8, sigma=60.0, lo=0, hi=1000):
    g = _rng(seed, 2)
    centres = g.integers(lo, hi + 1, size=(k, 2), dtype=np.int64).astype(np.float64)
    which = g.integers(0, k, size=n + 1)
    pts = centres[which] + g.normal(0.0, sigma, size=(n + 1, 2))
    pts = np.clip(np.rint(pts), lo, hi)
    return pts.astype(np.int32)


def processing_times(coords, variant, seed):
    n = coords.shape[0] - 1
    g = _rng(seed, 3)
    if variant in ("base", "2x", "5x"):
        base = g.integers(50, 151, size=n, dtype=np.int64)
        mult = {"base": 1, "2x": 2, "5x": 5}[variant]
        return (base * mult).astype(np.int32)
    dx = coords[1:, 0].astype(np.float64) - float(coords[0, 0])
    dy = coords[1:, 1].astype(np.float64) - float(coords[0, 1])
    mbar = float(np.mean(np.sqrt(dx * dx + dy * dy))) if n else 0.0
    if variant == "1R10":
        r = g.integers(1, 11, size=n, dtype=np.int64)
        return np.rint(r * mbar / 5.0).astype(np.int32)
    if variant == "1R20":
        r = g.integers(1, 21, size=n, dtype=np.int64)
        return np.rint(r * mbar / 10.0).astype(np.int32)
    raise ValueError(f"unknown processing-time variant {variant!r}")


def make_instance(n, m, R, Q, variant="base", layout="uniform", seed=0):
    if layout == "uniform":
        coords = uniform_coords(n, seed)
    elif layout == "clustered":
        coords = clustered_coords(n, seed)
    elif layout == "mixed":
        coords = uniform_coords(n, seed) if seed % 2 == 0 else clustered_coords(n, seed)
    else:
        raise ValueError(layout)
    p = processing_times(coords, variant, seed)
    return Instance(coords, p, m, R, Q, name=f"{layout}-n{n}-{variant}-s{seed}")


def paper_fleet(n):
    """Section 5.1 fleet: m = 3 vehicles of capacity 5 below 24 customers,
    m = 6 of capacity 4 from 24 on.  The paper has no depot pool, so R = mQ
    (every vehicle may leave full, the LOAD_FULL reading)."""
    m, Q = (3, 5) if n < 24 else (6, 4)
    return m, Q, m * Q


def paper_processing_times(coords, variant, seed):
    """Section 5.1 processing-time variants: base = U_int[d_min, d_max] over
    the instance's edge weights (distinct nodes); 2x and 5x scale it;
    1R10 / 1R20 multiply each base time by U_int[1, 10] / U_int[1, 20].  The
    base draws do not depend on the variant, so the variants of one seed pair
    up as in the paper.  Rounding to the nearest integer is monotone, so the
    extreme edge weights are the rounded extreme distances."""
    n = coords.shape[0] - 1
    if n < 1:
        return np.zeros(0, np.int32)
    xy = coords.astype(np.float64)
    diff = xy[:, None, :] - xy[None, :, :]
    dist = np.sqrt((diff * diff).sum(-1))
    off_diag = dist[~np.eye(n + 1, dtype=bool)]
    dmin = int(np.floor(off_diag.min() + 0.5)) if off_diag.size else 0
    dmax = int(np.floor(off_diag.max() + 0.5)) if off_diag.size else 0
    base = _rng(seed, 5).integers(dmin, dmax + 1, size=n, dtype=np.int64)
    mult = {"base": 1, "2x": 2, "5x": 5}
    if variant in mult:
        return (base * mult[variant]).astype(np.int32)
    hi = {"1R10": 10, "1R20": 20}.get(variant)
    if hi is None:
        raise ValueError(f"unknown processing-time variant {variant!r}")
    k = _rng(seed, 6).integers(1, hi + 1, size=n, dtype=np.int64)
    return (base * k).astype(np.int32)


def make_paper_instance(n, variant="base", layout="uniform", seed=0):
    """An instance under the paper's own rules (Section 5.1): its fleet and its
    processing-time variants; evaluate it with the LOAD_FULL flag."""
    coords = uniform_coords(n, seed) if layout == "uniform" else clustered_coords(n, seed)
    m, Q, R = paper_fleet(n)
    p = paper_processing_times(coords, variant, seed)
    return Instance(coords, p, m, R, Q, name=f"paper-{layout}-n{n}-{variant}-s{seed}")


def _cuts(g, total, m, count):
    """count x (m+1) offsets: m-1 sorted uniform cut points in [0,total]."""
    cuts = np.sort(g.integers(0, total + 1, size=(count, m - 1)), axis=1) if m > 1 else \
        np.zeros((count, 0), dtype=np.int64)
    off = np.zeros((count, m + 1), dtype=np.int64)
    off[:, 1:m] = cuts
    off[:, m] = total
    return off.astype(np.int32)


def random_candidates(n, m, count, seed):
    """Uniformly shuffled op order cut into m routes (mostly cyclic for n >> 1)."""
    g = _rng(seed, 4)
    ops = np.tile(np.arange(2, 2 * n + 2, dtype=np.int32), (count, 1))
    ops = g.permuted(ops, axis=1).astype(np.int32)
    return np.ascontiguousarray(ops), _cuts(g, 2 * n, m, count)


def precedence_candidates(n, m, count, seed):
    """Acyclic candidates: a random global op order with every drop before its
    pickup, each op sent to a uniformly random vehicle; route order is the
    global order restricted to the vehicle.  Every op gets simulated."""
    g = _rng(seed, 5)
    two_n = 2 * n
    ops = np.tile(np.arange(2, two_n + 2, dtype=np.int64), (count, 1))
    ops = g.permuted(ops, axis=1)
    # put each customer's drop before its pickup: the two positions of a
    # customer swap op codes when the pickup came first
    pos = np.argsort(ops, axis=1)              # pos[:, o-2] = position of op o
    pd = pos[:, 0::2]                          # drop positions, customer 1..n
    pp = pos[:, 1::2]                          # pickup positions
    first = np.minimum(pd, pp)
    second = np.maximum(pd, pp)
    cust = np.arange(1, n + 1, dtype=np.int64)[None, :]
    rows = np.arange(count)[:, None]
    ops[rows, first] = 2 * cust
    ops[rows, second] = 2 * cust + 1
    veh = g.integers(0, m, size=(count, two_n))
    # stable sort by vehicle keeps the global order inside each route
    order = np.argsort(veh, axis=1, kind="stable")
    ops = np.take_along_axis(ops, order, axis=1)
    counts = np.stack([(veh == v).sum(axis=1) for v in range(m)], axis=1)
    off = np.zeros((count, m + 1), dtype=np.int64)
    off[:, 1:] = np.cumsum(counts, axis=1)
    return np.ascontiguousarray(ops.astype(np.int32)), np.ascontiguousarray(off.astype(np.int32))


def random_keys(count, length, seed):
    """float32 random keys in [0,1) with 24 random bits each."""
    g = _rng(seed, 6)
    return (g.integers(0, 1 << 24, size=(count, length), dtype=np.int64)
            .astype(np.float32) * np.float32(2.0 ** -24))


def loguniform_sizes(count, lo, hi, seed):
    g = _rng(seed, 7)
    u = g.random(count)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64).clip(lo, hi)


# The five synthetic workloads, named by what they exercise and their size.
CONFIGS = {
    "tiny_n16": dict(n=16, m=2, R=4, Q=4, variant="base", layout="uniform", eval_batch=4096,
                     alns_iters=200),
    "alns_n100": dict(n=100, m=4, R=10, Q=5, variant="2x", layout="uniform", eval_batch=65536,
                      alns_iters=5000, q=10),
    "brkga_n200": dict(n=200, m=6, R=20, Q=6, variant="5x", layout="clustered", pop=1024,
                       elite=0.2, mutant=0.1, rho=0.7, generations=1000),
    "uneven_256": dict(instances=256, n_lo=17, n_hi=500, Q=8, variant="1R10", layout="uniform",
                       per_instance=4096),
    "serving_n1000": dict(n=1000, m=20, R=100, Q=10, variant="1R20", layout="mixed"),
}


def uneven_instances(count, n_lo, n_hi, Q, variant, seed, per_instance_seed=1000):
    """Configuration-4 style set: n log-uniform in [n_lo, n_hi], m = ceil(n/25),
    R = ceil(n/10), Q fixed, uniform coordinates."""
    sizes = loguniform_sizes(count, n_lo, n_hi, seed)
    out = []
    for i, n in enumerate(sizes):
        n = int(n)
        m = -(-n // 25)
        R = -(-n // 10)
        out.append(make_instance(n, m, R, Q, variant, "uniform", seed=per_instance_seed + i))
    return out
