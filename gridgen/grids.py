"""Synthetic grids and scenario batches (seeded, fixed draw order).

Bus-type codes follow the MATPOWER convention used by the paper (Sec. 3): 3 =
slack (reference), 2 = PV, 1 = PQ.  Branches are pi-models given by series
resistance r, series reactance x and total line charging b (half at each end),
with no taps, phase shifters or bus shunts.

Draw order for a meshed grid (one ``numpy.random.default_rng(seed)``):
  1. topology: ring (edge i -> i+1 mod n) or random recursive tree (bus i
     attaches to a uniform bus < i), then chords: uniform bus pairs, one pair
     per draw, rejecting self-loops and duplicates, until the branch count is
     reached;
  2. r, x, b vectors over all branches, in that order;
  3. PV buses: a uniform subset of the non-slack buses (bus 0 is the slack);
  4. base PV generation P (ascending PV bus order), then base PQ load P
     (ascending PQ bus order); Q = q_ratio * P.
Scenario factors: one ``default_rng(seed)`` drawing a [B, n] matrix of
per-bus factors; each factor scales that bus's generation and load alike.

The literal loadings of the large synthetic configurations do not admit a
flat-start Newton solution (the tree-plus-chords grids are far weaker than
real transmission grids), so every configuration carries one global load scale
``load_scale`` (lambda) applied to all injections.  The values below are the
largest 2**-k for which the FP64 reference Newton iteration converges from
flat start for the base case and at the top of the scenario range with
min |V| >= 0.8; they were found with ``oracle/calibrate_load_scale.py``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SLACK, PV, PQ = 3, 2, 1


@dataclass
class Grid:
    name: str
    n: int
    f: np.ndarray          # int32 [nbr] from-bus
    t: np.ndarray          # int32 [nbr] to-bus
    r: np.ndarray          # float64 [nbr] series resistance (p.u.)
    x: np.ndarray          # float64 [nbr] series reactance (p.u.)
    b: np.ndarray          # float64 [nbr] total line charging (p.u.)
    bus_type: np.ndarray   # int8 [n]
    p_gen: np.ndarray      # float64 [n] base generation P (PV buses)
    p_load: np.ndarray     # float64 [n] base load P (PQ buses)
    q_load: np.ndarray     # float64 [n] base load Q (PQ buses)
    v_set: np.ndarray      # float64 [n] |V| setpoint (slack, PV); 1.0 at PQ
    load_scale: float = 1.0

    @property
    def n_branch(self) -> int:
        return int(self.f.shape[0])


@dataclass
class Scenarios:
    factors: np.ndarray    # float64 [B, n]
    load_scale: float

    @property
    def batch(self) -> int:
        return int(self.factors.shape[0])

    def sbus(self, g: Grid) -> np.ndarray:
        """Complex injections [B, n] (generation minus load), p.u."""
        base = g.p_gen - g.p_load - 1j * g.q_load
        return (self.load_scale * self.factors) * base[None, :]

    def v0_flat(self, g: Grid) -> np.ndarray:
        """Flat start [B, n]: |V| = setpoint (1.0 at PQ buses), angle 0."""
        return np.broadcast_to(g.v_set.astype(np.complex128), (self.batch, g.n)).copy()


# Configuration table.  Keys name the workloads by what they are.
CONFIGS = {
    # 30-bus meshed grid, ring plus random chords, batch of 64 scenarios.
    "mesh30_b64": dict(n=30, topology="ring", n_branch=41, n_pv=5, pv_vset=1.02,
                       pv_p=(0.1, 0.5), pq_p=(0.05, 0.3), q_ratio=0.3,
                       r=(0.01, 0.05), x=(0.05, 0.2), bsh=(0.0, 0.02),
                       batch=64, scen=(0.7, 1.3), load_scale=1.0),
    # 2,000-bus meshed grid, spanning tree plus random chords, 10 % PV.
    "mesh2000_b10k": dict(n=2000, topology="tree", n_branch=2600, n_pv=200, pv_vset=1.02,
                          pv_p=(0.1, 0.5), pq_p=(0.05, 0.3), q_ratio=0.3,
                          r=(0.01, 0.05), x=(0.05, 0.2), bsh=(0.0, 0.02),
                          batch=10000, scen=(0.6, 1.4), load_scale=0.0625),
    # 9,000-bus meshed grid, spanning tree plus random chords, 15 % PV.
    "mesh9000_b10k": dict(n=9000, topology="tree", n_branch=14000, n_pv=1350, pv_vset=1.02,
                          pv_p=(0.1, 0.5), pq_p=(0.05, 0.3), q_ratio=0.3,
                          r=(0.01, 0.05), x=(0.05, 0.2), bsh=(0.0, 0.02),
                          batch=10000, scen=(0.6, 1.4), load_scale=0.03125),
}

FEEDERS = dict(count=256, size=(20, 400), r=(0.1, 0.6), x=(0.05, 0.3),
               pq_p=(0.002, 0.02), q_ratio=0.2, scen=(0.6, 1.4),
               per_feeder=100, load_scale=0.015625)


def _topology(rng, n, kind, n_branch):
    if kind == "ring":
        f = list(range(n))
        t = [(i + 1) % n for i in range(n)]
    elif kind == "tree":
        parents = rng.integers(0, np.arange(1, n))
        f = [int(p) for p in parents]
        t = list(range(1, n))
    else:
        raise ValueError(kind)
    seen = {(min(a, b), max(a, b)) for a, b in zip(f, t)}
    while len(f) < n_branch:
        a, b = (int(v) for v in rng.integers(0, n, size=2))
        key = (min(a, b), max(a, b))
        if a == b or key in seen:
            continue
        seen.add(key)
        f.append(a)
        t.append(b)
    return np.asarray(f, np.int32), np.asarray(t, np.int32)


def make_grid(name: str, seed: int = 0, **over) -> Grid:
    c = dict(CONFIGS[name])
    c.update(over)
    rng = np.random.default_rng(seed)
    n = c["n"]
    f, t = _topology(rng, n, c["topology"], c["n_branch"])
    nbr = f.shape[0]
    r = rng.uniform(*c["r"], size=nbr)
    x = rng.uniform(*c["x"], size=nbr)
    b = rng.uniform(*c["bsh"], size=nbr)
    pv = np.sort(rng.choice(np.arange(1, n), size=c["n_pv"], replace=False))
    bus_type = np.full(n, PQ, np.int8)
    bus_type[0] = SLACK
    bus_type[pv] = PV
    pq = np.flatnonzero(bus_type == PQ)
    p_gen = np.zeros(n)
    p_load = np.zeros(n)
    p_gen[pv] = rng.uniform(*c["pv_p"], size=pv.shape[0])
    p_load[pq] = rng.uniform(*c["pq_p"], size=pq.shape[0])
    q_load = c["q_ratio"] * p_load
    v_set = np.ones(n)
    v_set[pv] = c["pv_vset"]
    return Grid(name, n, f, t, r, x, b, bus_type, p_gen, p_load, q_load, v_set,
                float(c["load_scale"]))


def make_scenarios(g: Grid, batch: int, lo: float, hi: float, seed: int = 1,
                   load_scale: float | None = None) -> Scenarios:
    rng = np.random.default_rng(seed)
    fac = rng.uniform(lo, hi, size=(batch, g.n))
    return Scenarios(fac, g.load_scale if load_scale is None else load_scale)


def config_grid(name: str, seed: int = 0) -> Grid:
    return make_grid(name, seed)


def config_scenarios(name: str, g: Grid, batch: int | None = None, seed: int = 1) -> Scenarios:
    c = CONFIGS[name]
    return make_scenarios(g, c["batch"] if batch is None else batch, *c["scen"], seed=seed)


def make_feeders(seed: int = 0, count: int | None = None, **over) -> list[Grid]:
    """Radial low-voltage feeders: random recursive trees, slack at bus 0,
    every other bus a PQ load; no line charging."""
    c = dict(FEEDERS)
    c.update(over)
    count = c["count"] if count is None else count
    rng = np.random.default_rng(seed)
    sizes = rng.integers(c["size"][0], c["size"][1] + 1, size=count)
    out = []
    for k, n in enumerate(int(s) for s in sizes):
        parents = rng.integers(0, np.arange(1, n))
        f = parents.astype(np.int32)
        t = np.arange(1, n, dtype=np.int32)
        r = rng.uniform(*c["r"], size=n - 1)
        x = rng.uniform(*c["x"], size=n - 1)
        b = np.zeros(n - 1)
        bus_type = np.full(n, PQ, np.int8)
        bus_type[0] = SLACK
        p_load = np.zeros(n)
        p_load[1:] = rng.uniform(*c["pq_p"], size=n - 1)
        q_load = c["q_ratio"] * p_load
        out.append(Grid(f"feeder{k}", n, f, t, r, x, b, bus_type, np.zeros(n), p_load,
                        q_load, np.ones(n), float(c["load_scale"])))
    return out


def feeder_scenarios(feeders: list[Grid], per_feeder: int | None = None, seed: int = 1) -> list[Scenarios]:
    c = FEEDERS
    per = c["per_feeder"] if per_feeder is None else per_feeder
    rng = np.random.default_rng(seed)
    return [Scenarios(rng.uniform(*c["scen"], size=(per, g.n)), g.load_scale) for g in feeders]


# Static N-1 contingency batches: one instance per (branch outage, load level).
# Only outages that keep the grid connected are listed (a bridge outage would
# island buses).  The outaged branch keeps its place in the admittance
# pattern with zero admittance; every instance has the base injections times
# its load level (one injection profile per level, no per-bus draws).
N1_LEVELS = (0.8, 0.9, 1.0, 1.1, 1.2)


def bridges(n: int, f: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Boolean [nbr]: branch e is a bridge (its removal disconnects the graph).
    Parallel branches are never bridges.  Iterative DFS with low-link values
    (Tarjan), skipping only the branch used to enter a bus."""
    nbr = len(f)
    adj = [[] for _ in range(n)]
    for e in range(nbr):
        adj[int(f[e])].append((int(t[e]), e))
        adj[int(t[e])].append((int(f[e]), e))
    disc = [-1] * n
    low = [0] * n
    out = np.zeros(nbr, dtype=bool)
    timer = 0
    for root in range(n):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, 0)]  # (bus, entering branch, next adjacency index)
        while stack:
            u, pe, i = stack[-1]
            if i < len(adj[u]):
                stack[-1] = (u, pe, i + 1)
                w, e = adj[u][i]
                if e == pe:
                    continue
                if disc[w] < 0:
                    disc[w] = low[w] = timer
                    timer += 1
                    stack.append((w, e, 0))
                else:
                    low[u] = min(low[u], disc[w])
            else:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[u])
                    if low[u] > disc[p]:
                        out[pe] = True
    return out


def n1_contingencies(g: Grid) -> np.ndarray:
    """Indices of the branches whose single outage keeps the grid connected."""
    return np.flatnonzero(~bridges(g.n, g.f, g.t)).astype(np.int32)


def n1_batch(g: Grid, levels=N1_LEVELS):
    """(outage [B] branch index, level [B] load factor, in_service [B, nbr]
    bool, sbus [B, n] complex) for every connected single outage at every
    load level, level-major."""
    out = n1_contingencies(g)
    lv = np.asarray(levels, dtype=np.float64)
    outage = np.tile(out, len(lv))
    level = np.repeat(lv, len(out))
    ins = np.ones((len(outage), g.n_branch), dtype=bool)
    ins[np.arange(len(outage)), outage] = False
    base = g.p_gen - g.p_load - 1j * g.q_load
    sbus = (g.load_scale * level)[:, None] * base[None, :]
    return outage, level, ins, sbus
