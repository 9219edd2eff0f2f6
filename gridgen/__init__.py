"""Seeded synthetic power-grid networks (inputs only).

This module draws the networks that both the CPU oracle and the CUDA path
consume.  It holds none of the method's arithmetic: no admittances, no power
flow, no derivatives -- only topology, per-unit line parameters, generator
data and loads, drawn from fixed seeds.  Every quantity is in per unit.

Workload recipes (one per named workload):

* ``ring30``      -- 30-bus ring plus 11 random chords (41 lines), 6 generators,
                     every line flow-limited.
* ``lattice(nb)`` -- 2-D lattice with 20% of the edges dropped (connectivity
                     restored), plus short random chords; 10% of the buses
                     carry a generator; 10% of the lines are flow-limited.

Per-element distributions (shared by all recipes): r ~ U[0.005, 0.05],
x ~ U[0.02, 0.2], b ~ U[0, 0.05], rate ~ U[1, 3]; c2 ~ U[0.01, 0.1],
c1 ~ U[10, 40]; Pg in [0, Pmax], Pmax ~ U[0.5, 2]; Qg in [-Pmax, Pmax];
Vm in [0.94, 1.06]; loads P ~ U[0.1, 0.5], Q = 0.3 P.  Generators sit on
distinct buses; generator 0's bus is the slack (reference) bus.

The load and capacity distributions above, taken together, give more load
than generation capacity (expected 0.3 p.u. of load per bus against
0.125 p.u. of capacity per bus at 10% generator buses), which no dispatch can
serve.  The drawn loads are therefore rescaled by one common factor so that
total active load equals ``LOAD_TO_CAPACITY`` times total capacity; the shape
of the load distribution is kept.
"""
from __future__ import annotations

import dataclasses
from collections import deque

import numpy as np

SEED_BASE = 2203_11875
LOAD_TO_CAPACITY = 0.5


@dataclasses.dataclass
class Network:
    """A transmission network in per unit (host arrays, 0-based indices)."""

    name: str
    nb: int
    slack: int
    Pd: np.ndarray          # [nb] active load
    Qd: np.ndarray          # [nb] reactive load
    Vmin: np.ndarray        # [nb]
    Vmax: np.ndarray        # [nb]
    lf: np.ndarray          # [nl] int32 from-bus
    lt: np.ndarray          # [nl] int32 to-bus
    r: np.ndarray           # [nl] series resistance
    x: np.ndarray           # [nl] series reactance
    b: np.ndarray           # [nl] total line charging susceptance
    rate: np.ndarray        # [nl] apparent-power limit, 0 = unlimited
    gbus: np.ndarray        # [ng] int32 generator bus (distinct)
    Pmin: np.ndarray        # [ng]
    Pmax: np.ndarray        # [ng]
    Qmin: np.ndarray        # [ng]
    Qmax: np.ndarray        # [ng]
    c2: np.ndarray          # [ng] quadratic cost coefficient
    c1: np.ndarray          # [ng] linear cost coefficient

    @property
    def nl(self) -> int:
        return int(self.lf.shape[0])

    @property
    def ng(self) -> int:
        return int(self.gbus.shape[0])

    def copy(self) -> "Network":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy()
                              if isinstance(getattr(self, f.name), np.ndarray)
                              else getattr(self, f.name))
                     for f in dataclasses.fields(self)})

    def save(self, path: str) -> None:
        np.savez(path, **{f.name: getattr(self, f.name) for f in dataclasses.fields(self)})

    @staticmethod
    def load(path: str) -> "Network":
        z = np.load(path, allow_pickle=False)
        kw = {}
        for f in dataclasses.fields(Network):
            v = z[f.name]
            if f.name == "name":
                v = str(v)
            elif f.name in ("nb", "slack"):
                v = int(v)
            kw[f.name] = v
        return Network(**kw)


def _connected(nb: int, edges: list[tuple[int, int]]) -> bool:
    adj = [[] for _ in range(nb)]
    for a, c in edges:
        adj[a].append(c)
        adj[c].append(a)
    seen = np.zeros(nb, bool)
    seen[0] = True
    q = deque([0])
    while q:
        i = q.popleft()
        for j in adj[i]:
            if not seen[j]:
                seen[j] = True
                q.append(j)
    return bool(seen.all())


def _components(nb: int, edges) -> np.ndarray:
    parent = np.arange(nb)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a, c in edges:
        ra, rc = find(a), find(c)
        if ra != rc:
            parent[ra] = rc
    return np.array([find(i) for i in range(nb)])


def _finish(name, rng, nb, edges, ng, limited_frac, gen_buses=None) -> Network:
    nl = len(edges)
    lf = np.array([e[0] for e in edges], np.int32)
    lt = np.array([e[1] for e in edges], np.int32)
    r = rng.uniform(0.005, 0.05, nl)
    x = rng.uniform(0.02, 0.2, nl)
    b = rng.uniform(0.0, 0.05, nl)
    rate = rng.uniform(1.0, 3.0, nl)
    if limited_frac < 1.0:
        nlim = int(round(limited_frac * nl))
        keep = np.zeros(nl, bool)
        keep[rng.choice(nl, nlim, replace=False)] = True
        rate = np.where(keep, rate, 0.0)
    if gen_buses is None:
        gen_buses = rng.choice(nb, ng, replace=False)
    gbus = np.asarray(gen_buses, np.int32)
    Pmax = rng.uniform(0.5, 2.0, ng)
    c2 = rng.uniform(0.01, 0.1, ng)
    c1 = rng.uniform(10.0, 40.0, ng)
    Pd = rng.uniform(0.1, 0.5, nb)
    Pd *= LOAD_TO_CAPACITY * Pmax.sum() / Pd.sum()
    Qd = 0.3 * Pd
    return Network(
        name=name, nb=nb, slack=int(gbus[0]), Pd=Pd, Qd=Qd,
        Vmin=np.full(nb, 0.94), Vmax=np.full(nb, 1.06),
        lf=lf, lt=lt, r=r, x=x, b=b, rate=rate,
        gbus=gbus, Pmin=np.zeros(ng), Pmax=Pmax, Qmin=-Pmax.copy(), Qmax=Pmax.copy(),
        c2=c2, c1=c1)


def ring30(seed: int = SEED_BASE + 0) -> Network:
    """30-bus ring plus 11 distinct random chords; 6 generators; all lines limited."""
    rng = np.random.default_rng(seed)
    nb = 30
    edges = [(i, (i + 1) % nb) for i in range(nb)]
    have = {tuple(sorted(e)) for e in edges}
    while len(edges) < 41:
        a, c = rng.choice(nb, 2, replace=False)
        key = (int(min(a, c)), int(max(a, c)))
        if key in have:
            continue
        have.add(key)
        edges.append((int(a), int(c)))
    return _finish("ring30", rng, nb, edges, ng=6, limited_frac=1.0)


def _lattice_dims(nb: int) -> tuple[int, int]:
    best = (1, nb)
    for rows in range(1, int(np.sqrt(nb)) + 1):
        if nb % rows == 0:
            best = (rows, nb // rows)
    return best


def lattice(nb: int, seed: int, gen_frac: float = 0.10, name: str | None = None,
            load_scale: tuple[float, float] | None = None) -> Network:
    """Grid-like network: lattice, 20% edges dropped, short chords.

    Dropped edges that would disconnect the network are put back (the union-find
    pass below re-adds a dropped edge between any two components).  Chords join
    buses at lattice distance two (a diagonal or a two-step hop); their count is
    5% of the bus count.  With ``load_scale`` each bus load is further
    multiplied by its own draw from U[lo, hi].
    """
    rng = np.random.default_rng(seed)
    R, C = _lattice_dims(nb)
    idx = lambda i, j: i * C + j  # noqa: E731
    lat = []
    for i in range(R):
        for j in range(C):
            if j + 1 < C:
                lat.append((idx(i, j), idx(i, j + 1)))
            if i + 1 < R:
                lat.append((idx(i, j), idx(i + 1, j)))
    lat = np.array(lat, np.int64)
    drop = rng.random(len(lat)) < 0.20
    kept = [tuple(map(int, e)) for e in lat[~drop]]
    dropped = [tuple(map(int, e)) for e in lat[drop]]
    comp = _components(nb, kept)
    for e in dropped:             # restore connectivity with dropped edges
        if comp[e[0]] != comp[e[1]]:
            kept.append(e)
            comp = _components(nb, kept)
    have = {tuple(sorted(e)) for e in kept}
    nchord = int(round(0.05 * nb))
    offsets = [(1, 1), (1, -1), (2, 0), (0, 2)]
    added = 0
    while added < nchord:
        i, j = int(rng.integers(R)), int(rng.integers(C))
        di, dj = offsets[int(rng.integers(len(offsets)))]
        i2, j2 = i + di, j + dj
        if not (0 <= i2 < R and 0 <= j2 < C):
            continue
        key = tuple(sorted((idx(i, j), idx(i2, j2))))
        if key in have:
            continue
        have.add(key)
        kept.append((idx(i, j), idx(i2, j2)))
        added += 1
    assert _connected(nb, kept)
    ng = int(round(gen_frac * nb))
    net = _finish(name or f"lattice{nb}", rng, nb, kept, ng=ng, limited_frac=0.10)
    if load_scale is not None:
        f = rng.uniform(load_scale[0], load_scale[1], nb)
        net.Pd = net.Pd * f
        net.Qd = net.Qd * f
    return net


# ---------------------------------------------------------------- workloads
def grid2000() -> Network:
    """2,000-bus lattice network, 200 generators (nu = 399, nx = 3,799)."""
    return lattice(2000, SEED_BASE + 1, name="grid2000")


def grid10k() -> Network:
    """10,000-bus lattice network, 1,000 generators (nu = 1,999, nx = 18,999)."""
    return lattice(10000, SEED_BASE + 2, name="grid10k")


BATCH_SIZES = (500, 1500, 3000)


def batch96() -> list[Network]:
    """96 uneven instances: 32 networks each at 500, 1,500 and 3,000 buses.

    Network j (0..95) is drawn from seed SEED_BASE + 3 + 1000 j, with its
    bus loads scaled per bus by U[0.8, 1.2].
    """
    nets = []
    for k, nb in enumerate(BATCH_SIZES):
        for i in range(32):
            j = 32 * k + i
            nets.append(lattice(nb, SEED_BASE + 3 + 1000 * j, name=f"b{nb}_{i}",
                                load_scale=(0.8, 1.2)))
    return nets


def cotangents(ng: int, k: int = 256, seed: int = SEED_BASE + 4) -> np.ndarray:
    """k random unit vectors in R^ng (cotangents on the optimal dispatch)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((k, ng))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def lossless(net: Network) -> Network:
    """Same topology with r = b = 0 and every V, Q and flow limit made loose."""
    n = net.copy()
    n.name = net.name + "_lossless"
    n.r = np.zeros_like(n.r)
    n.b = np.zeros_like(n.b)
    n.rate = np.zeros_like(n.rate)
    n.Vmin = np.full(n.nb, 0.5)
    n.Vmax = np.full(n.nb, 1.5)
    n.Qmin = np.full(n.ng, -1e3)
    n.Qmax = np.full(n.ng, 1e3)
    return n


def tiny3() -> Network:
    """A 3-bus triangle with 2 generators (nx = 3, nu = 3), fixed values."""
    return Network(
        name="tiny3", nb=3, slack=0,
        Pd=np.array([0.0, 0.3, 0.9]), Qd=np.array([0.0, 0.09, 0.27]),
        Vmin=np.full(3, 0.94), Vmax=np.full(3, 1.06),
        lf=np.array([0, 1, 0], np.int32), lt=np.array([1, 2, 2], np.int32),
        r=np.array([0.01, 0.02, 0.015]), x=np.array([0.1, 0.15, 0.12]),
        b=np.array([0.02, 0.01, 0.0]), rate=np.array([1.5, 0.0, 1.2]),
        gbus=np.array([0, 1], np.int32), Pmin=np.zeros(2), Pmax=np.array([1.0, 1.0]),
        Qmin=np.array([-1.0, -1.0]), Qmax=np.array([1.0, 1.0]),
        c2=np.array([0.05, 0.02]), c1=np.array([20.0, 30.0]))


WORKLOADS = {"ring30": ring30, "grid2000": grid2000, "grid10k": grid10k, "tiny3": tiny3}
