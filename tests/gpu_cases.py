"""Shared inputs for the GPU parity tests: oracle iterates of the seeded
workloads (the oracle produces every input and expected value; nothing here
comes from the CUDA path)."""
import functools

import numpy as np

import gridgen
from oracle import ipm, model

RECORD_AT = 10


@functools.lru_cache(maxsize=None)
def oracle_iterate(name: str, record_at: int = RECORD_AT):
    """The oracle LinRed iterate at iteration record_at of a named workload:
    w, s, lam, y, Sigma_w, Sigma_s, the full-space right-hand side r, mu."""
    net = gridgen.WORKLOADS[name]()
    res = ipm.linred(net, record_at=record_at, max_iter=record_at + 1)
    rec = res.history[0]
    return net, rec


def random_point(name: str, seed: int = 0):
    """A random point near the flat start with random multipliers and Sigma."""
    net = gridgen.WORKLOADS[name]()
    lay = model.Layout(net)
    rng = np.random.default_rng(seed)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    lam = rng.standard_normal(lay.nx)
    y = rng.standard_normal(lay.m)
    sw = rng.uniform(0.1, 10.0, lay.nw)
    ss = rng.uniform(0.1, 10.0, lay.m)
    return net, lay, w, lam, y, sw, ss


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
