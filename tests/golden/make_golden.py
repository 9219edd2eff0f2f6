"""Writes the stored expected values for the 10,000-bus workload.

Calls only the CPU oracle.  Outputs, beside this script:
  grid10k_linred.json   objective, iterations and final error of the oracle's
                        linearize-then-reduce solve;
  grid10k_linred.npz    its converged point (w, s, lam, y, bound multipliers, mu)
                        for the dispatch-derivative parity test.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gridgen  # noqa: E402
from oracle import ipm  # noqa: E402


def main():
    net = gridgen.grid10k()
    t0 = time.time()
    res = ipm.linred(net, verbose=True)
    out = dict(workload="grid10k", variant="linred", status=res.status, iters=res.iters, obj=res.obj,
               err=res.err, mu=res.mu, seconds=time.time() - t0)
    with open(os.path.join(HERE, "grid10k_linred.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    np.savez_compressed(os.path.join(HERE, "grid10k_linred.npz"), w=res.w, s=res.s, lam=res.lam, y=res.y,
                        zwl=res.zl[0], zsl=res.zl[1], zwu=res.zu[0], zsu=res.zu[1], mu=res.mu)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
