"""Writes the stored mid-solve iterate of the 10,000-bus workload.

Calls only the CPU oracle.  Output, beside this script:
  grid10k_iterate.npz   the oracle's linearize-then-reduce iterate at iteration
                        RECORD_AT (w, s, lam, y, Sigma_w, Sigma_s, the full-space
                        right-hand side r, mu and the delta_w its inertia
                        correction chose).  The full-size parity tests condense,
                        factor and solve at this point and compare with the
                        oracle's definitions evaluated there.
Run from the repository root:  python tests/golden/make_grid10k_iterate.py
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

RECORD_AT = 3


def main():
    net = gridgen.grid10k()
    t0 = time.time()
    res = ipm.linred(net, record_at=RECORD_AT, max_iter=RECORD_AT + 1, verbose=True)
    rec = res.history[0]
    np.savez_compressed(os.path.join(HERE, "grid10k_iterate.npz"), it=rec["it"], w=rec["w"], s=rec["s"],
                        lam=rec["lam"], y=rec["y"], sig_w=rec["sig_w"], sig_s=rec["sig_s"], r=rec["r"],
                        mu=rec["mu"], delta=rec["delta"])
    print(json.dumps(dict(workload="grid10k", record_at=RECORD_AT, mu=rec["mu"], delta=rec["delta"],
                          seconds=time.time() - t0)))


if __name__ == "__main__":
    main()
