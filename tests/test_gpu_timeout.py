"""Failure detection without a GPU fault: every device-side wait is bounded by
opf_options.spin_limit.  With a limit of one poll, the sync-free LU
refactorisation's waits on other rows run out at once; the kernel records the
timeout in the device status word and returns, the call reports
OPF_ERR_TIMEOUT, and the context stays usable for the next handle."""
import numpy as np
import pytest

import gridgen
from oracle import kkt, model
from gpu_cases import random_point, rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


def test_expired_wait_reports_timeout_and_the_context_survives(pkg):
    net, lay, w, lam, y, sw, ss = random_point("grid2000", seed=3)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    u, x = dev(w[:lay.nu]), dev(w[lay.nu:])
    # column-parallel solves (no bulk copies), one poll per wait
    h = pkg.Handle(net, rhs_block=32, spin_limit=1)
    h.eval_derivatives(x, u, dev(lam), dev(y))
    with pytest.raises(pkg.OPFError) as err:
        h.condense(dev(sw[:lay.nu]), dev(sw[lay.nu:]), dev(ss))
    assert err.value.code == pkg.OPF_ERR_TIMEOUT
    h.close()
    # a new handle with the default limit condenses correctly on the same context
    h2 = pkg.Handle(net)
    h2.eval_derivatives(x, u, dev(lam), dev(y))
    K = torch.empty((lay.nu, lay.nu), dtype=torch.float64, device="cuda")
    h2.condense(dev(sw[:lay.nu]), dev(sw[lay.nu:]), dev(ss), K)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    ref = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    assert rel_err(K.cpu().numpy(), ref) <= 1e-9
