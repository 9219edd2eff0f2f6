"""Failure paths made on the host (no GPU fault, trap or hang): every one ends
in a status code, and the handle stays usable afterwards.

  * a network with a zero-impedance line is refused at opf_create (INVALID_ARG);
  * a non-finite iterate makes the G_x refactorisation report SINGULAR (the
    pivot test rejects non-finite pivots) instead of producing NaN factors;
  * Newton-Raphson on the state equation diverges under an infeasible load
    scale: opf_powerflow and the RedLin loop report PF_FAILED within their
    iteration caps;
  * an indefinite K_cond reports NOT_PD with the failing column, and a larger
    delta_w then factors it (the inertia-correction loop's two outcomes).
The expired bounded wait (TIMEOUT) is tests/test_gpu_timeout.py."""
import dataclasses

import numpy as np
import pytest

import gridgen
from oracle import kkt, model

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_zero_impedance_line_is_refused(pkg):
    net = gridgen.ring30()
    r, x = net.r.copy(), net.x.copy()
    r[3] = 0.0
    x[3] = 0.0
    with pytest.raises(pkg.OPFError) as e:
        pkg.Handle(dataclasses.replace(net, r=r, x=x))
    assert e.value.code == pkg.OPF_ERR_INVALID_ARG


def test_non_finite_iterate_reports_singular_and_the_handle_recovers(pkg):
    net = gridgen.ring30()
    lay = model.Layout(net)
    h = pkg.Handle(net)
    w = lay.flat_start()
    bad = w.copy()
    bad[lay.nu + 2] = np.nan
    zl, zy = np.zeros(lay.nx), np.zeros(lay.m)
    h.eval_derivatives(T(bad[lay.nu:]), T(bad[:lay.nu]), T(zl), T(zy))
    with pytest.raises(pkg.OPFError) as e:
        h.gx_factor()
    assert e.value.code == pkg.OPF_ERR_SINGULAR
    # a finite point on the same handle factors and solves again
    h.eval_derivatives(T(w[lay.nu:]), T(w[:lay.nu]), T(zl), T(zy))
    h.gx_factor()
    _, G, _ = model.jacobians(lay, w)
    b = np.random.default_rng(1).standard_normal(lay.nx)
    out = torch.zeros(lay.nx, dtype=torch.float64, device="cuda")
    h.gx_solve(0, T(b), out)
    ref = np.linalg.solve(G[:, lay.nu:].toarray(), b)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_infeasible_load_scale_reports_pf_failed(pkg):
    net = gridgen.ring30()
    heavy = dataclasses.replace(net, Pd=net.Pd * 25.0, Qd=net.Qd * 25.0)
    lay = model.Layout(heavy)
    h = pkg.Handle(heavy)
    w = lay.flat_start()
    x = T(w[lay.nu:])
    with pytest.raises(pkg.OPFError) as e:
        h.powerflow(T(w[:lay.nu]), x, tol=1e-10, max_iter=30)
    assert e.value.code == pkg.OPF_ERR_PF_FAILED
    with pytest.raises(pkg.OPFError) as e:
        pkg.Handle(heavy).solve("redlin", max_iter=50)
    assert e.value.code == pkg.OPF_ERR_PF_FAILED


def test_indefinite_kcond_then_regularised(pkg):
    net = gridgen.ring30()
    lay = model.Layout(net)
    rng = np.random.default_rng(4)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    lam, y = 30.0 * rng.standard_normal(lay.nx), 30.0 * rng.standard_normal(lay.m)
    sw, ss = rng.uniform(0.5, 5.0, lay.nw), rng.uniform(0.5, 5.0, lay.m)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Kc = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    lmin = float(np.linalg.eigvalsh(0.5 * (Kc + Kc.T))[0])
    assert lmin < 0
    h = pkg.Handle(net)
    h.eval_derivatives(T(w[lay.nu:]), T(w[:lay.nu]), T(lam), T(y))
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    assert h.kkt_factor(0.0) >= 0
    assert h.kkt_factor(-lmin + 1.0) == -1
