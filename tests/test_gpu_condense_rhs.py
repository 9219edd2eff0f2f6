"""opf_condense_rhs / opf_kkt_solve_condensed: the step's right-hand side
condensed as one extra column of the condensation (S_x solve, H = K Z, the
adjoint solve and the G_u^T product), then only the Cholesky solve and the
recovery products.  Checked against the oracle's full-space step (1e-9), the
plain opf_kkt_solve (1e-12), with delta_w, after a larger delta_w refactor,
with delta_c (plain recovery on the kept right-hand side), on the explicit
route (no column: plain recovery), and at the stored grid10k iterate."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
from oracle import kkt, model

from gpu_cases import rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid10k_iterate.npz")


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


def point(net, seed):
    lay = model.Layout(net)
    rng = np.random.default_rng(seed)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    lam, y = rng.standard_normal(lay.nx), rng.standard_normal(lay.m)
    sw, ss = rng.uniform(0.5, 5.0, lay.nw), rng.uniform(0.5, 5.0, lay.m)
    r = rng.standard_normal(lay.nw + 2 * lay.m + lay.nx)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Kc = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    dw = max(0.0, -np.linalg.eigvalsh(0.5 * (Kc + Kc.T))[0]) + 1.0
    return dict(lay=lay, w=w, lam=lam, y=y, sw=sw, ss=ss, r=r, G=G, A=A, W=W, dw=dw)


def ref_step(p, dw, dc=0.0):
    lay = p["lay"]
    Wd = p["W"] + sp.diags(np.r_[np.full(lay.nu, dw), np.zeros(lay.nx)])
    return np.concatenate(kkt.full_space_step(p["G"], p["A"], Wd, p["sw"], p["ss"], p["r"], delta_c=dc))


@pytest.mark.parametrize("name,route", [("ring30", 0), ("grid2000", 0), ("grid2000", 1),
                                        ("b3000", 0)])
def test_condensed_rhs_step(pkg, name, route):
    net = gridgen.lattice(3000, 7003, name="b3000") if name == "b3000" else gridgen.WORKLOADS[name]()
    p = point(net, 17)
    lay = p["lay"]
    h = pkg.Handle(net, route=route)
    h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
    sg = (T(p["sw"][:lay.nu]), T(p["sw"][lay.nu:]), T(p["ss"]))
    h.condense_rhs(*sg, T(p["r"]))
    assert h.kkt_factor(p["dw"]) == -1
    step = torch.zeros(len(p["r"]), dtype=torch.float64, device="cuda")
    h.kkt_solve_condensed(step)
    ref = ref_step(p, p["dw"])
    assert rel_err(N(step), ref) <= 1e-9
    plain = torch.zeros_like(step)
    h.kkt_solve(T(p["r"]), plain)
    assert rel_err(N(step), N(plain)) <= 1e-12
    # a larger delta_w after the condensation: the column stays valid
    assert h.kkt_factor(3.0 * p["dw"]) == -1
    h.kkt_solve_condensed(step)
    assert rel_err(N(step), ref_step(p, 3.0 * p["dw"])) <= 1e-9
    # delta_c re-forms K: the kept right-hand side goes through the plain recovery
    Kt = kkt.kred_definition(p["G"], p["A"], p["W"], p["sw"], kkt.regularized_sigma(p["ss"], 0.05), lay.nu)
    dwc = max(0.0, -np.linalg.eigvalsh(0.5 * (Kt + Kt.T))[0]) + 1.0
    assert h.kkt_factor(dwc, 0.05) == -1
    h.kkt_solve_condensed(step)
    assert rel_err(N(step), ref_step(p, dwc, 0.05)) <= 1e-9


def test_condensed_rhs_step_grid10k(pkg):
    d = dict(np.load(GOLDEN))
    net = gridgen.grid10k()
    lay = model.Layout(net)
    _, G, A = model.jacobians(lay, d["w"])
    W = model.lagrangian_hessian(lay, d["w"], d["lam"], d["y"])
    h = pkg.Handle(net)
    h.eval_derivatives(T(d["w"][lay.nu:]), T(d["w"][:lay.nu]), T(d["lam"]), T(d["y"]))
    sw, ss = d["sig_w"], d["sig_s"]
    h.condense_rhs(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss), T(d["r"]))
    delta = float(d["delta"])
    assert h.kkt_factor(delta) == -1
    step = torch.zeros(len(d["r"]), dtype=torch.float64, device="cuda")
    h.kkt_solve_condensed(step)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, d["r"]))
    assert rel_err(N(step), ref) <= 1e-9
    # the first one-vector solve timed the solve's cluster at 4, 8, 16 CTAs on
    # a copy of its right-hand side; the second runs on the size it kept
    cl, ms = h.chol_solve_choice()
    assert cl in (4, 8, 16) and all(t > 0 for t in ms.values())
    h.kkt_solve_condensed(step)
    assert rel_err(N(step), ref) <= 1e-9


def test_condensed_rhs_needs_the_condensation(pkg):
    net = gridgen.ring30()
    h = pkg.Handle(net)
    step = torch.zeros(h.n_kkt, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.OPFError):
        h.kkt_solve_condensed(step)


@pytest.mark.parametrize("width", [128, 256, 512])
def test_chunked_condensation_matches_one_pass(pkg, width):
    """The adjoint-route condensation in column chunks of N (Sec. 3.3's batch
    width) gives the one-pass Kred and the same step (grid2000, nu = 399: the
    last chunk is ragged, and carries the right-hand side's column)."""
    net = gridgen.grid2000()
    p = point(net, 23)
    lay = p["lay"]
    out = []
    for w in (0, width):
        h = pkg.Handle(net, rhs_width=w if w else 10 ** 6)
        h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
        K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
        h.condense_rhs(T(p["sw"][:lay.nu]), T(p["sw"][lay.nu:]), T(p["ss"]), T(p["r"]), K)
        assert h.kkt_factor(p["dw"]) == -1
        step = torch.zeros(len(p["r"]), dtype=torch.float64, device="cuda")
        h.kkt_solve_condensed(step)
        out.append((N(K), N(step), h.rhs_width()[0]))
    assert out[0][2] == lay.nu and out[1][2] == min(width, lay.nu)
    assert rel_err(out[1][0], out[0][0]) <= 1e-12
    assert rel_err(out[1][1], ref_step(p, p["dw"])) <= 1e-9


def test_width_autotune_on_grid10k(pkg):
    """rhs_width = 0 times the products at N = nu, 512, 256, 128 on the first
    condensation and keeps the fastest; the Kred is right whatever it picks."""
    d = dict(np.load(GOLDEN))
    net = gridgen.grid10k()
    lay = model.Layout(net)
    _, G, A = model.jacobians(lay, d["w"])
    W = model.lagrangian_hessian(lay, d["w"], d["lam"], d["y"])
    h = pkg.Handle(net)
    h.eval_derivatives(T(d["w"][lay.nu:]), T(d["w"][:lay.nu]), T(d["lam"]), T(d["y"]))
    sw, ss = d["sig_w"], d["sig_s"]
    K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.condense_rhs(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss), T(d["r"]), K)
    width, ms = h.rhs_width()
    assert width in (lay.nu, 512, 256, 128) and all(t > 0 for t in ms)
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    assert rel_err(N(K).reshape(lay.nu, lay.nu), 0.5 * (Ko + Ko.T)) <= 1e-9
