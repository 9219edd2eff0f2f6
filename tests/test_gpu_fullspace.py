"""The hybrid full-space solver (Sec. 4.3) against the oracle: the block LDL^T
of the slack-eliminated augmented matrix M through opf_fullspace_factor /
opf_fullspace_solve.

What is unique about any factorisation of M is compared: the Newton step
(against the sparse LU solve of M and the full K_aug solve, relative 1e-9),
the inertia (exactly, against Haynsworth additivity with the eigenvalues of
the oracle's K_cond, which the non-GPU pins tie to the eigenvalues of M), and
log|det M| (against the oracle's sparse LU, 1e-9 relative).  Points are random
iterates of uneven networks (3 to 3,000 buses, one definite and one indefinite
K_cond each), the dual regularisation delta_c, several right-hand sides (more
than one solve pass), and the stored grid10k iterate; the whole hybrid IPM is
checked against the condensed one (same iterations, objective 1e-6)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
from oracle import fullspace, kkt, model

from gpu_cases import rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-9
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


def point(net, seed, scale):
    lay = model.Layout(net)
    rng = np.random.default_rng(seed)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    lam = scale * rng.standard_normal(lay.nx)
    y = scale * rng.standard_normal(lay.m)
    sw = rng.uniform(0.5, 5.0, lay.nw)
    ss = rng.uniform(0.5, 5.0, lay.m)
    r = rng.standard_normal(lay.nw + 2 * lay.m + lay.nx)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    return dict(lay=lay, w=w, lam=lam, y=y, sw=sw, ss=ss, r=r, G=G, A=A, W=W)


def evaluated(pkg, net, p):
    lay = p["lay"]
    h = pkg.Handle(net)
    h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
    return h


def sig(p):
    lay = p["lay"]
    return T(p["sw"][:lay.nu]), T(p["sw"][lay.nu:]), T(p["ss"])


NETS = [("tiny3", gridgen.tiny3), ("ring30", gridgen.ring30),
        ("b500", lambda: gridgen.lattice(500, 7001, name="b500")),
        ("b3000", lambda: gridgen.lattice(3000, 7003, name="b3000")),
        ("grid2000", gridgen.grid2000)]


@pytest.mark.parametrize("name,make", NETS)
@pytest.mark.parametrize("delta_c", [0.0, 1e-2])
def test_fullspace_step_inertia_logdet(pkg, name, make, delta_c):
    net = make()
    p = point(net, 31, 1.0)
    lay = p["lay"]
    Kc0 = fullspace.kcond(p["G"], p["A"], p["W"], p["sw"], p["ss"], lay.nu, 0.0, delta_c)
    lmin = float(np.linalg.eigvalsh(Kc0)[0])
    h = evaluated(pkg, net, p)
    # an indefinite K_cond: the inertia is wrong and counted exactly
    for dw in (0.0, 0.5 * max(0.0, -lmin)):
        Kc = Kc0 + dw * np.eye(lay.nu)
        want = fullspace.inertia_by_reduction(Kc, lay.nx, lay.m)
        rc, inert = h.fullspace_factor(*sig(p), delta_w=dw, delta_c=delta_c)
        assert inert == want, (dw, inert, want)
        assert (rc == pkg.OPF_OK) == (want == (lay.nw, lay.nx + lay.m, 0))
    # a definite one: the inertia Theorem 3 asks for, the step and log|det|
    dw = max(0.0, -lmin) + 1.0
    rc, inert = h.fullspace_factor(*sig(p), delta_w=dw, delta_c=delta_c)
    assert rc == pkg.OPF_OK and inert == (lay.nw, lay.nx + lay.m, 0)
    M = fullspace.augmented(p["G"], p["A"], p["W"], p["sw"], p["ss"], lay.nu, dw, delta_c)
    st = h.fullspace_stats()
    ld = fullspace.logabsdet_lu(M)
    assert abs(st["logabsdet"] - ld) <= 1e-9 * max(1.0, abs(ld))
    ref = np.concatenate(fullspace.augmented_step(p["G"], p["A"], p["W"], p["sw"], p["ss"], p["r"], lay.nu, dw,
                                                  delta_c))
    Wd = p["W"] + sp.diags(np.r_[np.full(lay.nu, dw), np.zeros(lay.nx)])
    ref2 = np.concatenate(kkt.full_space_step(p["G"], p["A"], Wd, p["sw"], p["ss"], p["r"], delta_c=delta_c))
    assert rel_err(ref, ref2) <= 1e-10
    step = torch.zeros(len(p["r"]), dtype=torch.float64, device="cuda")
    for refine in (0, 3):
        h.fullspace_solve(T(p["r"]), step, 1, refine)
        assert rel_err(N(step), ref) <= TOL, refine


def test_fullspace_many_right_hand_sides(pkg):
    """Six right-hand sides (two solve passes of four columns) equal six single
    solves, and the oracle."""
    net = gridgen.lattice(500, 7001, name="b500")
    p = point(net, 5, 1.0)
    lay = p["lay"]
    Kc = fullspace.kcond(p["G"], p["A"], p["W"], p["sw"], p["ss"], lay.nu)
    dw = max(0.0, -float(np.linalg.eigvalsh(Kc)[0])) + 1.0
    h = evaluated(pkg, net, p)
    assert h.fullspace_factor(*sig(p), delta_w=dw)[0] == pkg.OPF_OK
    rng = np.random.default_rng(9)
    n = len(p["r"])
    R = rng.standard_normal((6, n))
    out = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    h.fullspace_solve(T(R.ravel()), out, 6, 0)
    out = N(out).reshape(6, n)
    one = torch.zeros(n, dtype=torch.float64, device="cuda")
    for j in range(6):
        h.fullspace_solve(T(R[j]), one, 1, 0)
        assert np.array_equal(N(one), out[j]), j
        ref = np.concatenate(fullspace.augmented_step(p["G"], p["A"], p["W"], p["sw"], p["ss"], R[j], lay.nu, dw))
        assert rel_err(out[j], ref) <= TOL, j


def test_fullspace_grid10k_at_oracle_iterate(pkg):
    """The stored grid10k iterate (nu = 1,999, 44,262 unknowns in M): the
    inertia at delta_w = 0 against Haynsworth with the oracle's K_cond, and at
    the iterate's own delta_w the step against the sparse K_aug solve."""
    d = dict(np.load(GOLDEN))
    net = gridgen.grid10k()
    lay = model.Layout(net)
    _, G, A = model.jacobians(lay, d["w"])
    W = model.lagrangian_hessian(lay, d["w"], d["lam"], d["y"])
    h = pkg.Handle(net)
    h.eval_derivatives(T(d["w"][lay.nu:]), T(d["w"][:lay.nu]), T(d["lam"]), T(d["y"]))
    sw, ss = d["sig_w"], d["sig_s"]
    sg = (T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    Kc = fullspace.kcond(G, A, W, sw, ss, lay.nu)
    rc, inert = h.fullspace_factor(*sg, delta_w=0.0)
    assert inert == fullspace.inertia_by_reduction(Kc, lay.nx, lay.m)
    delta = float(d["delta"])
    rc, inert = h.fullspace_factor(*sg, delta_w=delta)
    assert rc == pkg.OPF_OK and inert == (lay.nw, lay.nx + lay.m, 0)
    st = h.fullspace_stats()
    assert st["nblocks"] == net.nb + 2 * len(lay.lim)
    step = torch.zeros(len(d["r"]), dtype=torch.float64, device="cuda")
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, d["r"]))
    for refine in (0, 3):
        h.fullspace_solve(T(d["r"]), step, 1, refine)
        assert rel_err(N(step), ref) <= TOL, refine


@pytest.mark.parametrize("name,make", [("ring30", gridgen.ring30), ("grid2000", gridgen.grid2000)])
def test_hybrid_fullspace_ipm_matches_condensed(pkg, name, make):
    """The hybrid full-space IPM and LinRed are the same method in exact
    arithmetic (Sec. 4.3): same iteration count, objectives within 1e-6."""
    net = make()
    a = pkg.Handle(net).solve(linear_solver="condensed")
    b = pkg.Handle(net).solve(linear_solver="fullspace")
    assert a["status"] == 0 and b["status"] == 0
    assert abs(a["iters"] - b["iters"]) <= 1, (a["iters"], b["iters"])
    assert abs(a["obj"] - b["obj"]) <= 1e-6 * abs(a["obj"])
