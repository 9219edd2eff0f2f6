"""Dispatch derivative on the GPU (opf_vjp_prepare / opf_dispatch_vjp and the
autograd wrapper) against the oracle's implicit-function gradient.

* At a common point (the oracle's barrier solution, polished at fixed mu):
  element-wise parity to 1e-9 relative, for 1, 5 and 40 cotangents (40 spans two
  column blocks of the multi-RHS solves).
* From the GPU's own solve (both variants), through torch.autograd and
  torch.func.vmap: 1e-6 relative to the oracle gradient at the oracle's own
  solution (the two solutions agree to the IPM tolerance, not bit for bit).
* The 10,000-bus case with 256 unit cotangents, at the stored oracle solution.
The oracle gradient itself is pinned against finite differences of re-solved
barrier solutions in test_oracle_sens.py.
"""
import dataclasses
import functools
import json
import os

import numpy as np
import pytest

import gridgen
from oracle import ipm, sens

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_SAME_POINT = 1e-9
TOL_OWN_SOLVE = 1e-6


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_point(name):
    net = gridgen.WORKLOADS[name]()
    if name == "grid10k":
        z = np.load(os.path.join(GOLDEN, "grid10k_linred.npz"))
        start = sens.BarrierPoint(z["w"], z["s"], z["lam"], z["y"], z["zwl"], z["zwu"], z["zsl"], z["zsu"],
                                  float(z["mu"]))
    else:
        res = ipm.linred(net)
        assert res.status == "converged"
        start = sens.BarrierPoint.from_result(res)
    p = sens.barrier_solve(net, start)
    assert p.residual <= 1e-10
    return net, p


def at_mu(net, p, mu):
    if mu == p.mu:
        return p
    q = sens.barrier_solve(net, dataclasses.replace(p, mu=mu))
    assert q.residual <= 1e-10
    return q


def gpu_vjp(h, V):
    v = torch.tensor(V, dtype=torch.float64, device="cuda")
    gP = torch.empty((V.shape[0], h.nb), dtype=torch.float64, device="cuda")
    gQ = torch.empty_like(gP)
    h.dispatch_vjp(v, gP, gQ)
    return gP.cpu().numpy(), gQ.cpu().numpy()


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
@pytest.mark.parametrize("k", [1, 5, 40])
def test_vjp_parity_at_the_oracle_point(pkg, name, k):
    net, p = oracle_point(name)
    sw, ss = p.sigma(net)
    V = np.random.default_rng(k).standard_normal((k, net.ng))
    ref_P, ref_Q = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, V)
    h = pkg.Handle(net)
    h.vjp_prepare(p.w, p.lam, p.y, sw, ss)
    gP, gQ = gpu_vjp(h, V)
    scale = max(np.abs(ref_P).max(), np.abs(ref_Q).max())
    assert np.abs(gP - ref_P).max() <= TOL_SAME_POINT * scale
    assert np.abs(gQ - ref_Q).max() <= TOL_SAME_POINT * scale


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
@pytest.mark.parametrize("variant", ["linred", "redlin"])
def test_autograd_from_the_gpu_solve(pkg, name, variant):
    from paper_2203_11875_gb300 import autograd as ag
    net, p = oracle_point(name)
    h = pkg.Handle(net)
    Pd = torch.tensor(net.Pd, device="cuda", requires_grad=True)
    Qd = torch.tensor(net.Qd, device="cuda", requires_grad=True)
    Pg = ag.optimal_dispatch(h, Pd, Qd, variant=variant)
    # the derivative is that of the barrier solution at the solve's final mu:
    # the oracle's point is moved to the same mu
    p = at_mu(net, p, h.last_result["mu"])
    sw, ss = p.sigma(net)
    V = gridgen.cotangents(net.ng, 8, seed=7)
    ref_P, ref_Q = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, V)
    # one cotangent through .backward()
    (Pg * torch.tensor(V[0], device="cuda")).sum().backward()
    info = h.vjp_info()
    assert info["polish_iters"] >= 0 and info["kkt_residual"] <= 1e-10, info
    assert info["rel_residual"] <= 1e-13, info
    scale = max(np.abs(ref_P).max(), np.abs(ref_Q).max())
    assert np.abs(Pd.grad.cpu().numpy() - ref_P[0]).max() <= TOL_OWN_SOLVE * scale
    assert np.abs(Qd.grad.cpu().numpy() - ref_Q[0]).max() <= TOL_OWN_SOLVE * scale
    # all eight in one batched call
    _, vjp_fn = torch.func.vjp(lambda a, b: ag.optimal_dispatch(h, a, b, variant=variant),
                               Pd.detach(), Qd.detach())
    gP, gQ = torch.func.vmap(vjp_fn)(torch.tensor(V, device="cuda"))
    assert np.abs(gP.cpu().numpy() - ref_P).max() <= TOL_OWN_SOLVE * scale
    assert np.abs(gQ.cpu().numpy() - ref_Q).max() <= TOL_OWN_SOLVE * scale


def test_grid10k_256_cotangents_at_the_stored_solution(pkg):
    net, p = oracle_point("grid10k")
    sw, ss = p.sigma(net)
    V = gridgen.cotangents(net.ng)
    assert V.shape == (256, net.ng)
    ref_P, ref_Q = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, V)
    h = pkg.Handle(net)
    h.vjp_prepare(p.w, p.lam, p.y, sw, ss)
    gP, gQ = gpu_vjp(h, V)
    scale = max(np.abs(ref_P).max(), np.abs(ref_Q).max())
    assert np.abs(gP - ref_P).max() <= TOL_SAME_POINT * scale
    assert np.abs(gQ - ref_Q).max() <= TOL_SAME_POINT * scale


def test_grid10k_autograd_from_the_gpu_solve(pkg):
    from paper_2203_11875_gb300 import autograd as ag
    net, p = oracle_point("grid10k")
    with open(os.path.join(GOLDEN, "grid10k_linred.json")) as fh:
        gold = json.load(fh)
    h = pkg.Handle(net)
    Pd = torch.tensor(net.Pd, device="cuda")
    Qd = torch.tensor(net.Qd, device="cuda")
    _, vjp_fn = torch.func.vjp(lambda a, b: ag.optimal_dispatch(h, a, b), Pd, Qd)
    p = at_mu(net, p, h.last_result["mu"])
    sw, ss = p.sigma(net)
    V = gridgen.cotangents(net.ng)[:32]
    gP, gQ = torch.func.vmap(vjp_fn)(torch.tensor(V, device="cuda"))
    ref_P, ref_Q = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, V)
    scale = max(np.abs(ref_P).max(), np.abs(ref_Q).max())
    assert np.abs(gP.cpu().numpy() - ref_P).max() <= TOL_OWN_SOLVE * scale
    assert np.abs(gQ.cpu().numpy() - ref_Q).max() <= TOL_OWN_SOLVE * scale
    # the solve behind it reached the oracle's objective
    from oracle import model
    w, _, _, _ = h.solution()
    obj = model.objective(model.Layout(net), w)
    assert abs(obj - gold["obj"]) <= 1e-6 * abs(gold["obj"])


def test_vjp_argument_errors(pkg):
    net = gridgen.tiny3()
    h = pkg.Handle(net)
    V = np.ones((2, net.ng))
    with pytest.raises(pkg.OPFError):            # not prepared
        gpu_vjp(h, V)
    with pytest.raises(pkg.OPFError):            # no stored solution
        h.vjp_prepare()
    w0 = np.zeros(h.nw)
    with pytest.raises(pkg.OPFError):            # some but not all of the point
        h.vjp_prepare(w0)
    bad = net.Pd.copy()
    bad[1] = np.nan
    with pytest.raises(pkg.OPFError):
        h.set_loads(bad, net.Qd)
    # k = 0 after a solve is a no-op
    assert h.solve()["status"] == 0
    h.vjp_prepare()
    e = torch.empty((0, net.ng), dtype=torch.float64, device="cuda")
    out = torch.empty((0, net.nb), dtype=torch.float64, device="cuda")
    h.dispatch_vjp(e, out, out.clone())
