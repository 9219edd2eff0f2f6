"""Pins of the oracle's dispatch derivative (CPU only).

The derivative is the implicit-function formula written out with a sparse LU of
the whole K_aug (oracle.sens.dispatch_vjp).  It is pinned by routes that do not
go through that formula:
  * dF/dd and dPg/dd against differences of the model functions with the
    loads changed (F is affine in the loads, so central differences are exact
    up to rounding);
  * the whole vector-Jacobian product against central differences (h = 1e-6)
    of the barrier solution itself, re-solved by Newton's method at the same
    fixed mu for perturbed loads;
  * a closed form: on a lossless network with loose limits the OPF is economic
    dispatch, whose generators share any change of total demand in proportion
    to 1 / c2, wherever it is added, and ignore reactive loads.
"""
import dataclasses

import numpy as np
import pytest

import gridgen
from oracle import ipm, model, sens


def _kkt_F(net, p):
    lay = model.Layout(net)
    gf, G, A = model.jacobians(lay, p.w)
    return np.concatenate([gf + G.T @ p.lam + A.T @ p.y - p.zwl + p.zwu, p.y - p.zsl + p.zsu,
                           model.cons_g(lay, p.w), model.cons_h(lay, p.w) + p.s])


_SOLVED = {}


def _solved(name):
    if name not in _SOLVED:
        net = gridgen.WORKLOADS[name]()
        res = ipm.linred(net)
        assert res.status == "converged"
        p = sens.barrier_solve(net, sens.BarrierPoint.from_result(res))
        assert p.residual <= 1e-11
        _SOLVED[name] = (net, p)
    return _SOLVED[name]


@pytest.mark.parametrize("name", ["tiny3", "ring30"])
def test_load_jacobian_is_the_derivative_of_F(name):
    net, p = _solved(name)
    lay = model.Layout(net)
    dF = sens.load_jacobian(lay, p.w)
    rng = np.random.default_rng(3)
    for _ in range(4):
        dP, dQ = rng.standard_normal(net.nb), rng.standard_normal(net.nb)
        h = 1e-3
        Fp = _kkt_F(sens.with_loads(net, net.Pd + h * dP, net.Qd + h * dQ), p)
        Fm = _kkt_F(sens.with_loads(net, net.Pd - h * dP, net.Qd - h * dQ), p)
        fd = (Fp - Fm) / (2 * h)
        an = dF @ np.concatenate([dP, dQ])
        assert np.abs(fd - an).max() <= 1e-8 * max(1.0, np.abs(an).max())


@pytest.mark.parametrize("name", ["tiny3", "ring30"])
def test_output_jacobian_is_the_derivative_of_the_dispatch(name):
    net, p = _solved(name)
    lay = model.Layout(net)
    J, D = sens.output_jacobian(lay, p.w)
    rng = np.random.default_rng(4)
    nw = lay.nw
    dw = rng.standard_normal(nw)
    h = 1e-20
    # complex step in w: the dispatch is analytic in the voltages
    Pg_c, _ = model.dispatch(lay, p.w + 1j * h * dw)
    assert np.allclose(np.imag(Pg_c) / h, J[:, :nw] @ dw, rtol=1e-12, atol=1e-12)
    assert J[:, nw:].nnz == 0
    dP, dQ = rng.standard_normal(net.nb), rng.standard_normal(net.nb)
    Pp, _ = model.dispatch(model.Layout(sens.with_loads(net, net.Pd + dP, net.Qd + dQ)), p.w)
    P0, _ = model.dispatch(lay, p.w)
    assert np.allclose(Pp - P0, D @ np.concatenate([dP, dQ]), rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_vjp_matches_differences_of_the_barrier_solution(name):
    net, p = _solved(name)
    sw, ss = p.sigma(net)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((3, net.ng))
    gP, gQ = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, V)
    h = 1e-6
    for _ in range(2 if name == "grid2000" else 4):
        dP, dQ = rng.standard_normal(net.nb), rng.standard_normal(net.nb)
        Pp, pp = sens.solved_dispatch(net, p, net.Pd + h * dP, net.Qd + h * dQ)
        Pm, pm = sens.solved_dispatch(net, p, net.Pd - h * dP, net.Qd - h * dQ)
        assert pp.residual <= 1e-11 and pm.residual <= 1e-11
        fd = V @ (Pp - Pm) / (2 * h)
        an = gP @ dP + gQ @ dQ
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max()


def test_vjp_of_each_generator_matches_full_differences_tiny3():
    # brute force: every load perturbed on its own, all generators at once
    net, p = _solved("tiny3")
    sw, ss = p.sigma(net)
    gP, gQ = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, np.eye(net.ng))
    h = 1e-6
    for i in range(net.nb):
        for which in ("P", "Q"):
            e = np.zeros(net.nb)
            e[i] = h
            Pd_p, Qd_p = (net.Pd + e, net.Qd) if which == "P" else (net.Pd, net.Qd + e)
            Pd_m, Qd_m = (net.Pd - e, net.Qd) if which == "P" else (net.Pd, net.Qd - e)
            Pp, _ = sens.solved_dispatch(net, p, Pd_p, Qd_p)
            Pm, _ = sens.solved_dispatch(net, p, Pd_m, Qd_m)
            col = (Pp - Pm) / (2 * h)
            an = gP[:, i] if which == "P" else gQ[:, i]
            assert np.abs(col - an).max() <= 1e-6 * max(1.0, np.abs(an).max())


def test_lossless_dispatch_shares_demand_by_inverse_cost_curvature():
    net = gridgen.lossless(gridgen.ring30())
    net.c1 = np.full(net.ng, 20.0)           # equal marginal cost at zero output:
    net.Pmax = np.full(net.ng, 10.0)         # every generator ends inside its range
    res = ipm.linred(net, max_iter=80)
    p = sens.BarrierPoint.from_result(res)
    # follow the barrier path down to mu = 1e-9 (the voltage continuum slows the IPM)
    for mu in (1e-6, 1e-7, 1e-8, 1e-9):
        p = sens.barrier_solve(net, dataclasses.replace(p, mu=mu))
        assert p.residual <= 1e-10
    sw, ss = p.sigma(net)
    gP, gQ = sens.dispatch_vjp(net, p.w, p.lam, p.y, sw, ss, np.eye(net.ng))
    share = (1.0 / net.c2) / np.sum(1.0 / net.c2)
    # the barrier moves the solution by O(mu): 1e-7 leaves a wide margin at mu = 1e-9
    assert np.abs(gP - share[:, None]).max() <= 1e-7
    assert np.abs(gQ).max() <= 1e-7
