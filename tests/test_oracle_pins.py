"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (a printed table, a different formulation, the complex step,
finite differences, a library factorisation, a closed form, an independent
optimiser).  No GPU needed."""
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import gridgen
from oracle import ipm, kkt, model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ring_net(nb, ng):
    """Minimal ring network with ng generators on buses 0..ng-1 (counting only)."""
    z = np.zeros
    lf = np.arange(nb, dtype=np.int32)
    lt = ((np.arange(nb) + 1) % nb).astype(np.int32)
    one = np.ones(nb)
    return gridgen.Network(
        name="ring", nb=nb, slack=0, Pd=z(nb), Qd=z(nb), Vmin=0.9 * one, Vmax=1.1 * one,
        lf=lf, lt=lt, r=0.01 * one, x=0.1 * one, b=z(nb), rate=z(nb),
        gbus=np.arange(ng, dtype=np.int32), Pmin=z(ng), Pmax=np.ones(ng), Qmin=-np.ones(ng),
        Qmax=np.ones(ng), c2=np.ones(ng), c1=np.ones(ng))


# ----------------------------------------------------------------- sizes
def test_table1_variable_split():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_counts.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 7
    for name, nb, ng, nx, nu in rows:
        lay = model.Layout(_ring_net(int(nb), int(ng)))
        assert (lay.nx, lay.nu) == (int(nx), int(nu)), name


def test_ring30_sizes():
    # the 30-bus workload: 11 controls and 53 states, every one of 41 lines limited
    lay = model.Layout(gridgen.ring30())
    assert (lay.nu, lay.nx, lay.nl, lay.m) == (11, 53, 41, 1 + 6 + 2 * 41)


# ------------------------------------------------------------ the model
def _ybus(net):
    """Nodal admittance matrix from the pi-model, by plain loops."""
    Y = np.zeros((net.nb, net.nb), complex)
    for l in range(net.nl):
        f, t = net.lf[l], net.lt[l]
        ys = 1.0 / complex(net.r[l], net.x[l])
        Y[f, f] += ys + 0.5j * net.b[l]
        Y[t, t] += ys + 0.5j * net.b[l]
        Y[f, t] -= ys
        Y[t, f] -= ys
    return Y


@pytest.mark.parametrize("make", [gridgen.tiny3, gridgen.ring30])
def test_injections_match_nodal_form(make):
    net = make()
    lay = model.Layout(net)
    rng = np.random.default_rng(3)
    w = lay.flat_start() + 0.05 * rng.standard_normal(lay.nw)
    Vm, Va = lay.voltages(w)
    P, Q = model.injections(lay, Vm, Va)
    V = Vm * np.exp(1j * Va)
    S = V * np.conj(_ybus(net) @ V)
    np.testing.assert_allclose(P, S.real, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Q, S.imag, rtol=0, atol=1e-12)


def _complex_step_jac(fun, w, n_out, h=1e-30):
    J = np.zeros((n_out, len(w)))
    for j in range(len(w)):
        wc = w.astype(complex)
        wc[j] += 1j * h
        J[:, j] = np.atleast_1d(fun(wc)).imag / h
    return J


@pytest.mark.parametrize("make", [gridgen.tiny3, gridgen.ring30])
def test_first_derivatives_complex_step(make):
    lay = model.Layout(make())
    rng = np.random.default_rng(5)
    w = lay.flat_start() + 0.05 * rng.standard_normal(lay.nw)
    gf, G, A = model.jacobians(lay, w)
    Gcs = _complex_step_jac(lambda v: model.cons_g(lay, v), w, lay.nx)
    Acs = _complex_step_jac(lambda v: model.cons_h(lay, v), w, lay.m)
    fcs = _complex_step_jac(lambda v: model.objective(lay, v), w, 1)[0]
    assert np.abs(G.toarray() - Gcs).max() <= 1e-12 * max(1, np.abs(Gcs).max())
    assert np.abs(A.toarray() - Acs).max() <= 1e-12 * max(1, np.abs(Acs).max())
    assert np.abs(gf - fcs).max() <= 1e-12 * max(1, np.abs(fcs).max())


@pytest.mark.parametrize("make", [gridgen.tiny3, gridgen.ring30])
def test_hessian_matches_fd_of_gradient(make):
    lay = model.Layout(make())
    rng = np.random.default_rng(7)
    w = lay.flat_start() + 0.05 * rng.standard_normal(lay.nw)
    lam = rng.standard_normal(lay.nx)
    y = rng.standard_normal(lay.m)
    W = model.lagrangian_hessian(lay, w, lam, y).toarray()
    # gradient of f + lam^T g + y^T h by the complex step, differenced centrally
    def grad(v):
        return _complex_step_jac(
            lambda z: model.objective(lay, z) + lam @ model.cons_g(lay, z) + y @ model.cons_h(lay, z),
            v, 1)[0]
    h = 1e-5
    Wfd = np.zeros_like(W)
    for j in range(lay.nw):
        e = np.zeros(lay.nw)
        e[j] = h
        Wfd[:, j] = (grad(w + e) - grad(w - e)) / (2 * h)
    assert np.abs(W - W.T).max() <= 1e-12 * np.abs(W).max()
    assert np.abs(W - Wfd).max() <= 1e-7 * np.abs(W).max()


# ------------------------------------------------------------- the KKT
def _random_point(make, seed, scale_sig=(0.1, 10.0)):
    lay = model.Layout(make())
    rng = np.random.default_rng(seed)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    lam = rng.standard_normal(lay.nx)
    y = rng.standard_normal(lay.m)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    sw = rng.uniform(*scale_sig, lay.nw)
    ss = rng.uniform(*scale_sig, lay.m)
    r = rng.standard_normal(lay.nw + 2 * lay.m + lay.nx)
    return lay, G, A, W, sw, ss, r


@pytest.mark.parametrize("make,seed", [(gridgen.tiny3, 1), (gridgen.ring30, 2), (gridgen.ring30, 3)])
def test_condensed_step_equals_full_space_ldl(make, seed):
    """Theorems 1 and 2: the condensed route reaches the full-space Newton step."""
    lay, G, A, W, sw, ss, r = _random_point(make, seed)
    d = 0.0
    while True:
        out = kkt.condensed_step(G, A, W, sw, ss, r, lay.nu, delta_w=d)
        if out[-1]:
            break
        d = 1e-2 if d == 0 else d * 8
    Wd = W + sp.diags(np.r_[np.full(lay.nu, d), np.zeros(lay.nx)])
    Kfull = kkt.kaug(G, A, Wd, sw, ss).toarray()
    # full-space step through scipy's Bunch-Kaufman LDL^T: K = L D L^T, L[perm] lower
    import scipy.linalg as sla
    lu, dd, perm = sla.ldl(Kfull)
    tl = lu[perm]
    z = sla.solve_triangular(tl, -r[perm], lower=True, unit_diagonal=True)
    v = np.linalg.solve(dd, z)
    q = sla.solve_triangular(tl.T, v, lower=False, unit_diagonal=True)
    p_ref = np.empty_like(q)
    p_ref[perm] = q
    assert np.abs(Kfull @ p_ref + r).max() <= 1e-9 * np.abs(r).max()
    p = np.concatenate(out[:4])
    assert np.abs(p - p_ref).max() <= 1e-10 * np.abs(p_ref).max()


@pytest.mark.parametrize("make,seed", [(gridgen.tiny3, 1), (gridgen.ring30, 2)])
@pytest.mark.parametrize("delta_c", [1e-3, 0.7])
def test_condensed_step_with_dual_regularization_equals_full_space(make, seed, delta_c):
    """The dual regularisation -delta_c I on the (p_y, p_y) block of K_aug
    (Sec. 4.3, placed on the inequality rows): the condensed route with
    Sigma_t = (Sigma_s^{-1} + delta_c)^{-1} reaches the full-space step of that
    regularised K_aug, solved densely by LU; the step differs from the
    unregularised one, so a dropped delta_c term fails."""
    lay, G, A, W, sw, ss, r = _random_point(make, seed)
    d = 0.0
    while True:
        out = kkt.condensed_step(G, A, W, sw, ss, r, lay.nu, delta_w=d, delta_c=delta_c)
        if out[-1]:
            break
        d = 1e-2 if d == 0 else d * 8
    Wd = W + sp.diags(np.r_[np.full(lay.nu, d), np.zeros(lay.nx)])
    Kfull = kkt.kaug(G, A, Wd, sw, ss, delta_c=delta_c).toarray()
    m = lay.m
    yy = slice(Kfull.shape[0] - m, Kfull.shape[0])
    assert np.array_equal(np.diag(Kfull[yy, yy]), np.full(m, -delta_c))
    p_ref = np.linalg.solve(Kfull, -r)
    p = np.concatenate(out[:4])
    assert np.abs(p - p_ref).max() <= 1e-10 * np.abs(p_ref).max()
    p0 = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, r))
    assert np.abs(p - p0).max() > 1e-6 * np.abs(p0).max()
    # the condensed matrix is Kred by definition with Sigma_t in place of Sigma_s
    Kt = kkt.kred_definition(G, A, Wd, sw, kkt.regularized_sigma(ss, delta_c), lay.nu)
    assert np.abs(out[4] - Kt).max() <= 1e-12 * np.abs(Kt).max()


@pytest.mark.parametrize("delta_c", [0.05, 2.0])
@pytest.mark.parametrize("delta", [0.0, 10.0, 1e3])
def test_inertia_theorem3_with_dual_regularization(delta, delta_c):
    """Theorem 3 with -delta_c I in the (p_y, p_y) block: K_cond (with Sigma_t)
    is positive definite exactly when K_aug has inertia (nx+nu+m, nx+m, 0)."""
    lay, G, A, W, sw, ss, r = _random_point(gridgen.ring30, 11)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    Kr = kkt.kred_definition(G, A, Wd, sw, kkt.regularized_sigma(ss, delta_c), lay.nu)
    pd = np.linalg.eigvalsh(Kr).min() > 0
    inert = kkt.inertia_dense(kkt.kaug(G, A, Wd, sw, ss, delta_c=delta_c))
    assert pd == (inert == (lay.nw + lay.m, lay.nx + lay.m, 0))


def test_regularized_sigma_closed_form():
    """Sigma_t = (Sigma_s^{-1} + delta_c)^{-1}, its limits and its monotonicity."""
    ss = np.array([1e-8, 0.3, 1.0, 7.0, 1e8])
    for dc in (0.0, 1e-6, 0.5, 3.0):
        t = kkt.regularized_sigma(ss, dc)
        np.testing.assert_allclose(t, 1.0 / (1.0 / ss + dc), rtol=1e-15)
        assert np.all(t <= ss)
    assert np.array_equal(kkt.regularized_sigma(ss, 0.0), ss)
    assert abs(kkt.regularized_sigma(np.array([1e12]), 2.0)[0] - 0.5) <= 1e-12


@pytest.mark.parametrize("make,seed", [(gridgen.tiny3, 4), (gridgen.ring30, 5)])
def test_kred_definition_is_symmetric_and_matches_theorem1(make, seed):
    lay, G, A, W, sw, ss, r = _random_point(make, seed)
    Kr = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    assert np.abs(Kr - Kr.T).max() <= 1e-13 * np.abs(Kr).max()
    W_hat, A_hat, _, _, _ = kkt.reduced_blocks(G, A, W, sw, lay.nu)
    Kc = W_hat + np.diag(sw[:lay.nu]) + A_hat.T @ (ss[:, None] * A_hat)
    assert np.abs(Kr - Kc).max() <= 1e-12 * np.abs(Kr).max()


@pytest.mark.parametrize("delta", [0.0, 1.0, 10.0, 100.0, 1e3])
def test_inertia_theorem3(delta):
    """K_cond positive definite <=> inertia(K_aug) = (nx+nu+m, nx+m, 0)."""
    lay, G, A, W, sw, ss, r = _random_point(gridgen.ring30, 11)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    Kr = kkt.kred_definition(G, A, Wd, sw, ss, lay.nu)
    pd = np.linalg.eigvalsh(Kr).min() > 0
    inert = kkt.inertia_dense(kkt.kaug(G, A, Wd, sw, ss))
    assert pd == (inert == (lay.nw + lay.m, lay.nx + lay.m, 0))


def test_inertia_both_outcomes_occur():
    lay, G, A, W, sw, ss, r = _random_point(gridgen.ring30, 11)
    outs = set()
    for delta in (0.0, 1e3):
        Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
        outs.add(bool(np.linalg.eigvalsh(kkt.kred_definition(G, A, Wd, sw, ss, lay.nu)).min() > 0))
    assert outs == {True, False}


# ------------------------------------------------------------- the IPM
def _economic_dispatch(net):
    """min sum c2 P^2 + c1 P  s.t. sum P = sum Pd, Pmin <= P <= Pmax, by bisection
    on the marginal price."""
    def total(lmb):
        return np.clip((lmb - net.c1) / (2 * net.c2), net.Pmin, net.Pmax).sum()
    lo, hi = 0.0, 1e4
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if total(mid) < net.Pd.sum() else (lo, mid)
    P = np.clip((0.5 * (lo + hi) - net.c1) / (2 * net.c2), net.Pmin, net.Pmax)
    return float(np.sum(net.c2 * P * P + net.c1 * P))


@pytest.mark.parametrize("variant", ["linred", "redlin"])
def test_lossless_network_is_economic_dispatch(variant):
    # Losses vanish for every voltage profile, so the optimal voltages form a
    # continuum and the reduced Hessian is singular along it: near mu = 1e-9 the
    # infeasible-path variant can stall just above 1e-8 on the voltage continuum.
    # The objective, which the continuum does not move, is what is pinned.
    net = gridgen.lossless(gridgen.ring30())
    res = getattr(ipm, variant)(net, max_iter=60)
    assert res.err <= 1e-6
    ed = _economic_dispatch(net)
    assert abs(res.obj - ed) <= 1e-8 * abs(ed)


def test_tiny3_matches_independent_optimizer():
    net = gridgen.tiny3()
    lay = model.Layout(net)
    res = ipm.linred(net)
    assert res.status == "converged"
    cons = [dict(type="eq", fun=lambda v: model.cons_g(lay, v)),
            dict(type="ineq", fun=lambda v: lay.hu[np.isfinite(lay.hu)] - model.cons_h(lay, v)[np.isfinite(lay.hu)]),
            dict(type="ineq", fun=lambda v: model.cons_h(lay, v)[np.isfinite(lay.hl)] - lay.hl[np.isfinite(lay.hl)])]
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lay.wl, lay.wu)]
    best = np.inf
    rng = np.random.default_rng(0)
    for k in range(4):
        w0 = lay.flat_start() + (0 if k == 0 else 0.02 * rng.standard_normal(lay.nw))
        out = so.minimize(lambda v: model.objective(lay, v), w0, method="SLSQP", bounds=bounds,
                          constraints=cons, options=dict(ftol=1e-14, maxiter=500))
        if out.success and np.abs(model.cons_g(lay, out.x)).max() < 1e-9:
            best = min(best, out.fun)
    assert np.isfinite(best)
    assert abs(res.obj - best) <= 1e-6 * abs(best)


def test_variants_agree_and_power_balance_holds():
    net = gridgen.ring30()
    lay = model.Layout(net)
    a = ipm.linred(net)
    b = ipm.redlin(net)
    assert a.status == b.status == "converged"
    assert abs(a.obj - b.obj) <= 1e-8 * abs(a.obj)
    assert np.abs(model.cons_g(lay, a.w)).max() <= 1e-8
    assert np.abs(model.cons_g(lay, b.w)).max() <= 1e-10


def test_reduced_derivatives_through_projection():
    """Reduced-derivative theorem (Sec. 2.3): grad f_r and W_hat_uu against
    finite differences of f_r and of grad_u L_r through the Newton projection."""
    import scipy.sparse.linalg as spla
    net = gridgen.ring30()
    lay = model.Layout(net)
    nu = lay.nu
    w, _, ok = ipm.newton_projection(lay, lay.flat_start())
    assert ok
    rng = np.random.default_rng(9)
    y = rng.uniform(-1, 1, lay.m)

    def reduced(u):
        wt = w.copy()
        wt[:nu] = u
        wt, _, okp = ipm.newton_projection(lay, wt, tol=1e-14)
        assert okp
        gf, G, A = model.jacobians(lay, wt)
        Gx = G[:, nu:].tocsc()
        lam = -spla.splu(Gx).solve(gf[nu:] + A[:, nu:].T @ y, trans="T")
        grad = gf[:nu] + G[:, :nu].T @ lam + A[:, :nu].T @ y
        return wt, lam, grad, gf, G, A
    u0 = w[:nu].copy()
    wt, lam, grad0, gf, G, A = reduced(u0)
    W = model.lagrangian_hessian(lay, wt, lam, y)
    W_hat, _, _, _, _ = kkt.reduced_blocks(G, A, W, np.zeros(lay.nw), nu)
    Hfd = np.zeros((nu, nu))
    gfr_fd = np.zeros(nu)
    h = 1e-6
    for j in range(nu):
        e = np.zeros(nu)
        e[j] = h
        Hfd[:, j] = (reduced(u0 + e)[2] - reduced(u0 - e)[2]) / (2 * h)
        fp = model.objective(lay, reduced(u0 + e)[0])
        fm = model.objective(lay, reduced(u0 - e)[0])
        gfr_fd[j] = (fp - fm) / (2 * h)
    gfr, lam_f = kkt.reduced_gradient(G, gf, nu)
    assert np.abs(gfr - gfr_fd).max() <= 1e-6 * np.abs(gfr).max()
    # its adjoint is the multiplier that makes the state block of grad f + G^T lam vanish
    assert np.abs(gf[nu:] + G[:, nu:].T @ lam_f).max() <= 1e-12 * np.abs(gf[nu:]).max()
    # the same call on grad_w L reproduces the projection's reduced Lagrangian gradient
    gl, lam_l = kkt.reduced_gradient(G, gf + A.T @ y, nu)
    assert np.abs(gl - grad0).max() <= 1e-10 * np.abs(gl).max()
    assert np.abs(lam_l - lam).max() <= 1e-10 * np.abs(lam).max()
    assert np.abs(W_hat - Hfd).max() <= 1e-5 * np.abs(W_hat).max()


# ------------------------------------------------------------- the filter
def test_filter_rules():
    """The filter's dominance test and the acceptance rules of the filter line
    search (Wachter and Biegler 2006, Sec. 2.3), on hand-made values."""
    F = ipm.Filter(10.0)
    assert not F.acceptable(10.0, -1e30) and F.acceptable(9.9, 1e30)   # the initial half-plane
    F.add(5.0, 3.0)
    assert not F.acceptable(6.0, 4.0) and not F.acceptable(5.0, 3.0)   # dominated, boundary included
    assert F.acceptable(6.0, 2.9) and F.acceptable(4.9, 100.0)
    G = ipm.Filter(1e4)
    # no switching (dphi >= 0): sufficient decrease in theta or in phi
    assert ipm.filter_accepts(G, 1.0, 0.0, 0.5, 1.0, 1.0 - 2e-5, 1.0, 1e-4) == (True, False)
    assert ipm.filter_accepts(G, 1.0, 0.0, 0.5, 1.0, 1.0, -2e-8, 1e-4) == (True, False)
    assert ipm.filter_accepts(G, 1.0, 0.0, 0.5, 1.0, 1.0, 0.0, 1e-4) == (False, False)
    # switching (alpha (-dphi)^2.3 > theta^1.1) with theta <= theta_min: Armijo on phi only
    th = 1e-6
    assert ipm.filter_accepts(G, th, 0.0, -1.0, 1.0, th, -1e-4 * 0.99, 1e-4) == (False, True)
    assert ipm.filter_accepts(G, th, 0.0, -1.0, 1.0, th, -1e-4 * 1.01, 1e-4) == (True, True)
    # alpha_min: gamma_alpha gamma_theta without a descent direction
    assert abs(ipm.filter_alpha_min(1.0, 0.5, 1e-4) - 0.05 * 1e-5) <= 1e-20


def _counted_loads(net, scale):
    n = net.copy()
    n.Pd, n.Qd = scale * net.Pd, scale * net.Qd
    return n


@pytest.mark.parametrize("case", ["tiny3", "ring30", "lossless", "tiny3_loaded"])
def test_filter_line_search_reaches_the_pinned_optima(case):
    """The filter variant of the loop reaches the optimum the merit variant is
    pinned to: the same objective on tiny3 and ring30 (KKT tolerance 1e-8),
    the economic-dispatch closed form on the lossless network, and on tiny3
    with loads scaled by 1.3 -- a case whose first trial step raises the
    constraint violation -- through an accepted second-order correction."""
    if case == "lossless":
        net = gridgen.lossless(gridgen.ring30())
        res = ipm.linred(net, line_search="filter", max_iter=80)
        assert res.err <= 1e-6
        ed = _economic_dispatch(net)
        assert abs(res.obj - ed) <= 1e-8 * abs(ed)
        return
    net = _counted_loads(gridgen.tiny3(), 1.3) if case == "tiny3_loaded" else getattr(gridgen, case)()
    res = ipm.linred(net, line_search="filter")
    ref = ipm.linred(net)
    assert res.status == ref.status == "converged"
    assert abs(res.obj - ref.obj) <= 1e-8 * abs(ref.obj)
    lay = model.Layout(net)
    assert np.abs(model.cons_g(lay, res.w)).max() <= 1e-8
    if case == "tiny3_loaded":
        assert res.soc_steps >= 1


# ------------------------------------------------- feasibility restoration
def _scaled_loads(net, f):
    import dataclasses
    return dataclasses.replace(net, Pd=net.Pd * f, Qd=net.Qd * f)


def test_per_row_dual_regularisation_matches_kaug():
    """The restoration phase relaxes each inequality row with its own dual
    regularisation delta_i: the condensed step with Sigma_t,i = (Sigma_s,i^{-1}
    + delta_i)^{-1} against the sparse solve of K_aug with -diag(delta) in its
    (p_y, p_y) block."""
    net = gridgen.ring30()
    lay = model.Layout(net)
    rng = np.random.default_rng(77)
    w = lay.flat_start() + 0.02 * rng.standard_normal(lay.nw)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, rng.standard_normal(lay.nx), rng.standard_normal(lay.m))
    sw, ss = rng.uniform(0.5, 5.0, lay.nw), rng.uniform(0.5, 5.0, lay.m)
    dc = rng.uniform(1e-3, 2.0, lay.m)
    r = rng.standard_normal(lay.nw + 2 * lay.m + lay.nx)
    Kc0 = kkt.kred_definition(G, A, W, sw, kkt.regularized_sigma(ss, dc), lay.nu)
    dw = max(0.0, -np.linalg.eigvalsh(0.5 * (Kc0 + Kc0.T))[0]) + 1.0
    pw, ps, pl, py, _, ok = kkt.condensed_step(G, A, W, sw, ss, r, lay.nu, delta_w=dw, delta_c=dc)
    assert ok
    Wd = W + sp.diags(np.r_[np.full(lay.nu, dw), np.zeros(lay.nx)])
    ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, r, delta_c=dc))
    got = np.concatenate([pw, ps, pl, py])
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("make", [gridgen.tiny3, gridgen.ring30])
def test_restoration_from_the_start_reaches_the_same_optimum(make):
    """Ipopt's start-with-restoration: the restoration phase runs from the flat
    start, hands an acceptable point back, and the loop converges to the
    optimum of the plain filter solve."""
    net = make()
    a = ipm.linred(net, line_search="filter")
    b = ipm.linred(net, line_search="filter", restoration=True, start_with_resto=True)
    assert a.status == b.status == "converged"
    assert b.restorations == 1
    assert abs(a.obj - b.obj) <= 1e-8 * abs(a.obj)


def test_restoration_endpoint_is_acceptable():
    """The restoration phase returns a point whose violation of [g; h + s] is at
    most 0.9 of the starting one and that the original filter (holding the
    starting point) accepts; the bound multipliers are positive."""
    net = gridgen.ring30()
    lay = model.Layout(net)
    bw = ipm._Bounds(lay.wl, lay.wu)
    bs = ipm._Bounds(-lay.hu, -lay.hl)
    w = ipm._push(lay.flat_start(), lay.wl, lay.wu)
    s = ipm._push(-model.cons_h(lay, w), bs.lo, bs.hi)
    mu = 0.1

    def theta_phi(wt, st):
        c = np.concatenate([model.cons_g(lay, wt), model.cons_h(lay, wt) + st])
        return np.abs(c).sum(), model.objective(lay, wt) + bw.barrier(wt, mu) + bs.barrier(st, mu)
    t0, p0 = theta_phi(w, s)
    filt = ipm.Filter(1e4 * max(1.0, t0))
    filt.add(t0, p0)
    w2, s2, lam, y, zwl, zwu, zsl, zsu = ipm._restoration(lay, bw, bs, filt, w, s, mu, 1e-8, {})
    t1, p1 = theta_phi(w2, s2)
    assert t1 <= ipm.KAPPA_RESTO * t0 and filt.acceptable(t1, p1)
    assert (zwl[bw.fl] > 0).all() and (zwu[bw.fu] > 0).all() and (zsl[bs.fl] > 0).all()
    assert np.all(w2 >= lay.wl) and np.all(w2 <= lay.wu)


def test_restoration_fails_on_an_infeasible_case():
    """Loads of 1.7 x the 3-bus case exceed its generation capacity (total Pmax
    2.0 against 2.04 of load; losses are nonnegative), so no feasible point
    exists: the restoration phase cannot return one and the solve fails."""
    net = _scaled_loads(gridgen.tiny3(), 1.7)
    assert net.Pmax.sum() < net.Pd.sum()
    with pytest.raises(RuntimeError, match="restoration failed"):
        ipm.linred(net, line_search="filter", restoration=True)
