"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: model values and derivatives to 1e-12 normwise relative (same
closed-form expressions, different summation order); G_x solves to 1e-10;
the condensed matrix Kred and the Newton step to 1e-9 normwise relative (max
norm), the bar the method is held to; integer outputs (failing pivot column)
exactly."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import gridgen
from oracle import ipm, kkt, model

from gpu_cases import oracle_iterate, random_point, rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL_MODEL = 1e-12
TOL_SOLVE = 1e-10
TOL_KRED = 1e-9


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


def csr(h, which, vals):
    nr, nc, rp, ci = h.get_csr_pattern(which)
    return sp.csr_matrix((N(vals), ci, rp), shape=(nr, nc))


def gpu_eval(pkg, h, lay, w, lam=None, y=None):
    u, x = T(w[:lay.nu]), T(w[lay.nu:])
    h.eval_derivatives(x, u, None if lam is None else T(lam), None if y is None else T(y))
    return u, x


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_model_values_and_derivatives(pkg, name):
    net, lay, w, lam, y, _, _ = random_point(name, seed=1)
    h = pkg.Handle(net)
    gpu_eval(pkg, h, lay, w, lam, y)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(lay.nx, dtype=torch.float64, device="cuda")
    hv = torch.zeros(lay.m, dtype=torch.float64, device="cuda")
    gf = torch.zeros(lay.nw, dtype=torch.float64, device="cuda")
    h.get_vector(pkg.OPF_VEC_F, f)
    h.get_vector(pkg.OPF_VEC_G, g)
    h.get_vector(pkg.OPF_VEC_H, hv)
    h.get_vector(pkg.OPF_VEC_GRADF, gf)
    assert rel_err(N(f), [model.objective(lay, w)]) <= TOL_MODEL
    assert rel_err(N(g), model.cons_g(lay, w)) <= TOL_MODEL
    assert rel_err(N(hv), model.cons_h(lay, w)) <= TOL_MODEL
    gf_o, G_o, A_o = model.jacobians(lay, w)
    assert rel_err(N(gf), gf_o) <= TOL_MODEL
    vals = {}
    for which, ref in [(pkg.OPF_MAT_G, G_o), (pkg.OPF_MAT_A, A_o),
                       (pkg.OPF_MAT_W, model.lagrangian_hessian(lay, w, lam, y))]:
        nr, nc, rp, ci = h.get_csr_pattern(which)
        v = torch.zeros(max(1, len(ci)), dtype=torch.float64, device="cuda")
        h.get_csr_values(which, v)
        M = sp.csr_matrix((N(v)[:len(ci)], ci, rp), shape=(nr, nc)).toarray()
        assert rel_err(M, ref.toarray()) <= TOL_MODEL, which
        vals[which] = M
    # the Hessian is symmetric as stored
    assert np.abs(vals[pkg.OPF_MAT_W] - vals[pkg.OPF_MAT_W].T).max() <= 1e-13 * np.abs(vals[pkg.OPF_MAT_W]).max()


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
@pytest.mark.parametrize("rhs1", [0, 1, 64, 65, 66])
def test_gx_factor_and_solves(pkg, name, rhs1):
    """rhs1 = the one-right-hand-side kernel (0: staged until an autotune ran)."""
    net, lay, w, lam, y, _, _ = random_point(name, seed=2)
    h = pkg.Handle(net, rhs1_kernel=rhs1)
    gpu_eval(pkg, h, lay, w)
    h.gx_factor()
    _, G, _ = model.jacobians(lay, w)
    Gx = G[:, lay.nu:].tocsc()
    lu = spla.splu(Gx)
    rng = np.random.default_rng(3)
    for nrhs in (1, 3):
        B = rng.standard_normal((nrhs, lay.nx))
        for trans in (0, 1):
            X = torch.zeros(nrhs * lay.nx, dtype=torch.float64, device="cuda")
            h.gx_solve(trans, T(B.ravel()), X, nrhs)
            ref = np.stack([lu.solve(b, trans="T" if trans else "N") for b in B])
            assert rel_err(N(X).reshape(nrhs, lay.nx), ref) <= TOL_SOLVE


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
@pytest.mark.parametrize("route", [0, 1])
def test_condense_at_oracle_iterate(pkg, name, route):
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    h = pkg.Handle(net, route=route)
    w, lam, y = rec["w"], rec["lam"], rec["y"]
    gpu_eval(pkg, h, lay, w, lam, y)
    sw, ss = rec["sig_w"], rec["sig_s"]
    Kred = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss), Kred)
    Kg = N(Kred).reshape(lay.nu, lay.nu)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    assert np.array_equal(Kg, Kg.T)
    assert rel_err(Kg, Ko) <= TOL_KRED


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_route_autotune(pkg, name):
    """OPF_ROUTE_AUTO times the explicit and the adjoint route on the first
    condensation and keeps the faster; Kred and the step are right on the
    tuning call and on the next one with the pick."""
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    h = pkg.Handle(net, route=pkg.OPF_ROUTE_AUTO)
    assert h.route_choice()[0] == -1
    _, G, A = model.jacobians(lay, rec["w"])
    W = model.lagrangian_hessian(lay, rec["w"], rec["lam"], rec["y"])
    sw, ss, delta = rec["sig_w"], rec["sig_s"], rec["delta"]
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, rec["r"]))
    for call in range(2):
        gpu_eval(pkg, h, lay, rec["w"], rec["lam"], rec["y"])
        K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
        h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss), K)
        route, ms = h.route_choice()
        assert route in (0, 1) and ms["adjoint"] > 0 and ms["explicit"] > 0
        assert rel_err(N(K).reshape(lay.nu, lay.nu), Ko) <= TOL_KRED
        assert h.kkt_factor(delta) == -1
        step = torch.zeros(len(rec["r"]), dtype=torch.float64, device="cuda")
        h.kkt_solve(T(rec["r"]), step)
        assert rel_err(N(step), ref) <= TOL_KRED, call


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_rhs_block_and_route_invariance(pkg, name):
    """Kred does not depend on the multi-RHS solve kernel (staged with 1, 2, 4
    columns per CTA, column-parallel, level-blocked with a group barrier or on
    thread-block clusters, and its dataflow form; ragged
    column tails included: nu = 11, 399) nor on the route (explicit S^T H vs
    adjoint-adjoint).  The substitution kernels agree to 1e-12; the level-blocked
    kernels multiply by explicit inverses of the diagonal blocks, a different
    rounding, and are held to 1e-10 against them."""
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    outs = []
    for route in (0, 1):
        for cb in (1, 2, 4, 32, 64, 96, 128):
            h = pkg.Handle(net, route=route, rhs_block=cb)
            gpu_eval(pkg, h, lay, rec["w"], rec["lam"], rec["y"])
            K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
            h.condense(T(rec["sig_w"][:lay.nu]), T(rec["sig_w"][lay.nu:]), T(rec["sig_s"]), K)
            outs.append((cb, N(K)))
    ref = outs[0][1]
    for cb, o in outs[1:]:
        assert rel_err(o, ref) <= (1e-10 if cb in (64, 96, 128) else 1e-12), cb


def _first_failing_column(M):
    """Column at which the plain (unblocked, column-by-column) Cholesky meets a
    non-positive pivot, or -1."""
    A = np.array(M, dtype=np.float64)
    n = A.shape[0]
    for j in range(n):
        d = A[j, j] - A[j, :j] @ A[j, :j]
        if not d > 0:
            return j
        A[j, j] = np.sqrt(d)
        A[j + 1:, j] = (A[j + 1:, j] - A[j + 1:, :j] @ A[j, :j]) / A[j, j]
    return -1


@pytest.mark.parametrize("chol_form", [1, 2])
@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_kkt_factor_and_solve_match_full_space_step(pkg, name, chol_form):
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    h = pkg.Handle(net, chol_form=chol_form)
    w, lam, y = rec["w"], rec["lam"], rec["y"]
    gpu_eval(pkg, h, lay, w, lam, y)
    sw, ss, delta = rec["sig_w"], rec["sig_s"], rec["delta"]
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    assert h.kkt_factor(delta) == -1
    assert h.chol_choice()[0] == chol_form
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.get_factor(F)
    F = N(F).reshape(lay.nu, lay.nu)
    assert np.array_equal(F, np.tril(F))
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu) + delta * np.eye(lay.nu)
    assert rel_err(F @ F.T, Ko) <= TOL_KRED
    rng = np.random.default_rng(4)
    R = np.stack([rec["r"], rng.standard_normal(len(rec["r"])), -rec["r"]])
    step = torch.zeros(R.size, dtype=torch.float64, device="cuda")
    h.kkt_solve(T(R.ravel()), step, 3)
    step = N(step).reshape(3, -1)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    for k in range(3):
        ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, R[k]))
        assert rel_err(step[k], ref) <= TOL_KRED, k
    adj = torch.zeros(R.size, dtype=torch.float64, device="cuda")
    h.kkt_solve_adjoint(T(R.ravel()), adj, 3)
    assert rel_err(N(adj).reshape(3, -1), step) <= 1e-12


# (network, seed, multiplier scale): scaling lam and y makes W, hence Kred,
# indefinite; the grid2000 cases fail in tile columns 5 and 1 of the blocked
# factorisation (columns 169 and 47, pivots far from zero), the ring30 case in
# its first tile
@pytest.mark.parametrize("name,seed,scale", [("ring30", 11, 1.0), ("grid2000", 11, 3.0), ("grid2000", 11, 10.0)])
@pytest.mark.parametrize("chol_form", [1, 2])
def test_kkt_factor_reports_not_pd(pkg, name, seed, scale, chol_form):
    """An indefinite condensed matrix is reported with its failing column; a large
    enough delta_w then succeeds (the inertia-correction loop of Sec. 4.3)."""
    net, lay, w, lam, y, sw, ss = random_point(name, seed=seed)
    lam, y = scale * lam, scale * y
    h = pkg.Handle(net, chol_form=chol_form)
    gpu_eval(pkg, h, lay, w, lam, y)
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    S = 0.5 * (Ko + Ko.T)
    want = _first_failing_column(S)
    assert want >= 0
    assert h.kkt_factor(0.0) == want
    # an aborted factorisation does not tune the grid (its timings would be of a
    # partial factorisation); the forced form still ran.  With one tile (nu <= 32)
    # there is no grid to choose and nothing is timed.
    if lay.nu > 32:
        assert h.chol_choice()[0] == 0
    big = 2.0 * abs(np.linalg.eigvalsh(S)[0]) + 1.0
    assert h.kkt_factor(big) == -1
    assert h.chol_choice()[0] == chol_form
    # and the factor of the shifted matrix is right after the aborted one
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.get_factor(F)
    F = N(F).reshape(lay.nu, lay.nu)
    assert rel_err(F @ F.T, S + big * np.eye(lay.nu)) <= TOL_KRED


@pytest.mark.parametrize("route", [0, 1])
@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_dual_regularization_matches_full_space_step(pkg, name, route):
    """delta_c on the inequality rows (-delta_c I in the (p_y, p_y) block of
    K_aug, Sec. 4.3): the factor is that of Kred with (Sigma_s^{-1} +
    delta_c)^{-1} in place of Sigma_s, the step is the full-space step of the
    regularised K_aug, and delta_c = 0 afterwards gives back the plain factor."""
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    h = pkg.Handle(net, route=route)
    w, lam, y = rec["w"], rec["lam"], rec["y"]
    gpu_eval(pkg, h, lay, w, lam, y)
    sw, ss, delta = rec["sig_w"], rec["sig_s"], rec["delta"]
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(21)
    R = np.stack([rec["r"], rng.standard_normal(len(rec["r"]))])
    for dc in (0.3, 1e-3, 0.0):
        assert h.kkt_factor(delta, dc) == -1
        h.get_factor(F)
        Fm = N(F).reshape(lay.nu, lay.nu)
        Kt = kkt.kred_definition(G, A, W, sw, kkt.regularized_sigma(ss, dc), lay.nu) + delta * np.eye(lay.nu)
        assert rel_err(Fm @ Fm.T, Kt) <= TOL_KRED, dc
        step = torch.zeros(R.size, dtype=torch.float64, device="cuda")
        h.kkt_solve(T(R.ravel()), step, 2)
        step = N(step).reshape(2, -1)
        for k in range(2):
            ref = np.concatenate(kkt.full_space_step(G, A, Wd, sw, ss, R[k], delta_c=dc))
            assert rel_err(step[k], ref) <= TOL_KRED, (dc, k)
    with pytest.raises(pkg.OPFError):
        h.kkt_factor(delta, -1.0)


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_reduced_gradient_matches_oracle(pkg, name):
    """Eq. reduced:derivatives: grad f_r and the adjoint lam, from the handle's
    grad f and from a caller's gradient (here grad_w of f + y^T h)."""
    net, lay, w, lam, y, _, _ = random_point(name, seed=8)
    h = pkg.Handle(net)
    gpu_eval(pkg, h, lay, w)
    with pytest.raises(pkg.OPFError):
        h.reduced_gradient(None, torch.zeros(lay.nu, dtype=torch.float64, device="cuda"))
    h.gx_factor()
    gf, G, A = model.jacobians(lay, w)
    gr = torch.zeros(lay.nu, dtype=torch.float64, device="cuda")
    lm = torch.zeros(lay.nx, dtype=torch.float64, device="cuda")
    h.reduced_gradient(None, gr, lm)
    ref, lref = kkt.reduced_gradient(G, gf, lay.nu)
    assert rel_err(N(gr), ref) <= TOL_SOLVE
    assert rel_err(N(lm), lref) <= TOL_SOLVE
    gl = gf + A.T @ y
    h.reduced_gradient(T(gl), gr)
    ref, _ = kkt.reduced_gradient(G, gl, lay.nu)
    assert rel_err(N(gr), ref) <= TOL_SOLVE


def test_indefinite_first_factorisation_leaves_the_cholesky_untuned(pkg):
    """The Cholesky autotuner times complete factorisations only: a first call on
    an indefinite Kred reports NOT_PD and leaves the handle untuned (form 0, no
    timings), and the first positive definite factorisation tunes it."""
    net, lay, w, lam, y, sw, ss = random_point("grid2000", seed=11)
    lam, y = 3.0 * lam, 3.0 * y
    h = pkg.Handle(net)
    gpu_eval(pkg, h, lay, w, lam, y)
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss))
    assert h.kkt_factor(0.0) >= 0
    form, _, ms = h.chol_choice()
    assert form == 0 and all(v == 0 for v in ms.values())
    _, G, A = model.jacobians(lay, w)
    Ko = kkt.kred_definition(G, A, model.lagrangian_hessian(lay, w, lam, y), sw, ss, lay.nu)
    big = 2.0 * abs(np.linalg.eigvalsh(0.5 * (Ko + Ko.T))[0]) + 1.0
    assert h.kkt_factor(big) == -1
    form, _, ms = h.chol_choice()
    assert form in (1, 2) and any(v > 0 for v in ms.values())


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_powerflow_matches_oracle_projection(pkg, name):
    net = gridgen.WORKLOADS[name]()
    lay = model.Layout(net)
    w0 = ipm._push(lay.flat_start(), lay.wl, lay.wu)
    wo, _, ok = ipm.newton_projection(lay, w0)
    assert ok
    h = pkg.Handle(net)
    x = T(w0[lay.nu:])
    h.powerflow(T(w0[:lay.nu]), x, tol=1e-10, max_iter=30)
    assert np.abs(model.cons_g(lay, np.r_[w0[:lay.nu], N(x)])).max() <= 1e-10
    assert rel_err(N(x), wo[lay.nu:]) <= 1e-9


def test_full_size_grid10k_sampled_columns(pkg):
    """The 10,000-bus workload in the launch configuration the benchmark times:
    sampled columns of Kred against the oracle, each column from two sparse
    solves, K z_a = K [e_a; S_x e_a] and Z^T (K z_a)."""
    net, lay, w, lam, y, sw, ss = random_point("grid10k", seed=5)
    h = pkg.Handle(net)
    gpu_eval(pkg, h, lay, w, lam, y)
    Kred = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(ss), Kred)
    Kg = N(Kred).reshape(lay.nu, lay.nu)
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    K = (W + sp.diags(sw) + A.T @ sp.diags(ss) @ A).tocsr()
    Gu, Gx = G[:, :lay.nu].tocsc(), G[:, lay.nu:].tocsc()
    lu = spla.splu(Gx)
    rng = np.random.default_rng(6)
    cols = sorted({0, lay.nu - 1, *rng.choice(lay.nu, 6, replace=False).tolist()})
    for a in cols:
        z = np.zeros(lay.nw)
        z[a] = 1.0
        z[lay.nu:] = -lu.solve(Gu[:, a].toarray().ravel())
        Kz = K @ z
        col = Kz[:lay.nu] - Gu.T @ lu.solve(Kz[lay.nu:], trans="T")
        assert rel_err(Kg[:, a], col) <= TOL_KRED, a
    assert np.array_equal(Kg, Kg.T)
