"""Full-size parity on the 10,000-bus workload (nu = 1,999, nx = 18,999) in the
launch configuration the benchmark times: autotuned solve kernels, the
Cholesky forms at their tuned grids (the 32 x 32 full-tile update mode of the
dataflow form runs here, not at 2,000 buses), the 63-tile-step solves with the
dense factor and the one-vector G_x solves of the step recovery.

The point is the oracle's own LinRed iterate at iteration 3, stored by
tests/golden/make_grid10k_iterate.py (oracle only).  Expected values come from
the oracle's definitions at that point: Kred = Z^T K Z with Z = [I; -G_x^{-1}
G_u] (Eq. algo:reduction), the plain-definition Cholesky failing column
(LAPACK dpotrf's leading-minor test, checked to be a clearly negative pivot),
and the full-space Newton step from a sparse LU of K_aug (Theorems 1-2).  The
step is compared with no iterative refinement in the path.  Tolerance: the
1e-9 relative bar of Kred and the Newton step; integer outputs exactly."""
import functools
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.linalg.lapack as lapack
import scipy.sparse as sp

import gridgen
from oracle import kkt, model

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
    binding.load_library()
    return binding


@functools.lru_cache(maxsize=None)
def point():
    """(net, layout, iterate dict, G, A, W, oracle Kred) at the stored iterate."""
    d = dict(np.load(GOLDEN))
    net = gridgen.grid10k()
    lay = model.Layout(net)
    _, G, A = model.jacobians(lay, d["w"])
    W = model.lagrangian_hessian(lay, d["w"], d["lam"], d["y"])
    Ko = kkt.kred_definition(G, A, W, d["sig_w"], d["sig_s"], lay.nu)
    return net, lay, d, G, A, W, Ko


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


def condensed_handle(pkg, **opts):
    net, lay, d, _, _, _, _ = point()
    h = pkg.Handle(net, **opts)
    w = d["w"]
    h.eval_derivatives(T(w[lay.nu:]), T(w[:lay.nu]), T(d["lam"]), T(d["y"]))
    K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    sw = d["sig_w"]
    h.condense(T(sw[:lay.nu]), T(sw[lay.nu:]), T(d["sig_s"]), K)
    return h, N(K).reshape(lay.nu, lay.nu)


def oracle_failing_column(M):
    """First column whose Cholesky pivot is not positive (LAPACK's leading-minor
    test) and that pivot, recomputed from the leading factor."""
    c, info = lapack.dpotrf(M, lower=1, clean=1)
    if info == 0:
        return -1, None
    j = info - 1
    v = sla.solve_triangular(np.tril(c[:j, :j]), M[:j, j], lower=True) if j else np.zeros(0)
    return j, M[j, j] - v @ v


@pytest.mark.parametrize("route", [0, 1])
def test_grid10k_kred_at_oracle_iterate(pkg, route):
    """The whole 1,999 x 1,999 Kred, both routes, against Z^T K Z."""
    *_, Ko = point()
    h, Kg = condensed_handle(pkg, route=route)
    assert np.array_equal(Kg, Kg.T)
    assert rel_err(Kg, Ko) <= TOL
    if route == 0:
        kern, _, _ = h.trsm_choice()
        assert kern in (1, 2, 4, 32, 64, 96)


@pytest.mark.parametrize("chol_form", [1, 2])
def test_grid10k_factor_and_step_match_full_space(pkg, chol_form):
    """F F^T = Kred + delta I at the iterate's own delta, then three right-hand
    sides through opf_kkt_solve (no refinement) against the sparse full-space
    solve of K_aug."""
    net, lay, d, G, A, W, Ko = point()
    h, _ = condensed_handle(pkg, chol_form=chol_form)
    delta = float(d["delta"])
    assert h.kkt_factor(delta) == -1
    form, grid, _ = h.chol_choice()
    assert form == chol_form
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.get_factor(F)
    F = N(F).reshape(lay.nu, lay.nu)
    assert np.array_equal(F, np.tril(F))
    S = 0.5 * (Ko + Ko.T) + delta * np.eye(lay.nu)
    assert rel_err(F @ F.T, S) <= TOL
    rng = np.random.default_rng(12)
    R = np.stack([d["r"], rng.standard_normal(len(d["r"])), -d["r"]])
    step = torch.zeros(R.size, dtype=torch.float64, device="cuda")
    h.kkt_solve(T(R.ravel()), step, 3)
    step = N(step).reshape(3, -1)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    for k in range(3):
        ref = np.concatenate(kkt.full_space_step(G, A, Wd, d["sig_w"], d["sig_s"], R[k]))
        assert rel_err(step[k], ref) <= TOL, k
    # one right-hand side takes the one-vector kernels (cluster solves)
    one = torch.zeros(R.shape[1], dtype=torch.float64, device="cuda")
    h.kkt_solve(T(R[0]), one, 1)
    assert rel_err(N(one), step[0]) <= TOL


@pytest.mark.parametrize("chol_form", [1, 2])
def test_grid10k_not_pd_past_tile_column_20(pkg, chol_form):
    """Without enough primal regularisation the 1,999-column Kred is indefinite:
    the failing column is reported exactly, for failures in tile columns 33, 39
    and 52 of 63, and the factor of the corrected matrix is right afterwards."""
    net, lay, d, G, A, W, Ko = point()
    h, _ = condensed_handle(pkg, chol_form=chol_form)
    S = 0.5 * (Ko + Ko.T)
    for delta in (0.0, 10.0, 30.0):
        want, piv = oracle_failing_column(S + delta * np.eye(lay.nu))
        assert want >= 20 * 32 and piv < -1e-4 * S[want, want]
        assert h.kkt_factor(delta) == want, delta
    delta = float(d["delta"])
    assert h.kkt_factor(delta) == -1
    assert h.chol_choice()[0] == chol_form
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.get_factor(F)
    F = N(F).reshape(lay.nu, lay.nu)
    assert rel_err(F @ F.T, S + delta * np.eye(lay.nu)) <= TOL


def test_grid10k_dual_regularization(pkg):
    """delta_c on the inequality rows at full size: Kred with
    (Sigma_s^{-1} + delta_c)^{-1} and the step of K_aug with -delta_c I in its
    (p_y, p_y) block."""
    net, lay, d, G, A, W, _ = point()
    h, _ = condensed_handle(pkg)
    delta, dc = float(d["delta"]), 1e-2
    assert h.kkt_factor(delta, dc) == -1
    F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.get_factor(F)
    F = N(F).reshape(lay.nu, lay.nu)
    Kt = kkt.kred_definition(G, A, W, d["sig_w"], kkt.regularized_sigma(d["sig_s"], dc), lay.nu)
    assert rel_err(F @ F.T, 0.5 * (Kt + Kt.T) + delta * np.eye(lay.nu)) <= TOL
    step = torch.zeros(len(d["r"]), dtype=torch.float64, device="cuda")
    h.kkt_solve(T(d["r"]), step, 1)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, delta), np.zeros(lay.nx)])
    ref = np.concatenate(kkt.full_space_step(G, A, Wd, d["sig_w"], d["sig_s"], d["r"], delta_c=dc))
    assert rel_err(N(step), ref) <= TOL
