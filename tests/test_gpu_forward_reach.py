"""The condensation's forward sweep L Y = P G_u with the reach lists (Sec.
3.3's multi-RHS solve, passing by the rows of Y that are exactly zero): Kred
and the Newton step equal those of the sweep over every row (dense_forward=1)
to the last bit, and match the oracle, on the level-blocked kernel with a group
barrier (rhs_block=64) and on thread-block clusters (128), in one pass and in
column chunks of N (the chunks' 32-column blocks offset into G_u's), with the
condensed right-hand side's column riding along (a dense column, solved in
full), on a ragged column tail (nu = 399) and at the stored grid10k iterate."""
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
    return dict(lay=lay, w=w, lam=lam, y=y, sw=sw, ss=ss, r=r)


def golden():
    d = dict(np.load(GOLDEN))
    lay = model.Layout(gridgen.grid10k())
    return dict(lay=lay, w=d["w"], lam=d["lam"], y=d["y"], sw=d["sig_w"], ss=d["sig_s"], r=d["r"],
                dw=float(d["delta"]))


def oracle(p, dw):
    lay = p["lay"]
    _, G, A = model.jacobians(lay, p["w"])
    W = model.lagrangian_hessian(lay, p["w"], p["lam"], p["y"])
    Kc = kkt.kred_definition(G, A, W, p["sw"], p["ss"], lay.nu)
    Wd = W + sp.diags(np.r_[np.full(lay.nu, dw), np.zeros(lay.nx)])
    return 0.5 * (Kc + Kc.T), np.concatenate(kkt.full_space_step(G, A, Wd, p["sw"], p["ss"], p["r"]))


def run(pkg, net, p, dw, **opt):
    lay = p["lay"]
    h = pkg.Handle(net, **opt)
    h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
    K = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.condense_rhs(T(p["sw"][:lay.nu]), T(p["sw"][lay.nu:]), T(p["ss"]), T(p["r"]), K)
    assert h.kkt_factor(dw) == -1
    step = torch.zeros(len(p["r"]), dtype=torch.float64, device="cuda")
    h.kkt_solve_condensed(step)
    return h, N(K).reshape(lay.nu, lay.nu), N(step)


@pytest.mark.parametrize("rhs_block", [64, 128])
@pytest.mark.parametrize("width", [0, 128])
def test_reach_lists_grid2000(pkg, rhs_block, width):
    net = gridgen.grid2000()
    p = point(net, 41)
    lay = p["lay"]
    Ko, _ = oracle(p, 0.0)
    dw = max(0.0, -np.linalg.eigvalsh(Ko)[0]) + 1.0
    _, ref = oracle(p, dw)
    opt = dict(rhs_block=rhs_block, rhs_width=width if width else 10 ** 6)
    h0, K0, s0 = run(pkg, net, p, dw, dense_forward=1, **opt)
    h1, K1, s1 = run(pkg, net, p, dw, **opt)
    nblk, work = h1.forward_reach()
    assert nblk == lay.nu // 32 and 0 < work["listed"] < work["all"]
    assert h0.forward_reach()[0] == 0
    assert np.array_equal(K1, K0) and np.array_equal(s1, s0)
    assert rel_err(K1, Ko) <= 1e-9 and rel_err(s1, ref) <= 1e-9


@pytest.mark.parametrize("rhs_block,width", [(64, 0), (128, 0), (64, 256)])
def test_reach_lists_grid10k(pkg, rhs_block, width):
    p = golden()
    net = gridgen.grid10k()
    Ko, ref = oracle(p, p["dw"])
    opt = dict(rhs_block=rhs_block, rhs_width=width if width else 10 ** 6)
    _, K0, s0 = run(pkg, net, p, p["dw"], dense_forward=1, **opt)
    h1, K1, s1 = run(pkg, net, p, p["dw"], **opt)
    assert h1.forward_reach()[0] == p["lay"].nu // 32
    assert np.array_equal(K1, K0) and np.array_equal(s1, s0)
    assert rel_err(K1, Ko) <= 1e-9 and rel_err(s1, ref) <= 1e-9


def test_dense_forward_option_is_checked(pkg):
    with pytest.raises(pkg.OPFError) as e:
        pkg.Handle(gridgen.ring30(), dense_forward=2)
    assert e.value.code == pkg.OPF_ERR_INVALID_ARG
