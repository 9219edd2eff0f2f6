"""opf_batch_condense_factor -- the refactorisation, multi-RHS solves, Kred and
Cholesky of a whole batch in one launch per phase -- against the oracle and the
single-instance path.

Instances of uneven size (3 to 3,000 buses: nu = 3 .. 599, ragged column tails
included) at random points; one instance is made indefinite on purpose.  For
each: the factor against the oracle's Kred by definition plus delta_w I
(1e-9), the failing column of the indefinite one exactly (plain-definition
Cholesky), the Newton step through opf_kkt_solve against the full-space solve
of K_aug (1e-9), and the factor against the single-instance opf_condense +
opf_kkt_factor path (1e-11: the Cholesky forms differ in rounding order).  Two
batched calls in a row, at different Sigma, so that the reset of the
refactorisation flags and status words between calls is covered."""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
from oracle import kkt, model

from gpu_cases import rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


def networks():
    return [gridgen.tiny3(), gridgen.ring30(),
            gridgen.lattice(500, 7001, name="b500"), gridgen.lattice(1500, 7002, name="b1500"),
            gridgen.lattice(3000, 7003, name="b3000"), gridgen.grid2000()]


INDEFINITE = 3   # this instance gets scaled multipliers and delta_w = 0


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
    Ko = kkt.kred_definition(G, A, W, sw, ss, lay.nu)
    return dict(lay=lay, w=w, lam=lam, y=y, sw=sw, ss=ss, r=r, G=G, A=A, W=W, Ko=0.5 * (Ko + Ko.T))


def first_failing_column(M):
    A = np.array(M, dtype=np.float64)
    for j in range(A.shape[0]):
        d = A[j, j] - A[j, :j] @ A[j, :j]
        if not d > 0:
            return j
        A[j, j] = np.sqrt(d)
        A[j + 1:, j] = (A[j + 1:, j] - A[j + 1:, :j] @ A[j, :j]) / A[j, j]
    return -1


@pytest.mark.parametrize("call", [0, 1])
def test_batched_condense_factor(pkg, call):
    nets = networks()
    hs = [pkg.Handle(n) for n in nets]
    b = pkg.Batch(hs)
    pts, deltas = [], []
    for rep in range(2):
        pts = [point(n, 100 * rep + 10 * k + call, 1.0) for k, n in enumerate(nets)]
        # scale the multipliers of one instance until W makes its Kred indefinite
        for scale in (3.0, 10.0, 30.0, 100.0):
            pts[INDEFINITE] = point(nets[INDEFINITE], 100 * rep + 10 * INDEFINITE + call, scale)
            if np.linalg.eigvalsh(pts[INDEFINITE]["Ko"])[0] < 0:
                break
        deltas = []
        for k, p in enumerate(pts):
            lmin = float(np.linalg.eigvalsh(p["Ko"])[0])
            if k == INDEFINITE:
                assert lmin < 0
                deltas.append(0.0)
            else:
                deltas.append(max(0.0, -lmin) + 1.0)
        for h, p in zip(hs, pts):
            lay = p["lay"]
            h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
        sig = [[T(p["sw"][:p["lay"].nu]) for p in pts], [T(p["sw"][p["lay"].nu:]) for p in pts],
               [T(p["ss"]) for p in pts]]
        status, fcol = b.condense_factor(*sig, delta_w=deltas)
        for k, (h, p) in enumerate(zip(hs, pts)):
            lay = p["lay"]
            if k == INDEFINITE:
                assert status[k] == pkg.OPF_ERR_NOT_PD
                assert fcol[k] == first_failing_column(p["Ko"])
                continue
            assert status[k] == 0 and fcol[k] == -1, (k, status[k])
            F = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
            h.get_factor(F)
            F = N(F).reshape(lay.nu, lay.nu)
            assert np.array_equal(F, np.tril(F))
            ref = p["Ko"] + deltas[k] * np.eye(lay.nu)
            assert rel_err(F @ F.T, ref) <= TOL, k
            step = torch.zeros(len(p["r"]), dtype=torch.float64, device="cuda")
            h.kkt_solve(T(p["r"]), step)
            Wd = p["W"] + sp.diags(np.r_[np.full(lay.nu, deltas[k]), np.zeros(lay.nx)])
            full = np.concatenate(kkt.full_space_step(p["G"], p["A"], Wd, p["sw"], p["ss"], p["r"]))
            assert rel_err(N(step), full) <= TOL, k
            # the single-instance path on a handle of its own
            h1 = pkg.Handle(nets[k])
            h1.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
            h1.condense(T(p["sw"][:lay.nu]), T(p["sw"][lay.nu:]), T(p["ss"]))
            assert h1.kkt_factor(deltas[k]) == -1
            F1 = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
            h1.get_factor(F1)
            assert rel_err(F, N(F1).reshape(lay.nu, lay.nu)) <= 1e-11, k
        # the indefinite instance recovers on its own handle with a larger delta_w
        p = pts[INDEFINITE]
        big = 2.0 * abs(float(np.linalg.eigvalsh(p["Ko"])[0])) + 1.0
        assert hs[INDEFINITE].kkt_factor(big) == -1
    # the first call with every instance factored completely tunes the cluster
    # sizes; the first call (one instance indefinite) cannot, so the second tunes
    # and none is replayed from the captured graph yet
    st = b.stats()
    assert st["trsm_cl"] in (2, 4, 8, 16) or st["trsm_cl"] == 0
    b.close()


def test_batched_condense_factor_graph_replay(pkg):
    """After the tuning call, every call replays the captured graph of the whole
    batched sequence, with the same results as an eagerly enqueued call."""
    nets = networks()[:5]
    hs = [pkg.Handle(n) for n in nets]
    b = pkg.Batch(hs)
    outs = []
    for call in range(3):
        pts = [point(n, 500 + 10 * k, 1.0) for k, n in enumerate(nets)]
        deltas = [max(0.0, -float(np.linalg.eigvalsh(p["Ko"])[0])) + 1.0 for p in pts]
        for h, p in zip(hs, pts):
            lay = p["lay"]
            h.eval_derivatives(T(p["w"][lay.nu:]), T(p["w"][:lay.nu]), T(p["lam"]), T(p["y"]))
        sig = [[T(p["sw"][:p["lay"].nu]) for p in pts], [T(p["sw"][p["lay"].nu:]) for p in pts],
               [T(p["ss"]) for p in pts]]
        status, _ = b.condense_factor(*sig, delta_w=deltas)
        assert status == [0] * len(nets)
        Fs = []
        for h, p in zip(hs, pts):
            F = torch.zeros(p["lay"].nu ** 2, dtype=torch.float64, device="cuda")
            h.get_factor(F)
            Fs.append(N(F))
        outs.append(Fs)
    st = b.stats()
    assert st["trsm_cl"] > 0 and st["chol_cl"] > 0
    assert st["graph_calls"] == 2
    # the same point gives bitwise the same factors through the graph as through
    # the eagerly enqueued tuning call
    for k in range(len(nets)):
        assert np.array_equal(outs[0][k], outs[1][k]) and np.array_equal(outs[1][k], outs[2][k])
    b.close()
