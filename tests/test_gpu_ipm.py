"""End-to-end interior-point solves through the C ABI (opf_solve) against the
CPU oracle's IPM: final objective to 1e-6 relative, power balance at the
converged point (LinRed) and along the path (RedLin), both variants."""
import numpy as np
import pytest

import gridgen
from oracle import ipm, model

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL_OBJ = 1e-6


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
@pytest.mark.parametrize("variant", ["linred", "redlin"])
def test_solve_matches_oracle(pkg, name, variant):
    net = gridgen.WORKLOADS[name]()
    lay = model.Layout(net)
    ref = getattr(ipm, variant)(net)
    assert ref.status == "converged"
    h = pkg.Handle(net)
    res = h.solve(variant)
    assert res["status"] == 0, res
    assert abs(res["obj"] - ref.obj) <= TOL_OBJ * abs(ref.obj)
    w, lam, y, pg = h.solution()
    g = model.cons_g(lay, w)
    assert np.abs(g).max() <= (1e-10 if variant == "redlin" else 1e-8)
    pg_ref, _ = model.dispatch(lay, w)
    np.testing.assert_allclose(pg, pg_ref, rtol=0, atol=1e-8)
    assert abs(model.objective(lay, w) - res["obj"]) <= 1e-9 * abs(res["obj"])


def test_variants_agree_on_grid2000(pkg):
    net = gridgen.grid2000()
    a = pkg.Handle(net).solve("linred")
    b = pkg.Handle(net).solve("redlin")
    assert a["status"] == b["status"] == 0
    assert abs(a["obj"] - b["obj"]) <= TOL_OBJ * abs(a["obj"])


def test_solve_on_a_stream_replays_the_condensation_graph(pkg):
    """On a non-default stream the loop enqueues condensation + Cholesky as one
    captured graph from the second iteration on; the solve must not change."""
    net = gridgen.grid2000()
    a = pkg.Handle(net).solve("linred")
    h = pkg.Handle(net)
    st = torch.cuda.Stream()
    h.set_stream(st)
    b = h.solve("linred")
    assert a["status"] == b["status"] == 0
    assert a["graph_iters"] == 0 and b["graph_iters"] == b["iters"] - 1
    assert a["iters"] == b["iters"]
    assert abs(a["obj"] - b["obj"]) <= 1e-12 * abs(a["obj"])


@pytest.mark.parametrize("rhs1", [1, 64, 65, 66])
def test_one_rhs_kernels_give_the_same_solve(pkg, rhs1):
    """The Newton-step recovery's single-vector solves through each kernel: the
    loop must take the same path to the same optimum."""
    net = gridgen.grid2000()
    ref = pkg.Handle(net, rhs1_kernel=1).solve("linred")
    res = pkg.Handle(net, rhs1_kernel=rhs1).solve("linred")
    assert ref["status"] == res["status"] == 0
    assert abs(res["obj"] - ref["obj"]) <= 1e-9 * abs(ref["obj"])


def test_graph_is_recaptured_after_a_wide_vjp_grows_the_solve_buffers(pkg):
    """A derivative call with many cotangents (256 > the 32-column leading
    dimension of the 30-bus case) grows the solve scratch the captured
    condensation graph points into; the next solve on the same handle must
    capture again and reach the same optimum."""
    net = gridgen.ring30()
    ref = ipm.linred(net)
    h = pkg.Handle(net)
    st = torch.cuda.Stream()
    h.set_stream(st)
    a = h.solve("linred")
    assert a["status"] == 0 and a["graph_iters"] > 0
    h.vjp_prepare()
    V = torch.eye(net.ng, dtype=torch.float64, device="cuda").repeat(256 // net.ng + 1, 1)[:256].contiguous()
    gP = torch.empty((256, net.nb), dtype=torch.float64, device="cuda")
    gQ = torch.empty_like(gP)
    with torch.cuda.stream(st):
        h.dispatch_vjp(V, gP, gQ)
    b = h.solve("linred")
    assert b["status"] == 0 and b["graph_iters"] > 0
    assert b["iters"] == a["iters"]
    assert abs(b["obj"] - a["obj"]) <= 1e-12 * abs(a["obj"])
    assert abs(b["obj"] - ref.obj) <= TOL_OBJ * abs(ref.obj)


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000", "tiny3_loaded"])
def test_filter_line_search_matches_oracle(pkg, name):
    """The filter line search with second-order corrections (LinRed) reaches
    the oracle's filter-variant optimum; on tiny3 with loads x1.3 the first
    trial step raises the constraint violation and a correction is taken, as
    in the oracle."""
    if name == "tiny3_loaded":
        net = gridgen.tiny3()
        net.Pd, net.Qd = 1.3 * net.Pd, 1.3 * net.Qd
    else:
        net = gridgen.WORKLOADS[name]()
    ref = ipm.linred(net, line_search="filter")
    assert ref.status == "converged"
    res = pkg.Handle(net).solve("linred", line_search="filter")
    assert res["status"] == 0, res
    assert abs(res["obj"] - ref.obj) <= TOL_OBJ * abs(ref.obj)
    if name == "tiny3_loaded":
        assert ref.soc_steps >= 1 and res["soc_steps"] >= 1
    with pytest.raises(pkg.OPFError):
        pkg.Handle(net).solve("redlin", line_search="filter")


@pytest.mark.parametrize("name", ["tiny3", "ring30", "grid2000"])
def test_restoration_from_the_start_matches_oracle(pkg, name):
    """The feasibility restoration phase (filter line search, relaxation on the
    inequality rows as a per-row dual regularisation) run from the flat start
    hands back an acceptable point, and the loop reaches the oracle's optimum
    (which the non-GPU pins tie to the plain filter solve)."""
    net = gridgen.WORKLOADS[name]()
    ref = ipm.linred(net, line_search="filter", restoration=True, start_with_resto=True)
    assert ref.status == "converged" and ref.restorations == 1
    res = pkg.Handle(net).solve("linred", line_search="filter", restoration=True, start_with_resto=True)
    assert res["status"] == 0, res
    assert res["restorations"] == 1 and res["resto_iters"] >= 1
    assert abs(res["obj"] - ref.obj) <= TOL_OBJ * abs(ref.obj)


def test_restoration_reports_an_infeasible_case(pkg):
    """Loads of 1.7 x the 3-bus case exceed its generation capacity: the filter
    search runs out of step length, the restoration phase finds no acceptable
    point, and the solve ends with OPF_ERR_INFEASIBLE (the oracle fails the
    same way)."""
    net = gridgen.tiny3()
    net.Pd, net.Qd = 1.7 * net.Pd, 1.7 * net.Qd
    assert net.Pmax.sum() < net.Pd.sum()
    res = pkg.Handle(net).solve("linred", line_search="filter", restoration=True)
    assert res["status"] == pkg.OPF_ERR_INFEASIBLE and res["restorations"] >= 1
    with pytest.raises(RuntimeError, match="restoration failed"):
        ipm.linred(net, line_search="filter", restoration=True)
