"""Batched solves (opf_batch_*) of the 96 uneven instances: 32 networks each at
500, 1,500 and 3,000 buses with per-bus load scaling.  Every instance solved in
the batch -- in lockstep (one batched condensation per iteration for all
instances) and as concurrent independent loops -- must reach its own
single-instance objective to 1e-6 relative, and one instance per size class
must match the CPU oracle's objective to 1e-6."""
import numpy as np
import pytest

import gridgen
from oracle import ipm

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL_OBJ = 1e-6


@pytest.fixture(scope="module")
def pkg():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def runs(pkg):
    nets = gridgen.batch96()
    hs = [pkg.Handle(n) for n in nets]
    b = pkg.Batch(hs)
    b.autotune()
    single = [h.solve() for h in hs]
    batched, wall_ms = b.solve()
    calls = b.lockstep_calls()
    b.set_mode("concurrent")
    concurrent, _ = b.solve()
    b.close()
    return nets, single, batched, wall_ms, calls, concurrent


def test_every_batched_instance_matches_its_single_solve(runs):
    nets, single, batched, _, calls, concurrent = runs
    assert len(batched) == 96
    # lockstep: one batched condensation per iteration of the longest loop
    assert calls == max(r["iters"] for r in batched)
    for net, a, b, c in zip(nets, single, batched, concurrent):
        assert a["status"] == 0 and b["status"] == 0 and c["status"] == 0, (net.name, a["status"], b["status"])
        assert abs(a["obj"] - b["obj"]) <= TOL_OBJ * abs(a["obj"]), net.name
        assert abs(a["obj"] - c["obj"]) <= TOL_OBJ * abs(a["obj"]), net.name


@pytest.mark.parametrize("j", [0, 32, 64])
def test_one_instance_per_size_class_matches_the_oracle(runs, j):
    nets, _, batched, *_ = runs
    ref = ipm.linred(nets[j])
    assert ref.status == "converged"
    assert abs(batched[j]["obj"] - ref.obj) <= TOL_OBJ * abs(ref.obj)


def test_batch_rejects_a_repeated_handle(pkg):
    net = gridgen.tiny3()
    h = pkg.Handle(net)
    with pytest.raises(pkg.OPFError):
        pkg.Batch([h, h])


def test_small_batch_of_mixed_networks(pkg):
    nets = [gridgen.tiny3(), gridgen.ring30(), gridgen.tiny3()]
    hs = [pkg.Handle(n) for n in nets]
    ref = [pkg.Handle(n).solve() for n in nets]
    b = pkg.Batch(hs, nthreads=2)
    assert b.n == 3 and b.nthreads == 2
    # independent loops on streams reproduce the single solves
    b.set_mode("concurrent")
    out, ms = b.solve()
    assert ms > 0
    for r, o in zip(ref, out):
        assert o["status"] == 0
        assert abs(r["obj"] - o["obj"]) <= 1e-12 * abs(r["obj"])
    # lockstep: the same optima through the batched condensation
    b.set_mode("lockstep")
    out, ms = b.solve()
    assert b.lockstep_calls() == max(o["iters"] for o in out)
    for r, o in zip(ref, out):
        assert o["status"] == 0
        assert abs(r["obj"] - o["obj"]) <= TOL_OBJ * abs(r["obj"])
    # the handles get their own streams back and still work alone
    b.close()
    assert hs[1].solve()["status"] == 0
    assert np.isfinite(hs[1].solution()[3]).all()


def test_lockstep_redlin_batch_matches_single_solves(pkg):
    """Reduce-then-linearize loops in lockstep: each iteration's condensation of
    every instance still iterating goes through the batched call; every
    instance reaches its own single-instance RedLin optimum."""
    nets = [gridgen.tiny3(), gridgen.ring30(), gridgen.lattice(500, 7101, name="b500")]
    ref = [pkg.Handle(n).solve("redlin") for n in nets]
    hs = [pkg.Handle(n) for n in nets]
    b = pkg.Batch(hs)
    out, _ = b.solve(variant="redlin")
    assert b.lockstep_calls() == max(o["iters"] for o in out)
    for r, o in zip(ref, out):
        assert r["status"] == 0 and o["status"] == 0
        assert abs(r["obj"] - o["obj"]) <= TOL_OBJ * abs(r["obj"])
    b.close()
