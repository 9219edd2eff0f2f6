"""opf_chol_noalloc -- the dense Cholesky for callers that cannot allocate device
memory -- against the library's regular factorisation entry point.

The regular path (opf_condense + opf_kkt_factor) keeps its scratch in buffers
the handle allocated; the no-allocation path keeps it in a file-scope device
array and takes only caller buffers.  Both must give the same factor, on two
calls in a row (the second call finds the previous call's contents in the
shared array and has to clear what must start at zero)."""
import numpy as np
import pytest

from gpu_cases import oracle_iterate, rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("name", ["ring30", "grid2000"])
def test_chol_noalloc_matches_kkt_factor_twice(name):
    from oracle import model
    from paper_2203_11875_gb300 import binding, build
    build.build()
    net, rec = oracle_iterate(name)
    lay = model.Layout(net)
    h = binding.Handle(net)
    w = rec["w"]
    h.eval_derivatives(T(w[lay.nu:]), T(w[:lay.nu]), T(rec["lam"]), T(rec["y"]))
    Kred = torch.zeros(lay.nu * lay.nu, dtype=torch.float64, device="cuda")
    h.condense(T(rec["sig_w"][:lay.nu]), T(rec["sig_w"][lay.nu:]), T(rec["sig_s"]), Kred)
    delta = rec["delta"]
    assert h.kkt_factor(delta) == -1
    F = torch.zeros_like(Kred)
    h.get_factor(F)
    ref = F.cpu().numpy()
    Ls = [torch.full_like(Kred, 7.0) for _ in range(2)]
    torch.cuda.synchronize()
    for k in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        assert binding.chol_noalloc(Kred, lay.nu, delta, Ls[k]) == -1
        # no device memory taken by the call (the first one may load the module)
        if k == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        assert rel_err(Ls[k].cpu().numpy(), ref) <= 1e-9
        got = Ls[k].cpu().numpy().reshape(lay.nu, lay.nu)
        assert np.array_equal(got, np.tril(got))


def test_chol_noalloc_rejects_oversized_and_reports_not_pd():
    from paper_2203_11875_gb300 import binding, build
    build.build()
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.OPFError) as e:
        binding.chol_noalloc(big, 5000, 0.0, big)
    assert e.value.code == -1
    # indefinite matrix: failure reported with its column, twice in a row
    A = T(np.diag([4.0, 1.0, -2.0, 3.0]))
    L = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert binding.chol_noalloc(A, 4, 0.0, L) == 2
    assert binding.chol_noalloc(A, 4, 0.0, L) == 2
    assert binding.chol_noalloc(A, 4, 3.0, L) == -1
    np.testing.assert_allclose(L.cpu().numpy().reshape(4, 4), np.diag(np.sqrt([7.0, 4.0, 1.0, 6.0])), rtol=1e-14)
