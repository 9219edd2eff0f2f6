"""Host logic of the differentiable dispatch (CPU only).

The autograd wrapper only marshals tensors between torch and a handle; here it
drives a stand-in handle whose calls are answered by the oracle on the CPU, so
the plumbing (load hand-over, solve, preparation, single and batched backward)
is checked without a GPU.  The GPU handle is exercised by test_gpu_vjp.py.
"""
import numpy as np
import pytest
import torch

import gridgen
from oracle import ipm, model, sens
from paper_2203_11875_gb300 import autograd as ag


class OracleHandle:
    """The methods of binding.Handle that the autograd wrapper calls."""

    device = torch.device("cpu")

    def __init__(self, net):
        self.base = net
        self.net = net
        self.nb, self.ng = net.nb, net.ng
        self.vjp_shapes = []

    def set_loads(self, Pd, Qd):
        self.net = sens.with_loads(self.base, Pd, Qd)
        self.point = None

    def solve(self, variant="linred", tol=1e-8):
        res = ipm.linred(self.net, tol=tol)
        self.point = sens.BarrierPoint.from_result(res)
        return {"status": 0 if res.status == "converged" else -8}

    def solution(self):
        p = self.point
        Pg, _ = model.dispatch(model.Layout(self.net), p.w)
        return p.w, p.lam, p.y, Pg

    def vjp_prepare(self):
        self.sig = self.point.sigma(self.net)

    def dispatch_vjp(self, v, gP, gQ):
        self.vjp_shapes.append(tuple(v.shape))
        p = self.point
        a, b = sens.dispatch_vjp(self.net, p.w, p.lam, p.y, *self.sig, v.numpy())
        gP.copy_(torch.from_numpy(a))
        gQ.copy_(torch.from_numpy(b))


@pytest.fixture(scope="module")
def ring():
    net = gridgen.ring30()
    return net, OracleHandle(net)


def test_forward_returns_the_solved_dispatch(ring):
    net, hd = ring
    Pd = torch.tensor(net.Pd)
    Qd = torch.tensor(net.Qd)
    Pg = ag.optimal_dispatch(hd, Pd, Qd)
    res = ipm.linred(net)
    Pg_ref, _ = model.dispatch(model.Layout(net), res.w)
    assert Pg.dtype == torch.float64 and Pg.shape == (net.ng,)
    assert np.allclose(Pg.numpy(), Pg_ref, rtol=0, atol=1e-12)


def test_backward_is_one_vjp_call(ring):
    net, hd = ring
    Pd = torch.tensor(net.Pd, requires_grad=True)
    Qd = torch.tensor(net.Qd, requires_grad=True)
    Pg = ag.optimal_dispatch(hd, Pd, Qd)
    c = torch.linspace(-1.0, 1.0, net.ng, dtype=torch.float64)
    hd.vjp_shapes.clear()
    (Pg * c).sum().backward()
    assert hd.vjp_shapes == [(1, net.ng)]
    p = hd.point
    a, b = sens.dispatch_vjp(net, p.w, p.lam, p.y, *p.sigma(net), c.numpy()[None])
    assert np.allclose(Pd.grad.numpy(), a[0], rtol=0, atol=1e-12)
    assert np.allclose(Qd.grad.numpy(), b[0], rtol=0, atol=1e-12)


def test_batched_cotangents_run_as_one_call(ring):
    net, hd = ring
    Pd = torch.tensor(net.Pd)
    Qd = torch.tensor(net.Qd)
    V = torch.tensor(gridgen.cotangents(net.ng, 7, seed=11))
    _, vjp_fn = torch.func.vjp(lambda a, b: ag.optimal_dispatch(hd, a, b), Pd, Qd)
    hd.vjp_shapes.clear()
    gP, gQ = torch.func.vmap(vjp_fn)(V)
    assert hd.vjp_shapes == [tuple(V.shape)]
    p = hd.point
    a, b = sens.dispatch_vjp(net, p.w, p.lam, p.y, *p.sigma(net), V.numpy())
    assert np.allclose(gP.numpy(), a, rtol=0, atol=1e-12)
    assert np.allclose(gQ.numpy(), b, rtol=0, atol=1e-12)
    # the direct entry point gives the same
    gP2, gQ2 = ag.dispatch_vjp(hd, V)
    assert torch.equal(gP2, gP) and torch.equal(gQ2, gQ)
