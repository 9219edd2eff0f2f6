"""Derivative of the optimal dispatch with respect to the bus loads -- oracle side.

Test infrastructure: only tests, the package's smoke check and the benchmark's
CPU leg use this module.

The quantity.  At a point xi = (w, s, lambda, y, z) that solves the barrier KKT
system F(xi; d) = 0 at a fixed barrier parameter mu (Eq. 4 with the bound terms
of the primal-dual barrier method; d = (Pd, Qd) the bus loads), the
implicit-function theorem gives the derivative of the solution, and with it the
derivative of the dispatch Pg (every generator, the slack's Pg_0 = P_s + Pd_s
included):

    dPg/dd = dPg/dd|_xi fixed - J_out (dF/dxi)^{-1} dF/dd,   J_out = dPg/dxi.

Eliminating the bound multipliers z (their equations z (v - v_L) = mu do not
involve d) turns dF/dxi into the augmented matrix K_aug of Eq.
kktmatrix:normal with Sigma at the point, so for cotangents vbar

    zeta = K_aug^{-1} J_out^T vbar,     grad_d = -(dF/dd)^T zeta + (dPg/dd|_xi)^T vbar.

This module writes that definition out with a sparse LU of the whole K_aug
(no reduction or condensation), and supplies the independent route that pins
it: a Newton solve of the barrier system at fixed mu, from a warm start, for
perturbed loads, so that central differences of the solved dispatch can be
compared with the formula.  Choosing the derivative of the barrier solution at
the final mu, held fixed, is a reading: the paper does not differentiate its
solution.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import kkt, model
from .ipm import _Bounds


# --------------------------------------------------------------- the pieces
def load_jacobian(lay: model.Layout, w):
    """dF/dd (sparse, n_kkt x 2 nb) for F = [grad_w L; grad_s L; g; h + s] with
    columns d = [Pd (nb); Qd (nb)], rows in the unknown order [w, s, lambda, y].

    From the model: g has +Pd_i in the P row of a non-slack bus and +Qd_i in the
    Q row of a load bus; h_0 = P_s + Pd_s and h_{1+k} = Q_i + Qd_i at generator
    k's bus; the objective's slack term c2_0 Pg_0^2 + c1_0 Pg_0 has gradient
    (2 c2_0 Pg_0 + c1_0) grad P_s, whose derivative in Pd_s is 2 c2_0 grad P_s."""
    net = lay.net
    nb, nw, nx, m = lay.nb, lay.nw, lay.nx, lay.m
    r0_s, r0_lam, r0_y = nw, nw + m, nw + m + nx
    rows, cols, vals = [], [], []
    n_ns = len(lay.nonslack)
    for k, i in enumerate(lay.nonslack):
        rows.append(r0_lam + k); cols.append(i); vals.append(1.0)
    for k, i in enumerate(lay.load):
        rows.append(r0_lam + n_ns + k); cols.append(nb + i); vals.append(1.0)
    rows.append(r0_y); cols.append(net.slack); vals.append(1.0)
    for k, i in enumerate(net.gbus):
        rows.append(r0_y + 1 + k); cols.append(nb + i); vals.append(1.0)
    _, _, A = model.jacobians(lay, w)
    a0 = A[[0]].tocoo()
    for j, v in zip(a0.col, a0.data):
        rows.append(j); cols.append(net.slack); vals.append(2.0 * net.c2[0] * v)
    n_kkt = nw + 2 * m + nx
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_kkt, 2 * nb)).tocsr()


def output_jacobian(lay: model.Layout, w):
    """(J_out, D): J_out = dPg/dxi (ng x n_kkt; only the w block is non-zero) and
    D = dPg/dd at fixed xi (ng x 2 nb).  Pg_k (k >= 1) is a control; Pg_0 is row
    0 of h, whose w-gradient is row 0 of A, and it carries +Pd_s directly."""
    net = lay.net
    nb, nw, nx, m = lay.nb, lay.nw, lay.nx, lay.m
    _, _, A = model.jacobians(lay, w)
    a0 = A[[0]].tocoo()
    rows = list(np.zeros(len(a0.col), np.int64)) + list(range(1, lay.ng))
    cols = list(a0.col) + list(lay.pg_w[1:])
    vals = list(a0.data) + [1.0] * (lay.ng - 1)
    J = sp.coo_matrix((vals, (rows, cols)), shape=(lay.ng, nw + 2 * m + nx)).tocsr()
    D = sp.coo_matrix(([1.0], ([0], [net.slack])), shape=(lay.ng, 2 * nb)).tocsr()
    return J, D


def dispatch_vjp(net, w, lam, y, sig_w, sig_s, vbar):
    """grad_d = vbar^T dPg/dd for cotangents vbar (k x ng) at the point (w, lam,
    y) with Sigma = (sig_w, sig_s).  Returns (grad_Pd, grad_Qd), each k x nb.
    K_aug is assembled in full (Eq. kktmatrix:normal, +I slack coupling) and
    solved by a sparse LU."""
    lay = model.Layout(net)
    vbar = np.atleast_2d(np.asarray(vbar, dtype=np.float64))
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, lam, y)
    K = kkt.kaug(G, A, W, sig_w, sig_s)
    J, D = output_jacobian(lay, w)
    dF = load_jacobian(lay, w)
    zeta = spla.splu(sp.csc_matrix(K)).solve(np.ascontiguousarray((J.T @ vbar.T)))
    grad = -(dF.T @ zeta) + D.T @ vbar.T          # 2 nb x k
    return grad[: lay.nb].T.copy(), grad[lay.nb:].T.copy()


# ------------------------------------------------- the barrier solution itself
@dataclasses.dataclass
class BarrierPoint:
    w: np.ndarray
    s: np.ndarray
    lam: np.ndarray
    y: np.ndarray
    zwl: np.ndarray
    zwu: np.ndarray
    zsl: np.ndarray
    zsu: np.ndarray
    mu: float
    residual: float = np.inf
    iters: int = 0

    @classmethod
    def from_result(cls, res):
        """The converged state of oracle.ipm.linred."""
        (zwl, zsl), (zwu, zsu) = res.zl, res.zu
        return cls(res.w.copy(), res.s.copy(), res.lam.copy(), res.y.copy(), zwl.copy(), zwu.copy(),
                   zsl.copy(), zsu.copy(), float(res.mu))

    def sigma(self, net):
        lay = model.Layout(net)
        bw = _Bounds(lay.wl, lay.wu)
        bs = _Bounds(-lay.hu, -lay.hl)
        return bw.sigma(self.w, self.zwl, self.zwu), bs.sigma(self.s, self.zsl, self.zsu)


def barrier_residual(lay, p: BarrierPoint):
    """Max-norm of the barrier KKT residual: stationarity in w and s, g, h + s,
    and the perturbed complementarity z (v - v_L) = mu, z (v_U - v) = mu."""
    bw = _Bounds(lay.wl, lay.wu)
    bs = _Bounds(-lay.hu, -lay.hl)
    gf, G, A = model.jacobians(lay, p.w)
    parts = [gf + G.T @ p.lam + A.T @ p.y - p.zwl + p.zwu, p.y - p.zsl + p.zsu,
             model.cons_g(lay, p.w), model.cons_h(lay, p.w) + p.s,
             bw.compl(p.w, p.zwl, p.zwu, p.mu), bs.compl(p.s, p.zsl, p.zsu, p.mu)]
    return max(np.abs(x).max(initial=0.0) for x in parts)


def barrier_solve(net, start: BarrierPoint, tol=1e-12, max_iter=40):
    """Newton's method on the barrier KKT system of `net` at the fixed mu of
    `start`, from `start` (the full primal-dual step, bound multipliers
    recovered from their linearised equations, the step cut only to stay inside
    the bounds).  Stops at residual <= tol, or when the residual stops falling
    below 1e-9 (rounding level).  Returns a new BarrierPoint."""
    lay = model.Layout(net)
    bw = _Bounds(lay.wl, lay.wu)
    bs = _Bounds(-lay.hu, -lay.hl)
    p = dataclasses.replace(start)
    mu = p.mu
    prev = np.inf
    for it in range(max_iter + 1):
        res = barrier_residual(lay, p)
        p.residual, p.iters = res, it
        if res <= tol or (res < 1e-9 and res > 0.5 * prev) or it == max_iter:
            return p
        prev = res
        gf, G, A = model.jacobians(lay, p.w)
        W = model.lagrangian_hessian(lay, p.w, p.lam, p.y)
        sig_w = bw.sigma(p.w, p.zwl, p.zwu)
        sig_s = bs.sigma(p.s, p.zsl, p.zsu)
        r = np.concatenate([gf + G.T @ p.lam + A.T @ p.y + bw.barrier_grad(p.w, mu),
                            p.y + bs.barrier_grad(p.s, mu),
                            model.cons_g(lay, p.w), model.cons_h(lay, p.w) + p.s])
        pw, ps, plam, py = kkt.full_space_step(G, A, W, sig_w, sig_s, r)
        dzwl, dzwu = bw.dz(p.w, p.zwl, p.zwu, pw, mu)
        dzsl, dzsu = bs.dz(p.s, p.zsl, p.zsu, ps, mu)
        a = min(1.0, bw.max_step(p.w, pw, 0.995), bs.max_step(p.s, ps, 0.995))
        fl = [(p.zwl, dzwl, bw.fl), (p.zwu, dzwu, bw.fu), (p.zsl, dzsl, bs.fl), (p.zsu, dzsu, bs.fu)]
        for z, dz, mk in fl:
            neg = mk & (dz < 0)
            if neg.any():
                a = min(a, np.min(-0.995 * z[neg] / dz[neg]))
        p = BarrierPoint(p.w + a * pw, p.s + a * ps, p.lam + a * plam, p.y + a * py,
                         p.zwl + a * dzwl, p.zwu + a * dzwu, p.zsl + a * dzsl, p.zsu + a * dzsu, mu)
    return p


def with_loads(net, Pd, Qd):
    """A copy of `net` with the given bus loads."""
    n = net.copy()
    n.Pd = np.asarray(Pd, dtype=np.float64).copy()
    n.Qd = np.asarray(Qd, dtype=np.float64).copy()
    return n


def solved_dispatch(net, start: BarrierPoint, Pd, Qd, tol=1e-12):
    """Pg (all generators) of the barrier solution for loads (Pd, Qd) at the
    fixed mu of `start`, solved from `start`."""
    n = with_loads(net, Pd, Qd)
    p = barrier_solve(n, start, tol=tol)
    Pg, _ = model.dispatch(model.Layout(n), p.w)
    return Pg, p
