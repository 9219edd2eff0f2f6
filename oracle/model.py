"""Polar AC-OPF in state-control form -- oracle side (test infrastructure).

Formulation (the paper leaves the model equations out, Sec. 3.2, so this is
the reading used throughout; the variable split follows Table 1):

* state    x = (theta at the nb-1 non-slack buses, Vm at the nb-ng load buses)
* control  u = (Vm at the ng generator buses, Pg at the ng-1 non-slack gens)
* g(x,u)   = [P_i - Pg_i + Pd_i, i non-slack ; Q_i + Qd_i, i load bus]  (Eq. 1)
* h(x,u)   = [Pg_slack ; Qg_k for every gen k ; |S_f|^2, |S_t|^2 per limited
             line], with box bounds hL <= h <= hU
* f(x,u)   = sum_k c2_k Pg_k^2 + c1_k Pg_k, Pg_slack = P_s + Pd_s
* slack form h + s = 0 (Eq. 3), so s has bounds [-hU, -hL].

Lines are pi-models: series admittance y = 1/(r + j x), b/2 at each end, no
taps, no bus shunts.  P_i and Q_i are the sums over incident line ends of the
flow leaving bus i.

The full primal vector is ordered w = [u; x] as in the paper's block
partition (Sec. 2.1).  Functions evaluating f, g, h accept complex w so that
tests can differentiate them by the complex step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from gridgen import Network


class Layout:
    """Index maps between buses/generators and the (u, x) vectors."""

    def __init__(self, net: Network):
        self.net = net
        nb, ng = net.nb, net.ng
        self.nb, self.ng, self.nl = nb, ng, net.nl
        is_gen = np.zeros(nb, bool)
        is_gen[net.gbus] = True
        self.is_gen = is_gen
        self.nonslack = np.array([i for i in range(nb) if i != net.slack], np.int64)
        self.load = np.array([i for i in range(nb) if not is_gen[i]], np.int64)
        self.nx = len(self.nonslack) + len(self.load)
        self.nu = ng + (ng - 1)
        self.nw = self.nx + self.nu
        lim = np.nonzero(net.rate > 0)[0]
        self.lim = lim
        self.m = 1 + ng + 2 * len(lim)
        # w-index of theta_i (-1 for slack) and of Vm_i
        self.th_w = -np.ones(nb, np.int64)
        self.th_w[self.nonslack] = self.nu + np.arange(len(self.nonslack))
        self.vm_w = -np.ones(nb, np.int64)
        self.vm_w[net.gbus] = np.arange(ng)
        self.vm_w[self.load] = self.nu + len(self.nonslack) + np.arange(len(self.load))
        # w-index of Pg_k (-1 for the slack generator)
        self.pg_w = -np.ones(ng, np.int64)
        self.pg_w[1:] = ng + np.arange(ng - 1)
        self.gen_of_bus = -np.ones(nb, np.int64)
        self.gen_of_bus[net.gbus] = np.arange(ng)
        # bounds on w
        wl = np.full(self.nw, -np.inf)
        wu = np.full(self.nw, np.inf)
        wl[self.vm_w] = net.Vmin
        wu[self.vm_w] = net.Vmax
        wl[self.pg_w[1:]] = net.Pmin[1:]
        wu[self.pg_w[1:]] = net.Pmax[1:]
        self.wl, self.wu = wl, wu
        # bounds on h
        hl = np.concatenate([[net.Pmin[0]], net.Qmin, np.full(2 * len(lim), -np.inf)])
        hu = np.concatenate([[net.Pmax[0]], net.Qmax, np.tile(net.rate[lim] ** 2, 2)])
        self.hl, self.hu = hl, hu
        # line-end table: end e = (line l, this bus i, other bus k)
        L = net.nl
        self.end_line = np.concatenate([np.arange(L), np.arange(L)])
        self.end_i = np.concatenate([net.lf, net.lt]).astype(np.int64)
        self.end_k = np.concatenate([net.lt, net.lf]).astype(np.int64)
        y = 1.0 / (net.r + 1j * net.x)
        ys = y + 0.5j * net.b               # self admittance of a line end
        ym = -y                             # mutual admittance
        self.gs = np.concatenate([ys.real, ys.real])
        self.bs = np.concatenate([ys.imag, ys.imag])
        self.gm = np.concatenate([ym.real, ym.real])
        self.bm = np.concatenate([ym.imag, ym.imag])
        # local variable order per end: (theta_i, theta_k, Vm_i, Vm_k)
        self.end_w = np.stack([self.th_w[self.end_i], self.th_w[self.end_k],
                               self.vm_w[self.end_i], self.vm_w[self.end_k]], axis=1)
        # limited-line ends in h order: all from-ends then all to-ends
        self.lim_end = np.concatenate([lim, lim + L])

    # ------------------------------------------------------------- variables
    def split(self, w):
        return w[: self.nu], w[self.nu:]

    def voltages(self, w):
        net = self.net
        Vm = np.zeros(self.nb, dtype=w.dtype)
        Va = np.zeros(self.nb, dtype=w.dtype)
        Vm[:] = w[self.vm_w]
        Va[self.nonslack] = w[self.th_w[self.nonslack]]
        Va[net.slack] = 0.0
        return Vm, Va

    def flat_start(self):
        """theta = 0, Vm = 1 at load buses, Vm = 1.05 (clipped to the bounds) at
        generator buses, non-slack Pg at the middle of its range."""
        net = self.net
        w = np.zeros(self.nw)
        w[self.vm_w] = 1.0
        w[self.vm_w[net.gbus]] = np.clip(1.05, net.Vmin[net.gbus], net.Vmax[net.gbus])
        w[self.pg_w[1:]] = 0.5 * (net.Pmin[1:] + net.Pmax[1:])
        return w


# ------------------------------------------------------------------ values
def end_pq(lay: Layout, Vm, Va):
    """Flow (p, q) leaving bus i at every line end (i, k)."""
    Vi, Vk = Vm[lay.end_i], Vm[lay.end_k]
    t = Va[lay.end_i] - Va[lay.end_k]
    c, s = np.cos(t), np.sin(t)
    a = lay.gm * c + lay.bm * s
    bb = lay.gm * s - lay.bm * c
    p = Vi * Vi * lay.gs + Vi * Vk * a
    q = -Vi * Vi * lay.bs + Vi * Vk * bb
    return p, q


def injections(lay: Layout, Vm, Va):
    p, q = end_pq(lay, Vm, Va)
    P = np.zeros(lay.nb, dtype=p.dtype)
    Q = np.zeros(lay.nb, dtype=q.dtype)
    np.add.at(P, lay.end_i, p)
    np.add.at(Q, lay.end_i, q)
    return P, Q


def dispatch(lay: Layout, w):
    """Active and reactive generation of every generator at w."""
    net = lay.net
    Vm, Va = lay.voltages(w)
    P, Q = injections(lay, Vm, Va)
    Pg = np.zeros(lay.ng, dtype=P.dtype)
    Pg[0] = P[net.slack] + net.Pd[net.slack]
    Pg[1:] = w[lay.pg_w[1:]]
    Qg = Q[net.gbus] + net.Qd[net.gbus]
    return Pg, Qg


def objective(lay: Layout, w):
    net = lay.net
    Pg, _ = dispatch(lay, w)
    return np.sum(net.c2 * Pg * Pg + net.c1 * Pg)


def cons_g(lay: Layout, w, Pd=None, Qd=None):
    """State equation g(x, u) (Eq. 1), P rows then Q rows."""
    net = lay.net
    Pd = net.Pd if Pd is None else Pd
    Qd = net.Qd if Qd is None else Qd
    Vm, Va = lay.voltages(w)
    P, Q = injections(lay, Vm, Va)
    Pgb = np.zeros(lay.nb, dtype=w.dtype)
    Pgb[net.gbus[1:]] = w[lay.pg_w[1:]]
    gP = (P - Pgb + Pd)[lay.nonslack]
    gQ = (Q + Qd)[lay.load]
    return np.concatenate([gP, gQ])


def cons_h(lay: Layout, w, Pd=None, Qd=None):
    """Inequality functions h(x, u): slack Pg, every Qg, |S|^2 at limited ends."""
    net = lay.net
    Pd = net.Pd if Pd is None else Pd
    Qd = net.Qd if Qd is None else Qd
    Vm, Va = lay.voltages(w)
    p, q = end_pq(lay, Vm, Va)
    P = np.zeros(lay.nb, dtype=p.dtype)
    Q = np.zeros(lay.nb, dtype=q.dtype)
    np.add.at(P, lay.end_i, p)
    np.add.at(Q, lay.end_i, q)
    e = lay.lim_end
    return np.concatenate([[P[net.slack] + Pd[net.slack]], Q[net.gbus] + Qd[net.gbus],
                           p[e] * p[e] + q[e] * q[e]])


# ------------------------------------------------------------- derivatives
def _end_derivs(lay: Layout, Vm, Va):
    """Gradient (4) and Hessian (4x4) of p and q per end, local order
    (theta_i, theta_k, Vm_i, Vm_k)."""
    Vi, Vk = Vm[lay.end_i], Vm[lay.end_k]
    t = Va[lay.end_i] - Va[lay.end_k]
    c, s = np.cos(t), np.sin(t)
    a = lay.gm * c + lay.bm * s          # d a / d t = -bb
    bb = lay.gm * s - lay.bm * c         # d bb / d t = a
    gs, bs = lay.gs, lay.bs
    n = len(Vi)
    p = Vi * Vi * gs + Vi * Vk * a
    q = -Vi * Vi * bs + Vi * Vk * bb
    dp = np.stack([-Vi * Vk * bb, Vi * Vk * bb, 2 * Vi * gs + Vk * a, Vi * a], axis=1)
    dq = np.stack([Vi * Vk * a, -Vi * Vk * a, -2 * Vi * bs + Vk * bb, Vi * bb], axis=1)
    hp = np.zeros((n, 4, 4))
    hq = np.zeros((n, 4, 4))
    # p
    hp[:, 0, 0] = -Vi * Vk * a
    hp[:, 0, 1] = Vi * Vk * a
    hp[:, 1, 1] = -Vi * Vk * a
    hp[:, 0, 2] = -Vk * bb
    hp[:, 0, 3] = -Vi * bb
    hp[:, 1, 2] = Vk * bb
    hp[:, 1, 3] = Vi * bb
    hp[:, 2, 2] = 2 * gs
    hp[:, 2, 3] = a
    # q
    hq[:, 0, 0] = -Vi * Vk * bb
    hq[:, 0, 1] = Vi * Vk * bb
    hq[:, 1, 1] = -Vi * Vk * bb
    hq[:, 0, 2] = Vk * a
    hq[:, 0, 3] = Vi * a
    hq[:, 1, 2] = -Vk * a
    hq[:, 1, 3] = -Vi * a
    hq[:, 2, 2] = -2 * bs
    hq[:, 2, 3] = bb
    for H in (hp, hq):
        iu = np.triu_indices(4, 1)
        H[:, iu[1], iu[0]] = H[:, iu[0], iu[1]]
    return p, q, dp, dq, hp, hq


def _scatter_rows(lay, rows_of_end, dloc, nrows):
    """Sparse matrix with row rows_of_end[e] and local gradient dloc[e] scattered
    to the end's global w columns (fixed slack theta dropped)."""
    W = lay.end_w
    R = np.repeat(rows_of_end[:, None], 4, axis=1)
    mask = (W >= 0) & (R >= 0)
    return sp.coo_matrix((dloc[mask], (R[mask], W[mask])), shape=(nrows, lay.nw)).tocsr()


def jacobians(lay: Layout, w):
    """Return (grad f [nw], G [nx x nw], A [m x nw]) at w, hand-derived."""
    net = lay.net
    Vm, Va = lay.voltages(w)
    p, q, dp, dq, _, _ = _end_derivs(lay, Vm, Va)
    nb, ng = lay.nb, lay.ng
    # bus-level dP_i, dQ_i as sparse (nb x nw)
    bus_rows = lay.end_i
    dP = _scatter_rows(lay, bus_rows, dp, nb)
    dQ = _scatter_rows(lay, bus_rows, dq, nb)
    # G: P rows for non-slack buses, -Pg_i column; Q rows for load buses
    GP = dP[lay.nonslack].tolil()
    rowpos = -np.ones(nb, np.int64)
    rowpos[lay.nonslack] = np.arange(len(lay.nonslack))
    for k in range(1, ng):
        GP[rowpos[net.gbus[k]], lay.pg_w[k]] += -1.0
    G = sp.vstack([GP.tocsr(), dQ[lay.load]]).tocsr()
    # A: slack Pg row, Qg rows, |S|^2 rows
    e = lay.lim_end
    dS = 2 * p[e, None] * dp[e] + 2 * q[e, None] * dq[e]
    Wl = lay.end_w[e]
    R = np.repeat(np.arange(len(e))[:, None], 4, axis=1)
    mk = Wl >= 0
    Aflow = sp.coo_matrix((dS[mk], (R[mk], Wl[mk])), shape=(len(e), lay.nw)).tocsr()
    A = sp.vstack([dP[[net.slack]], dQ[net.gbus], Aflow]).tocsr()
    # grad f
    Pg, _ = dispatch(lay, w)
    gf = np.zeros(lay.nw)
    gf[lay.pg_w[1:]] = 2 * net.c2[1:] * Pg[1:] + net.c1[1:]
    gf += (2 * net.c2[0] * Pg[0] + net.c1[0]) * dP[net.slack].toarray().ravel()
    return gf, G, A


def lagrangian_hessian(lay: Layout, w, lam, y):
    """W = hess f + sum lam_i hess g_i + sum y_j hess h_j  (nw x nw sparse)."""
    net = lay.net
    Vm, Va = lay.voltages(w)
    p, q, dp, dq, hp, hq = _end_derivs(lay, Vm, Va)
    nb, ng = lay.nb, lay.ng
    Pg, _ = dispatch(lay, w)
    # per-bus weights on hess P_i and hess Q_i
    wP = np.zeros(nb)
    wQ = np.zeros(nb)
    wP[lay.nonslack] = lam[: len(lay.nonslack)]
    wQ[lay.load] = lam[len(lay.nonslack):]
    wP[net.slack] += 2 * net.c2[0] * Pg[0] + net.c1[0] + y[0]
    wQ[net.gbus] += y[1: 1 + ng]
    Hloc = wP[lay.end_i][:, None, None] * hp + wQ[lay.end_i][:, None, None] * hq
    # line-flow constraints: hess(p^2+q^2) = 2 dp dp^T + 2 p hp + 2 dq dq^T + 2 q hq
    e = lay.lim_end
    yl = y[1 + ng:]
    Hloc[e] += yl[:, None, None] * (
        2 * dp[e][:, :, None] * dp[e][:, None, :] + 2 * p[e][:, None, None] * hp[e]
        + 2 * dq[e][:, :, None] * dq[e][:, None, :] + 2 * q[e][:, None, None] * hq[e])
    Wl = lay.end_w
    I = np.repeat(Wl[:, :, None], 4, axis=2)
    J = np.repeat(Wl[:, None, :], 4, axis=1)
    mk = (I >= 0) & (J >= 0)
    W = sp.coo_matrix((Hloc[mk], (I[mk], J[mk])), shape=(lay.nw, lay.nw)).tocsr()
    # slack cost curvature 2 c2 dP_s dP_s^T and non-slack 2 c2 on Pg
    dP = _scatter_rows(lay, lay.end_i, dp, nb)
    ds = dP[[net.slack]]
    W = W + 2 * net.c2[0] * (ds.T @ ds)
    W = W + sp.coo_matrix((2 * net.c2[1:], (lay.pg_w[1:], lay.pg_w[1:])),
                          shape=(lay.nw, lay.nw))
    return W.tocsr()


def lagrangian_gradient(lay: Layout, w, lam, y):
    """grad_w of f + lam^T g + y^T h (the bound-multiplier terms excluded)."""
    gf, G, A = jacobians(lay, w)
    return gf + G.T @ lam + A.T @ y
