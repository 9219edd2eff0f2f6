"""Primal-dual barrier IPM around the condensed KKT step -- oracle side.

Test infrastructure.  The outer loop follows the published primal-dual
barrier method of Wachter and Biegler (2006), which the paper defers to
(Sec. 4.3): monotone barrier update, fraction-to-the-boundary rule, bound
multipliers eliminated into Sigma, Ipopt's scaled optimality error with
tolerance 1e-8, and y0 = 0.  The step comes from the condensed system
(Theorems 1-2), with inertia correction by a primal regularization on the
control block until K_cond is positive definite (Theorem 3; Sec. 4.3).  Step
acceptance uses backtracking on the l1 exact-penalty merit function
(Nocedal and Wright, Sec. 19.4) instead of Ipopt's filter.

linred(net)  -- Algorithm 1 (linearize-then-reduce).
redlin(net)  -- Algorithm 2 (reduce-then-linearize): Newton-Raphson projection
                to 1e-10 on the state equation at every trial control
                (Sec. 4.4), adjoint solve for lambda, state bounds moved into
                h_r (Eq. reduced:problem).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import kkt, model

TAU_MIN = 0.99
KAPPA_EPS = 10.0
KAPPA_MU = 0.2
THETA_MU = 1.5
ETA = 1e-4
KAPPA_SIGMA = 1e10

# filter line search (Wachter and Biegler 2006, their recommended constants)
GAMMA_THETA = 1e-5
GAMMA_PHI = 1e-8
SWITCH_DELTA = 1.0
S_THETA = 1.1
S_PHI = 2.3
ETA_PHI = 1e-4
GAMMA_ALPHA = 0.05
KAPPA_SOC = 0.99
SOC_MAX = 4
# feasibility restoration (Wachter and Biegler 2006, Sec. 3.3)
RHO_RESTO = 1000.0    # weight of the relaxation variables' l1 norm
KAPPA_RESTO = 0.9     # required reduction of the constraint violation
RESTO_MAX_ITER = 100


@dataclasses.dataclass
class Result:
    status: str
    iters: int
    obj: float
    w: np.ndarray
    s: np.ndarray
    lam: np.ndarray
    y: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    mu: float
    sig_w: np.ndarray = None
    sig_s: np.ndarray = None
    err: float = np.inf
    history: list = dataclasses.field(default_factory=list)
    soc_steps: int = 0          # accepted second-order corrections (filter line search)
    restorations: int = 0       # feasibility restoration phases (filter line search)


def _push(v, lo, hi, k1=1e-2, k2=1e-2):
    """Ipopt's initial bound push (Wachter-Biegler 2006, Sec. 3.6)."""
    v = v.copy()
    fl, fu = np.isfinite(lo), np.isfinite(hi)
    both = fl & fu
    pl = np.where(fl, k1 * np.maximum(1.0, np.abs(np.where(fl, lo, 0.0))), 0.0)
    pu = np.where(fu, k1 * np.maximum(1.0, np.abs(np.where(fu, hi, 0.0))), 0.0)
    rng = np.where(both, hi - lo, np.inf)
    pl = np.where(both, np.minimum(pl, k2 * rng), pl)
    pu = np.where(both, np.minimum(pu, k2 * rng), pu)
    v = np.where(fl, np.maximum(v, lo + pl), v)
    v = np.where(fu, np.minimum(v, hi - pu), v)
    return v


class _Bounds:
    """Finite-bound bookkeeping for a vector v with lo <= v <= hi."""

    def __init__(self, lo, hi):
        self.lo, self.hi = lo, hi
        self.fl, self.fu = np.isfinite(lo), np.isfinite(hi)

    def dl(self, v):
        return np.where(self.fl, v - np.where(self.fl, self.lo, 0.0), 1.0)

    def du(self, v):
        return np.where(self.fu, np.where(self.fu, self.hi, 0.0) - v, 1.0)

    def sigma(self, v, zl, zu):
        return np.where(self.fl, zl / self.dl(v), 0.0) + np.where(self.fu, zu / self.du(v), 0.0)

    def barrier_grad(self, v, mu):
        return np.where(self.fl, -mu / self.dl(v), 0.0) + np.where(self.fu, mu / self.du(v), 0.0)

    def barrier(self, v, mu):
        return -mu * (np.sum(np.log(self.dl(v)[self.fl])) + np.sum(np.log(self.du(v)[self.fu])))

    def dz(self, v, zl, zu, dv, mu):
        dzl = np.where(self.fl, mu / self.dl(v) - zl - zl / self.dl(v) * dv, 0.0)
        dzu = np.where(self.fu, mu / self.du(v) - zu + zu / self.du(v) * dv, 0.0)
        return dzl, dzu

    def max_step(self, v, dv, tau):
        a = 1.0
        m = self.fl & (dv < 0)
        if m.any():
            a = min(a, np.min(-tau * self.dl(v)[m] / dv[m]))
        m = self.fu & (dv > 0)
        if m.any():
            a = min(a, np.min(tau * self.du(v)[m] / dv[m]))
        return a

    def compl(self, v, zl, zu, mu):
        return np.concatenate([(self.dl(v) * zl - mu)[self.fl], (self.du(v) * zu - mu)[self.fu]])

    def safeguard(self, v, zl, zu, mu):
        zl = np.where(self.fl, np.clip(zl, mu / (KAPPA_SIGMA * self.dl(v)), KAPPA_SIGMA * mu / self.dl(v)), 0.0)
        zu = np.where(self.fu, np.clip(zu, mu / (KAPPA_SIGMA * self.du(v)), KAPPA_SIGMA * mu / self.du(v)), 0.0)
        return zl, zu


def _max_step_z(z, dz, mask, tau):
    m = mask & (dz < 0)
    if not m.any():
        return 1.0
    return min(1.0, np.min(-tau * z[m] / dz[m]))


def _opt_error(dual, primal, compl, mults, smax=100.0):
    n = max(1, sum(len(x) for x in mults))
    sd = max(smax, sum(np.abs(x).sum() for x in mults) / n) / smax
    e = max(np.abs(dual).max(initial=0.0) / sd, np.abs(primal).max(initial=0.0),
            np.abs(compl).max(initial=0.0) / sd)
    return e


class Filter:
    """The filter: pairs (theta_l, phi_l); a point (theta, phi) is acceptable when
    no pair dominates it, i.e. theta < theta_l or phi < phi_l for every pair.
    It starts as the half-plane theta >= theta_max (the pair (theta_max, -inf))."""

    def __init__(self, theta_max):
        self.pairs = [(theta_max, -np.inf)]

    def acceptable(self, theta, phi):
        return all(theta < tl or phi < pl for tl, pl in self.pairs)

    def add(self, theta, phi):
        self.pairs.append((theta, phi))


def filter_accepts(filt, theta0, phi0, dphi, alpha, theta_t, phi_t, theta_min):
    """Acceptance of a trial point (theta_t, phi_t) reached with step length
    alpha from (theta0, phi0), dphi the directional derivative of the barrier
    objective.  Returns (accepted, phi_type): with the switching condition
    alpha (-dphi)^s_phi > delta theta0^s_theta (dphi < 0) and theta0 <=
    theta_min the step must satisfy the Armijo condition on phi (a phi-type
    step, the filter is not augmented); otherwise sufficient decrease in theta
    or phi against the current point."""
    if not filt.acceptable(theta_t, phi_t):
        return False, False
    switching = dphi < 0 and alpha * (-dphi) ** S_PHI > SWITCH_DELTA * theta0 ** S_THETA
    if switching and theta0 <= theta_min:
        return phi_t <= phi0 + ETA_PHI * alpha * dphi, True
    return (theta_t <= (1.0 - GAMMA_THETA) * theta0 or phi_t <= phi0 - GAMMA_PHI * theta0), False


def filter_alpha_min(theta0, dphi, theta_min):
    """Smallest step length the filter line search tries before it gives up."""
    if dphi < 0:
        a = min(GAMMA_THETA, GAMMA_PHI * theta0 / -dphi)
        if theta0 <= theta_min:
            a = min(a, SWITCH_DELTA * theta0 ** S_THETA / (-dphi) ** S_PHI)
        return GAMMA_ALPHA * a
    return GAMMA_ALPHA * GAMMA_THETA


def _regularized(step_fn, delta_last):
    """Inertia correction: delta_w = 0, then 1e-4 (or delta_last/3) x 8 until PD."""
    out = step_fn(0.0)
    if out[-1]:
        return out, 0.0
    d = 1e-4 if delta_last == 0.0 else max(1e-20, delta_last / 3.0)
    while d < 1e40:
        out = step_fn(d)
        if out[-1]:
            return out, d
        d *= 8.0
    raise RuntimeError("inertia correction failed")


def _filter_search(lay, bw, bs, filt, G, A, W, sig_w, sig_s, r, nu, w, s, zwl, zwu, zsl, zsu, mu, tau,
                   pw, ps, plam, py, delta, theta_min, stats, restoration=False):
    """Filter line search with second-order corrections along the condensed
    step (Wachter and Biegler 2006, Algorithm A, steps A-5 to A-8).  theta is the
    l1 norm of c = [g; h + s], phi the barrier objective.  When the step length
    falls below alpha_min the step is shortened by a larger primal
    regularization and the search starts again, unless restoration is on:
    then the search gives up at once and returns None, and the caller runs the
    feasibility restoration phase.  Returns the primal-dual step, its primal
    and bound-multiplier lengths, the bound-multiplier steps and the delta_w in
    use."""
    nw, m = lay.nw, lay.m

    def cons(wt, st):
        return np.concatenate([model.cons_g(lay, wt), model.cons_h(lay, wt) + st])

    def phi(wt, st):
        return model.objective(lay, wt) + bw.barrier(wt, mu) + bs.barrier(st, mu)

    gf = model.jacobians(lay, w)[0]
    c0 = cons(w, s)
    theta0, phi0 = np.abs(c0).sum(), phi(w, s)
    for attempt in range(40):
        dphi = (gf + bw.barrier_grad(w, mu)) @ pw + bs.barrier_grad(s, mu) @ ps
        amax = min(bw.max_step(w, pw, tau), bs.max_step(s, ps, tau))
        amin = filter_alpha_min(theta0, dphi, theta_min)
        a, accepted, phi_type, pw_acc, ps_acc = amax, False, False, pw, ps
        while a >= amin and not accepted:
            wt, st = w + a * pw, s + a * ps
            ct = cons(wt, st)
            theta_t, phi_t = np.abs(ct).sum(), phi(wt, st)
            accepted, phi_type = filter_accepts(filt, theta0, phi0, dphi, a, theta_t, phi_t, theta_min)
            if not accepted and a == amax and theta_t >= theta0:
                # second-order corrections: the constraint part of the right-hand
                # side becomes c_soc = a c(x) + c(x + a d), accumulated
                c_soc, theta_prev = a * c0 + ct, theta0
                for _ in range(SOC_MAX):
                    r_soc = r.copy()
                    r_soc[nw + m:] = c_soc
                    qw, qs, _, _, _, ok = kkt.condensed_step(G, A, W, sig_w, sig_s, r_soc, nu, delta_w=delta)
                    if not ok:
                        break
                    a_soc = min(bw.max_step(w, qw, tau), bs.max_step(s, qs, tau))
                    w_soc, s_soc = w + a_soc * qw, s + a_soc * qs
                    c_new = cons(w_soc, s_soc)
                    theta_soc, phi_soc = np.abs(c_new).sum(), phi(w_soc, s_soc)
                    accepted, phi_type = filter_accepts(filt, theta0, phi0, dphi, a, theta_soc, phi_soc, theta_min)
                    if accepted:
                        pw_acc, ps_acc = a_soc * qw / a, a_soc * qs / a   # so that w + a pw_acc = w_soc
                        stats["soc"] += 1
                        break
                    if theta_soc > KAPPA_SOC * theta_prev:
                        break
                    theta_prev, c_soc = theta_soc, a_soc * c_soc + c_new
            if not accepted:
                a *= 0.5
        if accepted:
            if not phi_type:
                filt.add((1.0 - GAMMA_THETA) * theta0, phi0 - GAMMA_PHI * theta0)
            dzwl, dzwu = bw.dz(w, zwl, zwu, pw, mu)
            dzsl, dzsu = bs.dz(s, zsl, zsu, ps, mu)
            az = min(_max_step_z(zwl, dzwl, bw.fl, tau), _max_step_z(zwu, dzwu, bw.fu, tau),
                     _max_step_z(zsl, dzsl, bs.fl, tau), _max_step_z(zsu, dzsu, bs.fu, tau))
            return pw_acc, ps_acc, plam, py, a, az, dzwl, dzwu, dzsl, dzsu, delta
        if restoration:
            # out of step length: the current point goes into the filter and the
            # restoration phase takes over (Algorithm A, step A-9)
            filt.add(theta0, phi0)
            return None
        # out of step length: shorten the step by a larger primal regularization
        delta = max(1e-8, 10.0 * delta)
        pw, ps, plam, py, Kc, ok = kkt.condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=delta)
        if not ok:
            (pw, ps, plam, py, Kc, ok), delta = _regularized(
                lambda d: kkt.condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=d), delta)
    raise RuntimeError("filter line search failed")


def _restoration(lay, bw, bs, filt, w, s, mu, tol, stats, verbose=False):
    """Feasibility restoration phase (Wachter and Biegler 2006, Sec. 3.3) with
    the relaxation restricted to the inequality rows, as Sec. 4.3 describes for
    LinRed: the equality rows g(w) = 0 stay exact (so G_x and the reduction
    are unchanged) and each row of h + s = 0 gets two nonnegative variables,

        min  rho sum(p + n) + zeta/2 ||D_R (w - w_R)||^2
        s.t. g(w) = 0,  h(w) + s - p + n = 0,  bounds on w and s,  p, n >= 0,

    zeta = sqrt(mu), D_R = diag(min(1, 1/|w_R|)).  Its barrier Newton step is the
    condensed step of the same K_aug with W replaced by the Hessian of the
    constraint terms plus zeta D_R^2, and -delta I in the (p_y, p_y) block with
    delta_i = 1/Sigma_p,i + 1/Sigma_n,i: eliminating dp and dn folds the
    relaxation into a dual regularisation of the inequality rows.  Steps are
    accepted by backtracking on the l1 merit of the restoration barrier
    problem.  The phase ends at the first point whose violation theta of
    [g; h + s] is at most kappa theta(w_R, s_R) and that the original filter
    accepts (the current point was added to it before the call).
    Returns (w, s, lam, y, zwl, zwu, zsl, zsu) for the main loop or raises."""
    nu, nx, m, nw = lay.nu, lay.nx, lay.m, lay.nw

    def cons(wt, st):
        return np.concatenate([model.cons_g(lay, wt), model.cons_h(lay, wt) + st])

    def phi_main(wt, st):
        return model.objective(lay, wt) + bw.barrier(wt, mu) + bs.barrier(st, mu)

    theta_R = np.abs(cons(w, s)).sum()
    wR = w.copy()
    zeta = np.sqrt(mu)
    dr2 = np.minimum(1.0, 1.0 / np.maximum(np.abs(wR), 1e-300)) ** 2
    rho = RHO_RESTO
    c = model.cons_h(lay, w) + s
    mur = max(mu, np.abs(cons(w, s)).max())
    # p and n minimising the relaxed barrier terms for the current c (closed form)
    t = (mur - rho * c) / (2.0 * rho)
    n = t + np.sqrt(t * t + mur * c / (2.0 * rho))
    p = c + n
    zp, zn = mur / p, mur / n
    lam, y = np.zeros(nx), np.zeros(m)
    zwl, zwu = np.where(bw.fl, mur / bw.dl(w), 0.0), np.where(bw.fu, mur / bw.du(w), 0.0)
    zsl, zsu = np.where(bs.fl, mur / bs.dl(s), 0.0), np.where(bs.fu, mur / bs.du(s), 0.0)
    nu_pen = 1.0
    delta = 0.0
    for it in range(RESTO_MAX_ITER):
        gf, G, A = model.jacobians(lay, w)
        g = model.cons_g(lay, w)
        hv = model.cons_h(lay, w)
        Wc = (model.lagrangian_hessian(lay, w, lam, y) - model.lagrangian_hessian(lay, w, 0.0 * lam, 0.0 * y)
              + sp.diags(zeta * dr2))
        sig_w = bw.sigma(w, zwl, zwu)
        sig_s = bs.sigma(s, zsl, zsu)
        sp_, sn_ = zp / p, zn / n
        dcv = 1.0 / sp_ + 1.0 / sn_
        r_w = zeta * dr2 * (w - wR) + G.T @ lam + A.T @ y + bw.barrier_grad(w, mur)
        r_s = y + bs.barrier_grad(s, mur)
        r_y = hv + s - p + n
        r_p = rho - y - mur / p
        r_n = rho + y - mur / n
        r = np.concatenate([r_w, r_s, g, r_y + r_p / sp_ - r_n / sn_])
        (pw, ps, plam, py, Kc, ok), delta = _regularized(
            lambda d: kkt.condensed_step(G, A, Wc, sig_w, sig_s, r, nu, delta_w=d, delta_c=dcv), delta)
        pp = (py - r_p) / sp_
        pn = (-py - r_n) / sn_
        tau = max(TAU_MIN, 1.0 - mur)
        amax = min(bw.max_step(w, pw, tau), bs.max_step(s, ps, tau))
        for v, dv in ((p, pp), (n, pn)):
            neg = dv < 0
            if neg.any():
                amax = min(amax, np.min(-tau * v[neg] / dv[neg]))
        dzwl, dzwu = bw.dz(w, zwl, zwu, pw, mur)
        dzsl, dzsu = bs.dz(s, zsl, zsu, ps, mur)
        dzp = mur / p - zp - sp_ * pp
        dzn = mur / n - zn - sn_ * pn
        ones = np.ones(m, bool)
        az = min(_max_step_z(zwl, dzwl, bw.fl, tau), _max_step_z(zwu, dzwu, bw.fu, tau),
                 _max_step_z(zsl, dzsl, bs.fl, tau), _max_step_z(zsu, dzsu, bs.fu, tau),
                 _max_step_z(zp, dzp, ones, tau), _max_step_z(zn, dzn, ones, tau))
        nu_pen = max(nu_pen, 1.1 * max(np.abs(lam + plam).max(initial=0), np.abs(y + py).max(initial=0)))

        def merit(wt, st, pt, nt):
            cr = np.concatenate([model.cons_g(lay, wt), model.cons_h(lay, wt) + st - pt + nt])
            return (rho * np.sum(pt + nt) + 0.5 * zeta * np.sum(dr2 * (wt - wR) ** 2) + bw.barrier(wt, mur)
                    + bs.barrier(st, mur) - mur * np.sum(np.log(pt) + np.log(nt)) + nu_pen * np.abs(cr).sum())
        psi0 = merit(w, s, p, n)
        dpsi = (rho * np.sum(pp + pn) + zeta * np.sum(dr2 * (w - wR) * pw) + bw.barrier_grad(w, mur) @ pw
                + bs.barrier_grad(s, mur) @ ps - mur * np.sum(pp / p + pn / n)
                - nu_pen * np.abs(np.concatenate([g, r_y])).sum())
        a = amax
        while a > 1e-8 * amax and not (merit(w + a * pw, s + a * ps, p + a * pp, n + a * pn)
                                       <= psi0 + ETA * a * min(dpsi, 0.0)):
            a *= 0.5
        w, s, p, n = w + a * pw, s + a * ps, p + a * pp, n + a * pn
        lam, y = lam + a * plam, y + a * py
        zwl, zwu = bw.safeguard(w, zwl + az * dzwl, zwu + az * dzwu, mur)
        zsl, zsu = bs.safeguard(s, zsl + az * dzsl, zsu + az * dzsu, mur)
        zp = np.clip(zp + az * dzp, mur / (KAPPA_SIGMA * p), KAPPA_SIGMA * mur / p)
        zn = np.clip(zn + az * dzn, mur / (KAPPA_SIGMA * n), KAPPA_SIGMA * mur / n)
        theta = np.abs(cons(w, s)).sum()
        if verbose:
            print(f"  resto it {it:3d} theta {theta:.3e} (theta_R {theta_R:.3e}) mu_R {mur:.1e} a {a:.2e}")
        stats["resto_iters"] = stats.get("resto_iters", 0) + 1
        if theta <= KAPPA_RESTO * theta_R and filt.acceptable(theta, phi_main(w, s)):
            return w, s, lam, y, zwl, zwu, zsl, zsu
        # the restoration problem's own barrier parameter
        dual = np.concatenate([r_w, r_s, r_p, r_n])
        if np.abs(dual).max() <= KAPPA_EPS * mur and np.abs(np.concatenate([g, r_y])).max() <= KAPPA_EPS * mur:
            mur = max(0.1 * mu, min(KAPPA_MU * mur, mur ** THETA_MU))
    raise RuntimeError("feasibility restoration failed")


# ------------------------------------------------------------------ LinRed
def linred(net, tol=1e-8, max_iter=300, mu0=0.1, record_at=None, verbose=False, line_search="merit",
           restoration=False, start_with_resto=False):
    """Algorithm 1.  record_at: iteration index whose iterate (and the step
    inputs) is stored in Result.history as a dict.  line_search: "merit"
    (l1 exact-penalty backtracking) or "filter" (filter line search with
    second-order corrections); with the filter, restoration=True runs the
    feasibility restoration phase when the step length runs out (otherwise a
    larger primal regularisation shortens the step), and start_with_resto=True
    (Ipopt's option of that name) runs it once from the starting point before
    the first step."""
    lay = model.Layout(net)
    nu, nx, m, nw = lay.nu, lay.nx, lay.m, lay.nw
    bw = _Bounds(lay.wl, lay.wu)
    bs = _Bounds(-lay.hu, -lay.hl)
    w = _push(lay.flat_start(), lay.wl, lay.wu)
    s = _push(-model.cons_h(lay, w), bs.lo, bs.hi)
    lam = np.zeros(nx)
    y = np.zeros(m)
    zwl, zwu = bw.fl.astype(float), bw.fu.astype(float)
    zsl, zsu = bs.fl.astype(float), bs.fu.astype(float)
    mu = mu0
    nu_pen = 1.0
    delta = 0.0
    hist = []
    theta_init = np.abs(model.cons_g(lay, w)).sum() + np.abs(model.cons_h(lay, w) + s).sum()
    theta_max = 1e4 * max(1.0, theta_init)
    theta_min = 1e-4 * max(1.0, theta_init)
    filt, filt_mu = None, None
    stats = {"soc": 0}
    for it in range(max_iter + 1):
        gf, G, A = model.jacobians(lay, w)
        g = model.cons_g(lay, w)
        h = model.cons_h(lay, w)
        grad_w = gf + G.T @ lam + A.T @ y
        dual_w = grad_w - zwl + zwu
        dual_s = y - zsl + zsu
        primal = np.concatenate([g, h + s])
        mults = [lam, y, zwl[bw.fl], zwu[bw.fu], zsl[bs.fl], zsu[bs.fu]]
        err0 = _opt_error(np.concatenate([dual_w, dual_s]), primal,
                          np.concatenate([bw.compl(w, zwl, zwu, 0.0), bs.compl(s, zsl, zsu, 0.0)]), mults)
        if verbose:
            print(f"it {it:3d} obj {model.objective(lay, w):.10f} err {err0:.2e} mu {mu:.1e} "
                  f"inf_pr {np.abs(primal).max():.2e} delta {delta:.1e}")
        if err0 <= tol:
            return Result("converged", it, float(model.objective(lay, w)), w, s, lam, y,
                          (zwl, zsl), (zwu, zsu), mu, err=err0, history=hist, soc_steps=stats["soc"],
                          restorations=stats.get("restorations", 0))
        if it == max_iter:
            break
        while True:
            errmu = _opt_error(np.concatenate([dual_w, dual_s]), primal,
                               np.concatenate([bw.compl(w, zwl, zwu, mu), bs.compl(s, zsl, zsu, mu)]), mults)
            if errmu > KAPPA_EPS * mu or mu <= tol / 10:
                break
            mu = max(tol / 10, min(KAPPA_MU * mu, mu ** THETA_MU))
        tau = max(TAU_MIN, 1.0 - mu)
        if line_search == "filter" and restoration and start_with_resto and it == 0:
            # the restoration phase from the starting point, before any step
            filt, filt_mu = Filter(theta_max), mu
            filt.add(np.abs(primal).sum(), model.objective(lay, w) + bw.barrier(w, mu) + bs.barrier(s, mu))
            w, s, lam, y, zwl, zwu, zsl, zsu = _restoration(lay, bw, bs, filt, w, s, mu, tol, stats, verbose)
            stats["restorations"] = stats.get("restorations", 0) + 1
            continue
        W = model.lagrangian_hessian(lay, w, lam, y)
        sig_w = bw.sigma(w, zwl, zwu)
        sig_s = bs.sigma(s, zsl, zsu)
        r = np.concatenate([grad_w + bw.barrier_grad(w, mu), y + bs.barrier_grad(s, mu), g, h + s])
        (pw, ps, plam, py, Kc, ok), delta = _regularized(
            lambda d: kkt.condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=d), delta)
        if record_at is not None and it == record_at:
            hist.append(dict(it=it, w=w.copy(), s=s.copy(), lam=lam.copy(), y=y.copy(),
                             sig_w=sig_w.copy(), sig_s=sig_s.copy(), r=r.copy(), mu=mu,
                             delta=delta, pw=pw, ps=ps, plam=plam, py=py, Kc=Kc))
        phi0 = None
        if line_search == "filter":
            if filt is None or filt_mu != mu:      # a new barrier problem: a new filter
                filt, filt_mu = Filter(theta_max), mu

            res = _filter_search(
                lay, bw, bs, filt, G, A, W, sig_w, sig_s, r, nu, w, s, zwl, zwu, zsl, zsu, mu, tau,
                pw, ps, plam, py, delta, theta_min, stats, restoration)
            if res is None:
                w, s, lam, y, zwl, zwu, zsl, zsu = _restoration(lay, bw, bs, filt, w, s, mu, tol, stats, verbose)
                stats["restorations"] = stats.get("restorations", 0) + 1
                continue
            pw, ps, plam, py, a, az, dzwl, dzwu, dzsl, dzsu, delta = res
        for attempt in range(40 if line_search == "merit" else 0):
            dzwl, dzwu = bw.dz(w, zwl, zwu, pw, mu)
            dzsl, dzsu = bs.dz(s, zsl, zsu, ps, mu)
            amax = min(bw.max_step(w, pw, tau), bs.max_step(s, ps, tau))
            az = min(_max_step_z(zwl, dzwl, bw.fl, tau), _max_step_z(zwu, dzwu, bw.fu, tau),
                     _max_step_z(zsl, dzsl, bs.fl, tau), _max_step_z(zsu, dzsu, bs.fu, tau))
            # l1 merit  phi = f + barrier + nu ||c||_1
            nu_pen = max(nu_pen, 1.1 * max(np.abs(lam + plam).max(initial=0), np.abs(y + py).max(initial=0)))

            def merit(wt, st):
                c = np.concatenate([model.cons_g(lay, wt), model.cons_h(lay, wt) + st])
                return model.objective(lay, wt) + bw.barrier(wt, mu) + bs.barrier(st, mu) + nu_pen * np.abs(c).sum()
            phi0 = merit(w, s)
            dphi = (gf + bw.barrier_grad(w, mu)) @ pw + bs.barrier_grad(s, mu) @ ps - nu_pen * np.abs(primal).sum()
            a = amax
            while a > 1e-4 * amax:
                if merit(w + a * pw, s + a * ps) <= phi0 + ETA * a * min(dphi, 0.0):
                    break
                a *= 0.5
            if verbose:
                print(f"    amax {amax:.2e} a {a:.2e} dphi {dphi:.3e} |pw| {np.abs(pw).max():.2e}")
            if a > 1e-4 * amax:
                break
            # backtracking failed: shorten the step by a larger primal regularization
            delta = max(1e-8, 10.0 * delta)
            pw, ps, plam, py, Kc, ok = kkt.condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=delta)
            if not ok:
                (pw, ps, plam, py, Kc, ok), delta = _regularized(
                    lambda d: kkt.condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=d), delta)
        w = w + a * pw
        s = s + a * ps
        lam = lam + a * plam
        y = y + a * py
        zwl, zwu = zwl + az * dzwl, zwu + az * dzwu
        zsl, zsu = zsl + az * dzsl, zsu + az * dzsu
        zwl, zwu = bw.safeguard(w, zwl, zwu, mu)
        zsl, zsu = bs.safeguard(s, zsl, zsu, mu)
    return Result("max_iter", max_iter, float(model.objective(lay, w)), w, s, lam, y,
                  (zwl, zsl), (zwu, zsu), mu, err=err0, history=hist)


# ------------------------------------------------------------------ RedLin
def newton_projection(lay, w, tol=1e-10, max_iter=30):
    """Solve g(x, u) = 0 for x at fixed u by Newton-Raphson (Sec. 4.4).
    Returns (w with projected x, iterations, converged)."""
    w = w.copy()
    nu = lay.nu
    import scipy.sparse.linalg as spla
    for k in range(max_iter + 1):
        g = model.cons_g(lay, w)
        if np.abs(g).max() <= tol:
            return w, k, True
        if k == max_iter or not np.all(np.isfinite(g)):
            break
        _, G, _ = model.jacobians(lay, w)
        dx = spla.splu(G[:, nu:].tocsc()).solve(-g)
        w[nu:] += dx
    return w, max_iter, False


def redlin(net, tol=1e-8, max_iter=300, mu0=0.1, verbose=False, record_at=None):
    """Algorithm 2.  State bounds (Vm at load buses) become rows -x_b of h_r."""
    lay = model.Layout(net)
    nu, nx, m = lay.nu, lay.nx, lay.m
    xb = np.nonzero(np.isfinite(lay.wl[nu:]))[0]           # bounded states
    nb_ = len(xb)
    mr = m + nb_
    bu = _Bounds(lay.wl[:nu], lay.wu[:nu])
    bs = _Bounds(np.concatenate([-lay.hu, lay.wl[nu:][xb]]),
                 np.concatenate([-lay.hl, lay.wu[nu:][xb]]))
    w = _push(lay.flat_start(), lay.wl, lay.wu)
    w, _, ok = newton_projection(lay, w)
    if not ok:
        raise RuntimeError("initial power flow failed")

    def hr(wt):
        return np.concatenate([model.cons_h(lay, wt), -wt[nu:][xb]])

    s = _push(-hr(w), bs.lo, bs.hi)
    y = np.zeros(mr)
    zul, zuu = bu.fl.astype(float), bu.fu.astype(float)
    zsl, zsu = bs.fl.astype(float), bs.fu.astype(float)
    mu = mu0
    nu_pen = 1.0
    delta = 0.0
    hist = []
    import scipy.sparse as sp
    Eb = sp.coo_matrix((-np.ones(nb_), (np.arange(nb_), xb)), shape=(nb_, nx)).tocsr()
    for it in range(max_iter + 1):
        gf, G, A = model.jacobians(lay, w)
        blk = kkt.split_blocks(G, A, sp.csr_matrix((lay.nw, lay.nw)), nu)
        _, solveT = kkt._gx_solver(blk["Gx"])
        yh, yb = y[:m], y[m:]
        # adjoint step: lambda = -G_x^{-T} grad_x L
        lam = -solveT(gf[nu:] + blk["Ax"].T @ yh + Eb.T @ yb)
        grad_u = gf[:nu] + blk["Gu"].T @ lam + blk["Au"].T @ yh
        dual_u = grad_u - zul + zuu
        dual_s = y - zsl + zsu
        primal = hr(w) + s
        mults = [y, zul[bu.fl], zuu[bu.fu], zsl[bs.fl], zsu[bs.fu]]
        err0 = _opt_error(np.concatenate([dual_u, dual_s]), primal,
                          np.concatenate([bu.compl(w[:nu], zul, zuu, 0.0), bs.compl(s, zsl, zsu, 0.0)]), mults)
        if verbose:
            print(f"it {it:3d} obj {model.objective(lay, w):.10f} err {err0:.2e} mu {mu:.1e} delta {delta:.1e}")
        if err0 <= tol:
            return Result("converged", it, float(model.objective(lay, w)), w, s, lam, y,
                          (zul, zsl), (zuu, zsu), mu, err=err0, history=hist)
        if it == max_iter:
            break
        while True:
            errmu = _opt_error(np.concatenate([dual_u, dual_s]), primal,
                               np.concatenate([bu.compl(w[:nu], zul, zuu, mu), bs.compl(s, zsl, zsu, mu)]), mults)
            if errmu > KAPPA_EPS * mu or mu <= tol / 10:
                break
            mu = max(tol / 10, min(KAPPA_MU * mu, mu ** THETA_MU))
        tau = max(TAU_MIN, 1.0 - mu)
        W = model.lagrangian_hessian(lay, w, lam, yh)
        Ar = sp.vstack([A, sp.hstack([sp.csr_matrix((nb_, nu)), Eb])]).tocsr()
        sig_u = bu.sigma(w[:nu], zul, zuu)
        sig_s = bs.sigma(s, zsl, zsu)
        r1 = grad_u + bu.barrier_grad(w[:nu], mu)
        r2 = y + bs.barrier_grad(s, mu)
        r3 = primal

        def step(d):
            # Eq. reduced:kktsystem condensed by Theorem 2; W_hat without Sigma_x
            sig_w = np.concatenate([sig_u, np.zeros(nx)])
            W_hat, A_hat, _, _, _ = kkt.reduced_blocks(G, Ar, W, sig_w, nu)
            Kc = W_hat + np.diag(sig_u) + A_hat.T @ (sig_s[:, None] * A_hat) + d * np.eye(nu)
            try:
                L = np.linalg.cholesky(Kc)
            except np.linalg.LinAlgError:
                return None, None, None, Kc, False
            import scipy.linalg as sla
            rhs = -(r1 + A_hat.T @ (sig_s * r3) - A_hat.T @ r2)
            pu = sla.cho_solve((L, True), rhs)
            py = sig_s * (A_hat @ pu + r3) - r2
            ps = -(A_hat @ pu + r3)
            return pu, ps, py, Kc, True
        (pu, ps, py, Kc, ok), delta = _regularized(step, delta)
        if record_at is not None and it == record_at:
            hist.append(dict(it=it, w=w.copy(), s=s.copy(), lam=lam.copy(), y=y.copy(),
                             sig_u=sig_u.copy(), sig_s=sig_s.copy(), mu=mu, delta=delta,
                             pu=pu, ps=ps, py=py, Kc=Kc))
        dzul, dzuu = bu.dz(w[:nu], zul, zuu, pu, mu)
        dzsl, dzsu = bs.dz(s, zsl, zsu, ps, mu)
        amax = min(bu.max_step(w[:nu], pu, tau), bs.max_step(s, ps, tau))
        az = min(_max_step_z(zul, dzul, bu.fl, tau), _max_step_z(zuu, dzuu, bu.fu, tau),
                 _max_step_z(zsl, dzsl, bs.fl, tau), _max_step_z(zsu, dzsu, bs.fu, tau))
        nu_pen = max(nu_pen, 1.1 * np.abs(y + py).max(initial=0))

        def merit(wt, st):
            return (model.objective(lay, wt) + bu.barrier(wt[:nu], mu) + bs.barrier(st, mu)
                    + nu_pen * np.abs(hr(wt) + st).sum())
        phi0 = merit(w, s)
        # directional derivative of f_r along p_u: grad f_r = g_u - G_u^T G_x^{-T} g_x
        gfr = gf[:nu] - blk["Gu"].T @ solveT(gf[nu:])
        dphi = (gfr + bu.barrier_grad(w[:nu], mu)) @ pu + bs.barrier_grad(s, mu) @ ps \
            - nu_pen * np.abs(primal).sum()
        a = amax
        wn = None
        while a > 1e-12:
            wt = w.copy()
            wt[:nu] += a * pu
            wt, _, okp = newton_projection(lay, wt)
            if okp and merit(wt, s + a * ps) <= phi0 + ETA * a * min(dphi, 0.0):
                wn = wt
                break
            a *= 0.5
        if wn is None:
            return Result("line_search_failed", it, float(model.objective(lay, w)), w, s, lam, y,
                          (zul, zsl), (zuu, zsu), mu, err=err0, history=hist)
        w = wn
        s = s + a * ps
        y = y + a * py
        zul, zuu = zul + az * dzul, zuu + az * dzuu
        zsl, zsu = zsl + az * dzsl, zsu + az * dzsu
        zul, zuu = bu.safeguard(w[:nu], zul, zuu, mu)
        zsl, zsu = bs.safeguard(s, zsl, zsu, mu)
    return Result("max_iter", max_iter, float(model.objective(lay, w)), w, s, None, y,
                  (zul, zsl), (zuu, zsu), mu, err=err0, history=hist)
