"""Augmented, reduced and condensed KKT systems -- oracle side (test infrastructure).

Sign convention.  The slack form is h(x,u) + s = 0 (Eq. 3) and the
Lagrangian carries + y^T (h + s) (Eq. 4), so the blocks coupling p_s and p_y
in the augmented matrix are +I.  The printed matrices (Eq. kktmatrix:original
and kktmatrix:normal) show -I there, which corresponds to h - s = 0 instead.
The condensed matrix is unaffected (Sigma_s enters as (+-I) Sigma_s (+-I)),
and so are the right-hand side of Eq. kktmatrix:condensed and the p_y
recovery; the slack recovery becomes p_s = -(A_hat_u p_u + r_hat_3).

Sigma_u is kept in the condensed matrix (it appears in K_red of Theorem 1 and
is dropped in the statement of Theorem 2), and K in Eq. algo:reduction is read
as W + diag(Sigma_u, Sigma_x) + A^T Sigma_s A.

Dual regularisation.  The paper regularises until the condensed matrix is
positive definite (Sec. 4.3) without placing the terms.  The reading here: the
primal term delta_w sits on the u block (K_cond + delta_w I), and the dual term
delta_c sits on the inequality rows only, as -delta_c I in the (p_y, p_y) block
of K_aug (the equality rows of G stay exact, so the reduction on G_x is
unchanged).  Eliminating p_s and p_y then replaces Sigma_s by
Sigma_t = (Sigma_s^{-1} + delta_c)^{-1} in the condensed matrix.

All vectors over the primal variables are ordered w = [u; x].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _dense(M):
    return M.toarray() if sp.issparse(M) else np.asarray(M)


def split_blocks(G, A, W, nu):
    """Blocks of Sec. 2.1: G = [G_u G_x], A = [A_u A_x], W = [[W_uu W_ux],[W_xu W_xx]]."""
    G = sp.csr_matrix(G)
    A = sp.csr_matrix(A)
    W = sp.csr_matrix(W)
    return dict(Gu=G[:, :nu], Gx=G[:, nu:], Au=A[:, :nu], Ax=A[:, nu:],
                Wuu=W[:nu, :nu], Wux=W[:nu, nu:], Wxu=W[nu:, :nu], Wxx=W[nu:, nu:])


def kaug(G, A, W, sig_w, sig_s, delta_c=0.0):
    """K_aug of Eq. kktmatrix:normal (sparse), unknowns [p_w, p_s, p_lambda, p_y]
    with p_w = [p_u; p_x] and the +I slack coupling; delta_c > 0 puts
    -delta_c I in the (p_y, p_y) block (dual regularisation of the
    inequalities, Sec. 4.3); delta_c may also be one value per inequality row
    (the restoration phase's relaxation, oracle/ipm.py)."""
    G = sp.csr_matrix(G)
    A = sp.csr_matrix(A)
    W = sp.csr_matrix(W)
    nx, nw = G.shape
    m = A.shape[0]
    I = sp.identity(m, format="csr")
    dc = np.broadcast_to(np.asarray(delta_c, dtype=np.float64), (m,))
    Dyy = sp.diags(-dc, format="csr") if np.any(dc) else None
    return sp.bmat([
        [W + sp.diags(sig_w), None, G.T, A.T],
        [None, sp.diags(sig_s), None, I],
        [G, None, None, None],
        [A, I, None, Dyy],
    ], format="csc")


def full_space_step(G, A, W, sig_w, sig_s, r, delta_c=0.0):
    """Newton step p solving K_aug p = -r, r = [r1; r2; r3; r4; r5] with
    r1, r2 over w = [u; x].  Returns (p_w, p_s, p_lambda, p_y)."""
    K = kaug(G, A, W, sig_w, sig_s, delta_c)
    nx, nw = G.shape
    m = A.shape[0]
    if K.shape[0] <= 1500:
        p = np.linalg.solve(K.toarray(), -r)
    else:
        p = spla.splu(K).solve(-r)
    return p[:nw], p[nw:nw + m], p[nw + m:nw + m + nx], p[nw + m + nx:]


def inertia_dense(M):
    """(n+, n-, n0) of a symmetric matrix from its LDL^T factor (Sylvester's law)."""
    M = _dense(M)
    _, D, _ = sla.ldl(M)
    ev = np.linalg.eigvalsh(D)           # D is block diagonal (1x1 / 2x2)
    tol = 1e-12 * max(1.0, np.abs(ev).max())
    return int((ev > tol).sum()), int((ev < -tol).sum()), int((np.abs(ev) <= tol).sum())


def _gx_solver(Gx):
    Gx = sp.csc_matrix(Gx)
    if Gx.shape[0] <= 600:
        lu = sla.lu_factor(Gx.toarray())
        return (lambda B: sla.lu_solve(lu, B)), (lambda B: sla.lu_solve(lu, B, trans=1))
    lu = spla.splu(Gx)
    return (lambda B: lu.solve(np.asarray(B))), (lambda B: lu.solve(np.asarray(B), trans="T"))


def sensitivity(G, nu):
    """S_x = -G_x^{-1} G_u (the dense sensitivity matrix of Sec. 3.3), nx x nu."""
    b = split_blocks(G, sp.csr_matrix((G.shape[0], G.shape[0])), sp.csr_matrix((G.shape[1],) * 2), nu)
    solve, _ = _gx_solver(b["Gx"])
    return -solve(b["Gu"].toarray())


def regularized_sigma(sig_s, delta_c):
    """Sigma_t = (Sigma_s^{-1} + delta_c)^{-1}: the weight the inequality rows
    carry into the condensed matrix once -delta_c I sits in the (p_y, p_y)
    block of K_aug (written without forming Sigma_s^{-1})."""
    sig_s = np.asarray(sig_s, dtype=np.float64)
    return sig_s / (1.0 + delta_c * sig_s)


def reduced_gradient(G, grad_w, nu):
    """Reduced gradient of Eq. reduced:derivatives (Sec. 2.3) for any gradient
    grad_w = [grad_u; grad_x] over w = [u; x]:
        grad_r = grad_u - G_u^T G_x^{-T} grad_x = grad_u + G_u^T lam,
        lam = -G_x^{-T} grad_x (the adjoint step of Algorithm 2).
    Returns (grad_r, lam)."""
    G = sp.csr_matrix(G)
    _, solveT = _gx_solver(G[:, nu:])
    lam = -solveT(np.asarray(grad_w[nu:], dtype=np.float64))
    return grad_w[:nu] + G[:, :nu].T @ lam, lam


def kred_definition(G, A, W, sig_w, sig_s, nu, Sx=None):
    """K_hat_uu = Z^T (W + diag(Sigma_w) + A^T Sigma_s A) Z,  Z = [I; -G_x^{-1} G_u]
    (Eq. algo:reduction).  Dense nu x nu."""
    if Sx is None:
        Sx = sensitivity(G, nu)
    A = sp.csr_matrix(A)
    K = sp.csr_matrix(W) + sp.diags(sig_w) + A.T @ sp.diags(sig_s) @ A
    Z = np.vstack([np.eye(nu), Sx])
    return Z.T @ (K @ Z)


def reduced_blocks(G, A, W, sig_w, nu):
    """W_hat_uu and A_hat_u of Theorem 1 (with Sigma_x inside W_hat_uu)."""
    b = split_blocks(G, A, W, nu)
    solve, solveT = _gx_solver(b["Gx"])
    GxiGu = solve(b["Gu"].toarray())                  # G_x^{-1} G_u
    sx = sig_w[nu:]
    Wxx = b["Wxx"] + sp.diags(sx)
    Wuu = b["Wuu"].toarray()
    Wux = b["Wux"].toarray()
    Wxu = b["Wxu"].toarray()
    W_hat = (Wuu - Wux @ GxiGu - GxiGu.T @ Wxu + GxiGu.T @ (Wxx @ GxiGu))
    A_hat = b["Au"].toarray() - b["Ax"] @ GxiGu
    return W_hat, A_hat, GxiGu, (solve, solveT), b


def condensed_step(G, A, W, sig_w, sig_s, r, nu, delta_w=0.0, delta_c=0.0):
    """Newton step through Theorem 1 (reduce on G_x) then Theorem 2 (condense on
    Sigma_s), in the paper's notation.  Returns (p_w, p_s, p_lambda, p_y, K_cond,
    chol_ok).  delta_w is added to K_cond (primal regularization on u);
    delta_c > 0 is the dual regularization -delta_c I on the (p_y, p_y) block
    of K_aug, which Theorem 2's elimination of p_s and p_y turns into
    Sigma_t = (Sigma_s^{-1} + delta_c)^{-1} in place of Sigma_s."""
    nx = G.shape[0]
    m = A.shape[0]
    nw = nu + nx
    r1, r2 = r[:nu], r[nu:nw]
    r3 = r[nw:nw + m]
    r4 = r[nw + m:nw + m + nx]
    r5 = r[nw + m + nx:]
    W_hat, A_hat, GxiGu, (solve, solveT), b = reduced_blocks(G, A, W, sig_w, nu)
    su, sx = sig_w[:nu], sig_w[nu:]
    Wxx_s = b["Wxx"] + sp.diags(sx)
    # Theorem 1 right-hand sides
    Gxi_r4 = solve(r4)
    r1h = (r1 - b["Gu"].T @ solveT(r2)
           - (b["Wux"] @ Gxi_r4 - b["Gu"].T @ solveT(Wxx_s @ Gxi_r4)))
    r2h = r3
    r3h = r5 - b["Ax"] @ Gxi_r4
    # Theorem 2: condensed system.  The slack row gives p_s = -Sigma_s^{-1}(p_y + r2h);
    # with it the inequality row A_hat p_u + p_s - delta_c p_y = -r3h gives
    # p_y = Sigma_t (A_hat p_u + r3h - Sigma_s^{-1} r2h), and p_s follows from
    # that same row.
    sig_t = regularized_sigma(sig_s, delta_c)
    Kc = W_hat + np.diag(su) + A_hat.T @ (sig_t[:, None] * A_hat)
    Kc = Kc + delta_w * np.eye(nu)
    rhs = -(r1h + A_hat.T @ (sig_t * r3h) - A_hat.T @ (sig_t / sig_s * r2h))
    try:
        L = np.linalg.cholesky(Kc)
    except np.linalg.LinAlgError:
        return None, None, None, None, Kc, False
    pu = sla.cho_solve((L, True), rhs)
    py = sig_t * (A_hat @ pu + r3h - r2h / sig_s)
    ps = -(A_hat @ pu + r3h) + delta_c * py
    px = -solve(r4 + b["Gu"] @ pu)
    plam = -solveT(r2 + b["Ax"].T @ py + b["Wxu"] @ pu + Wxx_s @ px)
    return np.concatenate([pu, px]), ps, plam, py, Kc, True
