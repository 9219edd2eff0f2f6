"""The augmented system of the hybrid full-space IPM -- oracle side (test
infrastructure; only tests, the smoke check and the benchmark's CPU legs use it).

The hybrid full-space IPM of Sec. 4.3 runs the same interior-point loop as
LinRed but solves the augmented KKT system of Eq. kktmatrix:normal directly,
with a sparse symmetric-indefinite factorisation (MA27 in the paper) in place
of the reduction and the dense Cholesky.  With the slack step eliminated
(p_s = -Sigma_s^{-1}(r_s + p_y), from the +I slack coupling of the +s form
h + s = 0) the system over [p_w; p_lambda; p_y] is

    M = [[W + diag(Sigma_w) + delta_w E_u,  G^T,  A^T                        ],
         [G,                                0,    0                          ],
         [A,                                0,    -(Sigma_s^{-1} + delta_c) I]]

with the primal term delta_w on the u block (the same placement as LinRed's
K_cond + delta_w I) and the dual term delta_c on the inequality rows.

Whatever factorisation is used, three of its results are unique and are what
the oracle computes: the Newton step, the inertia of M (Sylvester's law: the
signs of any congruent block-diagonal D), and log|det M|.  The inertia is
given two ways:
  * from the eigenvalues of the dense M (small cases);
  * by Haynsworth's inertia additivity over the negative definite (p_y, p_y)
    block, then the saddle-point theorem for [[K, G^T], [G, 0]] with G_x
    nonsingular: In(M) = In(K_cond) + (n_x, n_x + m, 0).  With Theorem 3 this
    says the inertia is (n_w, n_x + m, 0) exactly when K_cond is positive
    definite.
log|det M| is given by a sparse LU of M and by the product formula
    |det M| = prod(Sigma_s^{-1} + delta_c) * det(G_x)^2 * det(K_cond)
(the Schur complements of the same two eliminations).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import kkt


def augmented(G, A, W, sig_w, sig_s, nu, delta_w=0.0, delta_c=0.0):
    """M above (sparse CSC), unknowns [p_w; p_lambda; p_y], p_w = [p_u; p_x]."""
    G = sp.csr_matrix(G)
    A = sp.csr_matrix(A)
    nx, nw = G.shape
    m = A.shape[0]
    dw = np.asarray(sig_w, dtype=np.float64).copy()
    dw[:nu] += delta_w
    H = sp.csr_matrix(W) + sp.diags(dw)
    Dy = sp.diags(-(1.0 / np.asarray(sig_s, dtype=np.float64) + delta_c))
    return sp.bmat([[H, G.T, A.T],
                    [G, sp.csr_matrix((nx, nx)), None],
                    [A, None, Dy]], format="csc")


def augmented_rhs(r, sig_s, nw, nx, m):
    """Right-hand side of M for K_aug p = -r, r = [r_w; r_s; r_lambda; r_y]."""
    r = np.asarray(r, dtype=np.float64)
    rw, rs = r[:nw], r[nw:nw + m]
    rl, ry = r[nw + m:nw + m + nx], r[nw + m + nx:]
    return np.concatenate([-rw, -rl, -ry + rs / np.asarray(sig_s, dtype=np.float64)])


def augmented_step(G, A, W, sig_w, sig_s, r, nu, delta_w=0.0, delta_c=0.0):
    """Newton step of K_aug p = -r through M (sparse LU), the slack step
    recovered from the slack row.  Returns (p_w, p_s, p_lambda, p_y) like
    kkt.full_space_step."""
    nx, nw = G.shape
    m = A.shape[0]
    M = augmented(G, A, W, sig_w, sig_s, nu, delta_w, delta_c)
    z = spla.splu(M).solve(augmented_rhs(r, sig_s, nw, nx, m))
    pw, pl, py = z[:nw], z[nw:nw + nx], z[nw + nx:]
    rs = np.asarray(r, dtype=np.float64)[nw:nw + m]
    ps = -(rs + py) / np.asarray(sig_s, dtype=np.float64)
    return pw, ps, pl, py


def inertia_eig(M):
    """(n+, n-, n0) of a symmetric matrix from its eigenvalues."""
    Md = M.toarray() if sp.issparse(M) else np.asarray(M)
    ev = np.linalg.eigvalsh(0.5 * (Md + Md.T))
    tol = 1e-12 * max(1.0, np.abs(ev).max())
    return int((ev > tol).sum()), int((ev < -tol).sum()), int((np.abs(ev) <= tol).sum())


def inertia_by_reduction(Kcond, nx, m):
    """In(M) = In(K_cond) + (n_x, n_x + m, 0) (Haynsworth additivity over the
    (p_y, p_y) block, then the saddle-point inertia with G_x nonsingular).
    Kcond must carry the same delta_w and delta_c as M."""
    p, n, z = inertia_eig(Kcond)
    return p + nx, n + nx + m, z


def logabsdet_lu(M):
    """log|det M| from a sparse LU (unit lower factor): sum of log|U_ii|."""
    lu = spla.splu(sp.csc_matrix(M))
    return float(np.sum(np.log(np.abs(lu.U.diagonal()))))


def logabsdet_by_reduction(G, Kcond, sig_s, nu, delta_c=0.0):
    """log|det M| = sum log(Sigma_s^{-1} + delta_c) + 2 log|det G_x| + log|det K_cond|."""
    Gx = sp.csc_matrix(sp.csr_matrix(G)[:, nu:])
    lg = logabsdet_lu(Gx)
    _, lk = np.linalg.slogdet(np.asarray(Kcond))
    ly = float(np.sum(np.log(1.0 / np.asarray(sig_s, dtype=np.float64) + delta_c)))
    return ly + 2.0 * lg + float(lk)


def kcond(G, A, W, sig_w, sig_s, nu, delta_w=0.0, delta_c=0.0):
    """K_cond + delta_w I with Sigma_t = (Sigma_s^{-1} + delta_c)^{-1} (the
    condensed matrix that goes with M)."""
    Kc = kkt.kred_definition(G, A, W, sig_w, kkt.regularized_sigma(sig_s, delta_c), nu)
    return 0.5 * (Kc + Kc.T) + delta_w * np.eye(nu)
