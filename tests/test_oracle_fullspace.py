"""Pins for the oracle of the hybrid full-space system (Sec. 4.3): the
slack-eliminated augmented matrix M, its step, inertia and log|det|, each tied
to a second route -- the full K_aug solve with the slack block kept, the
eigenvalues of the dense M, LAPACK's slogdet, and the product formula of the
two Schur complements.  A dropped delta term, a wrong sign or a missing inverse
on the (p_y, p_y) block, or a wrong right-hand-side fold fails one of them.
No GPU needed."""
import numpy as np
import pytest

import gridgen
from oracle import fullspace, kkt, model


def _point(net, seed, scale):
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
    return lay, G, A, W, sw, ss, r


NETS = [("tiny3", gridgen.tiny3), ("ring30", gridgen.ring30),
        ("b60", lambda: gridgen.lattice(60, 9101, name="b60"))]


@pytest.mark.parametrize("name,make", NETS)
@pytest.mark.parametrize("delta_w,delta_c", [(0.0, 0.0), (3.0, 0.0), (0.5, 1e-2)])
def test_augmented_step_matches_kaug(name, make, delta_w, delta_c):
    """The step through M (slack eliminated) equals the dense solve of K_aug
    with the slack block kept, delta_w added on the u diagonal of W."""
    lay, G, A, W, sw, ss, r = _point(make(), 11, 1.0)
    pw, ps, pl, py = fullspace.augmented_step(G, A, W, sw, ss, r, lay.nu, delta_w, delta_c)
    Wd = W.toarray() if hasattr(W, "toarray") else np.array(W)
    Wd[np.arange(lay.nu), np.arange(lay.nu)] += delta_w
    ref = kkt.full_space_step(G, A, Wd, sw, ss, r, delta_c=delta_c)
    got = np.concatenate([pw, ps, pl, py])
    want = np.concatenate(ref)
    assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("name,make", NETS)
def test_inertia_by_reduction_matches_eigenvalues(name, make):
    """Haynsworth + the saddle-point theorem against the eigenvalues of the
    dense M, at points where K_cond is indefinite and where it is definite;
    the count is (n_w, n_x + m, 0) exactly when K_cond is positive definite
    (Theorem 3)."""
    seen_bad = seen_good = False
    for scale, shift in ((30.0, None), (30.0, 1.0), (1.0, None), (1.0, 1e-3), (100.0, None)):
        lay, G, A, W, sw, ss, _ = _point(make(), 5, scale)
        # shift: delta_w just past (1 + shift) times the most negative eigenvalue
        lmin = np.linalg.eigvalsh(fullspace.kcond(G, A, W, sw, ss, lay.nu))[0]
        delta_w = 0.0 if shift is None else max(0.0, -lmin) * (1.0 + shift) + shift
        M = fullspace.augmented(G, A, W, sw, ss, lay.nu, delta_w)
        Kc = fullspace.kcond(G, A, W, sw, ss, lay.nu, delta_w)
        got = fullspace.inertia_by_reduction(Kc, lay.nx, lay.m)
        assert got == fullspace.inertia_eig(M)
        assert got == kkt.inertia_dense(M)
        pd = np.linalg.eigvalsh(Kc)[0] > 0
        assert (got == (lay.nw, lay.nx + lay.m, 0)) == pd
        seen_bad |= not pd
        seen_good |= pd
    assert seen_good and seen_bad


@pytest.mark.parametrize("name,make", NETS)
@pytest.mark.parametrize("delta_c", [0.0, 0.05])
def test_logabsdet_two_ways(name, make, delta_c):
    lay, G, A, W, sw, ss, _ = _point(make(), 7, 3.0)
    M = fullspace.augmented(G, A, W, sw, ss, lay.nu, 2.0, delta_c)
    Kc = fullspace.kcond(G, A, W, sw, ss, lay.nu, 2.0, delta_c)
    a = fullspace.logabsdet_lu(M)
    b = fullspace.logabsdet_by_reduction(G, Kc, ss, lay.nu, delta_c)
    _, c = np.linalg.slogdet(M.toarray())
    assert abs(a - c) <= 1e-9 * max(1.0, abs(c))
    assert abs(b - c) <= 1e-9 * max(1.0, abs(c))


def test_augmented_rhs_fold():
    """The slack row folded into the inequality rows: M z = rhs reproduces the
    y rows of K_aug p = -r once p_s = -Sigma_s^{-1}(r_s + p_y) is put back."""
    lay, G, A, W, sw, ss, r = _point(gridgen.ring30(), 3, 1.0)
    pw, ps, pl, py = fullspace.augmented_step(G, A, W, sw, ss, r, lay.nu, 0.0, 0.0)
    nw, m, nx = lay.nw, lay.m, lay.nx
    ry = r[nw + m + nx:]
    rs = r[nw:nw + m]
    assert np.allclose(A @ pw + ps, -ry, atol=1e-10)
    assert np.allclose(ss * ps + py, -rs, atol=1e-10)
