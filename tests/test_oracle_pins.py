"""Pins for the FP64 oracle: each test ties an oracle routine to something other
than itself (a closed form, an invariant, a theorem of the paper, brute force,
finite differences, or an independent library routine), chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in
``oracle/lasso_oracle.c`` fails at least one of them.

Citations are to arXiv 1905.11071.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dict(n, m, seed):
    return synth.gaussian_dictionary(n, m, np.random.default_rng(seed)).astype(np.float64)


def _lam_frac(D, X, frac):
    return frac * np.abs(X @ D).max()


# --------------------------------------------------------------------------
# Soft-thresholding (Section 1, after Eq. ista; sign(0) = 0 from Section 2)
# --------------------------------------------------------------------------

def test_st_closed_form_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "st_table.txt"), comments="#")
    for v, u, want in rows:
        assert oracle.st(v, u) == want, (v, u)


# --------------------------------------------------------------------------
# Gram quantities and lambda_max against independent numpy evaluations
# --------------------------------------------------------------------------

def test_gram_definition_matches_numpy():
    rng = np.random.default_rng(3)
    D = _dict(7, 13, 1)
    X = rng.standard_normal((9, 7))
    B, C, xsq = oracle.gram(D, X)
    np.testing.assert_allclose(B, D.T @ D, rtol=0, atol=1e-13)
    np.testing.assert_allclose(C, X @ D, rtol=0, atol=1e-13)
    np.testing.assert_allclose(xsq, (X * X).sum(axis=1), rtol=1e-14)
    # unit-norm columns: the Gram diagonal is exactly the squared column norms
    np.testing.assert_allclose(np.diag(B), 1.0, atol=1e-12)
    assert np.array_equal(B, B.T)


def test_lambda_max_matches_numpy():
    rng = np.random.default_rng(4)
    D = _dict(6, 11, 2)
    X = rng.standard_normal((5, 6))
    np.testing.assert_allclose(oracle.lambda_max(D, X), np.abs(X @ D).max(axis=1), rtol=1e-14)


# --------------------------------------------------------------------------
# Largest eigenvalues: L (Section 1) and L_S (Eq. spca)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 5, 17, 40])
def test_jacobi_matches_eigvalsh(k):
    rng = np.random.default_rng(k)
    A = rng.standard_normal((k, k))
    A = A + A.T  # symmetric, indefinite: the largest *algebraic* eigenvalue
    got = oracle.sym_max_eig(A)
    assert abs(got - np.linalg.eigvalsh(A).max()) <= 1e-11 * max(1.0, abs(got))


def test_lipschitz_and_support_lipschitz():
    D = _dict(10, 24, 5)
    L = oracle.lipschitz(D)
    assert abs(L - np.linalg.eigvalsh(D.T @ D).max()) < 1e-11
    rng = np.random.default_rng(6)
    for _ in range(5):
        mask = rng.random(24) < 0.3
        want = np.linalg.eigvalsh(D[:, mask].T @ D[:, mask]).max() if mask.any() else L
        assert abs(oracle.support_lipschitz(D, mask, L) - want) < 1e-11
    # |S| = 1: L_S is the squared column norm (1 for unit columns)
    for j in (0, 7, 23):
        mask = np.zeros(24, bool)
        mask[j] = True
        assert abs(oracle.support_lipschitz(D, mask, L) - D[:, j] @ D[:, j]) < 1e-14
    # convention L_empty = L (Eq. spca)
    assert oracle.support_lipschitz(D, np.zeros(24, bool), L) == L
    # L_S <= L for every S (Section 3)
    for _ in range(5):
        mask = rng.random(24) < 0.6
        assert oracle.support_lipschitz(D, mask, L) <= L + 1e-12


def test_marchenko_pastur_ratio():
    """Proposition 3.4: L_S / L -> ((1 + sqrt(zeta gamma)) / (1 + sqrt(gamma)))^2
    for i.i.d. N(0,1) entries, here at the paper's 200 x 600 illustration size
    (Fig. B.1), gamma = 3."""
    rng = np.random.default_rng(7)
    n, m = 200, 600
    D = rng.standard_normal((n, m))
    gamma = m / n
    L = oracle.sym_max_eig(D @ D.T)  # same non-zero spectrum as D^T D
    for zeta in (0.1, 0.25, 0.5, 0.75):
        k = int(zeta * m)
        S = np.sort(rng.choice(m, size=k, replace=False))
        if k <= n:
            mask = np.zeros(m, bool)
            mask[S] = True
            LS = oracle.support_lipschitz(D, mask, L)
        else:
            LS = oracle.sym_max_eig(D[:, S] @ D[:, S].T)
        want = ((1 + np.sqrt(zeta * gamma)) / (1 + np.sqrt(gamma))) ** 2
        assert abs(LS / L - want) < 0.06 * want, (zeta, LS / L, want)


# --------------------------------------------------------------------------
# Unfolded proximal gradient (Eq. ista, Eq. pgd, Eq. steprec)
# --------------------------------------------------------------------------

def test_zero_above_lambda_max_every_variant():
    """argmin F_x = {0} iff lam >= lam_max (Section 2); from z^(0) = 0 every
    layer returns exactly 0 because |alpha D^T x| <= alpha lam."""
    rng = np.random.default_rng(8)
    D = _dict(8, 16, 8)
    X = rng.standard_normal((6, 8))
    lam = np.abs(X @ D).max() * 1.0001
    L = oracle.lipschitz(D)
    alpha = np.array([0.3, 1.0, 2.0, 0.5]) / L
    assert not oracle.pgd(D, X, lam, alpha).any()
    assert not oracle.ista(D, X, lam, L, 7).any()
    Z, _, acc, _ = oracle.oista(D, X, lam, L, 7)
    assert not Z.any()


def test_ista_objective_monotone():
    """ISTA is a majorisation-minimisation step (Eq. majorization2), so
    F_x(z^(t+1)) <= F_x(z^(t)) when the step is 1/L (or smaller)."""
    w = synth.ista_10x20(N=20, T=60)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    for scale in (1.0, 0.5):
        Zall = oracle.pgd(D, w.X, w.lam, np.full(w.T, scale / L), keep_all=True)
        F = np.stack([oracle.objective(D, w.X, Zall[t], w.lam, with_gap=False) for t in range(w.T + 1)])
        assert (np.diff(F, axis=0) <= 1e-13).all()


def test_ista_kkt_at_convergence():
    """After 10^4 ISTA iterations (the paper's F* recipe, Appendix E) the KKT
    conditions of Lemma 2.1 hold to 1e-9."""
    w = synth.ista_10x20(N=5, T=10000)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    Z = oracle.ista(D, w.X, w.lam, L, w.T)
    for i in range(w.N):
        assert oracle.kkt_violation(D, w.X[i], Z[i], w.lam) < 1e-9


def _small_problem(seed, n=6, m=8, frac=0.25):
    rng = np.random.default_rng(seed)
    D = _dict(n, m, seed)
    x = rng.standard_normal(n)
    lam = frac * np.abs(D.T @ x).max()
    return D, x, lam


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bruteforce_matches_ista_limit_and_gap(seed):
    """Sign enumeration of the KKT system (Lemma 2.1) gives the unique z*
    (Assumption 2.2 holds a.s.); ISTA converges to it, its duality gap is 0
    and F* is below every ISTA iterate."""
    D, x, lam = _small_problem(seed)
    zstar, count = oracle.lasso_bruteforce(D, x, lam)
    assert count == 1
    L = oracle.lipschitz(D)
    z = oracle.ista(D, x[None, :], lam, L, 20000)[0]
    np.testing.assert_allclose(z, zstar, atol=1e-8)
    F, gap = oracle.objective(D, x[None, :], zstar[None, :], lam)
    assert abs(gap[0]) < 1e-12
    assert oracle.kkt_violation(D, x, zstar, lam) < 1e-12
    Zall = oracle.pgd(D, x[None, :], lam, np.full(50, 1.0 / L), keep_all=True)
    Fs = np.array([oracle.objective(D, x[None, :], Zall[t], lam, with_gap=False)[0] for t in range(51)])
    assert (Fs >= F[0] - 1e-14).all()
    # worst-case ISTA rate F(z^t) - F* <= L ||z*||^2 / (2t) (Section 3, after Prop. 3.2)
    t = np.arange(1, 51)
    assert (Fs[1:] - F[0] <= L * (zstar @ zstar) / (2 * t) + 1e-14).all()


def test_ista_linear_rate_strongly_convex():
    """The classical linear rate quoted with Prop. 3.2: with m < n, D^T D has
    smallest eigenvalue mu > 0 and ISTA satisfies
    F(z^t) - F* <= (1 - mu/L)^t (F(0) - F*)."""
    rng = np.random.default_rng(51)
    D = synth.gaussian_dictionary(30, 12, rng).astype(np.float64)
    X = rng.standard_normal((5, 30))
    lam = 0.2 * np.abs(X @ D).max()
    L = oracle.lipschitz(D)
    mu = np.linalg.eigvalsh(D.T @ D).min()
    assert mu > 0.05
    T = 200
    Zall = oracle.pgd(D, X, lam, np.full(T, 1.0 / L), keep_all=True)
    Fstar = oracle.objective(D, X, oracle.ista(D, X, lam, L, 5000), lam, with_gap=False)
    F = np.stack([oracle.objective(D, X, Zall[t], lam, with_gap=False) for t in range(T + 1)])
    t = np.arange(T + 1)[:, None]
    assert (F - Fstar <= (1 - mu / L) ** t * (F[0] - Fstar) + 1e-13).all()


def test_stability_closed_form():
    """Lemma 4.2: for unit columns, c = max_{l != j} |D_l^T D_j| and
    x = D_j + eps with eps orthogonal to D_j, ||eps|| < lam (1 - c), the Lasso
    solution is (1 - lam) e_j."""
    D = _dict(6, 8, 11)
    D /= np.linalg.norm(D, axis=0)  # exactly unit columns in float64
    rng = np.random.default_rng(12)
    lam = 0.6
    for j in range(8):
        c = np.max(np.abs(np.delete(D.T @ D[:, j], j)))
        assert c < 1
        e = rng.standard_normal(6)
        e -= (e @ D[:, j]) * D[:, j]
        e *= 0.9 * lam * (1 - c) / np.linalg.norm(e)
        x = D[:, j] + e
        want = np.zeros(8)
        want[j] = 1 - lam
        zstar, count = oracle.lasso_bruteforce(D, x, lam)
        assert count == 1
        np.testing.assert_allclose(zstar, want, atol=1e-12)
        assert oracle.kkt_violation(D, x, want, lam) < 1e-12
        L = oracle.lipschitz(D)
        z = oracle.ista(D, x[None, :], lam, L, 5000)[0]
        np.testing.assert_allclose(z, want, atol=1e-9)


def test_orthogonal_dictionary_one_step():
    """With D^T D = Id (L = 1), one ISTA step from 0 gives ST(D^T x, lam), which
    is already the Lasso solution (Section 3, before Prop. 3.3); OISTA takes the
    same step since every L_S equals 1."""
    rng = np.random.default_rng(13)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 8)))
    D = Q
    X = rng.standard_normal((4, 12))
    lam = 0.3
    L = oracle.lipschitz(D)
    assert abs(L - 1.0) < 1e-12
    z1 = oracle.ista(D, X, lam, L, 1)
    st = np.sign(X @ D) * np.maximum(np.abs(X @ D) - lam, 0)
    np.testing.assert_allclose(z1, st, atol=1e-14)
    for i in range(4):
        assert oracle.kkt_violation(D, X[i], z1[i], lam) < 1e-13
    z5 = oracle.ista(D, X, lam, L, 5)
    np.testing.assert_allclose(z5, z1, atol=1e-14)
    zo, LS, acc, dec = oracle.oista(D, X, lam, L, 5)
    np.testing.assert_allclose(zo, z1, atol=1e-14)


def test_pgd_step_sequence_is_layerwise():
    """Eq. steprec with a varying step sequence equals chaining single layers."""
    w = synth.slista_64x256(N=3, T=6)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    alpha = synth.step_sizes(6, 1.0 / L, 0.5, seed=1).astype(np.float64)
    Zall = oracle.pgd(D, w.X, w.lam, alpha, keep_all=True)
    # a single layer on an arbitrary start: recompute layer t from z^(t) by hand
    X = w.X.astype(np.float64)
    for t in range(6):
        z = Zall[t]
        u = z - alpha[t] * ((z @ D.T - X) @ D)
        want = np.sign(u) * np.maximum(np.abs(u) - alpha[t] * w.lam, 0)
        np.testing.assert_allclose(Zall[t + 1], want, atol=1e-13)


def test_lista_reduces_to_ista_and_step_lista():
    """Coupled LISTA (Eq. lista_layer): W = D with alpha = beta = 1/L is ISTA
    (Section 4); a layer (W, alpha, beta) is the Step-LISTA layer of step beta
    when (alpha / beta) W = D (Section 4, after Eq. steprec), and not in
    general otherwise; from z = 0 one layer returns 0 iff
    |alpha W^T x|_inf <= beta lam (ST's closed form)."""
    w = synth.ista_10x20(N=30, T=12)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    T = w.T
    Ws = np.repeat(D[None], T, axis=0)
    ista = oracle.ista(D, w.X, w.lam, L, T)
    np.testing.assert_allclose(oracle.lista(D, w.X, w.lam, Ws, np.full(T, 1 / L), np.full(T, 1 / L)), ista,
                               rtol=0, atol=1e-14)
    rng = np.random.default_rng(41)
    alpha = rng.uniform(0.3, 2.0, T) / L
    beta = rng.uniform(0.3, 1.5, T) / L
    Wc = Ws * (beta / alpha)[:, None, None]
    want = oracle.pgd(D, w.X, w.lam, beta)
    assert np.abs(want).max() > 0.1
    np.testing.assert_allclose(oracle.lista(D, w.X, w.lam, Wc, alpha, beta), want, rtol=0, atol=1e-12)
    Wp = Wc + 0.05 * rng.standard_normal(Wc.shape)
    assert np.abs(oracle.lista(D, w.X, w.lam, Wp, alpha, beta) - want).max() > 1e-4
    # one layer from 0: u = alpha W^T x
    W1 = rng.standard_normal((1, D.shape[0], D.shape[1]))
    a1, b1 = np.array([0.7]), np.array([0.4])
    top = np.abs(a1[0] * (w.X.astype(np.float64) @ W1[0])).max(axis=1)
    lam0 = top.max() / b1[0] * 1.0001
    assert not oracle.lista(D, w.X, lam0, W1, a1, b1).any()
    i = int(np.argmax(top))
    z = oracle.lista(D, w.X[i:i + 1], top[i] / b1[0] * 0.9999, W1, a1, b1)
    assert np.count_nonzero(z) == 1


# --------------------------------------------------------------------------
# Objective and duality gap (Eq. lasso; gap: standard Lasso dual)
# --------------------------------------------------------------------------

def test_objective_special_values_and_weak_duality():
    rng = np.random.default_rng(14)
    D = _dict(9, 30, 14)
    X = rng.standard_normal((10, 9))
    lam = 0.2 * np.abs(X @ D).max()
    F0, gap0 = oracle.objective(D, X, np.zeros((10, 30)), lam)
    np.testing.assert_allclose(F0, 0.5 * (X * X).sum(axis=1), rtol=1e-14)
    Z = rng.standard_normal((10, 30)) * (rng.random((10, 30)) < 0.2)
    F, gap = oracle.objective(D, X, Z, lam)
    assert (gap >= -1e-12).all()
    # lam above lam_max: z = 0 is optimal and the gap there is exactly zero
    big = np.abs(X @ D).max() * 1.01
    _, g0 = oracle.objective(D, X, np.zeros((10, 30)), big)
    assert np.abs(g0).max() < 1e-12
    # scaling: F(z) depends on lam only through lam ||z||_1
    F2 = oracle.objective(D, X, Z, 2 * lam, with_gap=False)
    np.testing.assert_allclose(F2 - F, lam * np.abs(Z).sum(axis=1), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Oracle-ISTA (Algorithm 1)
# --------------------------------------------------------------------------

def test_oista_monotone_and_safe_regime():
    """Every OISTA step decreases F_x (Section 3: both branches minimise a
    majoriser), and after finite support identification condition (star)
    always holds (Prop. 3.1).  Toy setup of Fig. 3: D 10 x 50, lam = 0.5, x in
    B_inf."""
    w = synth.paper_binf(10, 50, N=4, lam=0.5, T=400, seed=3)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    Zall, LS, acc, dec = oracle.oista(D, w.X, w.lam, L, w.T, keep_all=True)
    F = np.stack([oracle.objective(D, w.X, Zall[t], w.lam, with_gap=False) for t in range(w.T + 1)])
    assert (np.diff(F, axis=0) <= 1e-13).all()
    assert dec[-100:].all()
    assert acc[-1] == w.N
    # the L_S reported for the last layer is that of supp(z^(T-1))
    for i in range(w.N):
        mask = Zall[w.T - 1, i] != 0
        assert abs(LS[i] - oracle.support_lipschitz(D, mask, L)) < 1e-12


def test_oista_layer_margins_hand_case():
    """The per-layer decision margin of Oracle-ISTA on a case worked by hand.
    D = diag(2, 1) (L = 4; L_S = the largest d_j^2 on S; c = D^T x = (0.3, 0.6)),
    x = (0.15, 0.6), lam = 0.5, z^(0) = 0:
      layer 0: S empty, L_S = L = 4, u = c / 4 = (0.075, 0.15), threshold
               0.125: the local step gives (0, 0.025), code 1 leaves S, so
               condition (star) fails; margins |0.075 - 0.125| = 0.05 and
               |0.15 - 0.125| = 0.025 -> 0.025; the ISTA step (same 1/4)
               gives z^(1) = (0, 0.025).
      layer 1: S = {1}, L_S = 1, gradient B z - c = (-0.3, -0.575),
               u = (0.3, 0.6), threshold 0.5: the local step gives (0, 0.1),
               inside S (accepted); margin off S |0.3 - 0.5| = 0.2, on the
               step taken min(0.2, |0.6 - 0.5| = 0.1) -> 0.1; z^(2) = (0, 0.1).
      layer 2: z^(2) is the Lasso solution (|c_0 - (Bz)_0| = 0.3 <= lam and
               z_1 = ST(0.6, 0.5)); the same u, margin 0.1, accepted.
    A margin that used L instead of L_S, skipped the codes on S of an
    accepted step, or skipped the codes off S would differ."""
    D = np.diag([2.0, 1.0])
    X = np.array([[0.15, 0.6]])
    Zall, LS, acc, dec, lm = oracle.oista(D, X, 0.5, 4.0, 4, keep_all=True, layer_margins=True)
    np.testing.assert_allclose(lm[:, 0], [0.025, 0.1, 0.1, 0.1], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(dec[:, 0], [0, 1, 1, 1])
    np.testing.assert_allclose(Zall[1, 0], [0.0, 0.025], atol=1e-15)
    np.testing.assert_allclose(Zall[2, 0], [0.0, 0.1], atol=1e-15)
    assert LS[0] == 1.0
    # the per-sample trajectory margin is the smallest layer margin
    _, _, _, _, mg = oracle.oista(D, X, 0.5, 4.0, 4, with_margin=True)
    assert mg[0] == lm[:, 0].min()


def test_oista_layer_margin_vanishes_at_a_tie():
    """A code whose pre-threshold value sits exactly on its threshold has
    margin 0 at that layer (D = I, L = L_S = 1, u = x at every layer, so the
    margin is min_j ||x_j| - lam| at every layer)."""
    x = np.array([[0.9, -0.5, 0.2, -1.25]])
    _, _, _, _, lm = oracle.oista(np.eye(4), x, 0.5, 1.0, 3, layer_margins=True)
    np.testing.assert_allclose(lm[:, 0], 0.0, atol=1e-15)
    x2 = np.array([[0.9, -0.6, 0.2, -1.25]])
    _, _, _, _, lm2 = oracle.oista(np.eye(4), x2, 0.5, 1.0, 3, layer_margins=True)
    np.testing.assert_allclose(lm2[:, 0], 0.1, atol=1e-12)


def _support_identification(Zall, zstar_support):
    """T* of Prop. 3.1: the first iteration from which every iterate has the
    support of z*."""
    same = np.array([np.array_equal(z != 0, zstar_support) for z in Zall])
    off = np.where(~same)[0]
    assert len(off) and not same[0] and same[-1]
    return int(off.max()) + 1


def test_oista_rates_after_support_identification():
    """Prop. 3.2: for t > T*, F(z^t) - F* <= L_S* ||z* - z^T*||^2 / (2(t - T*))
    and, with mu* = min eig D_S*^T D_S* > 0, F(z^t) - F* <=
    (1 - mu*/L_S*)^(t - T*) (F(z^T*) - F*).  The linear bound has teeth:
    ISTA's 1/L steps, run through the same test, break it (the step on the
    identified support must be 1/L_S*, not 1/L)."""
    w = synth.paper_binf(10, 50, N=4, lam=0.5, T=300, seed=3)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    Zo, _, _, dec = oracle.oista(D, w.X, w.lam, L, w.T, keep_all=True)
    Zi = oracle.pgd(D, w.X, w.lam, np.full(w.T, 1.0 / L), keep_all=True)
    Zstar = oracle.oista(D, w.X, w.lam, L, 3000)[0]
    Fstar = oracle.objective(D, w.X, Zstar, w.lam, with_gap=False)

    def bounds(Zall, i):
        S = Zstar[i] != 0
        T0 = _support_identification(Zall[:, i], S)
        LS = oracle.support_lipschitz(D, S, L)
        mu = np.linalg.eigvalsh(D[:, S].T @ D[:, S]).min()
        assert mu > 0
        F = oracle.objective(D, np.repeat(w.X[i:i + 1], w.T + 1, 0), Zall[:, i], w.lam,
                             with_gap=False)
        t = np.arange(T0 + 1, w.T + 1)
        gap = F[t] - Fstar[i]
        sub = LS * np.sum((Zstar[i] - Zall[T0, i]) ** 2) / (2 * (t - T0))
        lin = (1 - mu / LS) ** (t - T0) * (F[T0] - Fstar[i])
        return T0, (gap <= sub + 1e-13).all(), (gap <= lin + 1e-13).all()

    for i in range(w.N):
        T0, sub_ok, lin_ok = bounds(Zo, i)
        assert T0 < w.T - 100 and dec[T0:, i].all()
        assert sub_ok and lin_ok, i
        assert not bounds(Zi, i)[2], i


def test_oista_orthogonal_support_one_step():
    """Prop. 3.3: if D_S*^T D_S* = L_S* Id, OISTA returns z* one iteration after
    it identifies S*.  Here S* holds 4 orthonormal columns (L_S* = 1, so
    z*_S* = ST(D_S*^T x, lam) by KKT) inside a 12 x 30 dictionary with L > 5;
    ISTA's 1/L step from the same support is still far from z*."""
    D, X, S = synth.orthogonal_support(N=3, dtype=np.float64)
    m = D.shape[1]
    lam = 0.3
    L = oracle.lipschitz(D)
    assert L > 5
    for i in range(X.shape[0]):
        zstar = np.zeros(m)
        zstar[S] = _st_by_hand(X[i] @ D[:, S], lam)
        assert (zstar[S] != 0).all()
        assert oracle.kkt_violation(D, X[i], zstar, lam) < 1e-13
        Zall, LS, _, dec = oracle.oista(D, X[i:i + 1], lam, L, 30, keep_all=True)
        T0 = next(t for t in range(31) if np.array_equal(np.nonzero(Zall[t, 0])[0], S))
        assert T0 >= 2
        np.testing.assert_allclose(Zall[T0 + 1, 0], zstar, rtol=0, atol=1e-14)
        assert np.abs(Zall[T0, 0] - zstar).max() > 1e-3
        assert abs(LS[0] - 1.0) < 1e-14
        # the same support reached with 1/L steps is not yet z*
        Zi = oracle.pgd(D, X[i:i + 1], lam, np.full(30, 1.0 / L), keep_all=True)
        assert np.abs(Zi[T0 + 1, 0] - zstar).max() > 0.1


def test_learned_steps_follow_support_steps_10x20():
    """Fig. 4 / Appendix E on the oracle: Step-LISTA (T = 20) trained by
    sub-gradient descent with backtracking on 10 x 20, lam = 0.2, N = 1000
    lowers the loss, and its steps alpha_t follow the distribution of
    1/L_S(x, t), S(x, t) = supp z^(t)(x): high rank correlation with its
    median, and median <= alpha_t <= maximum in the second half."""
    T = 20
    w = synth.paper_binf(10, 20, N=1000, lam=0.2, T=T, seed=0)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    alpha = np.full(T, 1.0 / L)
    grad, loss = oracle.slista_grad(D, w.X, w.lam, alpha)
    loss0 = loss
    lr = 0.1 * alpha.max() / np.abs(grad).max()
    for _ in range(60):
        for _h in range(20):
            trial = np.maximum(alpha - lr * grad, 1e-6)
            gt, lt = oracle.slista_grad(D, w.X, w.lam, trial)
            if lt <= loss:
                alpha, loss, grad = trial, lt, gt
                lr *= 1.2
                break
            lr *= 0.5
    assert loss < loss0
    Zall = oracle.pgd(D, w.X, w.lam, alpha, keep_all=True)
    med, top = [], []
    for t in range(T):
        inv = np.array([1.0 / oracle.support_lipschitz(D, Zall[t, i] != 0, L) for i in range(w.N)])
        med.append(np.median(inv))
        top.append(inv.max())
    med, top = np.array(med), np.array(top)
    rank = lambda v: np.argsort(np.argsort(v, kind="stable"), kind="stable")
    assert np.corrcoef(rank(alpha), rank(med))[0, 1] >= 0.8
    h = T // 2
    assert (med[h:] <= alpha[h:]).all() and (alpha[h:] <= top[h:]).all()
    assert alpha[h:].mean() > 2.0 / L


def _st_by_hand(v, theta):
    """Soft-thresholding written out for the test (Section 1)."""
    return np.sign(v) * np.maximum(np.abs(v) - theta, 0.0)


def test_oista_faster_than_ista():
    """Fig. B.2: OISTA reaches F* + 1e-13 in no more iterations than ISTA
    (D 100 x 200, samples in B_inf, high regularisation)."""
    w = synth.paper_binf(100, 200, N=2, lam=0.6, T=1500, seed=5)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    Fstar = oracle.objective(D, w.X, oracle.ista(D, w.X, w.lam, L, 20000), w.lam, with_gap=False)
    Zi = oracle.pgd(D, w.X, w.lam, np.full(w.T, 1.0 / L), keep_all=True)
    Zo, _, _, _ = oracle.oista(D, w.X, w.lam, L, w.T, keep_all=True)

    def first_hit(Zall):
        F = np.stack([oracle.objective(D, w.X, Zall[t], w.lam, with_gap=False) for t in range(w.T + 1)])
        ok = F < Fstar[None, :] + 1e-13
        return np.where(ok.any(axis=0), ok.argmax(axis=0), w.T + 1)

    hi, ho = first_hit(Zi), first_hit(Zo)
    assert (ho <= hi).all(), (ho, hi)
    assert (ho < w.T).all()


# --------------------------------------------------------------------------
# Step-LISTA sub-gradient (Eq. steprec, Appendix E)
# --------------------------------------------------------------------------

def _fd_check(D, X, lam, alpha, rel_tol):
    da, loss = oracle.slista_grad(D, X, lam, alpha)
    F = oracle.objective(D, X, oracle.pgd(D, X, lam, alpha), lam, with_gap=False)
    assert abs(loss - F.sum()) <= 1e-12 * abs(loss)
    checked = 0
    for t in range(len(alpha)):
        h = 1e-7 * alpha[t]
        for _ in range(6):
            ap = alpha.copy(); ap[t] += h
            am = alpha.copy(); am[t] -= h
            Zp = oracle.pgd(D, X, lam, ap, keep_all=True)
            Zm = oracle.pgd(D, X, lam, am, keep_all=True)
            if np.array_equal(Zp != 0, Zm != 0):
                break
            h *= 0.5
        else:
            continue  # a support change sits inside every window: skip
        lp = oracle.objective(D, X, Zp[-1], lam, with_gap=False).sum()
        lm = oracle.objective(D, X, Zm[-1], lam, with_gap=False).sum()
        fd = (lp - lm) / (2 * h)
        scale = max(np.abs(da).max(), 1e-12)
        assert abs(fd - da[t]) <= rel_tol * scale, (t, fd, da[t])
        checked += 1
    assert checked >= len(alpha) - 1


def test_slista_grad_finite_differences_small():
    """Hand adjoint vs central differences in FP64, N = 64 (10 x 20, T = 20)."""
    w = synth.paper_binf(10, 20, N=64, lam=0.2, T=20, seed=21)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    alpha = synth.step_sizes(w.T, 1.0 / L, 0.6, seed=22).astype(np.float64)
    _fd_check(D, w.X.astype(np.float64), w.lam, alpha, 1e-6)


def test_slista_grad_finite_differences_64x256():
    """Hand adjoint vs central differences on the 64 x 256 model (N = 8, T = 8)."""
    w = synth.slista_64x256(N=8, T=8)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    alpha = synth.step_sizes(w.T, 1.0 / L, 0.5, seed=23).astype(np.float64)
    _fd_check(D, w.X.astype(np.float64), w.lam, alpha, 1e-6)


def test_slista_grad_zero_when_output_zero():
    """lam >= lam_max: every layer outputs 0, every mask is empty, so the
    sub-gradient with respect to every step vanishes."""
    rng = np.random.default_rng(24)
    D = _dict(8, 16, 24)
    X = rng.standard_normal((5, 8))
    lam = np.abs(X @ D).max() * 1.01
    da, loss = oracle.slista_grad(D, X, lam, np.full(6, 0.1))
    assert not da.any()
    np.testing.assert_allclose(loss, 0.5 * (X * X).sum(), rtol=1e-14)


def test_convolutional_dictionary_is_the_convolution():
    """The dense matrix of a 1-D convolutional dictionary (Section 6's
    structured dictionaries), which the oracle iterates with, against the
    operator it stands for: D z = sum_k d_k * z_k (numpy's full convolution of
    each code map with its filter, length P + Lf - 1 = n) and
    (D^T r)_k = the valid correlation of r with d_k; unit-norm columns."""
    rng = np.random.default_rng(11)
    for (K, Lf, n) in [(3, 5, 37), (8, 16, 128), (2, 9, 9)]:
        F = synth.conv_filters(K, Lf, rng)
        D = synth.conv_dictionary(F, n).astype(np.float64)
        P = n - Lf + 1
        assert D.shape == (n, K * P)
        np.testing.assert_allclose(np.linalg.norm(D, axis=0), 1.0, rtol=1e-6)
        z = rng.standard_normal(K * P)
        r = rng.standard_normal(n)
        Dz = sum(np.convolve(z[k * P:(k + 1) * P], F[k].astype(np.float64)) for k in range(K))
        np.testing.assert_allclose(D @ z, Dz, rtol=1e-12, atol=1e-12)
        Dtr = np.concatenate([np.correlate(r, F[k].astype(np.float64), mode="valid") for k in range(K)])
        np.testing.assert_allclose(D.T @ r, Dtr, rtol=1e-12, atol=1e-12)


def test_2d_convolutional_dictionary_is_the_convolution():
    """The dense matrix of a 2-D convolutional dictionary against the operator
    it stands for: D z = sum_k d_k * z_k (scipy's full 2-D convolution of each
    code map with its filter, (Ph + Lh - 1) x (Pw + Lw - 1) = H x W) and
    (D^T r)_k = the valid 2-D correlation of r with d_k; unit-norm columns."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(12)
    for (K, Lh, Lw, H, W) in [(3, 3, 4, 9, 11), (4, 5, 5, 16, 16), (2, 7, 2, 7, 5)]:
        F = synth.conv2d_filters(K, Lh, Lw, rng)
        D = synth.conv2d_dictionary(F, H, W).astype(np.float64)
        Ph, Pw = H - Lh + 1, W - Lw + 1
        assert D.shape == (H * W, K * Ph * Pw)
        np.testing.assert_allclose(np.linalg.norm(D, axis=0), 1.0, rtol=1e-6)
        z = rng.standard_normal((K, Ph, Pw))
        r = rng.standard_normal((H, W))
        Fd = F.astype(np.float64)
        Dz = sum(signal.convolve2d(z[k], Fd[k], mode="full") for k in range(K))
        np.testing.assert_allclose(D @ z.reshape(-1), Dz.reshape(-1), rtol=1e-12, atol=1e-12)
        Dtr = np.stack([signal.correlate2d(r, Fd[k], mode="valid") for k in range(K)])
        np.testing.assert_allclose(D.T @ r.reshape(-1), Dtr.reshape(-1), rtol=1e-12, atol=1e-12)
