"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path):
  * codes z: |z_gpu - z_oracle| <= 2e-5 * max(1, max|z_oracle|) elementwise;
  * objective: |F_gpu - F_oracle| <= 1e-5 * F_oracle per sample, where F_gpu is
    the GPU objective kernel on the GPU codes and F_oracle the oracle's
    objective on its own codes (no GPU value is ever fed to the oracle);
  * support masks: bit-exact wherever the oracle's pre-threshold margin
    ||u| - alpha lam| exceeds 1e-4;
  * step-size sub-gradient: ||d_gpu - d_oracle||_2 <= 1e-4 ||d_oracle||_2;
  * Oracle-ISTA: the same bounds, layer by layer, on every sample up to its
    first layer whose oracle decision margin is at most 5e-6 (smaller margins
    can flip on rounding; tests/oista_layerwise.py);
  * L and L_S: relative error <= 1e-5 (FP32 Lanczos and Sturm multisection:
    rounding of the products and of the pivots, about k 2^-24 for k <= 64,
    plus the stopping rule's 2e-7).
"""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z_TOL = 2e-5
F_TOL = 1e-5
MASK_MARGIN = 1e-4
GRAD_TOL = 1e-4
OISTA_MARGIN = 5e-6
EIG_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib_ready():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1905_11071_gb300 import build, _lib
    build.build()
    _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def api():
    from paper_1905_11071_gb300 import api as A
    return A


def check_codes(Zg, Zo):
    tol = Z_TOL * max(1.0, float(np.abs(Zo).max()))
    err = np.abs(Zg.astype(np.float64) - Zo)
    assert err.max() <= tol, (err.max(), tol)


def check_objective(Fg, Fo):
    rel = np.abs(Fg - Fo) / np.abs(Fo)
    assert rel.max() <= F_TOL, rel.max()


def pre_threshold(D, X, Zt, alpha):
    """u^t = z^t - alpha D^T(D z^t - x) in FP64 (test-side, for margins)."""
    return Zt - alpha * ((Zt @ D.T - X) @ D)


def unpack_masks(words, T, N, m):
    """uint32 support words -> bool[T, N, m] (bit j % 32 of word j // 32)."""
    W = (m + 31) // 32
    w = words[: T * N * W].astype(np.uint64).reshape(T, N, W, 1)
    bits = (w >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(T, N, W * 32)[:, :, :m].astype(bool)


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,N", [(10, 20, 1000), (64, 256, 777), (12, 8, 5), (64, 100, 33)])
def test_gram_parity(n, m, N):
    rng = np.random.default_rng(n * 1000 + m)
    D = synth.gaussian_dictionary(n, m, rng)
    X = rng.standard_normal((N, n)).astype(np.float32)
    g = api().gram(dev(D), dev(X))
    Bo, Co, xo = oracle.gram(D, X)
    np.testing.assert_allclose(host(g.B), Bo, rtol=0, atol=2e-6)
    assert np.array_equal(host(g.B), host(g.B).T)
    np.testing.assert_allclose(host(g.C), Co, rtol=0, atol=2e-6 * max(1.0, np.abs(Co).max()))
    np.testing.assert_allclose(host(g.xsq), xo, rtol=1e-12)
    Lo = oracle.lipschitz(D)
    assert abs(float(host(g.L)[0]) - Lo) <= EIG_TOL * Lo
    L2 = api().lipschitz(g.B)
    assert abs(float(host(L2)[0]) - Lo) <= EIG_TOL * Lo


def test_ista_forward_parity_10x20():
    """Plain ISTA, FP64 oracle vs FP32 GPU: D 10 x 20, N = 1000, T = 100."""
    w = synth.ista_10x20()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Zg = A.ista(g.B, g.C, w.lam, g.L, w.T)
    Fg = host(A.objective(g.B, g.C, g.xsq, Zg, w.lam, with_gap=False))
    Lo = oracle.lipschitz(w.D)
    Zo = oracle.ista(w.D, w.X, w.lam, Lo, w.T)
    check_codes(host(Zg), Zo)
    check_objective(Fg, oracle.objective(w.D, w.X, Zo, w.lam, with_gap=False))


def _slista_case(N=700, T=40, seed=5):
    w = synth.slista_64x256(N=N, T=T)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(T, 1.0 / Lo, 0.3, seed=seed)
    return w, Lo, alpha


def test_slista_forward_parity_masks_and_checkpoints():
    w, Lo, alpha = _slista_case()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    K = 7
    Zg, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=K)
    Zall = oracle.pgd(w.D, w.X, w.lam, alpha, keep_all=True)
    check_codes(host(Zg), Zall[-1])
    Fg = host(A.objective(g.B, g.C, g.xsq, Zg, w.lam, with_gap=False))
    check_objective(Fg, oracle.objective(w.D, w.X, Zall[-1], w.lam, with_gap=False))
    # masks: bit-exact where the oracle's margin is not tiny
    masks = unpack_masks(host(st.masks).view(np.uint32), w.T, w.N, w.m)
    D = w.D.astype(np.float64)
    X = w.X.astype(np.float64)
    for t in range(w.T):
        u = pre_threshold(D, X, Zall[t], float(alpha[t]))
        safe = np.abs(np.abs(u) - float(alpha[t]) * w.lam) > MASK_MARGIN
        want = Zall[t + 1] != 0
        assert np.array_equal(masks[t][safe], want[safe]), t
    # checkpoints hold z^(sK) and g^(sK) = c - B z^(sK)
    ck = host(st.ckpt).reshape(-1, 2, w.N, w.m)
    Bo, Co, _ = oracle.gram(w.D, w.X)
    for s in range(ck.shape[0]):
        t = (s + 1) * K
        check_codes(ck[s, 0], Zall[t])
        g_or = Co - Zall[t] @ Bo
        assert np.abs(ck[s, 1] - g_or).max() <= Z_TOL * max(1.0, np.abs(g_or).max())


def test_ista_equals_slista_with_constant_step():
    """ISTA is Step-LISTA with alpha_t = 1/L (Section 4, after Eq. steprec):
    the two entry points run the same kernel and agree bitwise."""
    w = synth.slista_64x256(N=300, T=20)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    a = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    Zi = A.ista(g.B, g.C, w.lam, g.L, w.T)
    Zs = A.slista(g.B, g.C, w.lam, a)
    assert torch.equal(Zi, Zs)


@pytest.mark.parametrize("K", [1, 3, 7, 40, 64])
def test_slista_backward_parity(K):
    w, Lo, alpha = _slista_case(N=200, T=40, seed=7)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    _, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=K)
    dg = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st)).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert np.linalg.norm(dg - do) <= GRAD_TOL * np.linalg.norm(do), (dg, do)


def test_slista_backward_independent_of_checkpoint_spacing():
    """Recomputation between checkpoints repeats the forward's arithmetic
    exactly, so the sub-gradient does not depend on the spacing (bitwise)."""
    w, Lo, alpha = _slista_case(N=300, T=30, seed=9)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    outs = []
    for K in (1, 2, 5, 6, 30):
        _, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=K)
        outs.append(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st))
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_slista_backward_upstream_gradient_is_linear():
    w, Lo, alpha = _slista_case(N=100, T=12, seed=11)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=4)
    zero = torch.zeros_like(Z)
    d0 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=zero)
    assert not d0.any()
    rng = np.random.default_rng(3)
    G1 = dev(rng.standard_normal(Z.shape).astype(np.float32))
    d1 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=G1)
    d2 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=2 * G1)
    torch.testing.assert_close(d2, 2 * d1, rtol=1e-5, atol=1e-5 * float(d1.abs().max()))


def _oista_runner(A, g, lam, D=None):
    def run(t):
        Z, LS, acc = A.oista(g.B, g.C, lam, g.L, t, D=D)
        return host(Z), host(LS), host(acc)
    return run


def test_oista_parity_fig3_setup():
    """OISTA on the toy setup of Fig. 3 (D 10 x 50, lam = 0.5, x in B_inf),
    compared layer by layer (tests/oista_layerwise.py)."""
    from oista_layerwise import compare_layerwise
    w = synth.paper_binf(10, 50, N=400, lam=0.5, T=100, seed=2)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    r = compare_layerwise(_oista_runner(A, g, w.lam), w.D, w.X, w.lam, w.T, OISTA_MARGIN, Z_TOL, ls_rtol=EIG_TOL)
    assert r["frac"] >= 0.9
    done = r["first"] >= w.T
    Zg, _, _ = A.oista(g.B, g.C, w.lam, g.L, w.T)
    Fg = host(A.objective(g.B, g.C, g.xsq, Zg, w.lam, with_gap=False))
    check_objective(Fg[done], oracle.objective(w.D, w.X, r["Zo"], w.lam, with_gap=False)[done])


@pytest.mark.parametrize("with_D", [True, False])
def test_oista_parity_64x256(with_D):
    """Supports larger than 64 are solved on D_S D_S^T when D is given, else by
    Lanczos with the products read from global memory; layer by layer."""
    from oista_layerwise import compare_layerwise
    w = synth.slista_64x256(N=300, T=40)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    r = compare_layerwise(_oista_runner(A, g, w.lam, dev(w.D) if with_D else None), w.D, w.X, w.lam, w.T,
                          OISTA_MARGIN, Z_TOL, ls_rtol=EIG_TOL)
    print("fp32 oista 64x256: compared %.3f of (sample, layer) pairs, worst code error %.3g" % (r["frac"], r["worst"]))
    assert r["frac"] >= 0.9


def _pack_supports(mask):
    """Rows of a boolean N x m support array as N x ceil(m/32) int32 words
    (bit j % 32 of word j / 32 set iff code j is in the support)."""
    N, m = mask.shape
    words = np.zeros((N, (m + 31) // 32), dtype=np.uint32)
    for j in range(m):
        words[:, j // 32] |= mask[:, j].astype(np.uint32) << np.uint32(j % 32)
    return words.view(np.int32)


@pytest.mark.parametrize("with_D", [True, False])
def test_support_lipschitz_parity(with_D):
    """lasso_support_lipschitz (Eq. spca) on seeded supports of every solver
    class (|S| = 0, 1, <= 32, 33 - 64, > 64 on D_S D_S^T or from B) against
    the oracle's Jacobi value; L_empty = L."""
    w = synth.slista_64x256(N=8, T=1)
    rng = np.random.default_rng(31)
    sizes = [0, 1, 2, 3, 5, 9, 17, 31, 32, 33, 40, 57, 63, 64, 65, 80, 100, 140, 256]
    reps = [4 if k <= 64 else 2 for k in sizes]
    mask = np.zeros((sum(reps), w.m), dtype=bool)
    r = 0
    for k, c in zip(sizes, reps):
        for _ in range(c):
            mask[r, rng.choice(w.m, size=k, replace=False)] = True
            r += 1
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    LSg = host(A.support_lipschitz(g.B, dev(_pack_supports(mask)), g.L, D=dev(w.D) if with_D else None))
    Lo = oracle.lipschitz(w.D)
    LSo = np.array([oracle.support_lipschitz(w.D, mask[i], Lo) for i in range(len(mask))])
    np.testing.assert_allclose(LSg, LSo, rtol=EIG_TOL)
    assert LSg[0] == host(g.L)[0]  # empty support: L itself


def test_support_lipschitz_ignores_bits_past_m():
    """Bits of codes >= m in the last support word are not part of S."""
    w = synth.paper_binf(10, 50, N=8, lam=0.5, T=1, seed=2)
    rng = np.random.default_rng(32)
    mask = rng.random((64, 50)) < 0.3
    words = _pack_supports(mask).view(np.uint32).copy()
    dirty = words.copy()
    dirty[:, 1] |= np.uint32(0xFFFC0000)  # codes 50 .. 63
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    clean = host(A.support_lipschitz(g.B, dev(words.view(np.int32)), g.L))
    noisy = host(A.support_lipschitz(g.B, dev(dirty.view(np.int32)), g.L))
    assert np.array_equal(clean, noisy)
    Lo = oracle.lipschitz(w.D)
    np.testing.assert_allclose(clean, [oracle.support_lipschitz(w.D, mask[i], Lo) for i in range(64)], rtol=EIG_TOL)


def test_objective_and_gap_parity():
    """Objective/gap kernel on codes drawn by the test (not by the GPU)."""
    w = synth.slista_64x256(N=500, T=1)
    rng = np.random.default_rng(4)
    Z = (rng.standard_normal((w.N, w.m)) * (rng.random((w.N, w.m)) < 0.05)).astype(np.float32)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    F, gap = A.objective(g.B, g.C, g.xsq, dev(Z), w.lam)
    Fo, go = oracle.objective(w.D, w.X, Z, w.lam)
    check_objective(host(F), Fo)
    assert np.abs(host(gap) - go).max() <= 1e-5 * np.abs(Fo).max()
    # at an (oracle) converged point the gap is ~0
    Lo = oracle.lipschitz(w.D)
    Zc = oracle.ista(w.D, w.X[:20], w.lam, Lo, 3000).astype(np.float32)
    g2 = A.gram(dev(w.D), dev(w.X[:20]))
    _, gap2 = A.objective(g2.B, g2.C, g2.xsq, dev(Zc), w.lam)
    assert (host(gap2) >= -1e-5).all() and host(gap2).max() < 1e-4


# --------------------------------------------------------------------------- edge cases

def test_zero_solution_above_lambda_max():
    """lam >= lam_max: every variant returns exactly 0 (Section 2)."""
    w = synth.slista_64x256(N=100, T=10)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    assert not A.ista(g.B, g.C, lam, g.L, 10).any()
    a = dev(np.full(10, 0.1, np.float32))
    Z, st = A.slista(g.B, g.C, lam, a, keep_for_backward=True, ckpt_every=3)
    assert not Z.any()
    assert not st.masks.any()
    assert not A.slista_grad(g.B, g.C, lam, a, st).any()
    Zo, _, _ = A.oista(g.B, g.C, lam, g.L, 10)
    assert not Zo.any()


def test_identity_dictionary_is_exact():
    """D = Id: B = Id and C = X exactly, L = 1, and one ISTA layer is the
    closed form ST(x, lam) (Section 3, orthogonal case), bit for bit."""
    rng = np.random.default_rng(5)
    m = 64
    D = np.eye(m, dtype=np.float32)
    X = rng.standard_normal((77, m)).astype(np.float32)
    lam = 0.5
    A = api()
    g = A.gram(dev(D), dev(X))
    assert torch.equal(g.B, dev(D)) and torch.equal(g.C, dev(X))
    assert float(host(g.L)[0]) == 1.0
    Z = host(A.ista(g.B, g.C, lam, g.L, 1))
    want = np.sign(X) * np.maximum(np.abs(X) - np.float32(lam), 0)
    assert np.array_equal(Z, want)
    Zo, _, acc = A.oista(g.B, g.C, lam, g.L, 3)
    assert np.array_equal(host(Zo), want)


@pytest.mark.parametrize("N", [0, 1, 31, 33])
def test_small_and_ragged_batches(N):
    w, Lo, alpha = _slista_case(N=max(N, 1), T=9, seed=13)
    X = w.X[:N]
    A = api()
    g = A.gram(dev(w.D), dev(X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=3)
    da = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st)
    if N == 0:
        assert Z.numel() == 0 and not da.any()
        return
    check_codes(host(Z), oracle.pgd(w.D, X, w.lam, alpha))
    do, _ = oracle.slista_grad(w.D, X, w.lam, alpha)
    assert np.linalg.norm(host(da) - do) <= GRAD_TOL * max(np.linalg.norm(do), 1e-12)


def test_zero_layers():
    w = synth.slista_64x256(N=50, T=1)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    assert not A.ista(g.B, g.C, w.lam, g.L, 0).any()


def test_small_m_padding():
    """m = 20 is padded to 32 inside the kernels; padding stays zero."""
    w = synth.ista_10x20(N=300, T=30)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(w.T, 1.0 / Lo, 0.4, seed=3)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), keep_for_backward=True, ckpt_every=5)
    check_codes(host(Z), oracle.pgd(w.D, w.X, w.lam, alpha))
    da = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st))
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert np.linalg.norm(da - do) <= GRAD_TOL * np.linalg.norm(do)


# --------------------------------------------------------------------------- full size, sampled

def test_full_size_forward_sampled_rows():
    """The benchmark workload (64 x 256, N = 10000, T = 40) in the benchmark's
    launch configuration; 64 sampled rows against the oracle (samples are
    independent), every row checked for finiteness and F <= F(0)."""
    w = synth.slista_64x256()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    alpha = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    Z, st = A.slista(g.B, g.C, w.lam, alpha, keep_for_backward=True)
    F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
    assert np.isfinite(F).all() and (F <= 0.5 * host(g.xsq) + 1e-6).all()
    rows = np.random.default_rng(0).choice(w.N, size=64, replace=False)
    Lo = oracle.lipschitz(w.D)
    Zo = oracle.ista(w.D, w.X[rows], w.lam, Lo, w.T)
    check_codes(host(Z)[rows], Zo)
    check_objective(F[rows], oracle.objective(w.D, w.X[rows], Zo, w.lam, with_gap=False))
    # the sub-gradient is a sum over samples: full batch = sum of two halves
    da = A.slista_grad(g.B, g.C, w.lam, alpha, st).double()
    parts = []
    for sl in (slice(0, 4000), slice(4000, w.N)):
        C = g.C[sl].contiguous()
        _, s2 = A.slista(g.B, C, w.lam, alpha, keep_for_backward=True)
        parts.append(A.slista_grad(g.B, C, w.lam, alpha, s2).double())
    torch.testing.assert_close(da, parts[0] + parts[1], rtol=1e-5, atol=1e-5 * float(da.abs().max()))
