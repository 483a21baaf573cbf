"""Parity of the wide-dictionary path (256 < m <= 1024: per-layer tcgen05
kernels, column-blocked Gram and objective) with the FP64 oracle, through
the C ABI.  Tolerances are those of the resident tensor-core kernels
(test_gpu_tc.py): BF16X3 objective 1e-5, codes 1e-4 * max(1, max|z|),
gradient 1e-4 (relative 2-norm); BF16 objective 1e-3, codes 2e-2."""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": {"F": 1e-5, "Z": 1e-4, "grad": 1e-4}, "bf16": {"F": 1e-3, "Z": 2e-2, "grad": 3e-2}}


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


_L = {}


def lipschitz(D):
    """oracle.lipschitz, cached per dictionary (Jacobi on 1024 x 1024 takes seconds)."""
    key = (D.shape, hash(D.tobytes()))
    if key not in _L:
        _L[key] = oracle.lipschitz(D)
    return _L[key]


def _case(n, m, N, seed, density=0.05, frac=0.1):
    rng = np.random.default_rng(seed)
    D = synth.gaussian_dictionary(n, m, rng)
    X = synth.sparse_model_samples(D, N, density, 0.01, rng)
    return D, X, synth.lam_fraction(D, X, frac)


def _check(prec, Zg, Fg, Zo, Fo):
    zt = TOL[prec]["Z"] * max(1.0, float(np.abs(Zo).max()))
    zerr = float(np.abs(Zg.astype(np.float64) - Zo).max())
    ferr = float((np.abs(Fg - Fo) / np.abs(Fo)).max())
    assert zerr <= zt, (prec, zerr, zt)
    assert ferr <= TOL[prec]["F"], (prec, ferr)


@pytest.mark.parametrize("n,m", [(64, 320), (128, 512), (100, 400), (256, 1024)])
def test_gram_wide(n, m):
    D, X, _ = _case(n, m, 300, n + m)
    A = api()
    g = A.gram(dev(D), dev(X))
    Bo, Co, xo = oracle.gram(D, X)
    assert np.abs(host(g.B) - Bo).max() <= 2e-6 * max(1.0, np.abs(Bo).max())
    assert np.abs(host(g.C) - Co).max() <= 2e-6 * max(1.0, np.abs(Co).max())
    np.testing.assert_allclose(host(g.xsq), xo, rtol=1e-12)
    Lo = lipschitz(D)
    assert abs(float(host(g.L)[0]) - Lo) <= 1e-5 * Lo


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("n,m,N", [(64, 320, 300), (128, 512, 129), (100, 400, 1), (256, 1024, 260)])
def test_slista_forward_wide(prec, n, m, N):
    """Several row tiles with a ragged tail, m not a multiple of the 256-column block."""
    D, X, lam = _case(n, m, N, 7 * n + m)
    T = 20
    alpha = synth.step_sizes(T, 1.0 / lipschitz(D), 0.3, seed=5)
    A = api()
    g = A.gram(dev(D), dev(X))
    Z = A.slista(g.B, g.C, lam, dev(alpha), prec=prec)
    F = host(A.objective(g.B, g.C, g.xsq, Z, lam, with_gap=False))
    Zo = oracle.pgd(D, X, lam, alpha)
    _check(prec, host(Z), F, Zo, oracle.objective(D, X, Zo, lam, with_gap=False))


def test_wide_masks_bit_exact_where_safe():
    from paper_1905_11071_gb300 import _lib
    D, X, lam = _case(128, 512, 200, 3)
    T = 16
    alpha = synth.step_sizes(T, 1.0 / lipschitz(D), 0.3, seed=8)
    A = api()
    g = A.gram(dev(D), dev(X))
    N, m = X.shape[0], D.shape[1]
    W = m // 32
    Z = torch.empty((N, m), dtype=torch.float32, device="cuda")
    masks = torch.zeros(_lib.slista_mask_words(m, N, T), dtype=torch.int32, device="cuda")
    ws = A.workspace(_lib.slista_workspace_bytes(_lib.FN_SLISTA_FWD, m, N, T, _lib.PREC_BF16X3), Z.device, "w")
    _lib.slista_forward(g.B, g.C, lam, dev(alpha), _lib.PREC_BF16X3, Z, masks=masks, ws=ws)
    Zall = oracle.pgd(D, X, lam, alpha, keep_all=True)
    words = host(masks).view(np.uint32).astype(np.uint64).reshape(T, N, W, 1)
    bits = ((words >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).reshape(T, N, m).astype(bool)
    D64, X64 = D.astype(np.float64), X.astype(np.float64)
    for t in range(T):
        u = Zall[t] - float(alpha[t]) * ((Zall[t] @ D64.T - X64) @ D64)
        safe = np.abs(np.abs(u) - float(alpha[t]) * lam) > 1e-4
        assert np.array_equal(bits[t][safe], (Zall[t + 1] != 0)[safe]), t


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_wide_ista_matches_slista_constant_step(prec):
    D, X, lam = _case(64, 320, 200, 11)
    A = api()
    g = A.gram(dev(D), dev(X))
    T = 12
    a = (1.0 / g.L.double()).float().expand(T).contiguous()
    assert torch.equal(A.ista(g.B, g.C, lam, g.L, T, prec=prec), A.slista(g.B, g.C, lam, a, prec=prec))


def test_wide_zero_above_lambda_max():
    D, X, _ = _case(128, 512, 150, 13)
    lam = float(np.float32(np.abs(X.astype(np.float64) @ D.astype(np.float64)).max() * 1.001))
    A = api()
    g = A.gram(dev(D), dev(X))
    assert not A.ista(g.B, g.C, lam, g.L, 6, prec="bf16x3").any()


def test_wide_objective_and_gap():
    """FP32 objective / duality gap at m = 1024 on codes the oracle produced
    (the codes are an input here, not a GPU result)."""
    D, X, lam = _case(256, 1024, 200, 17)
    Zo = oracle.ista(D, X, lam, lipschitz(D), 10).astype(np.float32)
    A = api()
    g = A.gram(dev(D), dev(X))
    F, gap = A.objective(g.B, g.C, g.xsq, dev(Zo), lam)
    Fo, go = oracle.objective(D, X, Zo.astype(np.float64), lam)
    np.testing.assert_allclose(host(F), Fo, rtol=1e-5)
    assert np.all(host(gap) >= -1e-6 * np.abs(Fo))
    np.testing.assert_allclose(host(gap), go, rtol=1e-3, atol=1e-5 * np.abs(Fo).max())


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("n,m,K", [(64, 320, 3), (64, 320, 12), (256, 1024, 4)])
def test_wide_backward_matches_oracle_gradient(prec, n, m, K):
    D, X, lam = _case(n, m, 160, 19 + m)
    T = 12
    alpha = synth.step_sizes(T, 1.0 / lipschitz(D), 0.3, seed=7)
    A = api()
    g = A.gram(dev(D), dev(X))
    _, st = A.slista(g.B, g.C, lam, dev(alpha), prec=prec, keep_for_backward=True, ckpt_every=K)
    dg = host(A.slista_grad(g.B, g.C, lam, dev(alpha), st, prec=prec)).astype(np.float64)
    do, _ = oracle.slista_grad(D, X, lam, alpha)
    rel = np.linalg.norm(dg - do) / np.linalg.norm(do)
    assert rel <= TOL[prec]["grad"], (prec, K, rel)


def test_wide_backward_upstream_gradient_linear_and_deterministic():
    D, X, lam = _case(64, 320, 140, 23)
    T = 8
    alpha = synth.step_sizes(T, 1.0 / lipschitz(D), 0.3, seed=3)
    A = api()
    g = A.gram(dev(D), dev(X))
    Z, st = A.slista(g.B, g.C, lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=3)
    rng = np.random.default_rng(1)
    G1 = dev(rng.standard_normal(Z.shape).astype(np.float32))
    d1 = A.slista_grad(g.B, g.C, lam, dev(alpha), st, gZ=G1, prec="bf16x3")
    d2 = A.slista_grad(g.B, g.C, lam, dev(alpha), st, gZ=2 * G1, prec="bf16x3")
    torch.testing.assert_close(d2, 2 * d1, rtol=1e-5, atol=1e-5 * float(d1.abs().max()))
    assert torch.equal(d1, A.slista_grad(g.B, g.C, lam, dev(alpha), st, gZ=G1, prec="bf16x3"))
    assert not A.slista_grad(g.B, g.C, lam, dev(alpha), st, gZ=torch.zeros_like(Z), prec="bf16x3").any()


def test_large_256x1024_full_size_sampled_rows():
    """The large configuration (D 256 x 1024, N = 100000, T = 50, lam = 0.05 lam_max):
    forward on the full batch; 32 sampled rows against the oracle."""
    w = synth.large_256x1024()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    alpha = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    Z = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3")
    F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
    assert np.isfinite(F).all() and (F <= 0.5 * host(g.xsq) + 1e-6).all()
    rows = np.random.default_rng(4).choice(w.N, size=32, replace=False)
    Lo = lipschitz(w.D)
    Zo = oracle.ista(w.D, w.X[rows], w.lam, Lo, w.T)
    _check("bf16x3", host(Z)[rows], F[rows], Zo, oracle.objective(w.D, w.X[rows], Zo, w.lam, with_gap=False))


def test_wide_unaligned_c_matches_aligned():
    """m > 256 with C 4 bytes past a 16-byte boundary: scalar loads, same codes."""
    D, X, lam = _case(64, 320, 200, 29)
    A = api()
    g = A.gram(dev(D), dev(X))
    buf = torch.empty(g.C.numel() + 1, dtype=torch.float32, device="cuda")
    buf[1:] = g.C.reshape(-1)
    Cu = buf[1:].view(g.C.shape)
    assert Cu.data_ptr() % 16 != 0
    alpha = dev(synth.step_sizes(10, 1.0 / lipschitz(D), 0.3, seed=4))
    assert torch.equal(A.slista(g.B, g.C, lam, alpha, prec="bf16x3"), A.slista(g.B, Cu, lam, alpha, prec="bf16x3"))
