"""Parity of the tcgen05 tensor-core forward (SLISTA_PREC_BF16X3 and
SLISTA_PREC_BF16) with the FP64 oracle, through the C ABI.

Tolerances: relative objective error per sample <= 1e-5 for the split
BF16X3 product and <= 1e-3 for plain BF16 (the two precision classes the
method is held to); codes z elementwise <= 1e-4 * max(1, max|z|) (BF16X3) and
<= 2e-2 * max(1, max|z|) (BF16); support masks bit-exact where the oracle's
pre-threshold margin exceeds 1e-4 (BF16X3).
"""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": {"F": 1e-5, "Z": 1e-4}, "bf16": {"F": 1e-3, "Z": 2e-2}}


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


def _check(prec, Zg, Fg, Zo, Fo):
    zt = TOL[prec]["Z"] * max(1.0, float(np.abs(Zo).max()))
    zerr = float(np.abs(Zg.astype(np.float64) - Zo).max())
    ferr = float((np.abs(Fg - Fo) / np.abs(Fo)).max())
    assert zerr <= zt, (prec, zerr, zt)
    assert ferr <= TOL[prec]["F"], (prec, ferr)
    return zerr, ferr


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("N", [1, 127, 128, 700])
def test_slista_forward_tc_64x256(prec, N):
    w = synth.slista_64x256(N=N, T=40)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(w.T, 1.0 / Lo, 0.3, seed=5)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z = A.slista(g.B, g.C, w.lam, dev(alpha), prec=prec)
    F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
    Zo = oracle.pgd(w.D, w.X, w.lam, alpha)
    Fo = oracle.objective(w.D, w.X, Zo, w.lam, with_gap=False)
    _check(prec, host(Z), F, Zo, Fo)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("n,m", [(10, 20), (32, 64), (48, 100), (64, 128)])
def test_slista_forward_tc_small_m(prec, n, m):
    """m padded to 64 / 128 inside the kernel (B_lo resident)."""
    rng = np.random.default_rng(n + m)
    D = synth.gaussian_dictionary(n, m, rng)
    X = synth.sparse_model_samples(D, 300, 0.1, 0.01, rng)
    lam = synth.lam_fraction(D, X, 0.1)
    T = 30
    Lo = oracle.lipschitz(D)
    alpha = synth.step_sizes(T, 1.0 / Lo, 0.3, seed=6)
    A = api()
    g = A.gram(dev(D), dev(X))
    Z = A.slista(g.B, g.C, lam, dev(alpha), prec=prec)
    F = host(A.objective(g.B, g.C, g.xsq, Z, lam, with_gap=False))
    Zo = oracle.pgd(D, X, lam, alpha)
    _check(prec, host(Z), F, Zo, oracle.objective(D, X, Zo, lam, with_gap=False))


def test_tc_masks_bit_exact_where_safe():
    w = synth.slista_64x256(N=300, T=40)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(w.T, 1.0 / Lo, 0.3, seed=8)
    A = api()
    from paper_1905_11071_gb300 import _lib
    g = A.gram(dev(w.D), dev(w.X))
    Z = torch.empty((w.N, w.m), dtype=torch.float32, device="cuda")
    masks = torch.zeros(_lib.slista_mask_words(w.m, w.N, w.T), dtype=torch.int32, device="cuda")
    ws = A.workspace(_lib.slista_workspace_bytes(_lib.FN_SLISTA_FWD, w.m, w.N, w.T, _lib.PREC_BF16X3),
                     Z.device, "t")
    _lib.slista_forward(g.B, g.C, w.lam, dev(alpha), _lib.PREC_BF16X3, Z, masks=masks, ws=ws)
    Zall = oracle.pgd(w.D, w.X, w.lam, alpha, keep_all=True)
    words = host(masks).view(np.uint32).astype(np.uint64).reshape(w.T, w.N, 8, 1)
    bits = ((words >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).reshape(w.T, w.N, 256).astype(bool)
    D = w.D.astype(np.float64)
    X = w.X.astype(np.float64)
    for t in range(w.T):
        u = Zall[t] - float(alpha[t]) * ((Zall[t] @ D.T - X) @ D)
        safe = np.abs(np.abs(u) - float(alpha[t]) * w.lam) > 1e-4
        assert np.array_equal(bits[t][safe], (Zall[t + 1] != 0)[safe]), t


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_ista_matches_slista_constant_step(prec):
    w = synth.slista_64x256(N=260, T=25)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    a = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    assert torch.equal(A.ista(g.B, g.C, w.lam, g.L, w.T, prec=prec), A.slista(g.B, g.C, w.lam, a, prec=prec))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_identity_dictionary_one_layer_exact(prec):
    """D = Id: the first layer reads g = c exactly, so z^(1) = ST(x, lam) bit for bit."""
    rng = np.random.default_rng(9)
    D = np.eye(128, dtype=np.float32)
    X = rng.standard_normal((200, 128)).astype(np.float32)
    A = api()
    g = A.gram(dev(D), dev(X))
    Z = host(A.ista(g.B, g.C, 0.5, g.L, 1, prec=prec))
    want = np.sign(X) * np.maximum(np.abs(X) - np.float32(0.5), 0)
    assert np.array_equal(Z, want)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_zero_above_lambda_max(prec):
    w = synth.slista_64x256(N=200, T=10)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    assert not A.ista(g.B, g.C, lam, g.L, 10, prec=prec).any()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_tc_full_size_sampled_rows(prec):
    """The benchmark workload (64 x 256, N = 10000, T = 40), 64 sampled rows."""
    w = synth.slista_64x256()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    alpha = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    Z = A.slista(g.B, g.C, w.lam, alpha, prec=prec)
    F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
    assert np.isfinite(F).all()
    rows = np.random.default_rng(1).choice(w.N, size=64, replace=False)
    Lo = oracle.lipschitz(w.D)
    Zo = oracle.ista(w.D, w.X[rows], w.lam, Lo, w.T)
    Fo = oracle.objective(w.D, w.X[rows], Zo, w.lam, with_gap=False)
    _check(prec, host(Z)[rows], F[rows], Zo, Fo)


def test_tc_device_flag_clear_after_runs():
    from paper_1905_11071_gb300 import _lib
    _lib.slista_device_status()


def test_bounded_wait_expiry_is_reported_once():
    """Failure detection without a fault: a kernel waits with the library's
    bounded wait on an mbarrier that nothing arrives at, its limit lowered to
    a few thousand cycles; the wait expires, the device flag is raised,
    slista_device_status reports SLISTA_ERR_TIMEOUT once and clears the flag,
    and the context stays usable (the next status is OK and a layer call
    still gives the same codes)."""
    import ctypes
    from paper_1905_11071_gb300 import _lib
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    w = synth.slista_64x256(N=200, T=10)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    a = dev(synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.2, seed=3))
    Z0 = A.slista(g.B, g.C, w.lam, a, prec="bf16x3")
    assert lib.slista_device_status(st) == _lib.SLISTA_OK
    assert lib.slista_wait_probe(0, st) == _lib.SLISTA_ERR_ARG  # limits outside 1 .. 1e8 are refused
    assert lib.slista_wait_probe(4000, st) == _lib.SLISTA_OK
    assert lib.slista_device_status(st) == _lib.SLISTA_ERR_TIMEOUT
    assert "expired" in lib.slista_last_error().decode()
    assert lib.slista_device_status(st) == _lib.SLISTA_OK
    assert torch.equal(A.slista(g.B, g.C, w.lam, a, prec="bf16x3"), Z0)
    assert lib.slista_device_status(st) == _lib.SLISTA_OK


@pytest.mark.parametrize("K", [1, 7, 40])
def test_tc_forward_with_fp32_adjoint(K):
    """Step-size sub-gradient when the forward (masks, checkpoints) runs on the
    tensor cores (BF16X3) and the adjoint recomputes segments in FP32."""
    w = synth.slista_64x256(N=300, T=40)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(w.T, 1.0 / Lo, 0.3, seed=7)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=K)
    dg = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st)).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert np.linalg.norm(dg - do) <= 1e-4 * np.linalg.norm(do), (np.linalg.norm(dg - do) / np.linalg.norm(do))
    # the tensor-core checkpoints hold z^(t) and g^(t) = c - B z^(t)
    if st.ckpt is not None:
        Zall = oracle.pgd(w.D, w.X, w.lam, alpha, keep_all=True)
        Bo, Co, _ = oracle.gram(w.D, w.X)
        ck = host(st.ckpt).reshape(-1, 2, w.N, w.m)
        for s in range(ck.shape[0]):
            t = (s + 1) * K
            zt = TOL["bf16x3"]["Z"] * max(1.0, np.abs(Zall[t]).max())
            assert np.abs(ck[s, 0] - Zall[t]).max() <= zt
            g_or = Co - Zall[t] @ Bo
            assert np.abs(ck[s, 1] - g_or).max() <= TOL["bf16x3"]["Z"] * max(1.0, np.abs(g_or).max())


# --------------------------------------------------------------------------- tensor-core adjoint

GRAD_TOL = {"bf16x3": 1e-4, "bf16": 3e-2}


def _grad_case(N=300, T=40, seed=7):
    w = synth.slista_64x256(N=N, T=T)
    Lo = oracle.lipschitz(w.D)
    alpha = synth.step_sizes(w.T, 1.0 / Lo, 0.3, seed=seed)
    return w, alpha


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("K", [1, 3, 7, 40])
def test_tc_backward_matches_oracle_gradient(prec, K):
    """Forward and adjoint both on the tensor cores (Eq. steprec and its
    chain rule); the sub-gradient of sum_i F(z_i^(T)) against the FP64 oracle."""
    w, alpha = _grad_case()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    _, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec=prec, keep_for_backward=True, ckpt_every=K)
    dg = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec=prec)).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    rel = np.linalg.norm(dg - do) / np.linalg.norm(do)
    assert rel <= GRAD_TOL[prec], (prec, K, rel)


def test_tc_backward_deterministic():
    w, alpha = _grad_case(N=500, T=20, seed=3)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    _, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=5)
    d1 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3")
    d2 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3")
    assert torch.equal(d1, d2)


def test_tc_backward_upstream_gradient():
    """gZ = dF/dz^(T) formed on the host in FP64 from the returned codes gives
    the default gradient; gZ = 0 gives 0; the map gZ -> dalpha is linear."""
    w, alpha = _grad_case(N=256, T=12, seed=11)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    d_default = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3")).astype(np.float64)
    Bo, Co, _ = oracle.gram(w.D, w.X)
    Zh = host(Z).astype(np.float64)
    GT = Zh @ Bo - Co + w.lam * np.sign(Zh)
    d_gz = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=dev(GT.astype(np.float32)),
                              prec="bf16x3")).astype(np.float64)
    assert np.linalg.norm(d_gz - d_default) <= 1e-4 * np.linalg.norm(d_default)
    zero = torch.zeros_like(Z)
    assert not A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=zero, prec="bf16x3").any()
    rng = np.random.default_rng(3)
    G1 = dev(rng.standard_normal(Z.shape).astype(np.float32))
    d1 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=G1, prec="bf16x3")
    d2 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=2 * G1, prec="bf16x3")
    torch.testing.assert_close(d2, 2 * d1, rtol=1e-5, atol=1e-5 * float(d1.abs().max()))


@pytest.mark.parametrize("N", [1, 127, 129])
def test_tc_backward_small_and_ragged_batches(N):
    w, alpha = _grad_case(N=N, T=15, seed=13)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    _, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    dg = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3")).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert np.linalg.norm(dg - do) <= GRAD_TOL["bf16x3"] * max(np.linalg.norm(do), 1e-12), (dg, do)


@pytest.mark.parametrize("n,m", [(10, 20), (48, 100), (64, 128)])
def test_tc_backward_small_m(n, m):
    """m padded to 64 / 128 inside the kernels (B_lo resident)."""
    rng = np.random.default_rng(n + m)
    D = synth.gaussian_dictionary(n, m, rng)
    X = synth.sparse_model_samples(D, 300, 0.1, 0.01, rng)
    lam = synth.lam_fraction(D, X, 0.1)
    T = 30
    alpha = synth.step_sizes(T, 1.0 / oracle.lipschitz(D), 0.3, seed=6)
    A = api()
    g = A.gram(dev(D), dev(X))
    _, st = A.slista(g.B, g.C, lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=6)
    dg = host(A.slista_grad(g.B, g.C, lam, dev(alpha), st, prec="bf16x3")).astype(np.float64)
    do, _ = oracle.slista_grad(D, X, lam, alpha)
    assert np.linalg.norm(dg - do) <= GRAD_TOL["bf16x3"] * np.linalg.norm(do), (np.linalg.norm(dg - do) / np.linalg.norm(do))


def test_tc_backward_full_size_split_batch():
    """The benchmark workload (64 x 256, N = 10000, T = 40, checkpoints every
    7 layers): the sub-gradient is a sum over samples, so the full batch
    equals the sum over two halves; 256 sampled rows against the oracle."""
    w = synth.slista_64x256()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    alpha = dev(np.full(w.T, 1.0 / oracle.lipschitz(w.D), dtype=np.float32))
    _, st = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3", keep_for_backward=True)
    da = A.slista_grad(g.B, g.C, w.lam, alpha, st, prec="bf16x3").double()
    parts = []
    for sl in (slice(0, 4000), slice(4000, w.N)):
        C = g.C[sl].contiguous()
        _, s2 = A.slista(g.B, C, w.lam, alpha, prec="bf16x3", keep_for_backward=True)
        parts.append(A.slista_grad(g.B, C, w.lam, alpha, s2, prec="bf16x3").double())
    torch.testing.assert_close(da, parts[0] + parts[1], rtol=1e-4, atol=1e-4 * float(da.abs().max()))
    rows = np.random.default_rng(2).choice(w.N, size=256, replace=False)
    C = g.C[torch.from_numpy(rows).cuda()].contiguous()
    _, s3 = A.slista(g.B, C, w.lam, alpha, prec="bf16x3", keep_for_backward=True)
    dg = host(A.slista_grad(g.B, C, w.lam, alpha, s3, prec="bf16x3")).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X[rows], w.lam, host(alpha).astype(np.float32))
    assert np.linalg.norm(dg - do) <= GRAD_TOL["bf16x3"] * np.linalg.norm(do)


# --------------------------------------------------------------------------- Oracle-ISTA on the tensor cores

# Each sample is compared layer by layer up to its first layer whose oracle
# decision margin is at most OISTA_LAYER_MARGIN (tests/oista_layerwise.py);
# a decision with a larger margin that flipped would show as a code error.
OISTA_LAYER_MARGIN = 5e-6
# decisions along the whole trajectory, for the test against a closed form
TC_OISTA_MARGIN = 1e-4


@pytest.fixture(params=[True, False], ids=["fused", "two_kernel"])
def oista_impl(request):
    """Oracle-ISTA with split BF16 at 128 < m <= 256: the cooperative kernel
    (the default) and the two kernels per layer."""
    from paper_1905_11071_gb300 import _lib
    _lib.slista_set_oista_fused(request.param)
    yield request.param
    _lib.slista_set_oista_fused(True)


def _oista_runner(A, g, lam, D=None, prec="bf16x3"):
    def run(t):
        Z, LS, acc = A.oista(g.B, g.C, lam, g.L, t, D=D, prec=prec)
        return host(Z), host(LS), host(acc)
    return run


@pytest.mark.parametrize("with_D", [True, False])
def test_tc_oista_parity_64x256(with_D, oista_impl):
    """Algorithm 1 with the layer products on the tensor cores (BF16X3),
    compared layer by layer: at least 90 % of the (sample, layer) pairs are
    compared, the codes within the split product's tolerance."""
    from oista_layerwise import compare_layerwise
    w = synth.slista_64x256(N=300, T=40)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Dd = dev(w.D) if with_D else None
    r = compare_layerwise(_oista_runner(A, g, w.lam, Dd), w.D, w.X, w.lam, w.T, OISTA_LAYER_MARGIN,
                          TOL["bf16x3"]["Z"])
    print("tc oista 64x256: compared %.3f of (sample, layer) pairs, worst code error %.3g" % (r["frac"], r["worst"]))
    assert r["frac"] >= 0.9
    done = r["first"] >= w.T  # every decision safe: the objective after T layers
    Zg, _, _ = A.oista(g.B, g.C, w.lam, g.L, w.T, D=Dd, prec="bf16x3")
    Fg = host(A.objective(g.B, g.C, g.xsq, Zg, w.lam, with_gap=False))
    Fo = oracle.objective(w.D, w.X, r["Zo"], w.lam, with_gap=False)
    assert (np.abs(Fg[done] - Fo[done]) / np.abs(Fo[done])).max() <= TOL["bf16x3"]["F"]


def test_tc_oista_fig3_setup():
    """The toy setup of Fig. 3 (D 10 x 50, lam = 0.5, x in B_inf), m padded
    inside the kernel, compared layer by layer."""
    from oista_layerwise import compare_layerwise
    w = synth.paper_binf(10, 50, N=400, lam=0.5, T=100, seed=2)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    r = compare_layerwise(_oista_runner(A, g, w.lam), w.D, w.X, w.lam, w.T, OISTA_LAYER_MARGIN, TOL["bf16x3"]["Z"])
    assert r["frac"] >= 0.9


def test_tc_oista_zero_above_lambda_max():
    w = synth.slista_64x256(N=200, T=10)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, LS, acc = A.oista(g.B, g.C, lam, g.L, 10, D=dev(w.D), prec="bf16x3")
    assert not Z.any()


def test_tc_oista_full_size_sampled_rows(oista_impl):
    """The benchmark workload (N = 10000, T = 40) on the tensor cores: 48
    sampled rows against the oracle, layer by layer (samples are
    independent)."""
    from oista_layerwise import first_unsafe_layer
    w = synth.slista_64x256()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    rows = np.random.default_rng(3).choice(w.N, size=48, replace=False)
    Zall, LSo, acco, deco, lm = oracle.oista(w.D, w.X[rows], w.lam, oracle.lipschitz(w.D), w.T, keep_all=True,
                                             layer_margins=True)
    first = first_unsafe_layer(lm, OISTA_LAYER_MARGIN)
    zt = TOL["bf16x3"]["Z"] * max(1.0, float(np.abs(Zall).max()))
    compared = 0
    for t in range(1, w.T + 1):
        Zg, LSg, _ = A.oista(g.B, g.C, w.lam, g.L, t, D=dev(w.D), prec="bf16x3")
        ok = first >= t
        if ok.any():
            assert np.abs(host(Zg)[rows][ok].astype(np.float64) - Zall[t][ok]).max() <= zt
        compared += int(ok.sum())
        if t == w.T:
            ls_ok = first >= w.T - 1
            np.testing.assert_allclose(host(LSg)[rows][ls_ok], LSo[ls_ok], rtol=1e-5)
    assert compared >= 0.85 * w.T * len(rows)


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_oista_odd_batch(prec, oista_impl):
    """An odd batch size (N = 301) against the oracle, layer by layer: the
    per-sample state arrays of the workspace start on 256-byte boundaries
    whatever N is, as the layer kernels' 16-byte row loads need."""
    from oista_layerwise import compare_layerwise
    w = synth.slista_64x256(N=301, T=20)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    ztol = TOL["bf16x3"]["Z"] if prec == "bf16x3" else 2e-5
    r = compare_layerwise(_oista_runner(A, g, w.lam, dev(w.D), prec), w.D, w.X, w.lam, w.T, OISTA_LAYER_MARGIN,
                          ztol)
    assert r["frac"] >= 0.9


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_oista_orthogonal_support_one_step(prec):
    """Prop. 3.3 on the GPU: with 4 orthonormal columns S* (L_S* = 1) inside a
    12 x 30 dictionary (L ~ 5.5) and x_i = D_S* c_i, one layer after the
    oracle identifies S* the codes are z*_S* = ST(D_S*^T x, lam) (KKT), while
    ISTA's 1/L steps after as many layers are still far from it."""
    D, X, S = synth.orthogonal_support(N=64, seed=22)
    lam = 0.3
    Lo = oracle.lipschitz(D)
    Zall, _, _, _, marg = oracle.oista(D, X, lam, Lo, 30, keep_all=True, with_margin=True)
    T0 = [next(t for t in range(31) if np.array_equal(np.nonzero(Zall[t, i])[0], S)) for i in range(len(X))]
    T = max(T0) + 1
    safe = marg > TC_OISTA_MARGIN
    assert safe.sum() >= 48
    v = X.astype(np.float64) @ D[:, S].astype(np.float64)
    zstar = np.zeros((len(X), D.shape[1]))
    zstar[:, S] = np.sign(v) * np.maximum(np.abs(v) - lam, 0.0)
    zi = oracle.pgd(D, X, lam, np.full(T, 1.0 / Lo))
    assert (np.abs(zi - zstar).max(axis=1) > 0.1).all()
    A = api()
    g = A.gram(dev(D), dev(X))
    Zg, LSg, _ = A.oista(g.B, g.C, lam, g.L, T, prec=prec)
    zt = (TOL["bf16x3"]["Z"] if prec == "bf16x3" else 2e-5) * max(1.0, float(np.abs(zstar).max()))
    assert np.abs(host(Zg)[safe].astype(np.float64) - zstar[safe]).max() <= zt
    np.testing.assert_allclose(host(LSg)[safe], 1.0, rtol=1e-5)


def test_tc_unaligned_c_matches_aligned():
    """C passed at an address 4 bytes past a 16-byte boundary (a view into a
    larger buffer): the layer kernels fall back to scalar loads and give the
    same codes and gradient bit for bit."""
    w = synth.slista_64x256(N=300, T=12)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    buf = torch.empty(g.C.numel() + 1, dtype=torch.float32, device="cuda")
    buf[1:] = g.C.reshape(-1)
    Cu = buf[1:].view(g.C.shape)
    assert Cu.data_ptr() % 16 != 0
    alpha = dev(synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.3, seed=2))
    Z1, s1 = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    Z2, s2 = A.slista(g.B, Cu, w.lam, alpha, prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    assert torch.equal(Z1, Z2)
    d1 = A.slista_grad(g.B, g.C, w.lam, alpha, s1, prec="bf16x3")
    d2 = A.slista_grad(g.B, Cu, w.lam, alpha, s2, prec="bf16x3")
    assert torch.equal(d1, d2)


# --------------------------------------------------------------------------- one-pass backward (trajectory)

@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("N,T", [(300, 40), (129, 7), (1, 3)])
def test_tc_traj_backward_matches_oracle_gradient(prec, N, T):
    """The forward that keeps q_t and dF/dz^(T), then one reverse sweep: the
    sub-gradient against the FP64 oracle; codes and masks are those of the
    plain forward (same refresh schedule) bit for bit."""
    w, alpha = _grad_case(N=N, T=T, seed=17)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec=prec, keep_for_backward=True, trajectory=True)
    assert st.traj is not None and st.ckpt is None
    assert torch.equal(Z, A.slista(g.B, g.C, w.lam, dev(alpha), prec=prec))
    dg = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec=prec)).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    rel = np.linalg.norm(dg - do) / max(np.linalg.norm(do), 1e-12)
    assert rel <= GRAD_TOL[prec], (prec, N, T, rel)


def test_tc_traj_backward_upstream_gradient_and_determinism():
    w, alpha = _grad_case(N=256, T=12, seed=11)
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    Z, st = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, trajectory=True)
    d_default = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3")
    assert torch.equal(d_default, A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, prec="bf16x3"))
    Bo, Co, _ = oracle.gram(w.D, w.X)
    Zh = host(Z).astype(np.float64)
    GT = Zh @ Bo - Co + w.lam * np.sign(Zh)
    d_gz = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=dev(GT.astype(np.float32)),
                              prec="bf16x3")).astype(np.float64)
    dd = host(d_default).astype(np.float64)
    assert np.linalg.norm(d_gz - dd) <= 1e-4 * np.linalg.norm(dd)
    assert not A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=torch.zeros_like(Z), prec="bf16x3").any()
    G1 = dev(np.random.default_rng(5).standard_normal(Z.shape).astype(np.float32))
    d1 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=G1, prec="bf16x3")
    d2 = A.slista_grad(g.B, g.C, w.lam, dev(alpha), st, gZ=2 * G1, prec="bf16x3")
    torch.testing.assert_close(d2, 2 * d1, rtol=1e-5, atol=1e-5 * float(d1.abs().max()))
    # the checkpointed backward with the same upstream gradient
    _, sc = A.slista(g.B, g.C, w.lam, dev(alpha), prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    dc = host(A.slista_grad(g.B, g.C, w.lam, dev(alpha), sc, gZ=G1, prec="bf16x3")).astype(np.float64)
    assert np.linalg.norm(host(d1).astype(np.float64) - dc) <= 1e-4 * np.linalg.norm(dc)


def test_tc_traj_full_size_matches_checkpointed():
    """The benchmark workload (N = 10000, T = 40): the one-pass sub-gradient
    against the checkpointed one and, on 256 sampled rows, the oracle."""
    w = synth.slista_64x256()
    A = api()
    g = A.gram(dev(w.D), dev(w.X))
    alpha = dev(np.full(w.T, 1.0 / oracle.lipschitz(w.D), dtype=np.float32))
    _, st = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3", keep_for_backward=True, trajectory=True)
    dt = A.slista_grad(g.B, g.C, w.lam, alpha, st, prec="bf16x3").double()
    _, sc = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3", keep_for_backward=True)
    dc = A.slista_grad(g.B, g.C, w.lam, alpha, sc, prec="bf16x3").double()
    torch.testing.assert_close(dt, dc, rtol=1e-4, atol=1e-4 * float(dc.abs().max()))
    rows = np.random.default_rng(8).choice(w.N, size=256, replace=False)
    C = g.C[torch.from_numpy(rows).cuda()].contiguous()
    _, s3 = A.slista(g.B, C, w.lam, alpha, prec="bf16x3", keep_for_backward=True, trajectory=True)
    dg = host(A.slista_grad(g.B, C, w.lam, alpha, s3, prec="bf16x3")).astype(np.float64)
    do, _ = oracle.slista_grad(w.D, w.X[rows], w.lam, host(alpha).astype(np.float32))
    assert np.linalg.norm(dg - do) <= GRAD_TOL["bf16x3"] * np.linalg.norm(do)
