"""Step-LISTA and ISTA on a 1-D convolutional dictionary (Section 6's
structured dictionaries) through conv_slista_forward, against the FP64
oracle iterating with the equivalent dense dictionary:

* codes within the FP32 tolerance of the dense-path tests (2e-5 max(1, |z|)),
  the objective within 1e-5, for learned steps and for ISTA's 1/L;
* shapes with few positions per filter, odd sizes, a single position per map
  (Lf = n) and a single filter;
* lam above lam_max gives exactly zero codes;
* the fast operator and the dense tensor-core layers on the same dictionary
  agree within the split-BF16 tolerance;
* the step-size sub-gradient (conv_slista_forward_traj + conv_slista_backward)
  against the oracle's adjoint on the dense dictionary (relative 1e-4, the
  dense FP32 path's bound), its trajectory against the oracle's layers, its
  degenerate cases (zero codes, T = 1, N = 0) and its run-to-run identity;
  at the benchmark's size, additivity over samples and sampled rows;
* 2-D convolutional dictionaries (images): codes against the oracle on the
  equivalent dense dictionary for learned steps and ISTA's 1/L, odd shapes
  (non-square filters, one position per column of a map, 1 x 1 filters), zero
  codes above lam_max, and sampled rows of a 2000-image batch.
"""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z_TOL = 2e-5


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


def _close(Zg, Zo, tol=Z_TOL):
    t = tol * max(1.0, float(np.abs(Zo).max()))
    err = float(np.abs(host(Zg).astype(np.float64) - Zo).max())
    assert err <= t, (err, t)


def _workload(K, Lf, n, N, T, seed=0):
    return synth.conv_1d(seed=seed, N=N, T=T, K=K, Lf=Lf, n=n)


def test_conv_slista_matches_oracle():
    from paper_1905_11071_gb300 import api as A
    w = _workload(8, 16, 128, 300, 30)
    alpha = synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.3, seed=5)
    Z = A.conv_slista(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    Zo = oracle.pgd(w.D, w.X, w.lam, alpha)
    _close(Z, Zo)
    g = A.gram(dev(w.D), dev(w.X), with_L=False)
    F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
    Fo = oracle.objective(w.D, w.X, Zo, w.lam, with_gap=False)
    assert (np.abs(F - Fo) / np.abs(Fo)).max() <= 1e-5


def test_conv_ista_matches_oracle():
    from paper_1905_11071_gb300 import api as A
    w = _workload(8, 16, 128, 200, 40, seed=1)
    g = A.gram(dev(w.D), dev(w.X))  # L of the dictionary, on the GPU
    Z = A.conv_slista(dev(w.filters), dev(w.X), w.lam, L=g.L, T=w.T)
    Zo = oracle.ista(w.D, w.X, w.lam, oracle.lipschitz(w.D), w.T)
    _close(Z, Zo)


@pytest.mark.parametrize("K,Lf,n,N", [(3, 5, 37, 129), (5, 12, 12, 64), (1, 7, 200, 33), (16, 4, 20, 257)])
def test_conv_odd_shapes(K, Lf, n, N):
    from paper_1905_11071_gb300 import api as A
    w = _workload(K, Lf, n, N, 20, seed=K + n)
    alpha = synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.3, seed=K)
    Z = A.conv_slista(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    _close(Z, oracle.pgd(w.D, w.X, w.lam, alpha))


def test_conv_zero_above_lambda_max():
    from paper_1905_11071_gb300 import api as A
    w = _workload(8, 16, 128, 64, 10, seed=3)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    alpha = np.full(w.T, 1.0 / oracle.lipschitz(w.D), dtype=np.float32)
    Z = A.conv_slista(dev(w.filters), dev(w.X), lam, dev(alpha))
    assert not Z.any()


def test_conv_operator_agrees_with_dense_tensor_core_layers():
    from paper_1905_11071_gb300 import api as A
    w = _workload(8, 16, 128, 500, 30, seed=4)
    g = A.gram(dev(w.D), dev(w.X))
    alpha = (1.0 / g.L.double()).float().expand(w.T).contiguous()
    Zc = A.conv_slista(dev(w.filters), dev(w.X), w.lam, alpha)
    Zd = A.slista(g.B, g.C, w.lam, alpha, prec="bf16x3")
    tol = 1e-4 * max(1.0, float(Zd.abs().max()))
    assert float((Zc - Zd).abs().max()) <= tol


def test_conv_full_size_sampled_rows():
    """The benchmark's convolutional workload (N = 10000, T = 40): 64 sampled
    rows against the oracle (samples are independent)."""
    from paper_1905_11071_gb300 import api as A
    w = synth.conv_1d()
    alpha = synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.2, seed=9)
    Z = A.conv_slista(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    rows = np.random.default_rng(2).choice(w.N, size=64, replace=False)
    _close(Z[rows], oracle.pgd(w.D, w.X[rows], w.lam, alpha))


GRAD_TOL = 1e-4


def _grad_case(K, Lf, n, N, T, seed=0, spread=0.3):
    w = _workload(K, Lf, n, N, T, seed=seed)
    alpha = synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), spread, seed=seed + 5)
    return w, alpha


def _rel(dg, do):
    return float(np.linalg.norm(host(dg).astype(np.float64) - do) / np.linalg.norm(do))


def test_conv_backward_matches_oracle():
    from paper_1905_11071_gb300 import api as A
    w, alpha = _grad_case(8, 16, 128, 300, 30)
    Z, da = A.conv_slista_grad(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert _rel(da, do) <= GRAD_TOL, (host(da), do)
    # the trajectory forward repeats the forward's arithmetic exactly
    assert torch.equal(Z, A.conv_slista(dev(w.filters), dev(w.X), w.lam, dev(alpha)))


@pytest.mark.parametrize("K,Lf,n,N,T", [(3, 5, 37, 129, 17), (5, 12, 12, 64, 9), (1, 7, 200, 33, 25),
                                        (16, 4, 20, 257, 12), (4, 32, 96, 70, 10), (2, 3, 64, 1, 1)])
def test_conv_backward_odd_shapes(K, Lf, n, N, T):
    from paper_1905_11071_gb300 import api as A
    w, alpha = _grad_case(K, Lf, n, N, T, seed=K + n)
    _, da = A.conv_slista_grad(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    do, _ = oracle.slista_grad(w.D, w.X, w.lam, alpha)
    assert _rel(da, do) <= GRAD_TOL, (host(da), do)


def test_conv_trajectory_is_every_layer():
    """traj[:, t] = z^(t+1): the oracle run for t + 1 layers."""
    from paper_1905_11071_gb300 import _lib
    w, alpha = _grad_case(8, 13, 128, 100, 12, seed=2)  # P = 116: maps padded to 116
    K, Lf = w.filters.shape
    P = w.n - Lf + 1
    m = w.D.shape[1]
    shape = _lib.conv_traj_shape(K, Lf, w.n, w.N, w.T)
    assert shape[3] % 4 == 0 and shape[3] >= P
    assert _lib.conv_slista_traj_floats(K, Lf, w.n, w.N, w.T) == int(np.prod(shape))
    Z = torch.empty((w.N, m), dtype=torch.float32, device="cuda")
    traj = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    _lib.conv_slista_forward_traj(dev(w.filters), dev(w.X), w.lam, dev(alpha), Z, traj)
    assert not traj[..., P:].any()  # the padding is written, with zeros
    codes = traj[..., :P].reshape(w.N, w.T, m)
    assert torch.equal(codes[:, -1], Z)
    for t in (0, 1, 5, 11):
        _close(codes[:, t], oracle.pgd(w.D, w.X, w.lam, alpha[:t + 1]))


def test_conv_trajectory_padding_and_short_buffer():
    """P = 113 (maps padded to 116): the padding reads as zeros; a buffer one
    float short is refused before any launch."""
    from paper_1905_11071_gb300 import _lib
    w, alpha = _grad_case(8, 16, 128, 40, 5, seed=6)
    K, Lf = w.filters.shape
    P = w.n - Lf + 1
    shape = _lib.conv_traj_shape(K, Lf, w.n, w.N, w.T)
    assert shape[3] == 116
    Z = torch.empty((w.N, K * P), dtype=torch.float32, device="cuda")
    traj = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    _lib.conv_slista_forward_traj(dev(w.filters), dev(w.X), w.lam, dev(alpha), Z, traj)
    assert not traj[..., P:].any()
    lib = _lib.load()
    rc = lib.conv_slista_forward_traj(_lib._ptr(dev(w.filters)), K, Lf, _lib._ptr(dev(w.X)), w.N, w.n, w.lam,
                                      _lib._ptr(dev(alpha)), w.T, _lib._ptr(Z), _lib._ptr(traj), traj.numel() - 1, None)
    assert rc == _lib.SLISTA_ERR_WORKSPACE


def test_conv_backward_is_deterministic():
    from paper_1905_11071_gb300 import api as A
    w, alpha = _grad_case(8, 16, 128, 2000, 20, seed=4)
    outs = [A.conv_slista_grad(dev(w.filters), dev(w.X), w.lam, dev(alpha))[1] for _ in range(3)]
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_conv_backward_zero_codes_and_empty_batch():
    """Above lam_max every code is zero, so no layer has a support and the
    sub-gradient is exactly zero; N = 0 gives zeros too."""
    from paper_1905_11071_gb300 import api as A
    w, alpha = _grad_case(8, 16, 128, 64, 10, seed=3)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    Z, da = A.conv_slista_grad(dev(w.filters), dev(w.X), lam, dev(alpha))
    assert not Z.any() and not da.any()
    X0 = torch.empty((0, w.X.shape[1]), dtype=torch.float32, device="cuda")
    Z0, da0 = A.conv_slista_grad(dev(w.filters), X0, w.lam, dev(alpha))
    assert Z0.shape[0] == 0 and not da0.any()


def test_conv_backward_rejects_long_filters():
    from paper_1905_11071_gb300 import api as A, _lib
    w, alpha = _grad_case(2, 40, 128, 8, 4, seed=1)
    with pytest.raises(_lib.SlistaError) as e:
        A.conv_slista_grad(dev(w.filters), dev(w.X), w.lam, dev(alpha))
    assert e.value.code == _lib.SLISTA_ERR_UNSUPPORTED


def test_conv_backward_full_size():
    """The benchmark's convolutional workload (N = 10000, T = 40, one launch
    of each kernel): the sub-gradient is a sum over samples, so it equals the
    sum of the two halves' within FP32 rounding, and one 200-sample part
    matches the oracle."""
    from paper_1905_11071_gb300 import api as A
    w = synth.conv_1d()
    alpha = synth.step_sizes(w.T, 1.0 / oracle.lipschitz(w.D), 0.2, seed=9)
    F, X, a = dev(w.filters), dev(w.X), dev(alpha)
    _, da = A.conv_slista_grad(F, X, w.lam, a)
    _, d1 = A.conv_slista_grad(F, X[:5000].contiguous(), w.lam, a)
    _, d2 = A.conv_slista_grad(F, X[5000:].contiguous(), w.lam, a)
    s = (d1.double() + d2.double())
    assert float((da.double() - s).norm() / s.norm()) <= 1e-5
    rows = np.sort(np.random.default_rng(2).choice(w.N, size=200, replace=False))
    _, dr = A.conv_slista_grad(F, X[rows].contiguous(), w.lam, a)
    do, _ = oracle.slista_grad(w.D, w.X[rows], w.lam, alpha)
    assert _rel(dr, do) <= GRAD_TOL



# --- 2-D convolutional dictionaries

def _workload2d(K, Lh, Lw, H, W, N, T, seed=0):
    return synth.conv_2d(seed=seed, N=N, T=T, K=K, Lh=Lh, Lw=Lw, H=H, W=W)


def _images(w):
    return dev(w.X.reshape(w.X.shape[0], w.H, w.W))


def _L(D):
    """Largest eigenvalue of D^T D from the smaller Gram D D^T (numpy, FP64):
    the scale of the test's step sizes (the oracle's Jacobi works on the
    m x m Gram, too slow at m = 4608)."""
    D = D.astype(np.float64)
    return float(np.linalg.eigvalsh(D @ D.T)[-1])


def test_conv2d_slista_and_ista_match_oracle():
    from paper_1905_11071_gb300 import api as A
    w = _workload2d(4, 5, 5, 16, 16, 200, 20)
    alpha = synth.step_sizes(w.T, 1.0 / _L(w.D), 0.3, seed=3)
    Z = A.conv2d_slista(dev(w.filters), _images(w), w.lam, dev(alpha))
    assert Z.shape == (w.N, 4, 12, 12)
    _close(Z.reshape(w.N, -1), oracle.pgd(w.D, w.X, w.lam, alpha))
    g = A.gram(dev(w.D), dev(w.X))  # L of the dictionary, on the GPU
    Zi = A.conv2d_slista(dev(w.filters), _images(w), w.lam, L=g.L, T=w.T)
    _close(Zi.reshape(w.N, -1), oracle.ista(w.D, w.X, w.lam, oracle.lipschitz(w.D), w.T))  # m = 576


@pytest.mark.parametrize("K,Lh,Lw,H,W,N", [(3, 3, 4, 9, 11, 65), (2, 7, 2, 7, 5, 33), (5, 1, 1, 6, 6, 17),
                                           (16, 3, 3, 12, 10, 129)])
def test_conv2d_odd_shapes(K, Lh, Lw, H, W, N):
    from paper_1905_11071_gb300 import api as A
    w = _workload2d(K, Lh, Lw, H, W, N, 15, seed=K + H)
    alpha = synth.step_sizes(w.T, 1.0 / _L(w.D), 0.3, seed=K)
    Z = A.conv2d_slista(dev(w.filters), _images(w), w.lam, dev(alpha))
    _close(Z.reshape(w.N, -1), oracle.pgd(w.D, w.X, w.lam, alpha))


def test_conv2d_zero_above_lambda_max_and_empty_batch():
    from paper_1905_11071_gb300 import api as A
    w = _workload2d(4, 5, 5, 16, 16, 40, 8, seed=5)
    lam = float(np.float32(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.001))
    alpha = np.full(w.T, 1.0 / _L(w.D), dtype=np.float32)
    assert not A.conv2d_slista(dev(w.filters), _images(w), lam, dev(alpha)).any()
    X0 = torch.empty((0, w.H, w.W), dtype=torch.float32, device="cuda")
    assert A.conv2d_slista(dev(w.filters), X0, w.lam, dev(alpha)).shape == (0, 4, 12, 12)


def test_conv2d_batch_sampled_rows():
    """2000 images of 28 x 28 on 8 filters of 5 x 5 (m = 4608 codes), T = 30,
    one launch: 16 sampled images against the oracle (images are independent)."""
    from paper_1905_11071_gb300 import api as A
    w = synth.conv_2d()
    alpha = synth.step_sizes(w.T, 1.0 / _L(w.D), 0.2, seed=9)
    Z = A.conv2d_slista(dev(w.filters), _images(w), w.lam, dev(alpha))
    rows = np.random.default_rng(4).choice(w.N, size=16, replace=False)
    _close(Z.reshape(w.N, -1)[rows], oracle.pgd(w.D, w.X[rows], w.lam, alpha))
