"""Step-LISTA and ISTA on a 1-D convolutional dictionary (Section 6's
structured dictionaries) through conv_slista_forward, against the FP64
oracle iterating with the equivalent dense dictionary:

* codes within the FP32 tolerance of the dense-path tests (2e-5 max(1, |z|)),
  the objective within 1e-5, for learned steps and for ISTA's 1/L;
* shapes with few positions per filter, odd sizes, a single position per map
  (Lf = n) and a single filter;
* lam above lam_max gives exactly zero codes;
* the fast operator and the dense tensor-core layers on the same dictionary
  agree within the split-BF16 tolerance.
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
