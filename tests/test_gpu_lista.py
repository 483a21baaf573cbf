"""Coupled LISTA layers on the GPU (Eq. lista_layer, Section 4), through the
C ABI, against the FP64 oracle's coupled LISTA (oracle.lista):

* per-layer matrices W_t = D + perturbation and per-layer (alpha_t, beta_t):
  codes within the FP32 tolerance (both products of a layer use the
  FP32-class split);
* W_t = D, alpha_t = beta_t = 1/L is ISTA: against the oracle's ISTA;
* a layer whose (alpha_t / beta_t) W_t = D is the Step-LISTA layer of step
  beta_t: against the GPU's FP32 Step-LISTA forward;
* lam above every |alpha W^T x|_inf / beta gives exactly zero after one layer.
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


def _close(Zg, Zo):
    tol = Z_TOL * max(1.0, float(np.abs(Zo).max()))
    err = float(np.abs(Zg.cpu().numpy().astype(np.float64) - Zo).max())
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("n,m,N,T", [(64, 256, 700, 12), (10, 20, 300, 20), (32, 100, 129, 7)])
def test_lista_per_layer_weights(n, m, N, T):
    from paper_1905_11071_gb300 import api
    rng = np.random.default_rng(n + m + T)
    D = synth.gaussian_dictionary(n, m, rng)
    X = synth.sparse_model_samples(D, N, 0.05, 0.01, rng)
    lam = synth.lam_fraction(D, X, 0.1)
    L = oracle.lipschitz(D)
    W = (D[None] + 0.05 * rng.standard_normal((T, n, m))).astype(np.float32)
    alpha = (rng.uniform(0.6, 1.2, T) / L).astype(np.float32)
    beta = (rng.uniform(0.6, 1.2, T) / L).astype(np.float32)
    Zg = api.lista(dev(D), dev(X), dev(W), dev(alpha), dev(beta), lam)
    Zo = oracle.lista(D, X, lam, W, alpha, beta)
    _close(Zg, Zo)


def test_lista_with_dictionary_weights_is_ista():
    from paper_1905_11071_gb300 import api
    w = synth.ista_10x20(N=500, T=100)
    L = oracle.lipschitz(w.D)
    a = np.full(w.T, 1.0 / L, dtype=np.float32)
    W = np.repeat(w.D[None], w.T, axis=0)
    Zg = api.lista(dev(w.D), dev(w.X), dev(W), dev(a), dev(a), w.lam)
    _close(Zg, oracle.ista(w.D, w.X, w.lam, L, w.T))


def test_lista_coupled_to_step_lista():
    """(alpha_t / beta_t) W_t = D: the layer is z - beta_t D^T(Dz - x)
    thresholded at beta_t lam, the Step-LISTA layer of step beta_t."""
    from paper_1905_11071_gb300 import api
    w = synth.slista_64x256(N=400, T=10)
    L = oracle.lipschitz(w.D)
    rng = np.random.default_rng(3)
    beta = (rng.uniform(0.7, 1.3, w.T) / L).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, w.T)
    alpha = (beta * scale).astype(np.float32)
    W = (w.D[None] / (alpha.astype(np.float64) / beta.astype(np.float64))[:, None, None]).astype(np.float32)
    Zg = api.lista(dev(w.D), dev(w.X), dev(W), dev(alpha), dev(beta), w.lam)
    g = api.gram(dev(w.D), dev(w.X))
    Zs = api.slista(g.B, g.C, w.lam, dev(beta), prec="fp32")
    tol = 1e-4 * max(1.0, float(Zs.abs().max()))  # W_t rounded to FP32 after the division
    assert float((Zg - Zs).abs().max()) <= tol
    _close(Zg, oracle.lista(w.D, w.X, w.lam, W, alpha, beta))


def test_lista_zero_above_threshold():
    from paper_1905_11071_gb300 import api
    w = synth.slista_64x256(N=200, T=3)
    a = np.full(w.T, 0.1, dtype=np.float32)
    W = np.repeat(w.D[None], w.T, axis=0)
    lam = float(np.abs(w.X.astype(np.float64) @ w.D.astype(np.float64)).max() * 1.01)
    Zg = api.lista(dev(w.D), dev(w.X), dev(W), dev(a), dev(a), lam)
    assert not Zg.any()
