"""Seeded synthetic Lasso inputs shaped like the paper's workloads.

This module is the only code that both the oracle tests and the GPU path use:
it draws dictionaries and samples and nothing else.  It holds none of the
method's arithmetic (no ST, no gradient step, no Gram matrix, no eigenvalue);
the one quantity it evaluates, the regularisation level lam, is part of the
*input recipe*: a workload fixes lam as a fraction of the largest correlation
max_i ||D^T x_i||_inf of its own samples, evaluated once here in float64 and
rounded to float32, so both sides receive the identical scalar.

Recipes (arXiv 1905.11071, Section 5 and Appendix E):
  * dictionary: i.i.d. N(0, 1) entries, every column scaled to unit norm;
  * samples in B_inf: x = x_hat / ||D^T x_hat||_inf with x_hat ~ N(0, I_n);
  * unit samples: x ~ N(0, I_n) scaled to ||x|| = 1;
  * sparse-model samples: x = D z0 + sigma N(0, I_n) with z0 = Bernoulli(p) N(0, 1).
Everything is drawn in float64 from ``numpy.random.default_rng(seed)`` and
rounded once to float32; those float32 arrays are what both sides consume.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def gaussian_dictionary(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """n x m dictionary with N(0,1) entries and unit-norm columns (float32)."""
    Dh = rng.standard_normal((n, m))
    Dh /= np.linalg.norm(Dh, axis=0, keepdims=True)
    return Dh.astype(np.float32)


def unit_samples(N: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """N samples x ~ N(0, I_n), each scaled to unit Euclidean norm (float32)."""
    X = rng.standard_normal((N, n))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    return X.astype(np.float32)


def binf_samples(D: np.ndarray, N: int, rng: np.random.Generator) -> np.ndarray:
    """N samples scaled into B_inf = {x : ||D^T x||_inf = 1} (Appendix E)."""
    n = D.shape[0]
    Xh = rng.standard_normal((N, n))
    scale = np.abs(Xh @ D.astype(np.float64)).max(axis=1, keepdims=True)
    return (Xh / scale).astype(np.float32)


def sparse_model_samples(D: np.ndarray, N: int, density: float, noise: float,
                         rng: np.random.Generator) -> np.ndarray:
    """x = D z0 + noise * N(0, I_n), z0 = Bernoulli(density) * N(0, 1) (float32)."""
    n, m = D.shape
    support = rng.random((N, m)) < density
    z0 = np.where(support, rng.standard_normal((N, m)), 0.0)
    X = z0 @ D.astype(np.float64).T + noise * rng.standard_normal((N, n))
    return X.astype(np.float32)


def lam_fraction(D: np.ndarray, X: np.ndarray, frac: float) -> float:
    """frac * max_i ||D^T x_i||_inf, evaluated in float64, rounded to float32."""
    if X.shape[0] == 0:
        return float(np.float32(frac))
    top = np.abs(X.astype(np.float64) @ D.astype(np.float64)).max()
    return float(np.float32(frac * top))


@dataclasses.dataclass
class Workload:
    """One Lasso problem batch: float32 D (n x m), X (N x n), lam, depth T."""
    name: str
    D: np.ndarray
    X: np.ndarray
    lam: float
    T: int
    seed: int

    @property
    def n(self) -> int:
        return int(self.D.shape[0])

    @property
    def m(self) -> int:
        return int(self.D.shape[1])

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    def describe(self) -> dict:
        return {"workload": self.name, "n": self.n, "m": self.m, "N": self.N,
                "T": self.T, "lam": self.lam, "seed": self.seed}


def ista_10x20(seed: int = 0, N: int = 1000, T: int = 100) -> Workload:
    """Plain-ISTA case: D 10x20, unit-norm Gaussian samples, lam = 0.1 lam_max."""
    rng = np.random.default_rng(seed)
    D = gaussian_dictionary(10, 20, rng)
    X = unit_samples(N, 10, rng)
    return Workload("ista_10x20", D, X, lam_fraction(D, X, 0.1), T, seed)


def slista_64x256(seed: int = 0, N: int = 10000, T: int = 40, density: float = 0.05,
                  noise: float = 0.01, frac: float = 0.1) -> Workload:
    """SLISTA/OISTA case: D 64x256, x = D z0 + 0.01 noise, z0 ~ Bernoulli(0.05)N(0,1)."""
    rng = np.random.default_rng(seed)
    D = gaussian_dictionary(64, 256, rng)
    X = sparse_model_samples(D, N, density, noise, rng)
    return Workload("slista_64x256", D, X, lam_fraction(D, X, frac), T, seed)


def slista_train_64x256(N_train: int = 10000, N_test: int = 2000, T: int = 40):
    """Training split: one dictionary (seed 0); train samples seed 0, test seed 1."""
    train = slista_64x256(seed=0, N=N_train, T=T)
    rng = np.random.default_rng(1)
    Xt = sparse_model_samples(train.D, N_test, 0.05, 0.01, rng)
    test = Workload("slista_64x256_test", train.D, Xt, train.lam, T, 1)
    return train, test


def large_256x1024(seed: int = 0, N: int = 100000, T: int = 50) -> Workload:
    """Large SLISTA case: D 256x1024, z0 ~ Bernoulli(0.02), lam = 0.05 lam_max."""
    rng = np.random.default_rng(seed)
    D = gaussian_dictionary(256, 1024, rng)
    X = sparse_model_samples(D, N, 0.02, 0.01, rng)
    return Workload("large_256x1024", D, X, lam_fraction(D, X, 0.05), T, seed)


def ragged_problems(seed: int = 0, count: int = 64, T: int = 30, n_lo: int = 32,
                    n_hi: int = 128, N_lo: int = 100, N_hi: int = 20000):
    """Ragged batch: n ~ U{n_lo..n_hi}, m = 4n, N ~ floor(exp U[ln N_lo, ln N_hi])."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m = 4 * n
        N = int(math.floor(math.exp(rng.uniform(math.log(N_lo), math.log(N_hi)))))
        D = gaussian_dictionary(n, m, rng)
        X = sparse_model_samples(D, N, 0.05, 0.01, rng)
        out.append(Workload("ragged_%d" % p, D, X, lam_fraction(D, X, 0.1), T, seed))
    return out


def paper_binf(n: int, m: int, N: int, lam: float, T: int, seed: int = 0) -> Workload:
    """The paper's own synthetic setup: unit-column Gaussian D, samples in B_inf."""
    rng = np.random.default_rng(seed)
    D = gaussian_dictionary(n, m, rng)
    X = binf_samples(D, N, rng)
    return Workload("binf_%dx%d" % (n, m), D, X, float(np.float32(lam)), T, seed)


def orthogonal_support(n: int = 12, m: int = 30, k: int = 4, N: int = 2, leak: float = 0.15,
                       seed: int = 21, dtype=np.float32):
    """The setting of Prop. 3.3: k of the m unit columns (positions S, sorted)
    are orthonormal, the others lie mostly outside their span (a component of
    relative size ~leak inside it); sample i is x_i = D_S c_i with
    |c_i| ~ U[1.5, 2.5] and random signs.  Returns (D, X, S), D n x m and X
    N x n in ``dtype`` (drawn in float64, rounded once)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = np.empty((n, m))
    D[:, :k] = Q[:, :k]
    for j in range(k, m):
        v = Q[:, k:] @ rng.standard_normal(n - k) + leak * (Q[:, :k] @ rng.standard_normal(k))
        D[:, j] = v / np.linalg.norm(v)
    perm = rng.permutation(m)
    D = D[:, perm]
    S = np.sort(np.where(perm < k)[0])
    coef = rng.uniform(1.5, 2.5, size=(N, k)) * rng.choice([-1.0, 1.0], size=(N, k))
    X = coef @ D[:, S].T
    return D.astype(dtype), X.astype(dtype), S


def conv_filters(K: int, Lf: int, rng: np.random.Generator) -> np.ndarray:
    """K filters of length Lf with N(0,1) entries, each scaled to unit norm
    (float32, K x Lf)."""
    Fh = rng.standard_normal((K, Lf))
    Fh /= np.linalg.norm(Fh, axis=1, keepdims=True)
    return Fh.astype(np.float32)


def conv_dictionary(filters: np.ndarray, n: int) -> np.ndarray:
    """The dense n x K (n - Lf + 1) matrix of a 1-D convolutional dictionary
    (valid positions): column k (n - Lf + 1) + j holds filter k at rows
    j .. j + Lf - 1 and zeros elsewhere, so D z = sum_k d_k * z_k (the full
    convolution of each code map with its filter).  The entries are copies of
    the float32 filter values."""
    K, Lf = filters.shape
    P = n - Lf + 1
    D = np.zeros((n, K * P), dtype=np.float32)
    for k in range(K):
        for j in range(P):
            D[j:j + Lf, k * P + j] = filters[k]
    return D


@dataclasses.dataclass
class ConvWorkload(Workload):
    """A batch on a convolutional dictionary: filters (K x Lf) and the dense D
    they define (for the FP64 oracle and the dense kernels)."""
    filters: np.ndarray = None


def conv_1d(seed: int = 0, N: int = 10000, T: int = 40, K: int = 8, Lf: int = 16, n: int = 128,
            density: float = 0.02, frac: float = 0.1) -> ConvWorkload:
    """Structured-dictionary case (Section 6): K unit-norm filters of length Lf
    on signals of length n, m = K (n - Lf + 1) codes; x = D z0 + 0.01 noise
    with z0 = Bernoulli(density) N(0, 1); lam = frac lam_max."""
    rng = np.random.default_rng(seed)
    F = conv_filters(K, Lf, rng)
    D = conv_dictionary(F, n)
    X = sparse_model_samples(D, N, density, 0.01, rng)
    return ConvWorkload("conv1d_%dx%d_n%d" % (K, Lf, n), D, X, lam_fraction(D, X, frac), T, seed, F)


def conv2d_filters(K: int, Lh: int, Lw: int, rng: np.random.Generator) -> np.ndarray:
    """K filters of Lh x Lw taps with N(0,1) entries, each scaled to unit
    (Frobenius) norm (float32, K x Lh x Lw)."""
    Fh = rng.standard_normal((K, Lh, Lw))
    Fh /= np.linalg.norm(Fh.reshape(K, -1), axis=1)[:, None, None]
    return Fh.astype(np.float32)


def conv2d_dictionary(filters: np.ndarray, H: int, W: int) -> np.ndarray:
    """The dense (H W) x K Ph Pw matrix of a 2-D convolutional dictionary on
    H x W images (valid positions, Ph = H - Lh + 1, Pw = W - Lw + 1; images and
    code maps row-major): column (k Ph + p) Pw + q holds filter k with its
    top-left tap at pixel (p, q), so D z = sum_k d_k * z_k (the full 2-D
    convolution of each code map with its filter).  Entries are copies of the
    float32 filter values."""
    K, Lh, Lw = filters.shape
    Ph, Pw = H - Lh + 1, W - Lw + 1
    D = np.zeros((H * W, K * Ph * Pw), dtype=np.float32)
    img = np.zeros((H, W), dtype=np.float32)
    for k in range(K):
        for p in range(Ph):
            for q in range(Pw):
                img[:] = 0.0
                img[p:p + Lh, q:q + Lw] = filters[k]
                D[:, (k * Ph + p) * Pw + q] = img.reshape(-1)
    return D


@dataclasses.dataclass
class Conv2dWorkload(Workload):
    """A batch of H x W images on a 2-D convolutional dictionary: filters
    (K x Lh x Lw) and the dense D they define (for the FP64 oracle)."""
    filters: np.ndarray = None
    H: int = 0
    W: int = 0


def conv_2d(seed: int = 0, N: int = 2000, T: int = 30, K: int = 8, Lh: int = 5, Lw: int = 5, H: int = 28,
            W: int = 28, density: float = 0.01, frac: float = 0.1) -> Conv2dWorkload:
    """Structured-dictionary case on images (Section 6): K unit-norm Lh x Lw
    filters on H x W images, m = K (H - Lh + 1)(W - Lw + 1) codes;
    x = D z0 + 0.01 noise with z0 = Bernoulli(density) N(0, 1); lam = frac lam_max."""
    rng = np.random.default_rng(seed)
    F = conv2d_filters(K, Lh, Lw, rng)
    D = conv2d_dictionary(F, H, W)
    X = sparse_model_samples(D, N, density, 0.01, rng)
    return Conv2dWorkload("conv2d_%dx%dx%d_%dx%d" % (K, Lh, Lw, H, W), D, X, lam_fraction(D, X, frac), T, seed, F,
                          H, W)


def step_sizes(T: int, base: float, spread: float, seed: int) -> np.ndarray:
    """T positive step sizes base * U[1 - spread, 1 + spread] (float32)."""
    rng = np.random.default_rng(seed)
    return (base * rng.uniform(1.0 - spread, 1.0 + spread, size=T)).astype(np.float32)
