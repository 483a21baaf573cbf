"""FP64 CPU oracle for batched unfolded ISTA / Step-LISTA / Oracle-ISTA.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct statement
of what the GPU path computes (arXiv 1905.11071, Sections 1-4 and
Algorithm 1).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product package never does, and this module imports nothing from it.

All routines take numpy arrays (any float dtype; they are promoted to float64)
and return float64 numpy arrays.  The arithmetic lives in ``lasso_oracle.c``;
this wrapper only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lasso_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblasso_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lasso_oracle.c`` with gcc (plain -O2, IEEE semantics kept)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_ubyte)
            i = ctypes.c_int
            d = ctypes.c_double
            lib.orc_st.argtypes = [d, d]
            lib.orc_st.restype = d
            lib.orc_objective.argtypes = [dp, i, i, dp, i, dp, d, dp, dp]
            lib.orc_lambda_max.argtypes = [dp, i, i, dp, i, dp]
            lib.orc_gram.argtypes = [dp, i, i, dp, i, dp, dp, dp]
            lib.orc_sym_max_eig.argtypes = [dp, i, dp]
            lib.orc_sym_max_eig.restype = d
            lib.orc_lipschitz.argtypes = [dp, i, i]
            lib.orc_lipschitz.restype = d
            lib.orc_support_lipschitz.argtypes = [dp, i, i, up, d]
            lib.orc_support_lipschitz.restype = d
            lib.orc_pgd.argtypes = [dp, i, i, dp, i, d, dp, i, dp, dp]
            lib.orc_lista.argtypes = [dp, i, i, dp, i, d, dp, dp, dp, i, dp]
            lib.orc_oista.argtypes = [dp, i, i, dp, i, d, d, i, dp, dp, ip, up, dp, dp]
            lib.orc_slista_grad.argtypes = [dp, i, i, dp, i, d, dp, i, dp, dp]
            lib.orc_lasso_bruteforce.argtypes = [dp, i, i, dp, d, dp]
            lib.orc_lasso_bruteforce.restype = i
            lib.orc_kkt_violation.argtypes = [dp, i, i, dp, dp, d]
            lib.orc_kkt_violation.restype = d
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def st(v: float, u: float) -> float:
    """Soft-thresholding ST(v, u) = sign(v) max(|v| - u, 0) (Section 1)."""
    return float(_load().orc_st(float(v), float(u)))


def gram(D, X):
    """B = D^T D, C = X D (row i = D^T x_i), xsq_i = ||x_i||^2, by definition."""
    D = _f64(D); X = _f64(X)
    n, m = D.shape
    N = X.shape[0]
    B = np.empty((m, m)); C = np.empty((N, m)); xsq = np.empty(N)
    _load().orc_gram(_p(D), n, m, _p(X), N, _p(B), _p(C), _p(xsq))
    return B, C, xsq


def objective(D, X, Z, lam, with_gap: bool = True):
    """Per-sample F_x(z) (Eq. lasso) and the standard Lasso duality gap."""
    D = _f64(D); X = _f64(X); Z = _f64(Z)
    n, m = D.shape
    N = X.shape[0]
    F = np.empty(N)
    gap = np.empty(N) if with_gap else None
    _load().orc_objective(_p(D), n, m, _p(X), N, _p(Z), float(lam), _p(F),
                          _p(gap) if with_gap else None)
    return (F, gap) if with_gap else F


def lambda_max(D, X):
    """||D^T x_i||_inf per sample (Section 2)."""
    D = _f64(D); X = _f64(X)
    n, m = D.shape
    N = X.shape[0]
    out = np.empty(N)
    _load().orc_lambda_max(_p(D), n, m, _p(X), N, _p(out))
    return out


def sym_max_eig(A) -> float:
    """Largest eigenvalue of a symmetric matrix by cyclic Jacobi rotations."""
    A = _f64(A)
    k = A.shape[0]
    work = np.empty(max(k * k, 1))
    return float(_load().orc_sym_max_eig(_p(A), k, _p(work)))


def lipschitz(D) -> float:
    """L = largest eigenvalue of D^T D (Section 1)."""
    D = _f64(D)
    n, m = D.shape
    return float(_load().orc_lipschitz(_p(D), n, m))


def support_lipschitz(D, mask, L_empty: float) -> float:
    """L_S = largest eigenvalue of D_S^T D_S, L_{empty} = L (Eq. spca)."""
    D = _f64(D)
    n, m = D.shape
    mk = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
    return float(_load().orc_support_lipschitz(
        _p(D), n, m, mk.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), float(L_empty)))


def pgd(D, X, lam, alpha, keep_all: bool = False):
    """T layers of Eq. pgd / Eq. steprec from z^(0) = 0.

    ``alpha`` is the length-T step sequence (ISTA: every entry 1/L).
    Returns z^(T) (N x m), or every iterate ((T+1) x N x m) if ``keep_all``.
    """
    D = _f64(D); X = _f64(X); alpha = _f64(np.atleast_1d(alpha))
    n, m = D.shape
    N = X.shape[0]
    T = alpha.shape[0]
    Z = np.empty((N, m))
    Zall = np.empty((T + 1, N, m)) if keep_all else None
    _load().orc_pgd(_p(D), n, m, _p(X), N, float(lam), _p(alpha), T, _p(Z),
                    _p(Zall) if keep_all else None)
    return Zall if keep_all else Z


def lista(D, X, lam, W, alpha, beta):
    """T layers of coupled LISTA (Eq. lista_layer) from z^(0) = 0:
    z <- ST(z - alpha_t W_t^T (D z - x), beta_t lam).  W: T x n x m (one
    matrix per layer), alpha, beta: T positive scalars.  Returns z^(T) (N x m)."""
    D = _f64(D); X = _f64(X); W = _f64(W); alpha = _f64(np.atleast_1d(alpha)); beta = _f64(np.atleast_1d(beta))
    n, m = D.shape
    N = X.shape[0]
    T = alpha.shape[0]
    assert W.shape == (T, n, m) and beta.shape == (T,)
    Z = np.empty((N, m))
    _load().orc_lista(_p(D), n, m, _p(X), N, float(lam), _p(W), _p(alpha), _p(beta), T, _p(Z))
    return Z


def ista(D, X, lam, L, T):
    """ISTA (Eq. ista): Eq. pgd with every step equal to 1/L."""
    return pgd(D, X, lam, np.full(T, 1.0 / L))


def oista(D, X, lam, L, T, keep_all: bool = False, with_margin: bool = False,
          layer_margins: bool = False):
    """Oracle-ISTA, Algorithm 1.

    Returns (Z, LS, accepted, decision): z^(T) (or every iterate,
    (T+1) x N x m, if ``keep_all``); the L_S of the last support the method
    evaluated, per sample; per-layer count of samples whose local step met
    condition (star); and the per-layer, per-sample (star) outcome (T x N,
    uint8).  With ``with_margin`` one more value: per sample, the smallest
    decision margin along its trajectory (N).  With ``layer_margins`` one
    more value (after that one when both are asked for): the decision margin
    of every layer and sample (T x N) -- the smallest distance of a
    pre-threshold value to its threshold among the codes off the support
    under the local step 1/L_S and every code under the step taken.
    """
    D = _f64(D); X = _f64(X)
    n, m = D.shape
    N = X.shape[0]
    Z = np.empty((N, m)); LS = np.empty(N)
    acc = np.zeros(T, dtype=np.int32)
    dec = np.zeros((T, N), dtype=np.uint8)
    Zall = np.empty((T + 1, N, m)) if keep_all else None
    marg = np.empty((T, N)) if (with_margin or layer_margins) else None
    _load().orc_oista(_p(D), n, m, _p(X), N, float(lam), float(L), int(T), _p(Z), _p(LS),
                      acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      dec.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                      _p(Zall) if keep_all else None, _p(marg) if marg is not None else None)
    out = ((Zall if keep_all else Z), LS, acc, dec)
    if with_margin:
        out = out + ((marg.min(axis=0) if T > 0 else np.full(N, np.inf)),)
    if layer_margins:
        out = out + (marg,)
    return out


def slista_grad(D, X, lam, alpha):
    """Sub-gradient of sum_i F_{x_i}(z_i^(T)) w.r.t. the step sizes (Eq. steprec).

    Returns (dalpha (T,), loss).
    """
    D = _f64(D); X = _f64(X); alpha = _f64(np.atleast_1d(alpha))
    n, m = D.shape
    N = X.shape[0]
    T = alpha.shape[0]
    da = np.empty(T)
    loss = ctypes.c_double(0.0)
    _load().orc_slista_grad(_p(D), n, m, _p(X), N, float(lam), _p(alpha), T, _p(da),
                            ctypes.byref(loss))
    return da, float(loss.value)


def lasso_bruteforce(D, x, lam):
    """Exact Lasso solution by enumerating sign patterns (Lemma 2.1), m <= 12.

    Returns (z*, number of KKT-consistent patterns).
    """
    D = _f64(D); x = _f64(x)
    n, m = D.shape
    z = np.zeros(m)
    cnt = _load().orc_lasso_bruteforce(_p(D), n, m, _p(x), float(lam), _p(z))
    if cnt < 0:
        raise ValueError("brute force needs 1 <= m <= 12")
    return z, int(cnt)


def kkt_violation(D, x, z, lam) -> float:
    """Largest violation of the KKT conditions (Lemma 2.1) at z."""
    D = _f64(D); x = _f64(x); z = _f64(z)
    n, m = D.shape
    return float(_load().orc_kkt_violation(_p(D), n, m, _p(x), _p(z), float(lam)))
