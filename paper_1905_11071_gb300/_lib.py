"""ctypes binding of libslista.so (include/slista.h).

Argument marshalling only: every function here forwards torch tensors' device
pointers and sizes to the C entry point of the same name and raises
``SlistaError`` on a non-zero status.  There is no fallback: if the CUDA
library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libslista.so")

SLISTA_OK = 0
SLISTA_ERR_ARG = -1
SLISTA_ERR_UNSUPPORTED = -2
SLISTA_ERR_WORKSPACE = -3
SLISTA_ERR_CUDA = -4
SLISTA_ERR_TIMEOUT = -5

PREC_FP32 = 0
PREC_TF32 = 1
PREC_BF16 = 2
PREC_BF16X3 = 3
PRECISIONS = {"fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16, "bf16x3": PREC_BF16X3}

FN_GRAM = 0
FN_ISTA = 1
FN_SLISTA_FWD = 2
FN_SLISTA_BWD = 3
FN_OISTA = 4
FN_OBJECTIVE = 5
FN_SLISTA_BWD_TRAJ = 6
FN_SUPPORT_LIPSCHITZ = 7

EXPORTS = [
    "slista_last_error", "slista_device_status", "slista_workspace_bytes", "slista_ckpt_floats",
    "slista_mask_words", "lasso_gram", "lasso_lipschitz", "ista_forward", "slista_forward",
    "slista_backward", "oista_forward", "lasso_objective", "slista_forward_noalloc",
    "slista_batched_workspace_bytes", "slista_forward_batched", "slista_backward_batched",
    "slista_traj_floats", "slista_forward_traj", "slista_backward_traj", "lasso_support_lipschitz",
    "slista_wait_probe", "lista_workspace_bytes", "lista_forward", "slista_set_tile_rows",
    "slista_get_tile_rows", "slista_set_oista_fused", "slista_get_oista_fused", "conv_slista_forward",
    "conv_slista_backward_workspace_bytes", "conv_slista_forward_traj", "conv_slista_backward",
    "conv_slista_traj_floats", "conv2d_slista_forward",
]


# entry points that return a size (size_t): every other one returns an int status
SIZE_RETURNING = ("slista_workspace_bytes", "slista_ckpt_floats", "slista_mask_words",
                  "slista_batched_workspace_bytes", "slista_traj_floats", "lista_workspace_bytes",
                  "conv_slista_backward_workspace_bytes", "conv_slista_traj_floats")


class Problem(ctypes.Structure):
    """slista_problem_t: one problem of a ragged batch (device pointers)."""
    _fields_ = [("B", ctypes.c_void_p), ("C", ctypes.c_void_p), ("m", ctypes.c_int), ("N", ctypes.c_int),
                ("lam", ctypes.c_float), ("alpha", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("masks", ctypes.c_void_p), ("mask_words", ctypes.c_size_t), ("ckpt", ctypes.c_void_p),
                ("ckpt_floats", ctypes.c_size_t), ("gZ", ctypes.c_void_p), ("dalpha", ctypes.c_void_p)]


class SlistaError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__("%s failed with status %d: %s" % (fn, code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads the library (once) and declares the C signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libslista.so not found at %s: build it with "
                               "paper_1905_11071_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i = ctypes.c_int
        f = ctypes.c_float
        sz = ctypes.c_size_t
        lib.slista_last_error.restype = ctypes.c_char_p
        lib.slista_last_error.argtypes = []
        lib.slista_device_status.argtypes = [vp]
        lib.slista_wait_probe.argtypes = [ctypes.c_longlong, vp]
        lib.slista_set_tile_rows.argtypes = [i]
        lib.slista_get_tile_rows.argtypes = []
        lib.slista_set_oista_fused.argtypes = [i]
        lib.slista_get_oista_fused.argtypes = []
        lib.slista_workspace_bytes.restype = sz
        lib.slista_workspace_bytes.argtypes = [i, i, i, i, i, i]
        lib.slista_ckpt_floats.restype = sz
        lib.slista_ckpt_floats.argtypes = [i, i, i, i]
        lib.slista_mask_words.restype = sz
        lib.slista_mask_words.argtypes = [i, i, i]
        lib.lasso_gram.argtypes = [vp, i, i, vp, i, vp, vp, vp, vp, vp]
        lib.lasso_lipschitz.argtypes = [vp, i, vp, vp]
        lib.ista_forward.argtypes = [vp, vp, i, i, f, vp, i, i, vp, vp, sz, vp]
        lib.slista_forward.argtypes = [vp, vp, i, i, f, vp, i, i, vp, vp, sz, vp, sz, i, vp, sz, vp]
        lib.slista_backward.argtypes = [vp, vp, i, i, f, vp, i, i, vp, sz, vp, sz, i, vp, vp, vp, sz, vp]
        lib.slista_forward_noalloc.argtypes = [vp, vp, i, i, f, vp, i, i, vp, vp, sz, vp]
        lib.slista_traj_floats.argtypes = [i, i, i]
        lib.slista_traj_floats.restype = sz
        lib.slista_forward_traj.argtypes = [vp, vp, i, i, f, vp, i, i, vp, vp, sz, vp, sz, vp, sz, vp]
        lib.slista_backward_traj.argtypes = [vp, i, i, f, vp, i, i, vp, sz, vp, sz, vp, vp, vp, sz, vp]
        lib.oista_forward.argtypes = [vp, vp, vp, i, i, i, f, vp, i, i, vp, vp, vp, vp, sz, vp]
        lib.lasso_objective.argtypes = [vp, vp, vp, vp, i, i, f, vp, vp, vp]
        lib.lasso_support_lipschitz.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp, sz, vp]
        lib.lista_workspace_bytes.restype = sz
        lib.lista_workspace_bytes.argtypes = [i, i, i]
        lib.lista_forward.argtypes = [vp, i, i, vp, i, vp, vp, vp, f, i, vp, vp, sz, vp]
        lib.conv_slista_forward.argtypes = [vp, i, i, vp, i, i, f, vp, vp, i, vp, vp]
        lib.conv_slista_backward_workspace_bytes.restype = sz
        lib.conv_slista_backward_workspace_bytes.argtypes = [i, i, i, i, i]
        lib.conv2d_slista_forward.argtypes = [vp, i, i, i, vp, i, i, i, f, vp, vp, i, vp, vp]
        lib.conv_slista_traj_floats.restype = sz
        lib.conv_slista_traj_floats.argtypes = [i, i, i, i, i]
        lib.conv_slista_forward_traj.argtypes = [vp, i, i, vp, i, i, f, vp, i, vp, vp, sz, vp]
        lib.conv_slista_backward.argtypes = [vp, i, i, vp, i, i, f, vp, i, vp, sz, vp, vp, sz, vp]
        pp = ctypes.POINTER(Problem)
        lib.slista_batched_workspace_bytes.restype = sz
        lib.slista_batched_workspace_bytes.argtypes = [i, pp, i, i, i, i]
        lib.slista_forward_batched.argtypes = [pp, i, i, i, i, vp, sz, vp]
        lib.slista_backward_batched.argtypes = [pp, i, i, i, i, vp, sz, vp]
        for name in EXPORTS:
            if name not in SIZE_RETURNING + ("slista_last_error",):
                getattr(lib, name).restype = i
        _lib = lib
        return lib


def _check(rc: int, fn: str):
    if rc != SLISTA_OK:
        msg = load().slista_last_error()
        raise SlistaError(rc, fn, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a tensor (None -> NULL)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, shape, name):
    import torch
    if t is None:
        raise ValueError("%s is required" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s (got %s)" % (name, tuple(shape), tuple(t.shape)))
    return t


def _opt(t, dtype, shape, name):
    return None if t is None else _need(t, dtype, shape, name)


def _len(t) -> int:
    """Length in elements of an optional buffer (0 for None)."""
    return 0 if t is None else int(t.numel())


def slista_last_error() -> str:
    msg = load().slista_last_error()
    return msg.decode() if msg else ""


def slista_device_status(stream=None) -> None:
    _check(load().slista_device_status(_stream(stream)), "slista_device_status")


def slista_wait_probe(limit_cycles: int, stream=None) -> None:
    """Launches the bounded-wait check kernel (its wait expires after
    limit_cycles and raises the device flag)."""
    _check(load().slista_wait_probe(int(limit_cycles), _stream(stream)), "slista_wait_probe")


def slista_set_tile_rows(rows: int) -> None:
    """Rows per tile of the persistent layer kernels (0: even spread)."""
    _check(load().slista_set_tile_rows(int(rows)), "slista_set_tile_rows")


def slista_get_tile_rows() -> int:
    return int(load().slista_get_tile_rows())


def slista_set_oista_fused(enable: bool) -> None:
    """Oracle-ISTA with split BF16: the cooperative kernel where it applies
    (True, the default) or two kernels per layer (False)."""
    _check(load().slista_set_oista_fused(1 if enable else 0), "slista_set_oista_fused")


def slista_get_oista_fused() -> bool:
    return bool(load().slista_get_oista_fused())


def slista_workspace_bytes(fn: int, m: int, N: int, T: int, prec: int, ckpt_every: int = 1) -> int:
    return int(load().slista_workspace_bytes(fn, m, N, T, prec, ckpt_every))


def slista_ckpt_floats(m: int, N: int, T: int, ckpt_every: int) -> int:
    return int(load().slista_ckpt_floats(m, N, T, ckpt_every))


def slista_mask_words(m: int, N: int, T: int) -> int:
    return int(load().slista_mask_words(m, N, T))


def lasso_gram(D, X, B, C, xsq, L=None, stream=None) -> None:
    import torch
    n, m = D.shape
    N = X.shape[0]
    _need(D, torch.float32, (n, m), "D")
    _need(X, torch.float32, (N, n), "X")
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(xsq, torch.float64, (N,), "xsq")
    _opt(L, torch.float64, (1,), "L")
    _check(load().lasso_gram(_ptr(D), n, m, _ptr(X), N, _ptr(B), _ptr(C), _ptr(xsq), _ptr(L),
                             _stream(stream)), "lasso_gram")


def lasso_lipschitz(B, L, stream=None) -> None:
    import torch
    m = B.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(L, torch.float64, (1,), "L")
    _check(load().lasso_lipschitz(_ptr(B), m, _ptr(L), _stream(stream)), "lasso_lipschitz")


def ista_forward(B, C, lam, L, T, prec, Z, ws=None, stream=None) -> None:
    import torch
    m = B.shape[0]
    N = C.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(L, torch.float64, (1,), "L")
    _need(Z, torch.float32, (N, m), "Z")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().ista_forward(_ptr(B), _ptr(C), m, N, float(lam), _ptr(L), int(T), int(prec), _ptr(Z),
                               _ptr(ws), wsb, _stream(stream)), "ista_forward")


def slista_forward(B, C, lam, alpha, prec, Z, masks=None, ckpt=None, ckpt_every=1, ws=None,
                   stream=None) -> None:
    import torch
    m = B.shape[0]
    N = C.shape[0]
    T = alpha.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(Z, torch.float32, (N, m), "Z")
    _opt(masks, torch.int32, None, "masks")
    _opt(ckpt, torch.float32, None, "ckpt")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_forward(_ptr(B), _ptr(C), m, N, float(lam), _ptr(alpha), T, int(prec), _ptr(Z),
                                 _ptr(masks), _len(masks), _ptr(ckpt), _len(ckpt), int(ckpt_every), _ptr(ws), wsb,
                                 _stream(stream)),
           "slista_forward")


def slista_forward_noalloc(B, C, lam, alpha, prec, Z, masks=None, stream=None) -> None:
    """Tensor-core Step-LISTA forward without workspace (static device scratch)."""
    import torch
    m = B.shape[0]
    N = C.shape[0]
    T = alpha.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(Z, torch.float32, (N, m), "Z")
    _opt(masks, torch.int32, None, "masks")
    _check(load().slista_forward_noalloc(_ptr(B), _ptr(C), m, N, float(lam), _ptr(alpha), T, int(prec), _ptr(Z),
                                         _ptr(masks), _len(masks), _stream(stream)), "slista_forward_noalloc")


def slista_backward(B, C, lam, alpha, prec, masks, ckpt, ckpt_every, dalpha, gZ=None, ws=None,
                    stream=None) -> None:
    import torch
    m = B.shape[0]
    N = C.shape[0]
    T = alpha.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(masks, torch.int32, None, "masks")
    _opt(ckpt, torch.float32, None, "ckpt")
    _opt(gZ, torch.float32, (N, m), "gZ")
    _need(dalpha, torch.float32, (T,), "dalpha")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_backward(_ptr(B), _ptr(C), m, N, float(lam), _ptr(alpha), T, int(prec), _ptr(masks),
                                  _len(masks), _ptr(ckpt), _len(ckpt), int(ckpt_every), _ptr(gZ), _ptr(dalpha),
                                  _ptr(ws), wsb, _stream(stream)), "slista_backward")


def slista_traj_floats(m: int, N: int, T: int) -> int:
    return int(load().slista_traj_floats(int(m), int(N), int(T)))


def slista_forward_traj(B, C, lam, alpha, prec, Z, masks, traj, ws=None, stream=None) -> None:
    """Tensor-core forward that also writes the one-pass backward's trajectory."""
    import torch
    m = B.shape[0]
    N = C.shape[0]
    T = alpha.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(Z, torch.float32, (N, m), "Z")
    _need(masks, torch.int32, None, "masks")
    _need(traj, torch.float32, None, "traj")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_forward_traj(_ptr(B), _ptr(C), m, N, float(lam), _ptr(alpha), T, int(prec), _ptr(Z),
                                      _ptr(masks), _len(masks), _ptr(traj), _len(traj), _ptr(ws), wsb,
                                      _stream(stream)),
           "slista_forward_traj")


def slista_backward_traj(B, N, lam, alpha, prec, masks, traj, dalpha, gZ=None, ws=None, stream=None) -> None:
    """One reverse sweep over the trajectory of slista_forward_traj."""
    import torch
    m = B.shape[0]
    T = alpha.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(masks, torch.int32, None, "masks")
    _need(traj, torch.float32, None, "traj")
    _opt(gZ, torch.float32, (N, m), "gZ")
    _need(dalpha, torch.float32, (T,), "dalpha")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_backward_traj(_ptr(B), m, int(N), float(lam), _ptr(alpha), T, int(prec), _ptr(masks),
                                       _len(masks), _ptr(traj), _len(traj), _ptr(gZ), _ptr(dalpha), _ptr(ws), wsb,
                                       _stream(stream)),
           "slista_backward_traj")


def oista_forward(B, C, lam, L, T, prec, Z, LS=None, accepted=None, ws=None, D=None, stream=None) -> None:
    import torch
    m = B.shape[0]
    N = C.shape[0]
    n = 0 if D is None else D.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _opt(D, torch.float32, (n, m), "D")
    _need(C, torch.float32, (N, m), "C")
    _need(L, torch.float64, (1,), "L")
    _need(Z, torch.float32, (N, m), "Z")
    _opt(LS, torch.float64, (N,), "LS")
    _opt(accepted, torch.int32, (T,), "accepted")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().oista_forward(_ptr(B), _ptr(C), _ptr(D), n, m, N, float(lam), _ptr(L), int(T), int(prec), _ptr(Z),
                                _ptr(LS), _ptr(accepted), _ptr(ws), wsb, _stream(stream)), "oista_forward")


def lasso_support_lipschitz(B, S, L, LS, ws=None, D=None, stream=None) -> None:
    """L_S for the N supports given as rows of S (N x ceil(m/32) int32 words)."""
    import torch
    m = B.shape[0]
    N = S.shape[0]
    n = 0 if D is None else D.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _opt(D, torch.float32, (n, m), "D")
    _need(S, torch.int32, (N, (m + 31) // 32), "S")
    _need(L, torch.float64, (1,), "L")
    _need(LS, torch.float64, (N,), "LS")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().lasso_support_lipschitz(_ptr(B), _ptr(D), n, m, N, _ptr(S), _ptr(L), _ptr(LS), _ptr(ws), wsb,
                                          _stream(stream)), "lasso_support_lipschitz")


def lista_workspace_bytes(n: int, m: int, N: int) -> int:
    return int(load().lista_workspace_bytes(int(n), int(m), int(N)))


def conv_slista_forward(filters, X, lam, alpha, L, T, Z, stream=None) -> None:
    """Layers on a 1-D convolutional dictionary: filters K x Lf, X N x n,
    Z N x K (n - Lf + 1); alpha (T steps) or, when None, 1/L (L: 1 double)."""
    import torch
    K, Lf = filters.shape
    N, n = X.shape
    _need(filters, torch.float32, (K, Lf), "filters")
    _need(X, torch.float32, (N, n), "X")
    if alpha is not None:
        _need(alpha, torch.float32, (T,), "alpha")
    if L is not None:
        _need(L, torch.float64, (1,), "L")
    _need(Z, torch.float32, (N, K * (n - Lf + 1)), "Z")
    _check(load().conv_slista_forward(_ptr(filters), K, Lf, _ptr(X), N, n, float(lam), _ptr(alpha), _ptr(L), int(T),
                                      _ptr(Z), _stream(stream)), "conv_slista_forward")


def conv_slista_backward_workspace_bytes(K: int, Lf: int, n: int, N: int, T: int) -> int:
    return int(load().conv_slista_backward_workspace_bytes(int(K), int(Lf), int(n), int(N), int(T)))


def conv2d_slista_forward(filters, X, lam, alpha, L, T, Z, stream=None) -> None:
    """Layers on a 2-D convolutional dictionary: filters K x Lh x Lw, X N x H
    x W, Z N x K x (H - Lh + 1) x (W - Lw + 1); alpha (T steps) or, when None,
    1/L (L: 1 double)."""
    import torch
    K, Lh, Lw = filters.shape
    N, H, W = X.shape
    _need(filters, torch.float32, (K, Lh, Lw), "filters")
    _need(X, torch.float32, (N, H, W), "X")
    if alpha is not None:
        _need(alpha, torch.float32, (T,), "alpha")
    if L is not None:
        _need(L, torch.float64, (1,), "L")
    _need(Z, torch.float32, (N, K, H - Lh + 1, W - Lw + 1), "Z")
    _check(load().conv2d_slista_forward(_ptr(filters), K, Lh, Lw, _ptr(X), N, H, W, float(lam), _ptr(alpha), _ptr(L),
                                        int(T), _ptr(Z), _stream(stream)), "conv2d_slista_forward")


def conv_slista_traj_floats(K: int, Lf: int, n: int, N: int, T: int) -> int:
    return int(load().conv_slista_traj_floats(int(K), int(Lf), int(n), int(N), int(T)))


def conv_traj_shape(K: int, Lf: int, n: int, N: int, T: int):
    """Shape of the trajectory buffer: N x T x K x PQ, PQ = P rounded up to 4."""
    P = n - Lf + 1
    return (N, T, K, (P + 3) // 4 * 4)


def conv_slista_forward_traj(filters, X, lam, alpha, Z, traj, stream=None) -> None:
    """conv_slista_forward with steps alpha that also writes traj
    (conv_traj_shape: z^(t+1) of every layer t, maps padded to PQ)."""
    import torch
    K, Lf = filters.shape
    N, n = X.shape
    T = alpha.shape[0]
    m = K * (n - Lf + 1)
    _need(filters, torch.float32, (K, Lf), "filters")
    _need(X, torch.float32, (N, n), "X")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(Z, torch.float32, (N, m), "Z")
    _need(traj, torch.float32, conv_traj_shape(K, Lf, n, N, T), "traj")
    _check(load().conv_slista_forward_traj(_ptr(filters), K, Lf, _ptr(X), N, n, float(lam), _ptr(alpha), T, _ptr(Z),
                                           _ptr(traj), traj.numel(), _stream(stream)), "conv_slista_forward_traj")


def conv_slista_backward(filters, X, lam, alpha, traj, dalpha, ws=None, stream=None) -> None:
    """dalpha (T) = d sum_i F_{x_i}(z_i^(T)) / d alpha from traj."""
    import torch
    K, Lf = filters.shape
    N, n = X.shape
    T = alpha.shape[0]
    _need(filters, torch.float32, (K, Lf), "filters")
    _need(X, torch.float32, (N, n), "X")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(traj, torch.float32, conv_traj_shape(K, Lf, n, N, T), "traj")
    _need(dalpha, torch.float32, (T,), "dalpha")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().conv_slista_backward(_ptr(filters), K, Lf, _ptr(X), N, n, float(lam), _ptr(alpha), T, _ptr(traj),
                                       traj.numel(), _ptr(dalpha), _ptr(ws), wsb, _stream(stream)),
           "conv_slista_backward")


def lista_forward(D, X, W, alpha, beta, lam, Z, ws=None, stream=None) -> None:
    """Coupled LISTA layers (Eq. lista_layer): W is T x n x m."""
    import torch
    n, m = D.shape
    N = X.shape[0]
    T = alpha.shape[0]
    _need(D, torch.float32, (n, m), "D")
    _need(X, torch.float32, (N, n), "X")
    _need(W, torch.float32, (T, n, m), "W")
    _need(alpha, torch.float32, (T,), "alpha")
    _need(beta, torch.float32, (T,), "beta")
    _need(Z, torch.float32, (N, m), "Z")
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().lista_forward(_ptr(D), n, m, _ptr(X), N, _ptr(W), _ptr(alpha), _ptr(beta), float(lam), T,
                                _ptr(Z), _ptr(ws), wsb, _stream(stream)), "lista_forward")


def lasso_objective(B, C, xsq, Z, lam, F, gap=None, stream=None) -> None:
    import torch
    m = B.shape[0]
    N = C.shape[0]
    _need(B, torch.float32, (m, m), "B")
    _need(C, torch.float32, (N, m), "C")
    _need(xsq, torch.float64, (N,), "xsq")
    _need(Z, torch.float32, (N, m), "Z")
    _need(F, torch.float64, (N,), "F")
    _opt(gap, torch.float64, (N,), "gap")
    _check(load().lasso_objective(_ptr(B), _ptr(C), _ptr(xsq), _ptr(Z), m, N, float(lam), _ptr(F), _ptr(gap),
                                  _stream(stream)), "lasso_objective")


def _problems(probs, T, backward):
    """ctypes array of slista_problem_t from dicts of tensors (keys B, C, lam,
    alpha, Z, masks, ckpt, gZ, dalpha; m and N from C)."""
    import torch
    arr = (Problem * max(len(probs), 1))()
    for i, q in enumerate(probs):
        C = q["C"]
        N, m = C.shape
        _need(q["B"], torch.float32, (m, m), "B")
        _need(C, torch.float32, (N, m), "C")
        _need(q["alpha"], torch.float32, (T,), "alpha")
        _opt(q.get("masks"), torch.int32, None, "masks")
        _opt(q.get("ckpt"), torch.float32, None, "ckpt")
        if backward:
            _opt(q.get("gZ"), torch.float32, (N, m), "gZ")
            _need(q["dalpha"], torch.float32, (T,), "dalpha")
        else:
            _need(q["Z"], torch.float32, (N, m), "Z")
        p = arr[i]
        p.B = q["B"].data_ptr()
        p.C = C.data_ptr()
        p.m = m
        p.N = N
        p.lam = float(q["lam"])
        p.alpha = q["alpha"].data_ptr()
        for k in ("Z", "masks", "ckpt", "gZ", "dalpha"):
            t = q.get(k)
            setattr(p, k, None if t is None else t.data_ptr())
        p.mask_words = _len(q.get("masks"))
        p.ckpt_floats = _len(q.get("ckpt"))
    return arr


def slista_batched_workspace_bytes(fn: int, probs, T: int, prec: int, ckpt_every: int) -> int:
    arr = (Problem * max(len(probs), 1))()
    for i, q in enumerate(probs):
        arr[i].m, arr[i].N = int(q["m"]), int(q["N"])
    return int(load().slista_batched_workspace_bytes(fn, arr, len(probs), T, prec, ckpt_every))


def slista_forward_batched(probs, T, prec, ckpt_every, ws=None, stream=None) -> None:
    arr = _problems(probs, T, backward=False)
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_forward_batched(arr, len(probs), T, int(prec), int(ckpt_every), _ptr(ws), wsb,
                                         _stream(stream)), "slista_forward_batched")


def slista_backward_batched(probs, T, prec, ckpt_every, ws=None, stream=None) -> None:
    arr = _problems(probs, T, backward=True)
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _check(load().slista_backward_batched(arr, len(probs), T, int(prec), int(ckpt_every), _ptr(ws), wsb,
                                          _stream(stream)), "slista_backward_batched")
