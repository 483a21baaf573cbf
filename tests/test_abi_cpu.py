"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/slista.h declares, sizes its
buffers as documented, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1905_11071_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SLISTA_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) <= set(names)


def test_size_returning_entry_points_keep_size_t(lib):
    """The binding types every size_t result as such (a 32-bit int would
    truncate, e.g., a 10^10-float trajectory and under-allocate it)."""
    import ctypes
    for name in _lib.SIZE_RETURNING:
        assert getattr(lib, name).restype is ctypes.c_size_t, name
    for name in _lib.EXPORTS:
        if name not in _lib.SIZE_RETURNING + ("slista_last_error",):
            assert getattr(lib, name).restype is ctypes.c_int, name
    assert _lib.slista_mask_words(256, 10 ** 6, 10 ** 4) == 256 // 32 * 10 ** 10  # > 2^32
    # trajectory sizes of large batches exceed 2^32 floats (device-dependent tiling: >= the plain size)
    assert _lib.slista_traj_floats(256, 10 ** 6, 40) >= 41 * 10 ** 6 * 256


def test_sizes(lib):
    assert _lib.slista_mask_words(256, 10000, 40) == 40 * 10000 * 8
    assert _lib.slista_mask_words(20, 7, 3) == 3 * 7 * 1
    assert _lib.slista_mask_words(33, 7, 3) == 3 * 7 * 2
    # ceil(40 / 7) - 1 = 5 checkpoints, each z and g
    assert _lib.slista_ckpt_floats(256, 10000, 40, 7) == 2 * 10000 * 256 * 5
    assert _lib.slista_ckpt_floats(256, 100, 40, 40) == 0
    assert _lib.slista_ckpt_floats(256, 100, 40, 50) == 0
    assert _lib.slista_workspace_bytes(_lib.FN_SLISTA_FWD, 256, 1000, 40, _lib.PREC_FP32) == 0
    ws = _lib.slista_workspace_bytes(_lib.FN_SLISTA_BWD, 256, 1000, 40, _lib.PREC_FP32, 7)
    assert ws >= 4 * 7 * 1000 * 256
    assert _lib.slista_workspace_bytes(_lib.FN_OBJECTIVE, 256, 1000, 40, 0) == 0


def _err(lib):
    return lib.slista_last_error().decode()


def test_argument_validation_without_gpu(lib):
    vp = ctypes.c_void_p(1)  # never dereferenced: validation fails first
    # null dictionary
    assert lib.lasso_gram(None, 4, 8, vp, 3, vp, vp, vp, None, None) == _lib.SLISTA_ERR_ARG
    assert "D and B" in _err(lib)
    # bad sizes
    assert lib.lasso_gram(vp, 0, 8, vp, 3, vp, vp, vp, None, None) == _lib.SLISTA_ERR_ARG
    # negative / NaN lambda
    for lam in (-1.0, float("nan"), float("inf")):
        rc = lib.slista_forward(vp, vp, 8, 4, lam, vp, 3, 0, vp, None, 0, None, 0, 1, None, 0, None)
        assert rc == _lib.SLISTA_ERR_ARG, lam
        assert "lam" in _err(lib)
    # unknown precision and unbuilt TF32
    assert lib.slista_forward(vp, vp, 8, 4, 0.1, vp, 3, 9, vp, None, 0, None, 0, 1, None, 0, None) == _lib.SLISTA_ERR_ARG
    assert lib.slista_forward(vp, vp, 8, 4, 0.1, vp, 3, _lib.PREC_TF32, vp, None, 0, None, 0, 1, None, 0,
                              None) == _lib.SLISTA_ERR_UNSUPPORTED
    # FP32 path limit
    assert lib.slista_forward(vp, vp, 300, 4, 0.1, vp, 3, 0, vp, None, 0, None, 0, 1, None, 0,
                              None) == _lib.SLISTA_ERR_UNSUPPORTED
    # checkpoint spacing
    assert lib.slista_forward(vp, vp, 8, 4, 0.1, vp, 3, 0, vp, vp, 1 << 40, vp, 1 << 40, 0, None, 0, None) == _lib.SLISTA_ERR_ARG
    # backward: workspace too small, missing checkpoints, precision
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, 0, vp, 1 << 40, vp, 1 << 40, 3, None, vp, None, 0,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, 0, vp, 1 << 40, None, 0, 3, None, vp, vp, 1 << 30,
                               None) == _lib.SLISTA_ERR_ARG
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, _lib.PREC_TF32, vp, 1 << 40, vp, 1 << 40, 3, None, vp, vp, 1 << 30,
                               None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, 9, vp, 1 << 40, vp, 1 << 40, 3, None, vp, vp, 1 << 30,
                               None) == _lib.SLISTA_ERR_ARG
    # tensor-core adjoint: at most 256 layers per recompute segment, and its own workspace size
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 300, _lib.PREC_BF16X3, vp, 1 << 40, None, 0, 300, None, vp, vp, 1 << 30,
                               None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert "256" in _err(lib)
    need = _lib.slista_workspace_bytes(_lib.FN_SLISTA_BWD, 8, 4, 10, _lib.PREC_BF16X3, 3)
    assert need >= 64 * 64 * 4 + 4 * 3 * 4 * 8
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, _lib.PREC_BF16X3, vp, 1 << 40, vp, 1 << 40, 3, None, vp, vp, need - 1,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    # a workspace off a 256-byte boundary (large enough) is refused before any launch
    odd = ctypes.c_void_p(0x1010)
    assert lib.slista_backward(vp, vp, 8, 4, 0.1, vp, 10, _lib.PREC_BF16X3, vp, 1 << 40, vp, 1 << 40, 3, None, vp, odd, need,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    assert "256-byte" in _err(lib)
    assert lib.slista_forward(vp, vp, 8, 4, 0.1, vp, 3, _lib.PREC_BF16X3, vp, None, 0, None, 0, 1, odd, 1 << 30,
                              None) == _lib.SLISTA_ERR_WORKSPACE
    # one-pass backward: precision, width and depth limits, workspace
    assert lib.slista_forward_traj(vp, vp, 8, 4, 0.1, vp, 3, _lib.PREC_FP32, vp, vp, 1 << 40, vp, 1 << 40, odd, 1 << 30,
                                   None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.slista_forward_traj(vp, vp, 300, 4, 0.1, vp, 3, _lib.PREC_BF16X3, vp, vp, 1 << 40, vp, 1 << 40, odd, 1 << 30,
                                   None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.slista_backward_traj(vp, 8, 4, 0.1, vp, 300, _lib.PREC_BF16X3, vp, 1 << 40, vp, 1 << 40, None, vp, odd, 1 << 30,
                                    None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.slista_forward_traj(vp, vp, 8, 4, 0.1, vp, 3, _lib.PREC_BF16X3, vp, None, 0, vp, 1 << 40, odd, 1 << 30,
                                   None) == _lib.SLISTA_ERR_ARG
    assert lib.slista_forward_traj(vp, vp, 8, 4, 0.1, vp, 3, _lib.PREC_BF16X3, vp, vp, 1 << 40, vp, 1 << 40, odd, 1 << 30,
                                   None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward_traj(vp, 8, 4, 0.1, vp, 3, _lib.PREC_BF16X3, vp, 1 << 40, vp, 1 << 40, None, vp, odd, 1 << 30,
                                    None) == _lib.SLISTA_ERR_WORKSPACE
    assert _lib.slista_traj_floats(300, 4, 3) == 0 and _lib.slista_traj_floats(8, 4, 300) == 0
    # OISTA and objective null pointers
    assert lib.oista_forward(vp, vp, None, 0, 8, 4, 0.1, None, 3, 0, vp, None, None, None, 0, None) == _lib.SLISTA_ERR_ARG
    assert lib.oista_forward(vp, vp, vp, 4, 8, 4, 0.1, vp, 3, 0, vp, None, None, None, 0,
                             None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.lasso_objective(vp, vp, None, vp, 8, 4, 0.1, vp, None, None) == _lib.SLISTA_ERR_ARG
    assert lib.lasso_lipschitz(vp, 0, vp, None) == _lib.SLISTA_ERR_ARG
    assert lib.ista_forward(vp, vp, 8, 4, 0.1, None, 3, 0, vp, None, 0, None) == _lib.SLISTA_ERR_ARG
    # standalone L_S: width limit, null pointers, n with D, workspace size and alignment
    assert lib.lasso_support_lipschitz(vp, None, 0, 300, 4, vp, vp, vp, odd, 1 << 30,
                                       None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.lasso_support_lipschitz(vp, None, 0, 8, 4, None, vp, vp, odd, 1 << 30, None) == _lib.SLISTA_ERR_ARG
    assert lib.lasso_support_lipschitz(vp, vp, 0, 8, 4, vp, vp, vp, odd, 1 << 30, None) == _lib.SLISTA_ERR_ARG
    need = _lib.slista_workspace_bytes(_lib.FN_SUPPORT_LIPSCHITZ, 40, 1000, 0, 0)
    assert need >= 4 * (2 * 1000 * 2 + 1000 + 6 * 1000)
    assert lib.lasso_support_lipschitz(vp, None, 0, 40, 1000, vp, vp, vp, ctypes.c_void_p(0x1000), need - 1,
                                       None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.lasso_support_lipschitz(vp, None, 0, 40, 1000, vp, vp, vp, odd, need,
                                       None) == _lib.SLISTA_ERR_WORKSPACE
    assert _lib.slista_workspace_bytes(_lib.FN_SUPPORT_LIPSCHITZ, 300, 1000, 0, 0) == 0
    # N = 0 needs no workspace and launches nothing
    assert lib.lasso_support_lipschitz(vp, None, 0, 40, 0, None, None, None, None, 0, None) == _lib.SLISTA_OK


def test_conv_gradient_validation_without_gpu(lib):
    """The convolutional trajectory forward and adjoint refuse bad sizes,
    filters longer than 32 taps, T = 0 and a short workspace before any
    launch (the pointers are never dereferenced)."""
    vp = ctypes.c_void_p(1)
    big = 1 << 40
    # n < Lf, T = 0
    assert lib.conv_slista_forward_traj(vp, 4, 16, vp, 8, 10, 0.1, vp, 5, vp, vp, big, None) == _lib.SLISTA_ERR_ARG
    assert lib.conv_slista_forward_traj(vp, 4, 16, vp, 8, 128, 0.1, vp, 0, vp, vp, big, None) == _lib.SLISTA_ERR_ARG
    # 33 taps
    assert lib.conv_slista_forward_traj(vp, 4, 33, vp, 8, 128, 0.1, vp, 5, vp, vp, big,
                                        None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.conv_slista_backward(vp, 4, 33, vp, 8, 128, 0.1, vp, 5, vp, big, vp, vp, 1 << 20,
                                    None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert _lib.conv_slista_backward_workspace_bytes(4, 33, 128, 8, 5) == 0
    # steps are required (no 1/L form of the adjoint); a null trajectory
    assert lib.conv_slista_backward(vp, 4, 16, vp, 8, 128, 0.1, None, 5, vp, big, vp, vp, 1 << 20,
                                    None) == _lib.SLISTA_ERR_ARG
    assert lib.conv_slista_backward(vp, 4, 16, vp, 8, 128, 0.1, vp, 5, None, big, vp, vp, 1 << 20,
                                    None) == _lib.SLISTA_ERR_ARG
    # the trajectory: maps padded to a multiple of 4 (P = 113 -> 116), its length checked, 16-byte aligned
    assert _lib.conv_slista_traj_floats(4, 16, 128, 8, 5) == 8 * 5 * 4 * 116
    assert _lib.conv_slista_traj_floats(4, 13, 128, 8, 5) == 8 * 5 * 4 * 116
    tf = _lib.conv_slista_traj_floats(4, 16, 128, 8, 5)
    aligned = ctypes.c_void_p(0x1000)
    assert lib.conv_slista_forward_traj(vp, 4, 16, vp, 8, 128, 0.1, vp, 5, vp, aligned, tf - 1,
                                        None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.conv_slista_forward_traj(vp, 4, 16, vp, 8, 128, 0.1, vp, 5, vp, ctypes.c_void_p(0x1004), tf,
                                        None) == _lib.SLISTA_ERR_ARG
    assert lib.conv_slista_backward(vp, 4, 16, vp, 8, 128, 0.1, vp, 5, aligned, tf - 1, vp, vp, 1 << 20,
                                    None) == _lib.SLISTA_ERR_WORKSPACE
    # workspace: one per-CTA partial per layer
    need = _lib.conv_slista_backward_workspace_bytes(4, 16, 128, 8, 5)
    assert need >= 5 * 4
    assert lib.conv_slista_backward(vp, 4, 16, vp, 8, 128, 0.1, vp, 5, aligned, tf, vp, vp, need - 1,
                                    None) == _lib.SLISTA_ERR_WORKSPACE
    # negative lambda
    assert lib.conv_slista_backward(vp, 4, 16, vp, 8, 128, -0.1, vp, 5, aligned, tf, vp, vp, need,
                                    None) == _lib.SLISTA_ERR_ARG


def test_conv2d_validation_without_gpu(lib):
    """The 2-D convolutional forward refuses bad sizes, images too large for
    its shared memory, missing steps and a negative lambda before any launch."""
    vp = ctypes.c_void_p(1)
    assert lib.conv2d_slista_forward(vp, 4, 5, 5, vp, 8, 4, 16, 0.1, vp, None, 5, vp, None) == _lib.SLISTA_ERR_ARG
    assert lib.conv2d_slista_forward(vp, 4, 5, 0, vp, 8, 16, 16, 0.1, vp, None, 5, vp, None) == _lib.SLISTA_ERR_ARG
    assert lib.conv2d_slista_forward(vp, 4, 5, 5, vp, 8, 256, 256, 0.1, vp, None, 5, vp,
                                     None) == _lib.SLISTA_ERR_UNSUPPORTED
    assert lib.conv2d_slista_forward(vp, 4, 5, 5, vp, 8, 16, 16, 0.1, None, None, 5, vp, None) == _lib.SLISTA_ERR_ARG
    assert lib.conv2d_slista_forward(vp, 4, 5, 5, vp, 8, 16, 16, -0.1, vp, None, 5, vp, None) == _lib.SLISTA_ERR_ARG


def test_python_binding_rejects_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    D = torch.zeros(4, 8)
    X = torch.zeros(3, 4)
    with pytest.raises(ValueError):
        _lib.lasso_gram(D, X, torch.zeros(8, 8), torch.zeros(3, 8), torch.zeros(3, dtype=torch.float64))


def test_conv_gradient_binding_layout_and_host_tensors(lib):
    """conv_traj_shape pads each map to a multiple of 4 codes, and the
    bindings of the convolutional trajectory forward and adjoint refuse host
    tensors before calling the library."""
    torch = pytest.importorskip("torch")
    assert _lib.conv_traj_shape(8, 16, 128, 10, 5) == (10, 5, 8, 116)
    assert _lib.conv_traj_shape(3, 5, 37, 2, 1) == (2, 1, 3, 36)
    F, X, a = torch.zeros(8, 16), torch.zeros(10, 128), torch.full((5,), 0.1)
    with pytest.raises(ValueError, match="CUDA"):
        _lib.conv_slista_forward_traj(F, X, 0.1, a, torch.zeros(10, 8 * 113), torch.zeros(10, 5, 8, 116))
    with pytest.raises(ValueError, match="CUDA"):
        _lib.conv_slista_backward(F, X, 0.1, a, torch.zeros(10, 5, 8, 116), torch.zeros(5))


def test_support_lipschitz_binding_rejects_host_tensors(lib):
    """The binding of lasso_support_lipschitz refuses host tensors before any
    call into the library."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="CUDA"):
        _lib.lasso_support_lipschitz(torch.zeros(40, 40), torch.zeros(5, 2, dtype=torch.int32),
                                     torch.ones(1, dtype=torch.float64), torch.zeros(5, dtype=torch.float64))


def test_short_caller_buffers_are_refused_before_any_launch(lib):
    """Masks, checkpoints and the trajectory are passed with their lengths;
    a length one element short of slista_mask_words / slista_ckpt_floats /
    slista_traj_floats returns SLISTA_ERR_WORKSPACE without touching the GPU
    (the pointers below are never dereferenced).  A binding that under-sized
    the trajectory of a 10^6-sample batch (a 32-bit truncation of
    slista_traj_floats) once made the forward write past its end; the C ABI
    now refuses such a buffer itself."""
    vp = ctypes.c_void_p(1)
    ws = ctypes.c_void_p(0x1000)  # 256-byte aligned, never dereferenced
    m, N, T, K = 64, 100, 10, 3
    mw = _lib.slista_mask_words(m, N, T)
    cf = _lib.slista_ckpt_floats(m, N, T, K)
    assert mw == T * N * 2 and cf == 2 * N * m * 3
    P3 = _lib.PREC_BF16X3
    big = 1 << 40
    # forward: masks one word short, then checkpoints one float short
    assert lib.slista_forward(vp, vp, m, N, 0.1, vp, T, P3, vp, vp, mw - 1, None, 0, 1, ws, big,
                              None) == _lib.SLISTA_ERR_WORKSPACE
    assert "masks" in _err(lib)
    assert lib.slista_forward(vp, vp, m, N, 0.1, vp, T, P3, vp, vp, mw, vp, cf - 1, K, ws, big,
                              None) == _lib.SLISTA_ERR_WORKSPACE
    assert "ckpt" in _err(lib)
    # the no-workspace forward checks its masks the same way
    assert lib.slista_forward_noalloc(vp, vp, m, N, 0.1, vp, T, P3, vp, vp, mw - 1, None) == _lib.SLISTA_ERR_WORKSPACE
    # backward
    assert lib.slista_backward(vp, vp, m, N, 0.1, vp, T, P3, vp, mw - 1, vp, cf, K, None, vp, ws, big,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward(vp, vp, m, N, 0.1, vp, T, P3, vp, mw, vp, cf - 1, K, None, vp, ws, big,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward(vp, vp, m, N, 0.1, vp, T, 0, vp, mw, vp, cf - 1, K, None, vp, ws, big,
                               None) == _lib.SLISTA_ERR_WORKSPACE
    # one-pass forward / backward: the trajectory's length follows the
    # device's tile layout, so it is queried and passed one float short
    tf = _lib.slista_traj_floats(m, N, T)
    assert tf >= (T + 1) * N * m
    assert lib.slista_forward_traj(vp, vp, m, N, 0.1, vp, T, P3, vp, vp, mw, vp, tf - 1, ws, big,
                                   None) == _lib.SLISTA_ERR_WORKSPACE
    assert "traj" in _err(lib)
    assert lib.slista_forward_traj(vp, vp, m, N, 0.1, vp, T, P3, vp, vp, mw - 1, vp, tf, ws, big,
                                   None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward_traj(vp, m, N, 0.1, vp, T, P3, vp, mw, vp, tf - 1, None, vp, ws, big,
                                    None) == _lib.SLISTA_ERR_WORKSPACE
    assert lib.slista_backward_traj(vp, m, N, 0.1, vp, T, P3, vp, mw - 1, vp, tf, None, vp, ws, big,
                                    None) == _lib.SLISTA_ERR_WORKSPACE
    # ragged batches: per-problem lengths in the descriptor
    arr = (_lib.Problem * 1)()
    p = arr[0]
    p.B, p.C, p.m, p.N, p.lam, p.alpha, p.Z = 1, 1, m, N, 0.1, 1, 1
    p.masks, p.mask_words, p.ckpt, p.ckpt_floats = 1, mw - 1, 1, cf
    assert lib.slista_forward_batched(arr, 1, T, P3, K, ws, big, None) == _lib.SLISTA_ERR_WORKSPACE
    assert "problem 0 masks" in _err(lib)
    p.mask_words, p.ckpt_floats = mw, cf - 1
    assert lib.slista_forward_batched(arr, 1, T, P3, K, ws, big, None) == _lib.SLISTA_ERR_WORKSPACE
    assert "problem 0 ckpt" in _err(lib)
