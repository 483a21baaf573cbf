"""slista_forward_noalloc: the tensor-core Step-LISTA forward for callers that
cannot allocate device memory at call time (their device memory belongs to
another allocator or is reserved up front, or they cannot pay for the
synchronisation cudaMalloc implies).  Its scratch is a static device array of
the library, so it takes no workspace; its results must equal those of
slista_forward with a caller-provided workspace.

The entry point is called through the C ABI (ctypes); torch only provides the
caller's input and output buffers.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {3: 1e-4, 2: 2e-2}  # relative to max(1, max|z|): BF16X3, BF16 (as in the tensor-core tests)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1905_11071_gb300 import build, _lib
    build.build()
    return _lib.load()


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _problem(n, m, N, T, seed):
    from paper_1905_11071_gb300 import api, synth
    rng = np.random.default_rng(seed)
    D = synth.gaussian_dictionary(n, m, rng)
    X = synth.sparse_model_samples(D, N, 0.05, 0.01, rng)
    lam = synth.lam_fraction(D, X, 0.1)
    g = api.gram(torch.from_numpy(D).cuda(), torch.from_numpy(X).cuda())
    alpha = ((1.0 / g.L.double()) * torch.linspace(0.8, 1.2, T, dtype=torch.float64, device="cuda")).float()
    return g, lam, alpha.contiguous()


def _masks(lib, m, N, T, fill):
    from paper_1905_11071_gb300 import _lib
    nw = _lib.slista_mask_words(m, N, T)
    return torch.full((nw,), fill, dtype=torch.int32, device="cuda"), nw


def _with_workspace(lib, g, lam, alpha, prec):
    from paper_1905_11071_gb300 import _lib
    N, m = g.C.shape
    T = alpha.shape[0]
    Z = torch.empty((N, m), dtype=torch.float32, device="cuda")
    masks, nw = _masks(lib, m, N, T, 0)
    nb = _lib.slista_workspace_bytes(_lib.FN_SLISTA_FWD, m, N, T, prec)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    rc = lib.slista_forward(_p(g.B), _p(g.C), m, N, lam, _p(alpha), T, prec, _p(Z), _p(masks), nw, None, 0, 1,
                            _p(ws), nb, _stream())
    assert rc == 0, lib.slista_last_error()
    return Z, masks


def _noalloc(lib, g, lam, alpha, prec, with_masks=True):
    N, m = g.C.shape
    T = alpha.shape[0]
    Z = torch.full((N, m), float("nan"), dtype=torch.float32, device="cuda")
    masks, nw = _masks(lib, m, N, T, -1) if with_masks else (None, 0)
    rc = lib.slista_forward_noalloc(_p(g.B), _p(g.C), m, N, lam, _p(alpha), T, prec, _p(Z), _p(masks), nw,
                                    _stream())
    assert rc == 0, lib.slista_last_error()
    return Z, masks


def _close(got, ref, prec):
    """Codes within the tensor-core tolerance; support masks bit for bit (the
    same kernel runs, so the decisions are identical)."""
    (Z, mk), (Zr, mkr) = got, ref
    torch.cuda.synchronize()
    tol = TOL[prec] * max(1.0, float(Zr.abs().max()))
    err = float((Z - Zr).abs().max())
    assert err <= tol, (prec, err, tol)
    if mk is not None:
        assert torch.equal(mk, mkr)


@pytest.mark.parametrize("prec", [3, 2])
def test_noalloc_matches_workspace_forward_twice(lib, prec):
    g, lam, alpha = _problem(64, 256, 700, 40, seed=11)
    ref = _with_workspace(lib, g, lam, alpha, prec)
    for _ in range(2):  # the static scratch keeps the previous call's contents
        _close(_noalloc(lib, g, lam, alpha, prec), ref, prec)
    # a smaller problem in between (m padded to 128), then the first again,
    # with and without masks
    g2, lam2, alpha2 = _problem(32, 100, 300, 20, seed=12)
    _close(_noalloc(lib, g2, lam2, alpha2, prec), _with_workspace(lib, g2, lam2, alpha2, prec), prec)
    _close(_noalloc(lib, g, lam, alpha, prec), ref, prec)
    _close(_noalloc(lib, g, lam, alpha, prec, with_masks=False), ref, prec)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    vp = ctypes.c_void_p(1)  # never dereferenced: the size check fails first
    rc = lib.slista_forward_noalloc(vp, vp, 300, 4, 0.1, vp, 3, 3, vp, None, 0, None)
    assert rc == -2
    assert b"m <= 256" in lib.slista_last_error()
    rc = lib.slista_forward_noalloc(vp, vp, 64, 4, 0.1, vp, 3, 0, vp, None, 0, None)  # FP32 has no such variant
    assert rc == -2
