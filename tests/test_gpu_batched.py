"""Ragged batches of independent Lasso problems (slista_forward_batched /
slista_backward_batched): one persistent launch for the forward of all
problems and one (plus a reduction) for the backward.  Parity of
every problem with the FP64 oracle (BF16X3 tolerances of the tensor-core
tests), agreement with the single-problem calls, and replay under a CUDA
graph."""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"F": 1e-5, "Z": 1e-4, "grad": 1e-4}


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


def _small_batch(T, seed=0):
    """Six problems: widths 64 .. 400 (several below, several above 256),
    batch sizes 1 .. 300 (ragged row tiles)."""
    rng = np.random.default_rng(seed)
    spec = [(16, 64, 37), (40, 160, 300), (64, 256, 1), (72, 288, 130), (100, 400, 129), (24, 96, 0)]
    out = []
    for k, (n, m, N) in enumerate(spec):
        D = synth.gaussian_dictionary(n, m, rng)
        X = synth.sparse_model_samples(D, N, 0.05, 0.01, rng)
        lam = synth.lam_fraction(D, X, 0.1) if N > 0 else 0.1
        L = oracle.lipschitz(D)
        alpha = synth.step_sizes(T, 1.0 / L, 0.3, seed=seed + k)
        out.append((D, X, lam, alpha))
    return out


def _device_problems(batch):
    A = api()
    probs = []
    for D, X, lam, alpha in batch:
        g = A.gram(dev(D), dev(X), with_L=False)
        probs.append({"B": g.B, "C": g.C, "lam": lam, "alpha": dev(alpha), "xsq": g.xsq})
    return probs


def test_batched_forward_matches_oracle():
    T = 14
    batch = _small_batch(T)
    A = api()
    probs = _device_problems(batch)
    Zs = A.slista_batched(probs, prec="bf16x3")
    for (D, X, lam, alpha), q, Z in zip(batch, probs, Zs):
        if X.shape[0] == 0:
            assert Z.numel() == 0
            continue
        Zo = oracle.pgd(D, X, lam, alpha)
        zt = TOL["Z"] * max(1.0, float(np.abs(Zo).max()))
        assert np.abs(host(Z).astype(np.float64) - Zo).max() <= zt, D.shape
        F = host(A.objective(q["B"], q["C"], q["xsq"], Z, lam, with_gap=False))
        Fo = oracle.objective(D, X, Zo, lam, with_gap=False)
        assert (np.abs(F - Fo) / np.abs(Fo)).max() <= TOL["F"], D.shape


@pytest.mark.parametrize("K", [3, 14])
def test_batched_backward_matches_oracle(K):
    T = 14
    batch = _small_batch(T, seed=5)
    A = api()
    probs = _device_problems(batch)
    _, st, Kused = A.slista_batched(probs, prec="bf16x3", keep_for_backward=True, ckpt_every=K)
    das = A.slista_grad_batched(st, Kused, prec="bf16x3")
    for (D, X, lam, alpha), da in zip(batch, das):
        if X.shape[0] == 0:
            assert not da.any()
            continue
        do, _ = oracle.slista_grad(D, X, lam, alpha)
        rel = np.linalg.norm(host(da).astype(np.float64) - do) / np.linalg.norm(do)
        assert rel <= TOL["grad"], (D.shape, rel)


def test_batched_equals_single_calls_for_wide_problems():
    """For m > 256 the single-problem calls run the same layer arithmetic: the
    batch reproduces their codes bit for bit and their sub-gradients up to
    the order of the per-item sums."""
    T = 10
    batch = [b for b in _small_batch(T, seed=9) if b[0].shape[1] > 256]
    A = api()
    probs = _device_problems(batch)
    Zs, st, K = A.slista_batched(probs, prec="bf16x3", keep_for_backward=True, ckpt_every=4)
    das = A.slista_grad_batched(st, K, prec="bf16x3")
    for q, Z, da in zip(probs, Zs, das):
        Z1, s1 = A.slista(q["B"], q["C"], q["lam"], q["alpha"], prec="bf16x3", keep_for_backward=True,
                          ckpt_every=4)
        assert torch.equal(Z, Z1)
        # (the per-item partial sums may be grouped differently)
        torch.testing.assert_close(da, A.slista_grad(q["B"], q["C"], q["lam"], q["alpha"], s1, prec="bf16x3"),
                                   rtol=1e-5, atol=0.0)


def test_batched_forward_replays_under_cuda_graph():
    T = 8
    batch = _small_batch(T, seed=3)
    A = api()
    probs = _device_problems(batch)
    ref = A.slista_batched(probs, prec="bf16x3")  # eager; also sets up the kernels
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            out = A.slista_batched(probs, prec="bf16x3")
    torch.cuda.current_stream().wait_stream(s)
    for Z in out:
        Z.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for Zr, Zg in zip(ref, out):
        assert torch.equal(Zr, Zg)


def test_ragged_64_problems_sampled_rows():
    """The ragged configuration: 64 problems, n ~ U{32..128}, m = 4n,
    N ~ logU[100, 20000], lam = 0.1 lam_max each, T = 30, split BF16, forward
    and backward through the persistent batch kernels; sampled rows of 8 problems against
    the oracle, the gradient of every problem finite and the batch's gradient
    of the 8 problems against their single-problem calls."""
    problems = synth.ragged_problems()
    T = problems[0].T
    A = api()
    probs = []
    for w in problems:
        g = A.gram(dev(w.D), dev(w.X))
        alpha = (1.0 / g.L.double()).float().expand(T).contiguous()
        probs.append({"B": g.B, "C": g.C, "lam": w.lam, "alpha": alpha, "xsq": g.xsq, "L": g.L})
    Zs, st, K = A.slista_batched(probs, prec="bf16x3", keep_for_backward=True)
    das = A.slista_grad_batched(st, K, prec="bf16x3")
    assert all(torch.isfinite(d).all() for d in das)
    rng = np.random.default_rng(0)
    for p in rng.choice(len(problems), size=8, replace=False):
        w, q, Z = problems[p], probs[p], Zs[p]
        rows = rng.choice(w.N, size=min(16, w.N), replace=False)
        Zo = oracle.ista(w.D, w.X[rows], w.lam, oracle.lipschitz(w.D), T)
        zt = TOL["Z"] * max(1.0, float(np.abs(Zo).max()))
        assert np.abs(host(Z)[rows].astype(np.float64) - Zo).max() <= zt, (p, w.D.shape)
        Z1, s1 = A.slista(q["B"], q["C"], q["lam"], q["alpha"], prec="bf16x3", keep_for_backward=True,
                          ckpt_every=K)
        d1 = host(A.slista_grad(q["B"], q["C"], q["lam"], q["alpha"], s1, prec="bf16x3")).astype(np.float64)
        d = host(das[p]).astype(np.float64)
        assert np.linalg.norm(d - d1) <= TOL["grad"] * np.linalg.norm(d1), (p, w.D.shape)
