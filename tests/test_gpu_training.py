"""Step-size training of a 40-layer Step-LISTA network on the 64 x 256
workload (Section 4, Eq. unsupervised; Appendix E's backtracking descent),
with the forward and the hand-written adjoint at each precision of the
tensor-core path and on the CUDA cores.

* The training loss never increases (backtracking accepts a step only when
  the loss does not grow).
* The learned steps generalise: on 2000 held-out samples the unsupervised
  loss of the trained network is no larger than ISTA's with the same number
  of layers (ISTA is the network at its initialisation alpha_t = 1/L; the
  squeeze argument of Section 4 makes Step-LISTA at least as good as ISTA
  once trained).
* The held-out losses are GPU objectives of GPU forwards; ISTA's held-out
  loss is also evaluated by the FP64 oracle on its own (oracle L, no GPU
  value as input), which pins the GPU's evaluation path.
"""
import numpy as np
import pytest

import oracle
from paper_1905_11071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_ready():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1905_11071_gb300 import build, _lib
    build.build()
    _lib.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def split():
    return synth.slista_train_64x256(N_train=10000, N_test=2000, T=40)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "fp32"])
def test_training_lowers_train_and_held_out_loss(split, prec):
    from paper_1905_11071_gb300 import api
    train, test = split
    g = api.gram(dev(train.D), dev(train.X))
    gt = api.gram(dev(test.D), dev(test.X))
    Lo = oracle.lipschitz(train.D)
    alpha0 = (1.0 / g.L.double()).float().expand(train.T).contiguous()
    alpha, hist = api.train_step_sizes(alpha0, g, train.lam, steps=12, prec=prec)
    assert len(hist) >= 2
    assert all(b <= a for a, b in zip(hist, hist[1:])), hist
    assert hist[-1] < hist[0]
    assert (alpha > 0).all()
    # held-out loss on 400 rows: trained network vs ISTA (alpha_t = 1/L) at equal T
    rows = np.random.default_rng(7).choice(test.N, size=400, replace=False)
    F = lambda Z: api.objective(gt.B, gt.C, gt.xsq, Z, test.lam, with_gap=False).cpu().numpy()[rows].sum()
    F_tr = F(api.slista(gt.B, gt.C, test.lam, alpha, prec=prec))
    F_ista_gpu = F(api.ista(gt.B, gt.C, test.lam, gt.L, test.T, prec=prec))
    assert F_tr <= F_ista_gpu, (prec, F_tr, F_ista_gpu)
    # the GPU's ISTA held-out loss against the oracle's (its own inputs only)
    F_ista = oracle.objective(test.D, test.X[rows], oracle.ista(test.D, test.X[rows], test.lam, Lo, test.T),
                              test.lam, with_gap=False).sum()
    tol = 1e-3 if prec == "bf16" else 1e-5
    assert abs(F_ista_gpu - F_ista) <= tol * abs(F_ista), (prec, F_ista_gpu, F_ista)
