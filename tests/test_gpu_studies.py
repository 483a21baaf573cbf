"""Two studies of the paper run on the GPU path and checked against the FP64
oracle:

* Oracle-ISTA's accept / fall-back pattern (Section 3, Appendix B): on the
  paper's 100 x 200 setup (x in B_inf), per layer the number of samples whose
  step 1/L_S is accepted by condition (star) is the oracle's, up to the
  samples that met a decision margin below the FP32 rounding scale at or
  before that layer; and the
  objective reached after T layers matches the oracle's.
* Learned steps (Section 4, Appendix E): Step-LISTA trained on 10 x 20,
  lam = 0.2, N = 1000 (T = 20) lowers the unsupervised loss monotonically and
  learns steps larger than ISTA's 1/L in the later layers (the supports of
  late layers are small, and 1/L_S > 1/L on them).  As in Fig. 4, the
  learned alpha_t follow the distribution of 1/L_S(x, t) over the training
  samples, S(x, t) = supp z^(t)(x), with L_S from lasso_support_lipschitz.
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


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("lam", [0.2, 0.5])
def test_oista_accept_pattern_100x200(lam):
    """Per layer, the accepted count differs from the oracle's by at most the
    samples that met a decision with margin <= 5e-6 at or before that layer."""
    from paper_1905_11071_gb300 import api as A
    from oista_layerwise import first_unsafe_layer
    w = synth.paper_binf(100, 200, N=32, lam=lam, T=300, seed=4)
    g = A.gram(dev(w.D), dev(w.X))
    Zg, LSg, accg = A.oista(g.B, g.C, w.lam, g.L, w.T, D=dev(w.D))
    Lo = oracle.lipschitz(w.D)
    Zo, LSo, acco, deco, lm = oracle.oista(w.D, w.X, w.lam, Lo, w.T, layer_margins=True)
    first = first_unsafe_layer(lm, 5e-6)
    accg = host(accg)
    for t in range(w.T):
        assert abs(int(accg[t]) - int(acco[t])) <= int((first <= t).sum()), t
    # Oracle-ISTA accepts its step at most layers once supports settle
    assert acco[-50:].mean() >= 0.5 * w.N
    safe = first >= w.T
    Fg = host(A.objective(g.B, g.C, g.xsq, Zg, w.lam, with_gap=False))
    Fo = oracle.objective(w.D, w.X, Zo, w.lam, with_gap=False)
    assert (np.abs(Fg[safe] - Fo[safe]) / np.abs(Fo[safe])).max() <= 1e-5


def test_learned_steps_10x20():
    from paper_1905_11071_gb300 import api as A
    T = 20
    w = synth.paper_binf(10, 20, N=1000, lam=0.2, T=T, seed=0)
    g = A.gram(dev(w.D), dev(w.X))
    L = float(host(g.L)[0])
    alpha0 = torch.full((T,), 1.0 / L, dtype=torch.float32, device="cuda")
    alpha, hist = A.train_step_sizes(alpha0, g, w.lam, steps=60)
    hist = np.asarray(hist)
    assert np.all(np.diff(hist) <= 1e-9 * np.abs(hist[:-1]))  # backtracking never increases the loss
    assert hist[-1] < hist[0]
    a = host(alpha).astype(np.float64)
    assert a[T // 2:].mean() > 1.0 / L
    # the starting point is ISTA itself: its loss (hist[0]) against the oracle
    Zi = oracle.ista(w.D, w.X, w.lam, oracle.lipschitz(w.D), T)
    F_ista = oracle.objective(w.D, w.X, Zi, w.lam, with_gap=False).sum()
    assert abs(hist[0] - F_ista) <= 1e-5 * abs(F_ista)


def _rank(v):
    r = np.empty(len(v))
    r[np.argsort(v, kind="stable")] = np.arange(len(v))
    return r


def test_learned_steps_follow_support_steps_10x20():
    """Fig. 4: the steps learned on 10 x 20 (lam = 0.2, T = 20, N = 1000) grow
    with the per-layer distribution of 1/L_S(x, t): their rank correlation
    with its median is high, and in the second half of the network every
    alpha_t lies between that median and its maximum."""
    from paper_1905_11071_gb300 import api as A
    T = 20
    w = synth.paper_binf(10, 20, N=1000, lam=0.2, T=T, seed=0)
    g = A.gram(dev(w.D), dev(w.X))
    L = float(host(g.L)[0])
    alpha0 = torch.full((T,), 1.0 / L, dtype=torch.float32, device="cuda")
    alpha, _ = A.train_step_sizes(alpha0, g, w.lam, steps=60)
    _, st = A.slista(g.B, g.C, w.lam, alpha, keep_for_backward=True)
    masks = st.masks.view(T, w.N, -1)
    med, top = [1.0 / L], [1.0 / L]  # layer 0 acts on z^(0) = 0: S empty, L_empty = L
    for t in range(1, T):
        inv = 1.0 / host(A.support_lipschitz(g.B, masks[t - 1].contiguous(), g.L))
        med.append(float(np.median(inv)))
        top.append(float(inv.max()))
    a = host(alpha).astype(np.float64)
    med, top = np.array(med), np.array(top)
    assert np.corrcoef(_rank(a), _rank(med))[0, 1] >= 0.8
    h = T // 2
    assert (med[h:] <= a[h:]).all() and (a[h:] <= top[h:]).all()


@pytest.mark.parametrize("method", ["ista", "oista"])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_objective_never_increases_along_gpu_layers(method, prec):
    """The descent property that Sections 2 and 3 rest on, on the GPU's own
    iterates: with the step 1/L (ISTA, Eq. majorization2) or 1/L_S when
    condition (star) holds (Oracle-ISTA, Section 3), F(z^(t+1)) <= F(z^(t))
    for every sample and layer.  An L or L_S from the FP32 Lanczos that came
    out too small would make a step too long and could break it.  The
    objective is the GPU's FP64-reduced one; the allowance is its rounding
    (1e-6 relative)."""
    from paper_1905_11071_gb300 import api as A
    w = synth.slista_64x256(N=400, T=30)
    g = A.gram(dev(w.D), dev(w.X))
    prev = host(g.xsq) * 0.5  # F(0) = ||x||^2 / 2
    for t in range(1, w.T + 1):
        if method == "ista":
            Z = A.ista(g.B, g.C, w.lam, g.L, t, prec=prec)
        else:
            Z, _, _ = A.oista(g.B, g.C, w.lam, g.L, t, D=dev(w.D), prec=prec)
        F = host(A.objective(g.B, g.C, g.xsq, Z, w.lam, with_gap=False))
        assert (F <= prev + 1e-6 * np.abs(prev)).all(), (method, prec, t, float((F - prev).max()))
        prev = F
