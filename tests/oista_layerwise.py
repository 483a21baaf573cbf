"""Layer-by-layer comparison of the GPU's Oracle-ISTA (Algorithm 1) with the
FP64 oracle, shared by the GPU test modules.

Algorithm 1 takes discrete decisions at every layer: condition (star) (does
the local step 1/L_S keep the support?) and the thresholds of ST.  Where the
oracle's decision margin at a layer is below the arithmetic's error scale, the
GPU may decide the other way, and from the next layer on that sample follows
another (equally valid) trajectory.  So each sample is compared with the
oracle layer by layer, up to its first layer whose margin is at most `tol`:

* codes z^(t) elementwise for every t <= first(s) (z^(t) depends only on the
  decisions of layers 0 .. t-1, all of them safe);
* the per-layer accepted counts: layer t may differ by at most the number of
  samples with first(s) <= t (the others take the oracle's decision there);
* L_S of the last evaluated support, on the samples whose decisions up to
  layer T - 2 are safe (that support is supp z^(T-1)).

The GPU's z^(t) is taken from a separate GPU call with T = t layers (the
iteration does not depend on T), so no GPU value is ever fed to the oracle.
"""
import numpy as np

import oracle


def first_unsafe_layer(layer_margin, tol):
    """Per sample, the first layer whose decision margin is <= tol (T if none)."""
    T, N = layer_margin.shape
    unsafe = layer_margin <= tol
    return np.where(unsafe.any(axis=0), unsafe.argmax(axis=0), T)


def compare_layerwise(run_gpu, D, X, lam, T, tol, z_tol, ls_rtol=1e-5, L=None):
    """run_gpu(t) -> (Z, LS, accepted) as numpy arrays for a t-layer GPU call.

    Asserts the comparisons listed in the module docstring and returns a dict
    with the fraction of (sample, layer) pairs whose codes were compared and
    the largest code error seen on them."""
    Lo = oracle.lipschitz(D) if L is None else L
    Zall, LSo, acco, deco, lm = oracle.oista(D, X, lam, Lo, T, keep_all=True, layer_margins=True)
    N = X.shape[0]
    first = first_unsafe_layer(lm, tol)
    ztol = z_tol * max(1.0, float(np.abs(Zall).max()))
    compared = 0
    worst = 0.0
    for t in range(1, T + 1):
        Zg, LSg, accg = run_gpu(t)
        rows = first >= t
        if rows.any():
            err = float(np.abs(Zg[rows].astype(np.float64) - Zall[t][rows]).max())
            worst = max(worst, err)
            assert err <= ztol, ("codes after layer", t, err, ztol)
        compared += int(rows.sum())
        if t == T:
            for u in range(T):
                bound = int((first <= u).sum())
                assert abs(int(accg[u]) - int(acco[u])) <= bound, ("accepted", u, accg[u], acco[u], bound)
            ls_rows = first >= T - 1
            if ls_rows.any():
                np.testing.assert_allclose(LSg[ls_rows], LSo[ls_rows], rtol=ls_rtol)
    frac = compared / float(T * N) if T * N else 1.0
    return {"frac": frac, "worst": worst, "first": first, "Zo": Zall[T], "acco": acco}
