"""Tensor-level API over the C ABI: allocates outputs and workspaces with torch
and calls the entry points of ``_lib`` (every computation runs in the CUDA
library).  Also provides the autograd function that trains Step-LISTA step
sizes on the unsupervised loss sum_i F_{x_i}(Phi(x_i)) (Eq. unsupervised).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import torch

from . import _lib


def default_ckpt_every(T: int) -> int:
    """Checkpoint spacing ceil(sqrt(T)): memory ~ sqrt(T) states, ~1 recompute."""
    return max(1, int(math.ceil(math.sqrt(max(T, 1)))))


def _prec(prec) -> int:
    if isinstance(prec, str):
        return _lib.PRECISIONS[prec]
    return int(prec)


_ws_cache: dict = {}


def workspace(nbytes: int, device, tag: str = "default") -> Optional[torch.Tensor]:
    """A cached uint8 device buffer of at least nbytes (None if nbytes == 0)."""
    if nbytes <= 0:
        return None
    key = (str(device), tag)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


@dataclass
class Gram:
    B: torch.Tensor      # m x m float32
    C: torch.Tensor      # N x m float32
    xsq: torch.Tensor    # N float64
    L: torch.Tensor      # 1 float64 (device)


def gram(D: torch.Tensor, X: torch.Tensor, with_L: bool = True, stream=None) -> Gram:
    n, m = D.shape
    N = X.shape[0]
    dev = D.device
    B = torch.empty((m, m), dtype=torch.float32, device=dev)
    C = torch.empty((N, m), dtype=torch.float32, device=dev)
    xsq = torch.empty((N,), dtype=torch.float64, device=dev)
    L = torch.empty((1,), dtype=torch.float64, device=dev) if with_L else None
    _lib.lasso_gram(D, X, B, C, xsq, L, stream=stream)
    return Gram(B, C, xsq, L)


def lipschitz(B: torch.Tensor, stream=None) -> torch.Tensor:
    L = torch.empty((1,), dtype=torch.float64, device=B.device)
    _lib.lasso_lipschitz(B, L, stream=stream)
    return L


def ista(B, C, lam, L, T, prec="fp32", stream=None) -> torch.Tensor:
    N, m = C.shape
    p = _prec(prec)
    Z = torch.empty((N, m), dtype=torch.float32, device=C.device)
    ws = workspace(_lib.slista_workspace_bytes(_lib.FN_ISTA, m, N, T, p), C.device, "fwd")
    _lib.ista_forward(B, C, lam, L, T, p, Z, ws=ws, stream=stream)
    return Z


@dataclass
class ForwardState:
    """What slista_backward needs from a forward call: masks and checkpoints,
    or (trajectory forward) masks and the trajectory."""
    masks: torch.Tensor
    ckpt: Optional[torch.Tensor]
    ckpt_every: int
    traj: Optional[torch.Tensor] = None
    tile_rows: int = 0   # the layer kernels' tile setting the buffers were laid out for


def slista(B, C, lam, alpha, prec="fp32", keep_for_backward: bool = False,
           ckpt_every: Optional[int] = None, trajectory: bool = False, stream=None):
    """Step-LISTA forward (Eq. steprec).  Returns Z, or (Z, ForwardState).
    trajectory=True (tensor-core precisions, m <= 256, T <= 256) keeps the
    adjoint's inputs instead of checkpoints: more memory, no recompute in
    slista_grad."""
    N, m = C.shape
    T = alpha.shape[0]
    p = _prec(prec)
    dev = C.device
    Z = torch.empty((N, m), dtype=torch.float32, device=dev)
    ws = workspace(_lib.slista_workspace_bytes(_lib.FN_SLISTA_FWD, m, N, T, p), dev, "fwd")
    if not keep_for_backward:
        _lib.slista_forward(B, C, lam, alpha, p, Z, ws=ws, stream=stream)
        return Z
    if trajectory:
        masks = torch.empty((max(1, _lib.slista_mask_words(m, N, T)),), dtype=torch.int32, device=dev)
        nt = _lib.slista_traj_floats(m, N, T)
        if nt == 0:
            raise ValueError("trajectory forward: m <= 256 and 1 <= T <= 256 on the tensor cores")
        traj = torch.empty((nt,), dtype=torch.float32, device=dev)
        _lib.slista_forward_traj(B, C, lam, alpha, p, Z, masks, traj, ws=ws, stream=stream)
        return Z, ForwardState(masks, None, T, traj, _lib.slista_get_tile_rows())
    K = ckpt_every or default_ckpt_every(T)
    masks = torch.empty((max(1, _lib.slista_mask_words(m, N, T)),), dtype=torch.int32, device=dev)
    nck = _lib.slista_ckpt_floats(m, N, T, K)
    ckpt = torch.empty((nck,), dtype=torch.float32, device=dev) if nck > 0 else None
    _lib.slista_forward(B, C, lam, alpha, p, Z, masks=masks, ckpt=ckpt, ckpt_every=K, ws=ws, stream=stream)
    return Z, ForwardState(masks, ckpt, K, None, _lib.slista_get_tile_rows())


def slista_grad(B, C, lam, alpha, state: ForwardState, gZ=None, prec="fp32", stream=None) -> torch.Tensor:
    """Sub-gradient of sum_i F(z_i^(T)) (or of <gZ, z^(T)>) w.r.t. alpha."""
    N, m = C.shape
    T = alpha.shape[0]
    p = _prec(prec)
    if state.tile_rows != _lib.slista_get_tile_rows():
        raise ValueError("the layer kernels' tile setting changed between the forward and the backward")
    dalpha = torch.empty((T,), dtype=torch.float32, device=C.device)
    if state.traj is not None:
        ws = workspace(_lib.slista_workspace_bytes(_lib.FN_SLISTA_BWD_TRAJ, m, N, T, p, 1), C.device, "bwd")
        _lib.slista_backward_traj(B, N, lam, alpha, p, state.masks, state.traj, dalpha, gZ=gZ, ws=ws,
                                  stream=stream)
        return dalpha
    ws = workspace(_lib.slista_workspace_bytes(_lib.FN_SLISTA_BWD, m, N, T, p, state.ckpt_every), C.device,
                   "bwd")
    _lib.slista_backward(B, C, lam, alpha, p, state.masks, state.ckpt, state.ckpt_every, dalpha, gZ=gZ,
                         ws=ws, stream=stream)
    return dalpha


def slista_batched(problems, prec="bf16x3", keep_for_backward: bool = False, ckpt_every: Optional[int] = None,
                   stream=None):
    """Step-LISTA forward of a ragged batch (one launch per layer for all
    problems).  problems: list of dicts with B (m x m), C (N x m), lam and
    alpha (T steps, the same T for all).  Returns the list of Z, and with
    keep_for_backward the per-problem masks / checkpoints (added to the dicts
    under "masks", "ckpt") and the checkpoint spacing."""
    T = int(problems[0]["alpha"].shape[0]) if problems else 0
    p = _prec(prec)
    K = ckpt_every or default_ckpt_every(T)
    dev = problems[0]["C"].device if problems else None
    probs = []
    for q in problems:
        N, m = q["C"].shape
        d = dict(q)
        d["Z"] = torch.empty((N, m), dtype=torch.float32, device=dev)
        if keep_for_backward:
            d["masks"] = torch.empty((max(1, _lib.slista_mask_words(m, N, T)),), dtype=torch.int32, device=dev)
            nck = _lib.slista_ckpt_floats(m, N, T, K)
            d["ckpt"] = torch.empty((nck,), dtype=torch.float32, device=dev) if nck > 0 else None
        else:
            d.pop("masks", None)
            d.pop("ckpt", None)
        probs.append(d)
    sizes = [{"m": int(q["C"].shape[1]), "N": int(q["C"].shape[0])} for q in problems]
    ws = workspace(_lib.slista_batched_workspace_bytes(_lib.FN_SLISTA_FWD, sizes, T, p, K), dev, "bfwd") \
        if problems else None
    _lib.slista_forward_batched(probs, T, p, K, ws=ws, stream=stream)
    Zs = [d["Z"] for d in probs]
    return (Zs, probs, K) if keep_for_backward else Zs


def slista_grad_batched(probs, ckpt_every: int, prec="bf16x3", gZs=None, stream=None):
    """Step-size sub-gradients of a batch from slista_batched(...,
    keep_for_backward=True)'s problem dicts.  Returns the list of dalpha."""
    T = int(probs[0]["alpha"].shape[0])
    p = _prec(prec)
    dev = probs[0]["C"].device
    qs = []
    for i, d in enumerate(probs):
        q = dict(d)
        q["dalpha"] = torch.empty((T,), dtype=torch.float32, device=dev)
        q["gZ"] = None if gZs is None else gZs[i]
        qs.append(q)
    sizes = [{"m": int(q["C"].shape[1]), "N": int(q["C"].shape[0])} for q in probs]
    ws = workspace(_lib.slista_batched_workspace_bytes(_lib.FN_SLISTA_BWD, sizes, T, p, ckpt_every), dev, "bbwd")
    _lib.slista_backward_batched(qs, T, p, ckpt_every, ws=ws, stream=stream)
    return [q["dalpha"] for q in qs]


def oista(B, C, lam, L, T, D=None, prec="fp32", stream=None):
    """Oracle-ISTA (Algorithm 1).  Returns (Z, LS, accepted).  D (optional)
    lets supports larger than 64 be solved on the n x n matrix D_S D_S^T.
    prec: "fp32" (CUDA-core layers) or "bf16x3" / "bf16" (tensor-core layers)."""
    N, m = C.shape
    p = _prec(prec)
    dev = C.device
    Z = torch.empty((N, m), dtype=torch.float32, device=dev)
    LS = torch.empty((N,), dtype=torch.float64, device=dev)
    acc = torch.empty((max(T, 1),), dtype=torch.int32, device=dev)
    ws = workspace(_lib.slista_workspace_bytes(_lib.FN_OISTA, m, N, T, p), dev, "oista")
    _lib.oista_forward(B, C, lam, L, T, p, Z, LS=LS, accepted=acc[:T] if T > 0 else None,
                       ws=ws, D=D, stream=stream)
    return Z, LS, acc[:T]


def support_lipschitz(B, S, L, D=None, stream=None):
    """L_S (Eq. spca) for the N supports given as rows of S, N x ceil(m/32)
    int32 words (bit j % 32 of word j / 32 set iff code j is in the support;
    one layer of the support masks).  Returns LS (N doubles)."""
    N, m = S.shape[0], B.shape[0]
    LS = torch.empty((N,), dtype=torch.float64, device=B.device)
    ws = workspace(_lib.slista_workspace_bytes(_lib.FN_SUPPORT_LIPSCHITZ, m, N, 0, 0), B.device, "support_ls")
    _lib.lasso_support_lipschitz(B, S, L, LS, ws=ws, D=D, stream=stream)
    return LS


def lista(D, X, W, alpha, beta, lam, stream=None) -> torch.Tensor:
    """Coupled LISTA (Eq. lista_layer): T layers with per-layer (W_t, alpha_t,
    beta_t); W is T x n x m.  Returns z^(T) (N x m)."""
    n, m = D.shape
    N = X.shape[0]
    Z = torch.empty((N, m), dtype=torch.float32, device=D.device)
    ws = workspace(_lib.lista_workspace_bytes(n, m, N), D.device, "lista")
    _lib.lista_forward(D, X, W, alpha, beta, lam, Z, ws=ws, stream=stream)
    return Z


def conv_slista(filters, X, lam, alpha=None, L=None, T=None, stream=None) -> torch.Tensor:
    """Step-LISTA (alpha: T steps) or ISTA (alpha None, step 1/L) on a 1-D
    convolutional dictionary (Section 6): filters K x Lf, X N x n.  Returns
    the codes, N x K (n - Lf + 1), map k in columns [k P, (k + 1) P)."""
    K, Lf = filters.shape
    N, n = X.shape
    T = int(alpha.shape[0]) if alpha is not None else int(T)
    Z = torch.empty((N, K * (n - Lf + 1)), dtype=torch.float32, device=X.device)
    _lib.conv_slista_forward(filters, X, lam, alpha, L, T, Z, stream=stream)
    return Z


def conv2d_slista(filters, X, lam, alpha=None, L=None, T=None, stream=None) -> torch.Tensor:
    """Step-LISTA (alpha: T steps) or ISTA (alpha None, step 1/L) on a 2-D
    convolutional dictionary (Section 6): filters K x Lh x Lw, X N x H x W
    images.  Returns the codes, N x K x (H - Lh + 1) x (W - Lw + 1)."""
    K, Lh, Lw = filters.shape
    N, H, W = X.shape
    T = int(alpha.shape[0]) if alpha is not None else int(T)
    Z = torch.empty((N, K, H - Lh + 1, W - Lw + 1), dtype=torch.float32, device=X.device)
    _lib.conv2d_slista_forward(filters, X, lam, alpha, L, T, Z, stream=stream)
    return Z


def conv_slista_grad(filters, X, lam, alpha, stream=None):
    """Step-LISTA on a 1-D convolutional dictionary and the sub-gradient of
    sum_i F_{x_i}(z_i^(T)) with respect to its steps alpha (Eq. steprec).
    Returns (Z, dalpha); the trajectory (N x T x K x P rounded up to 4
    floats) lives only for the call."""
    K, Lf = filters.shape
    N, n = X.shape
    T = int(alpha.shape[0])
    m = K * (n - Lf + 1)
    Z = torch.empty((N, m), dtype=torch.float32, device=X.device)
    traj = torch.empty(_lib.conv_traj_shape(K, Lf, n, N, T), dtype=torch.float32, device=X.device)
    dalpha = torch.empty((T,), dtype=torch.float32, device=X.device)
    ws = workspace(_lib.conv_slista_backward_workspace_bytes(K, Lf, n, N, T), X.device, "conv_bwd")
    _lib.conv_slista_forward_traj(filters, X, lam, alpha, Z, traj, stream=stream)
    _lib.conv_slista_backward(filters, X, lam, alpha, traj, dalpha, ws=ws, stream=stream)
    if stream is not None:
        traj.record_stream(stream)  # freed here, still read on that stream
    return Z, dalpha


def objective(B, C, xsq, Z, lam, with_gap: bool = True, stream=None):
    N = C.shape[0]
    F = torch.empty((N,), dtype=torch.float64, device=C.device)
    gap = torch.empty((N,), dtype=torch.float64, device=C.device) if with_gap else None
    _lib.lasso_objective(B, C, xsq, Z, lam, F, gap, stream=stream)
    return (F, gap) if with_gap else F


def _traj_ok(prec, m: int, T: int) -> bool:
    """Whether the one-pass (trajectory) backward exists for this case."""
    return _prec(prec) in (_lib.PREC_BF16, _lib.PREC_BF16X3) and m <= 256 and 1 <= T <= 256


class SlistaLoss(torch.autograd.Function):
    """sum_i F_{x_i}(Phi_alpha(x_i)) with Phi the T-layer Step-LISTA network
    (the empirical form of Eq. unsupervised).

    forward(alpha, B, C, xsq, lam, ckpt_every, prec) -> scalar loss (float64)
    backward -> d loss / d alpha from the hand-written adjoint kernel at the
    same precision: on the tensor cores ("bf16x3", "bf16") the forward keeps
    the adjoint's inputs (one reverse sweep, m <= 256) or checkpoints; on the
    CUDA cores ("fp32") checkpoints and a recompute.
    """

    @staticmethod
    def forward(ctx, alpha, B, C, xsq, lam, ckpt_every=None, prec="fp32"):
        m, T = C.shape[1], alpha.shape[0]
        traj = _traj_ok(prec, m, T)
        Z, st = slista(B, C, lam, alpha, prec=prec, keep_for_backward=True, ckpt_every=ckpt_every,
                       trajectory=traj)
        F = objective(B, C, xsq, Z, lam, with_gap=False)
        ctx.save_for_backward(alpha, B, C)
        ctx.state = st
        ctx.lam = lam
        ctx.prec = prec
        return F.sum()

    @staticmethod
    def backward(ctx, grad_out):
        alpha, B, C = ctx.saved_tensors
        da = slista_grad(B, C, ctx.lam, alpha, ctx.state, prec=ctx.prec)
        return (da * grad_out.to(da.dtype)), None, None, None, None, None, None


def slista_loss(alpha, g: Gram, lam, ckpt_every=None, prec="fp32"):
    return SlistaLoss.apply(alpha, g.B, g.C, g.xsq, lam, ckpt_every, prec)


def train_step_sizes(alpha0: torch.Tensor, g: Gram, lam: float, steps: int = 50, lr0: Optional[float] = None,
                     grow: float = 1.2, max_halvings: int = 20, min_alpha: float = 1e-6, prec="fp32",
                     group=None, loss_fn=None):
    """Full-batch sub-gradient descent with backtracking on the step sizes
    (Appendix E).  A trial step alpha - lr * dalpha is accepted when the loss
    does not increase; otherwise lr is halved (at most max_halvings times).
    After an accepted step lr grows by `grow`.  Steps stay >= min_alpha.
    prec: precision of the forward and of the adjoint ("fp32", "bf16x3",
    "bf16").  Returns (alpha, history of losses).

    group: a torch.distributed process group whose ranks each hold their own
    samples (their own g): the loss of every trial and the gradient of every
    accepted step are summed over the ranks (an all-reduce of 1 and of T
    values), so every rank takes the same decisions and ends with the same
    steps - data-parallel training of the loss over all the ranks' samples.
    loss_fn(alpha) -> scalar loss, differentiable in alpha, replaces the
    Step-LISTA loss on g (default)."""
    if loss_fn is None:
        def loss_fn(a):
            return slista_loss(a, g, lam, prec=prec)
    if group is not None:
        import torch.distributed as dist

    def total(v: torch.Tensor) -> torch.Tensor:
        """v summed over the ranks of group (float64)."""
        v = v.detach().double().clone()
        if group is not None:
            dist.all_reduce(v, group=group)
        return v

    alpha = alpha0.detach().clone()
    hist = []
    a = alpha.clone().requires_grad_(True)
    loss = loss_fn(a)
    loss.backward()
    cur = float(total(loss.reshape(1)))
    grad = total(a.grad).to(alpha.dtype)
    hist.append(cur)
    if lr0 is None:
        gmax = float(grad.abs().max())
        lr0 = 0.1 * float(alpha.abs().max()) / gmax if gmax > 0 else 0.0
    lr = lr0
    for _ in range(steps):
        accepted = False
        for _h in range(max_halvings):
            trial = torch.clamp(alpha - lr * grad, min=min_alpha)
            t = trial.clone().requires_grad_(True)
            tl = loss_fn(t)
            tv = float(total(tl.reshape(1)))
            if tv <= cur:
                tl.backward()
                alpha, cur, grad = trial, tv, total(t.grad).to(alpha.dtype)
                lr *= grow
                accepted = True
                break
            lr *= 0.5
        hist.append(cur)
        if not accepted:
            break
    return alpha, hist
