"""Fitting a triangle mesh to a reference measure by gradient descent on D.

D(verts) = sum_k W_k |mu^(xi_k) - nu^(xi_k)|^2 is the truncated squared
H^{-s} distance between the mesh's surface measure mu and nu (by default the
unit sphere), W_k = w_k (1 + |xi_k|^2)^{-s}. Each step evaluates D and
dD/dverts in the library's forward and adjoint kernels, through the
torch.autograd.Function in `autograd`, and moves every vertex against the
gradient with a fixed step: v <- v - lr * dD/dv.

The step defaults to 1/L, L the largest eigenvalue of the Hessian of D at the
starting mesh, estimated by power iteration on central-difference
Hessian-vector products of the adjoint gradient; gradient descent on a
function whose Hessian stays below L decreases it for any step below 2/L.

The only state of the loop is the step count and the vertices (plus the
history of D for reporting). A checkpoint file (torch.save of a dict) holds
them; a later call with the same checkpoint path resumes from it and, since
the library's distance and gradient are bitwise reproducible, continues along
exactly the trajectory an uninterrupted run takes.
"""
from __future__ import annotations

import os
import zlib
from dataclasses import dataclass, field
from typing import Callable, Optional

import torch

from . import WD_MIXED, wd_rule_info
from .autograd import weak_distance

ValueAndGrad = Callable[[torch.Tensor], "tuple[float, torch.Tensor]"]


@dataclass
class FitResult:
    verts: torch.Tensor          # vertices after `step` steps
    step: int                    # number of steps taken in total
    lr: float                    # step size used
    history: list = field(default_factory=list)  # D at steps 0..step
    resumed_from: int = 0        # step the last call started from


def hessian_max_eig(value_and_grad: ValueAndGrad, v0: torch.Tensor, iters: int = 8, eps: float = 1e-4,
                    seed: int = 0) -> float:
    """Largest Hessian eigenvalue of D at v0: power iteration with
    Hv ~ (g(v0 + eps u) - g(v0 - eps u)) / (2 eps), u a unit vector, started
    from a seeded Gaussian direction; returns the last Rayleigh quotient."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    u = torch.randn(v0.shape, generator=gen, dtype=torch.float64).to(v0.device)
    u /= u.norm()
    lam = 0.0
    for _ in range(iters):
        _, gp = value_and_grad(v0 + eps * u)
        _, gm = value_and_grad(v0 - eps * u)
        hv = (gp - gm) / (2.0 * eps)
        lam = float(torch.dot(u.flatten(), hv.flatten()))
        nrm = hv.norm()
        if not torch.isfinite(nrm) or nrm == 0:
            break
        u = hv / nrm
    return lam


def _save(path: str, state: dict) -> None:
    tmp = path + ".tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)  # atomic: a crash leaves the previous checkpoint intact


def gradient_descent(value_and_grad: ValueAndGrad, v0: torch.Tensor, steps: int, lr: float,
                     checkpoint: Optional[str] = None, checkpoint_every: int = 10,
                     meta: Optional[dict] = None, callback=None) -> FitResult:
    """`steps` total steps of v <- v - lr g(v) from v0.

    With `checkpoint`, the state is saved every `checkpoint_every` steps and at
    the end; if the file already exists the loop resumes from it instead of v0
    (its `meta` and `lr` must equal the ones given, else ValueError). `steps`
    counts from the start of the whole run, so a resumed call with the same
    arguments finishes the same run.
    """
    if steps < 0:
        raise ValueError("steps must be >= 0")
    if not (lr > 0.0) or lr != lr or lr == float("inf"):
        raise ValueError("lr must be finite and > 0")
    meta = dict(meta or {})
    v = v0.detach().clone()
    step, history = 0, []
    if checkpoint is not None and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location="cpu", weights_only=False)
        if st.get("meta") != meta:
            raise ValueError("checkpoint %s belongs to another problem: %r != %r" % (checkpoint, st.get("meta"), meta))
        if st.get("lr") != lr:
            raise ValueError("checkpoint %s was written with lr=%r, not %r" % (checkpoint, st.get("lr"), lr))
        if tuple(st["verts"].shape) != tuple(v0.shape):
            raise ValueError("checkpoint %s has vertices of shape %s" % (checkpoint, tuple(st["verts"].shape)))
        step = int(st["step"])
        if step > steps:
            raise ValueError("checkpoint %s is at step %d, past the requested %d" % (checkpoint, step, steps))
        v = st["verts"].to(device=v0.device, dtype=v0.dtype)
        history = list(st["history"])
    start = step

    def state():
        return {"step": step, "verts": v.detach().cpu(), "history": list(history), "lr": lr, "meta": meta}

    while step < steps:
        d, g = value_and_grad(v)
        if len(history) == step:
            history.append(float(d))
        v = v - lr * g
        step += 1
        if callback is not None:
            callback(step, history[-1])
        if checkpoint is not None and checkpoint_every > 0 and step % checkpoint_every == 0:
            _save(checkpoint, state())
    if len(history) == step:
        d, _ = value_and_grad(v)
        history.append(float(d))
    if checkpoint is not None:
        _save(checkpoint, state())
    return FitResult(verts=v, step=step, lr=lr, history=history, resumed_from=start)


def distance_value_and_grad(ctx, rule, tris: torch.Tensor, s: float = 1.0, precision: int = WD_MIXED,
                            nu=None) -> ValueAndGrad:
    """Closure v -> (D(v), dD/dv) through the autograd Function (forward and
    adjoint in the library's kernels)."""
    t = tris.to(torch.int32).contiguous()

    def f(v: torch.Tensor):
        x = v.detach().clone().requires_grad_(True)
        D = weak_distance(ctx, rule, x, t, s, precision, nu)
        D.backward()
        return float(D.detach()), x.grad

    return f


def fit_mesh(ctx, rule, verts: torch.Tensor, tris: torch.Tensor, steps: int = 200, s: float = 1.0,
             precision: int = WD_MIXED, nu=None, lr: Optional[float] = None, lr_scale: float = 1.0,
             checkpoint: Optional[str] = None, checkpoint_every: int = 10, callback=None) -> FitResult:
    """Gradient descent of the mesh (verts: (V, 3) float64 CUDA tensor, tris:
    (T, 3) int tensor on the same device) toward nu (None: the unit sphere).
    lr None: lr_scale / L with L from `hessian_max_eig` at the starting mesh,
    or, when resuming, the step stored in the checkpoint."""
    f = distance_value_and_grad(ctx, rule, tris, s, precision, nu)
    if lr is None and checkpoint is not None and os.path.exists(checkpoint):
        lr = torch.load(checkpoint, map_location="cpu", weights_only=False)["lr"]
    if lr is None:
        lr = lr_scale / hessian_max_eig(f, verts.detach())
    n_eval, n_total = wd_rule_info(rule)
    tb = tris.detach().to(torch.int32).cpu().contiguous().numpy().tobytes()
    meta = {"n_eval": int(n_eval), "n_total": int(n_total), "s": float(s), "precision": int(precision),
            "n_verts": int(verts.shape[0]), "n_tris": int(tris.shape[0]), "tris_crc32": zlib.crc32(tb),
            "nu": repr(nu)}
    return gradient_descent(f, verts, steps, lr, checkpoint, checkpoint_every, meta, callback)
