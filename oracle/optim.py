"""FP64 CPU oracle of the training update over the model's parameters (test
infrastructure).

This file is test infrastructure: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path
never calls it, and it imports nothing from the product package.

What it computes.  HelixFold's tensor fusion (Sec. 3.2, Fig. "Tensor Fusion"
and the table of kernel launches per stage) keeps the parameters, gradients
and Adam moments of the whole model in a few large buffers, so that the
stages after the backward -- gradient clipping by global norm, the Adam
update and the exponential moving average (EMA) of the parameters -- each
take O(1) launches instead of one or two per tensor.  Fusion changes the
launch count, not the arithmetic: the result is the same as running each
stage tensor by tensor.  This oracle is that unfused form, one named tensor at
a time, in the order the paper lists the stages:

  1. global gradient norm  G = sqrt(sum over all tensors of sum g^2);
  2. clip by global norm:  g <- g * c / max(G, c)  for a threshold c > 0
     (c <= 0: no clipping);
  3. Adam (Kingma and Ba 2015, Algorithm 1) at step t = 1, 2, ...:
     m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
     w <- w - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  4. EMA of the updated parameters:  e <- d e + (1 - d) w.

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository):
  * the clip factor is c / max(G, c) (1 when G <= c), the form of the
    PaddlePaddle global-norm clip the paper's system uses;
  * eps is added to the square root of the bias-corrected second moment, not
    inside the root; no weight decay;
  * the EMA follows the parameter update and averages the updated values;
  * default hyper-parameters are AlphaFold2's training settings (Jumper et
    al. 2021, supplement 1.11.3): lr 1e-3, b1 0.9, b2 0.999, eps 1e-6, clip
    0.1, EMA decay 0.999.

Parity pins (tests/test_oracle_optim.py): torch.optim.Adam over several steps,
the closed form of Adam under a constant gradient, the clipped norm equal to
the threshold, the EMA closed form with a frozen parameter, and the order of
the EMA after the update.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

DT = torch.float64


@dataclass(frozen=True)
class AdamHyper:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-6
    clip_norm: float = 0.1
    ema_decay: float = 0.999


def _t(x):
    return torch.as_tensor(np.asarray(x)).to(DT) if not isinstance(x, torch.Tensor) else x.to(DT)


def global_norm(grads: dict) -> float:
    """Stage 1: the L2 norm of all gradients together."""
    return math.sqrt(sum(float((_t(g) ** 2).sum()) for g in grads.values()))


def clip_by_global_norm(grads: dict, clip_norm: float):
    """Stage 2: every gradient scaled by c / max(G, c); returns (grads, G)."""
    G = global_norm(grads)
    if clip_norm <= 0:
        return {k: _t(g) for k, g in grads.items()}, G
    s = clip_norm / max(G, clip_norm)
    return {k: _t(g) * s for k, g in grads.items()}, G


def adam_update(w, g, m, v, step: int, h: AdamHyper):
    """Stage 3 for one tensor: returns (w, m, v) after step number `step` (>= 1)."""
    w, g, m, v = _t(w), _t(g), _t(m), _t(v)
    m = h.beta1 * m + (1.0 - h.beta1) * g
    v = h.beta2 * v + (1.0 - h.beta2) * g * g
    m_hat = m / (1.0 - h.beta1 ** step)
    v_hat = v / (1.0 - h.beta2 ** step)
    w = w - h.lr * m_hat / (torch.sqrt(v_hat) + h.eps)
    return w, m, v


def ema_update(e, w, decay: float):
    """Stage 4 for one tensor: the moving average moves towards w."""
    return decay * _t(e) + (1.0 - decay) * _t(w)


def train_update(params: dict, grads: dict, exp_avg: dict, exp_avg_sq: dict, ema: dict | None, step: int,
                 h: AdamHyper = AdamHyper()):
    """The four stages over named tensors, each tensor on its own.

    Returns (params, exp_avg, exp_avg_sq, ema, G) as FP64 tensors; ema is None
    when not given.  G is the global norm before clipping."""
    if step < 1:
        raise ValueError("Adam steps count from 1")
    g_clip, G = clip_by_global_norm(grads, h.clip_norm)
    P, M, V, E = {}, {}, {}, ({} if ema is not None else None)
    for k in params:
        P[k], M[k], V[k] = adam_update(params[k], g_clip[k], exp_avg[k], exp_avg_sq[k], step, h)
        if ema is not None:
            E[k] = ema_update(ema[k], P[k], h.ema_decay)
    return P, M, V, E, G
