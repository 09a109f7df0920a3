"""Learned warm start: training pairs from the solver, training, and use.

Orchestration only -- every step runs in the library's kernels through the C
ABI (gf.py).  A training pair for one field U:

1. FP32 12-real overrelaxation of U with gauge tracking until theta < switch
   (the FP32 phase of the mixed policy);
2. the FP64 field g U g^dagger at the switch; s = sqrt(theta) there;
   inputs = gf_features(s) (BF16 [V][80]);
3. FP64 overrelaxation to theta < label_theta with a fresh tracked g;
   label = gf_gauge_algebra(s): the algebra coefficients of the remaining
   transformation divided by s (FP32 [V][8]).

The network learns the remaining transformation from the field at the switch;
at inference the mixed policy applies its prediction at the switch and plain
overrelaxation finishes (gf_set_net).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gf

OMEGA = 1.7


def make_pair(ctx, U, theta_switch=1e-6, label_theta=1e-12, max_iter=200_000, check_every=25):
    """(features BF16 [V][80], labels FP32 [V][8], s) for field U (device tensor)."""
    V = ctx.volume
    dev = U.device
    gf.gf_set_option(ctx, "check_every", check_every)
    gf.gf_set_option(ctx, "track", 1)
    gf.gf_upload(ctx, U, gf.GF_FP32)
    gf.gf_gauge_reset(ctx)
    gf.gf_converge(ctx, OMEGA, theta_switch, max_iter)
    gf.gf_apply_tracked_gauge(ctx, U)
    _, th = gf.gf_measure(ctx)
    s = math.sqrt(th)
    feats = torch.empty(V, gf.GF_NET_CIN, dtype=torch.bfloat16, device=dev)
    gf.gf_features(ctx, s, feats)
    gf.gf_gauge_reset(ctx)
    gf.gf_converge(ctx, OMEGA, label_theta, max_iter)
    labels = torch.empty(V, gf.GF_NET_COUT, dtype=torch.float32, device=dev)
    gf.gf_gauge_algebra(ctx, s, labels)
    gf.gf_set_option(ctx, "track", 0)
    torch.cuda.synchronize()
    return feats, labels, s


def init_params(seed: int = 0, scale_last: float = 0.1) -> np.ndarray:
    """He-initialised parameters (flat FP32, the library's layout)."""
    rng = np.random.default_rng(seed)
    ch = gf.NET_CHANNELS
    parts = []
    for l in range(4):
        fan_in = 81 * ch[l]
        std = math.sqrt(2.0 / fan_in) * (scale_last if l == 3 else 1.0)
        parts.append(rng.standard_normal(81 * ch[l + 1] * ch[l]) * std)
        parts.append(np.zeros(ch[l + 1]))
    return np.concatenate(parts).astype(np.float32)


def train(net, pairs, epochs: int, lr: float = 1e-3, lr_decay: float = 1.0, log=None):
    """Adam over the pairs (each a (features, labels, s) tuple); returns loss history."""
    hist = []
    for ep in range(epochs):
        tot = 0.0
        for feats, labels, _ in pairs:
            tot += gf.gf_net_train_step(net, feats, labels, lr)
        hist.append(tot / max(1, len(pairs)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
        lr *= lr_decay
    return hist


def validation_loss(net, pairs) -> float:
    tot = 0.0
    for feats, labels, _ in pairs:
        tot += gf.gf_net_gradient(net, feats, labels)
    return tot / max(1, len(pairs))
