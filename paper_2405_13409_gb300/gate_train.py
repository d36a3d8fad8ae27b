"""Training recipe of the learned gate, on top of the C ABI.

Labels come from the plain FP64 solve (a chain is positive when its solve
returns a path); features and training run in the library's kernels.  The
threshold is calibrated on held-out scenes for a target recall of positive
chains.  Host orchestration only: every step runs on the GPU.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding


def _device_inputs(torch, s):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]


def labelled_features(ctx, torch, scene, mode, camera=None):
    """Candidates of `scene` (built with `mode`), their features [n, 24] and
    labels [n] (device tensors), from one plain FP64 solve without a pixel
    filter."""
    d = _device_inputs(torch, scene)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, mode, camera=camera)
    try:
        n = ctx.spoly_chains_count(ch)
        feat = torch.empty((n, binding.MLP_FEATURES), dtype=torch.float32, device="cuda")
        labels = torch.zeros(n, dtype=torch.uint8, device="cuda")
        if n:
            ctx.spoly_mlp_features(mesh, q, ch, feat)
            sol = ctx.spoly_solve(mesh, q, ch, precision=binding.PLAIN_FP64)
            try:
                ctx.spoly_chain_labels(sol, n, labels)
            finally:
                ctx.spoly_solution_free(sol)
    finally:
        ctx.spoly_chains_free(ch)
    return feat, labels


def train_gate(ctx, torch, train_scenes, val_scenes, mode, camera=None, target_recall=1.0, margin=1.0, steps=3000,
               batch=8192, lr=3e-3, lr_final=1e-4, pos_fraction=0.25, seed=0):
    """Trains a gate network on `train_scenes` and calibrates its threshold
    on `val_scenes`: the largest logit that keeps target_recall of the
    validation positives, lowered by `margin` (logit units) against the
    spread of the calibration statistic.  Returns (mlp handle, tau_logit,
    info dict)."""
    t0 = time.perf_counter()
    parts = [labelled_features(ctx, torch, s, mode, camera) for s in train_scenes]
    feat = torch.cat([p[0] for p in parts])
    labels = torch.cat([p[1] for p in parts])
    del parts
    t1 = time.perf_counter()
    mlp = ctx.spoly_mlp_create(seed=seed)
    loss = ctx.spoly_mlp_train(mlp, feat, labels, steps=steps, batch=batch, lr=lr, lr_final=lr_final,
                               pos_fraction=pos_fraction, seed=seed)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    n_train, n_pos = int(labels.numel()), int(labels.sum().item())
    del feat, labels
    vparts = [labelled_features(ctx, torch, s, mode, camera) for s in val_scenes]
    vf = torch.cat([p[0] for p in vparts])
    vl = torch.cat([p[1] for p in vparts])
    tau_cal, _ = ctx.spoly_mlp_calibrate(mlp, vf, vl, target_recall)
    tau = tau_cal - margin
    z = torch.empty(vf.shape[0], dtype=torch.float32, device="cuda")
    ctx.spoly_mlp_forward(mlp, vf, z)
    pass_frac = float((z >= tau).float().mean().item())
    info = {"train_rows": n_train, "train_positive": n_pos, "final_loss": loss, "val_rows": int(vl.numel()),
            "val_positive": int(vl.sum().item()), "val_pass_fraction": pass_frac, "tau_logit": tau,
            "tau_calibrated": tau_cal, "margin": margin, "target_recall": target_recall,
            "label_s": t1 - t0, "train_s": t2 - t1, "steps": steps, "batch": batch}
    return mlp, tau, info
