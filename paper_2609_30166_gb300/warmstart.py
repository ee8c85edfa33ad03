"""Learned warm start vs plain SIRT on the sparse-view workload (128^3
textured phantoms, 60 views, 192^2 detector): trains the U-Net on
(5-iteration SIRT, phantom) pairs made by the library, then measures wall time
and iterations to relative data residual 1e-3 on held-out phantoms.

    python -m paper_2609_30166_gb300.warmstart [--steps 1200] [--train 56] [--test 8]
prints one JSON object.
"""

from __future__ import annotations

import argparse
import json
import statistics
import time

import torch

from . import ctrex, inputs, unet


def run(n_train=56, n_test=8, steps=1200, batch=2, tol=1e-3, max_iter=4000, seed=0, log=None):
    cfg = inputs.SPARSE_128
    ctx = ctrex.context_for(cfg)
    t0 = time.perf_counter()
    x_tr, y_tr, _ = unet.make_pairs(cfg, range(0, n_train), ctx)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    model = unet.UNet3D(seed=seed).cuda()
    t0 = time.perf_counter()
    losses = unet.train(model, x_tr, y_tr, steps=steps, batch=batch, seed=seed, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x_tr, y_tr
    rows = unet.compare_warm_start(model, cfg, ctx, range(56, 56 + n_test), tol=tol, max_iter=max_iter)
    mean = lambda k: statistics.mean(r[k] for r in rows)  # noqa: E731
    return {
        "workload": cfg.name, "tol": tol, "train_phantoms": n_train, "test_phantoms": n_test,
        "train_steps": steps, "batch": batch, "data_s": t_data, "train_s": t_train,
        "loss_first": statistics.mean(losses[:10]), "loss_last": statistics.mean(losses[-10:]),
        "plain_s": mean("plain_s"), "warm_s": mean("warm_s"),
        "plain_iters": mean("plain_iters"), "warm_iters": mean("warm_iters"),
        "sirt_in_err": mean("sirt_in_err"), "net_err": mean("net_err"),
        "warm_over_plain_time": mean("warm_s") / mean("plain_s"),
        "per_phantom": rows,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1200)
    ap.add_argument("--train", type=int, default=56)
    ap.add_argument("--test", type=int, default=8)
    a = ap.parse_args()
    print(json.dumps(run(a.train, a.test, a.steps)))


if __name__ == "__main__":
    main()
