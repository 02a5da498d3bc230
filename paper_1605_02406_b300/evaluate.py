"""Evaluation of the filter against synthetic ground truth (the experiments of Sect. VIII).

For every frame of a seeded scene, the ground truth of scene.label_cells (which cells
belong to which object, which objects move, their true velocities) is compared with the
filter's cell estimates through the library's evaluation calls:

  * velocity of each object's cell cluster S: mean (Eq. mean_cluster) and variance of the
    Gaussian mixture of its cells (Eq. gaussian_mixture_x), and the normalised estimation
    error squared against the true velocity (Eq. NEES_x), x and y;
  * classification of occupied object cells into static and dynamic by the Mahalanobis
    distance of their velocity estimate from v = 0 (Eq. mahadist), over a sweep of
    thresholds: the ROC curve (true-positive rate over dynamic cells, false-positive rate
    over static cells).

    python -m paper_1605_02406_b300.evaluate --workload plain_128 --frames 40
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import native as N
from . import scene
from .filter import DogFilter

CHI2_1_95 = 3.841458820694124  # 95 % quantile of chi-square with one degree of freedom


class Evaluator:
    """Device buffers for the evaluation calls of one filter."""

    def __init__(self, f: DogFilter, n_objects: int, thresholds):
        self.f = f
        self.n_objects = max(1, int(n_objects))
        dev = f.device
        self.thr = torch.tensor(np.sort(np.asarray(thresholds, np.float32)), device=dev)
        self.scratch = torch.zeros(self.n_objects * 5, dtype=torch.int64, device=dev)
        self.stats = torch.zeros(self.n_objects * 5, dtype=torch.float64, device=dev)
        self.counts = torch.zeros(2 * (len(self.thr) + 1), dtype=torch.int64, device=dev)
        self.m = torch.zeros(f.C, dtype=torch.float32, device=dev)
        f.stream.wait_stream(torch.cuda.current_stream(dev))

    def clusters(self, cell_object) -> np.ndarray:
        """[n_objects, 5]: |S|, mean vx, mean vy, var vx, var vy."""
        obj = torch.as_tensor(np.asarray(cell_object, np.int32), device=self.f.device)
        self.f.stream.wait_stream(torch.cuda.current_stream(self.f.device))  # the upload
        N.dog_eval_clusters(self.f.h, obj.data_ptr(), self.n_objects, self.scratch.data_ptr(),
                            self.stats.data_ptr())
        self.f.sync()
        return self.stats.view(self.n_objects, 5).cpu().numpy()

    def classification(self, label, min_occ: float = 0.5):
        """(histogram [2, n_thresholds + 1], m [C]) -- see dog_eval_mahalanobis."""
        lab = torch.as_tensor(np.asarray(label, np.uint8), device=self.f.device)
        self.f.stream.wait_stream(torch.cuda.current_stream(self.f.device))  # the upload
        N.dog_eval_mahalanobis(self.f.h, lab.data_ptr(), min_occ, self.thr.data_ptr(), len(self.thr),
                               self.counts.data_ptr(), self.m.data_ptr())
        self.f.sync()
        return self.counts.view(2, -1).cpu().numpy(), self.m.cpu().numpy()


def detections(hist: np.ndarray) -> np.ndarray:
    """[2, n_thresholds]: cells detected dynamic at each threshold (m >= t_j), per class,
    from the histogram over the number of thresholds <= m."""
    return np.cumsum(hist[:, ::-1], axis=1)[:, ::-1][:, 1:]


def run(cfg: dict, frames: int, seed: int = 1001, thresholds=None, min_occ: float = 0.5,
        warmup: int = 10, **params_over) -> dict:
    """Run the filter over a scene and evaluate every frame after `warmup`."""
    if thresholds is None:
        thresholds = np.concatenate([[0.0], np.logspace(-2, 3, 41)])
    params = scene.filter_params(cfg, **params_over)
    seq = scene.frame_sequence_with_truth(cfg, frames, seed)
    f = DogFilter(params)
    n_obj = len(seq[0][1]["velocity"])
    ev = Evaluator(f, n_obj, thresholds)
    moving = [k for k in range(n_obj) if np.any(seq[0][1]["velocity"][k] != 0)]
    nees_x, nees_y, err = [], [], []
    tp = np.zeros(len(thresholds), np.int64)
    fp = np.zeros(len(thresholds), np.int64)
    n_dyn = n_stat = 0
    for t, (grid, truth) in enumerate(seq):
        f.set_measurement_grid(**grid)
        f.step(cfg["dt"])
        if t < warmup:
            continue
        st = ev.clusters(truth["object"])
        for k in moving:
            n, mx, my, vx, vy = st[k]
            if n < 3:
                continue
            tx, ty = truth["velocity"][k]
            nees_x.append((mx - tx) ** 2 / vx if vx > 0 else np.inf)
            nees_y.append((my - ty) ** 2 / vy if vy > 0 else np.inf)
            err.append(float(np.hypot(mx - tx, my - ty)))
        hist, _ = ev.classification(truth["dynamic"], min_occ)
        det = detections(hist)
        tp += det[0]
        fp += det[1]
        n_dyn += int(hist[0].sum())
        n_stat += int(hist[1].sum())
    f.close()
    tpr = tp / max(n_dyn, 1)
    fpr = fp / max(n_stat, 1)
    order = np.argsort(fpr)
    auc = float(np.trapezoid(np.concatenate([[0.0], tpr[order], [1.0]]),
                             np.concatenate([[0.0], fpr[order], [1.0]])))
    nx, ny = np.asarray(nees_x), np.asarray(nees_y)
    return {
        "workload": cfg["name"], "frames": frames, "warmup": warmup, "p_B": params["p_B"],
        "moving_objects": len(moving),
        "velocity_error_mean": float(np.mean(err)) if err else None,
        "nees_x_mean": float(np.mean(nx[np.isfinite(nx)])) if nx.size else None,
        "nees_within_95pct": float(np.mean(np.concatenate([nx, ny]) <= CHI2_1_95)) if nx.size else None,
        "roc": {"thresholds": [float(x) for x in np.sort(np.asarray(thresholds, np.float32))],
                "tpr": [float(x) for x in tpr], "fpr": [float(x) for x in fpr],
                "dynamic_cells": n_dyn, "static_cells": n_stat, "auc": auc},
    }


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="plain_128", choices=sorted(scene.CONFIGS))
    ap.add_argument("--frames", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--p-B", type=float, default=None)
    args = ap.parse_args()
    over = {} if args.p_B is None else {"p_B": args.p_B}
    out = run(scene.CONFIGS[args.workload], args.frames, warmup=args.warmup, **over)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
