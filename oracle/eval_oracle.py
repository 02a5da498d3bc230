"""CPU oracle of the evaluation of Sect. VIII -- TEST INFRASTRUCTURE ONLY.

Plain numpy, written from the paper's equations, one function per quantity:

  cluster_stats      Eq. mean_cluster (mean of the cells' mean velocities over a cluster S)
                     and Eq. gaussian_mixture_x (variance of the Gaussian mixture of the
                     cells), summed in binary64
  nees               Eq. NEES_x, (cluster mean - true velocity)^2 / cluster variance
  mahalanobis0       Eq. mahadist, m = v P^-1 v^T from v = 0; computed in binary32 with the
                     operation order the kernel uses, because m decides an integer (the
                     static/dynamic class at each threshold), and pinned by the tests
                     against the binary64 definition
  classify_counts    the number of cells detected dynamic (m >= threshold) per class

Only tests/ and bench.py's CPU legs use this module.
"""
from __future__ import annotations

import numpy as np


def cluster_stats(cells: dict, cell_object: np.ndarray, n_objects: int) -> np.ndarray:
    """[n_objects, 5]: |S|, mean vx, mean vy, var vx, var vy of each object's cells."""
    out = np.zeros((n_objects, 5))
    mx = cells["mean_vx"].astype(np.float64)
    my = cells["mean_vy"].astype(np.float64)
    vx = cells["var_vx"].astype(np.float64)
    vy = cells["var_vy"].astype(np.float64)
    for k in range(1, n_objects + 1):
        S = np.flatnonzero(cell_object == k)
        n = S.size
        out[k - 1, 0] = n
        if n == 0:
            continue
        cx = mx[S].sum() / n                      # Eq. mean_cluster
        cy = my[S].sum() / n
        out[k - 1, 1] = cx
        out[k - 1, 2] = cy
        out[k - 1, 3] = (vx[S] + mx[S] ** 2).sum() / n - cx ** 2   # Eq. gaussian_mixture_x
        out[k - 1, 4] = (vy[S] + my[S] ** 2).sum() / n - cy ** 2
    return out


def nees(mean: float, var: float, truth: float) -> float:
    """Eq. NEES_x."""
    return (mean - truth) ** 2 / var if var > 0 else float("inf")


def mahalanobis0(mean_vx, mean_vy, var_vx, var_vy, cov_vxy) -> np.ndarray:
    """Eq. mahadist in binary32, (var_y vx^2 - 2 cov vx vy + var_x vy^2) / det P with
    det P = var_x var_y - cov^2, every operation rounded; a singular P gives 0 for v = 0
    and +inf otherwise."""
    f = np.float32
    vx, vy = np.asarray(mean_vx, f), np.asarray(mean_vy, f)
    sx, sy, cv = np.asarray(var_vx, f), np.asarray(var_vy, f), np.asarray(cov_vxy, f)
    a, b, c = vx * vx, vy * vy, vx * vy
    t2 = cv * c
    num = (sy * a - (t2 + t2)) + sx * b
    det = sx * sy - cv * cv
    with np.errstate(divide="ignore", invalid="ignore"):
        zero_v = (vx == 0) & (vy == 0)
        m = np.where(det > 0, num / np.where(det > 0, det, f(1)), np.where(zero_v, f(0), f(np.inf)))
    return m.astype(f)


def classify_counts(m: np.ndarray, label: np.ndarray, m_occ: np.ndarray, min_occ: float,
                    thresholds: np.ndarray) -> np.ndarray:
    """[2, n_thresholds]: cells detected dynamic (m >= t) among label 1 (dynamic) and label 2
    (static) cells with m_occ >= min_occ."""
    sel = m_occ >= np.float32(min_occ)
    out = np.zeros((2, len(thresholds)), np.int64)
    for li in (1, 2):
        mm = m[sel & (label == li)]
        for j, t in enumerate(thresholds):
            out[li - 1, j] = int((mm >= np.float32(t)).sum())
    return out
