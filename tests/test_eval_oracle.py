"""CPU pins of the evaluation oracle (oracle/eval_oracle.py, the experiments of Sect. VIII)
against hand computations and the binary64 definitions."""
import numpy as np

from oracle import eval_oracle as E


def _cells(mx, my, vx, vy, cov=None):
    n = len(mx)
    f = lambda a: np.asarray(a, np.float32)
    return dict(mean_vx=f(mx), mean_vy=f(my), var_vx=f(vx), var_vy=f(vy),
                cov_vxy=f(cov if cov is not None else np.zeros(n)))


def test_cluster_mixture_by_hand():
    # two cells of object 1: N(1, 0.5) and N(3, 1.5) -> mixture mean 2, variance
    # (0.5 + 1 + 1.5 + 9) / 2 - 4 = 2; object 2 one cell; cell 3 in no object
    c = _cells([1.0, 3.0, -2.0, 7.0], [0.0, 0.0, 4.0, 7.0], [0.5, 1.5, 0.25, 9.0], [1.0, 1.0, 0.5, 9.0])
    st = E.cluster_stats(c, np.array([1, 1, 2, 0]), 3)
    assert np.allclose(st[0], [2, 2.0, 0.0, 2.0, 1.0])
    assert np.allclose(st[1], [1, -2.0, 4.0, 0.25, 0.5])
    assert np.allclose(st[2], [0, 0, 0, 0, 0])


def test_cluster_variance_is_variance_of_pooled_samples():
    # equal-size samples per cell: the mixture variance equals the variance of the pooled samples
    rng = np.random.default_rng(0)
    samples = [rng.normal(rng.uniform(-5, 5), rng.uniform(0.1, 2), 4000) for _ in range(6)]
    c = _cells([s.mean() for s in samples], [0.0] * 6, [s.var() for s in samples], [0.0] * 6)
    st = E.cluster_stats(c, np.ones(6, np.int64), 1)
    pooled = np.concatenate(samples)
    assert abs(st[0, 1] - pooled.mean()) < 1e-5
    assert abs(st[0, 3] - pooled.var()) < 1e-4 * pooled.var()


def test_nees():
    assert E.nees(2.0, 4.0, 1.0) == 0.25
    assert E.nees(1.0, 0.0, 0.0) == float("inf")


def test_mahalanobis_matches_binary64_definition():
    rng = np.random.default_rng(1)
    n = 20000
    mx, my = rng.normal(0, 3, n), rng.normal(0, 3, n)
    a, b, r = rng.uniform(0.05, 4, n), rng.uniform(0.05, 4, n), rng.uniform(-0.95, 0.95, n)
    vx, vy = a * a, b * b
    cv = r * a * b
    m32 = E.mahalanobis0(mx, my, vx, vy, cv)
    # binary64 definition on the same binary32 inputs: v P^-1 v^T by a linear solve
    f = lambda x: np.asarray(x, np.float32).astype(np.float64)
    P = np.stack([np.stack([f(vx), f(cv)], -1), np.stack([f(cv), f(vy)], -1)], -2)
    v = np.stack([f(mx), f(my)], -1)
    m64 = np.einsum("ni,ni->n", v, np.linalg.solve(P, v[..., None])[..., 0])
    cond = (f(vx) * f(vy)) / (f(vx) * f(vy) - f(cv) ** 2)  # relative error grows with the conditioning
    assert np.all(np.abs(m32 - m64) <= 1e-5 * cond * (1 + np.abs(m64)))


def test_mahalanobis_special_cases():
    # diagonal P: m = vx^2 / var_x + vy^2 / var_y; singular P: 0 at v = 0, inf otherwise
    m = E.mahalanobis0([3.0, 0.0, 1.0, 0.0], [4.0, 0.0, 0.0, 0.0], [9.0, 0.0, 0.0, 1.0],
                       [16.0, 0.0, 0.0, 1.0], [0.0, 0.0, 0.0, 1.0])
    assert m[0] == np.float32(2.0)
    assert m[1] == 0.0 and m[2] == np.inf and m[3] == 0.0


def test_classify_counts_monotone():
    rng = np.random.default_rng(2)
    m = rng.exponential(5, 5000).astype(np.float32)
    lab = rng.integers(0, 3, 5000).astype(np.uint8)
    occ = rng.uniform(0, 1, 5000).astype(np.float32)
    thr = np.array([0, 0.5, 1, 5, 50], np.float32)
    c = E.classify_counts(m, lab, occ, 0.5, thr)
    assert np.all(np.diff(c, axis=1) <= 0)
    assert c[0, 0] == ((lab == 1) & (occ >= 0.5)).sum()  # every cell has m >= 0
