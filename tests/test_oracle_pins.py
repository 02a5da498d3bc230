"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU needed).

Each test pins one part of the oracle to something other than itself:
  * Philox4x32-10 against the published known-answer vectors,
  * the FP32 mirror's ln / sin / cos / exp against libm,
  * Box-Muller draws against N(0, 1) (moments and a KS test),
  * the per-cell update against brute-force Dempster combination over the power set,
  * the newborn/persistent split against the ratio of Eq. DS_relation_masses,
  * the whole recursion against the binary Bayes filter (Prop. in Sect. IV-G: a static
    process model reduces the filter to Eq. BBF_gen),
  * sorting against a stable argsort and cell ranges against brute force,
  * normalised weights against Eq. DSnormalization's sum rule (sum in cell = rho_p),
  * newborn allocation and systematic resampling against their integer floor/ceil bounds,
  * velocity moments against the textbook weighted mean / variance,
  * end-to-end behaviour stated in Sect. VIII (static cells -> zero velocity, a moving
    object's velocity is recovered with a bias toward zero that grows with p_B).
"""
import math
import os

import numpy as np
import pytest

from oracle import OracleFilter, box_muller, cell_update, exp_f32, ln_f32, philox4x32_10, sincos2pi_f32
from paper_1605_02406_b300 import scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NO_RESAMPLE = 0x2
MODES = ["f32", "f64"]


def q40(w):
    """Exact fixed-point quantisation of weights (truncation at 2^-40); float32 and float64
    inputs scale exactly by the power of two."""
    w = np.asarray(w)
    if w.dtype != np.float64:
        w = w.astype(np.float32).astype(np.float64)
    return np.where(w > 0, np.floor(w * 2.0 ** 40), 0).astype(np.uint64)


def small_params(W=16, H=16, nu=4096, nu_b=1024, **kw):
    p = dict(width=W, height=H, cell_size=0.5, nu=nu, nu_b=nu_b, p_S=0.99, p_B=0.02, alpha=0.9,
             sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0, sensor_x=W * 0.25,
             sensor_y=H * 0.25, seed=123, flags=0)
    p.update(kw)
    return p


# ---------------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_ln_f32_against_libm():
    ks = np.unique(np.concatenate([np.arange(1, 4096), np.linspace(1, 2 ** 24, 200001).astype(np.int64)]))
    worst = 0.0
    for k in ks[::7]:
        u = float(np.float32(k * 2.0 ** -24))
        ref = math.log(u)
        err = abs(ln_f32(u) - ref)
        worst = max(worst, err / max(abs(ref) * 2.0 ** -23, 2.0 ** -24))
    assert worst <= 4.0, worst  # within 4 ulp of the true value (or 4 * 2^-24 near 0)


def test_sincos2pi_f32_against_libm():
    ks = np.linspace(0, 2 ** 24 - 1, 100003).astype(np.int64)
    errs = []
    for k in ks[::3]:
        u = k * 2.0 ** -24
        s, c = sincos2pi_f32(u)
        errs.append(max(abs(s - math.sin(2 * math.pi * u)), abs(c - math.cos(2 * math.pi * u))))
    assert max(errs) < 3e-7


def test_exp_f32_against_libm():
    xs = np.concatenate([np.linspace(-86.9, 0.0, 40001), -np.logspace(-8, 1.9, 2000)]).astype(np.float32)
    worst = 0.0
    for x in xs[::3]:
        ref = math.exp(float(x))
        worst = max(worst, abs(exp_f32(float(x)) - ref) / ref)
    assert worst < 5e-7, worst
    assert exp_f32(-90.0) == 0.0


@pytest.mark.parametrize("mode", MODES)
def test_box_muller_is_standard_normal(mode):
    from scipy import stats
    n = []
    for i in range(30000):
        r = philox4x32_10([i, 5, 1, 0], [77, 0])
        n.extend(box_muller(int(r[0]), int(r[1]), mode))
        n.extend(box_muller(int(r[2]), int(r[3]), mode))
    n = np.array(n)
    assert abs(n.mean()) < 0.01
    assert abs(n.var() - 1.0) < 0.015
    assert stats.kstest(n, "norm").pvalue > 1e-3
    # the two outputs of one pair are uncorrelated
    assert abs(np.corrcoef(n[0::2], n[1::2])[0, 1]) < 0.02


# ------------------------------------------------------------------------ cell update
def _fit(a, b):
    """largest float32 b' <= b with a + b' <= 1 (a valid BBA after rounding)"""
    b = np.float32(b)
    while float(a) + float(b) > 1.0:
        b = np.nextafter(b, np.float32(0))
    return float(b)


def _dempster_bruteforce(m, z):
    """Dempster's rule by enumeration of focal-set pairs over 2^{O,F}."""
    O, F = frozenset("O"), frozenset("F")
    T = O | F
    out = {O: 0.0, F: 0.0, T: 0.0}
    K = 0.0
    for A, ma in m.items():
        for B, zb in z.items():
            I = A & B
            if not I:
                K += ma * zb
            else:
                out[I] += ma * zb
    return out[O] / (1 - K), out[F] / (1 - K), K


@pytest.mark.parametrize("mode,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_dempster_against_power_set_enumeration(mode, tol):
    rng = np.random.default_rng(0)
    O, F = frozenset("O"), frozenset("F")
    T = O | F
    for _ in range(3000):
        mO, mF = rng.dirichlet([1, 1, 1])[:2]
        zO, zF = rng.dirichlet([1, 1, 1])[:2]
        if rng.uniform() < 0.2:
            zF, zO = 1 - zO, zO  # Bayesian measurement
        mO, mF, zO, zF = (float(np.float32(v)) for v in (mO, mF, zO, zF))
        mF, zF = _fit(mO, mF), _fit(zO, zF)
        ref_o, ref_f, K = _dempster_bruteforce({O: mO, F: mF, T: 1 - mO - mF},
                                               {O: zO, F: zF, T: 1 - zO - zF})
        if 1 - K < 1e-5:
            continue
        out = cell_update(mO, mF, zO, zF, 1.0, 0.0, mode)
        assert abs(out["m_occ"] - ref_o) < tol and abs(out["m_free"] - ref_f) < tol
        assert out["m_occ"] >= 0 and out["m_free"] >= 0 and out["m_occ"] + out["m_free"] <= 1 + tol


def test_total_conflict_keeps_prediction():
    out = cell_update(1.0, 0.0, 0.0, 1.0, 1.0, 0.0, "f64")
    assert out["m_occ"] == 1.0 and out["m_free"] == 0.0


@pytest.mark.parametrize("mode,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_free_mass_prediction_is_discounted_and_capped(mode, tol):
    # Eq. DS_freespace_pred: min(alpha m_F, 1 - m_O,pred)
    for mp, mf, a in [(0.2, 0.7, 0.9), (0.6, 0.7, 0.9), (0.0, 1.0, 0.5), (1.0, 0.3, 1.0)]:
        out = cell_update(mp, mf, 0.0, 0.0, a, 0.0, mode)
        assert abs(out["m_free_pred"] - min(a * mf, 1 - mp)) < tol


@pytest.mark.parametrize("mode,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_birth_split_follows_mass_ratio(mode, tol):
    # Eq. DS_resulting_masses1/2: rho_b + rho_p = m_O and rho_b/rho_p = p_B (1-m_pred)/m_pred
    rng = np.random.default_rng(1)
    for _ in range(2000):
        mp = float(rng.uniform(0.01, 1.0))
        pB = float(rng.choice([0.005, 0.02, 0.1, 0.5]))
        zO = float(rng.uniform(0.01, 0.99))
        zF = float(rng.uniform(0, 1 - zO))
        out = cell_update(mp, 0.0, zO, zF, 0.9, pB, mode)
        assert abs(out["rho_b"] + out["rho_p"] - out["m_occ"]) < tol
        mp32 = float(np.float32(mp)) if mode == "f32" else mp
        ratio = pB * (1 - mp32) / mp32
        assert abs(out["rho_b"] - ratio * out["rho_p"]) < 10 * tol * max(1.0, ratio)
    # no births where the measurement has no occupied mass
    out = cell_update(0.3, 0.1, 0.0, 0.6, 0.9, 0.5, mode)
    assert out["rho_b"] == 0.0 and out["rho_p"] == out["m_occ"]
    # an empty prediction with m_z(O) > 0 hands all occupied mass to the newborn part
    out = cell_update(0.0, 0.0, 0.8, 0.0, 0.9, 0.02, mode)
    assert abs(out["rho_b"] - out["m_occ"]) < tol and abs(out["rho_p"]) < tol


# ------------------------------------------------------------- binary Bayes reduction
@pytest.mark.parametrize("mode,tol", [("f64", 1e-8), ("f32", 3e-5)])
def test_static_recursion_reduces_to_binary_bayes_filter(mode, tol):
    """Prop. (Sect. IV-G): static deterministic process, p_S = 1, no births, Bayesian
    measurement BBAs -> m_O follows Eq. BBF_gen with alpha_z = z(O)/z(F).

    Tolerance: FP64 mode differs from the closed form only by the fixed-point truncation
    of the cell sum (at most K 2^-40 per frame for K particles), which the log-odds
    recursion amplifies near 0 and 1 to ~1e-9 over 12 frames; the FP32 mirror carries
    ~1e-7 relative rounding per operation."""
    W = H = 8
    C, K = W * H, 16
    rng = np.random.default_rng(2)
    p = small_params(W, H, nu=C * K, nu_b=64, p_S=1.0, p_B=0.0, alpha=1.0, sigma_pos=0.0,
                     sigma_vel=0.0, flags=NO_RESAMPLE)
    cells = np.repeat(np.arange(C), K)
    m0 = rng.uniform(0.05, 0.95, C).astype(np.float32).astype(np.float64)
    st = dict(x=((cells % W) + rng.uniform(0.1, 0.9, C * K)) * 0.5,
              y=((cells // W) + rng.uniform(0.1, 0.9, C * K)) * 0.5,
              vx=np.zeros(C * K), vy=np.zeros(C * K), w=np.repeat(m0 / K, K),
              m_free=(1 - m0), frame=0)
    o = OracleFilter(p, mode)
    o.set_state(st)
    logit = np.log(m0 / (1 - m0.astype(np.float64)))
    for _ in range(12):
        zO = rng.uniform(0.05, 0.95, C).astype(np.float32).astype(np.float64)
        zF = 1 - zO if mode == "f64" else (1 - zO).astype(np.float32).astype(np.float64)
        o.set_measurement_grid(zO, zF)
        o.step(0.1)
        logit += np.log(zO / zF)
        expect = 1 / (1 + np.exp(-logit))
        got = o.cells()["m_occ"].astype(np.float64)
        assert np.max(np.abs(got - expect)) < tol


# ------------------------------------------------------------------- sort / assignment
@pytest.mark.parametrize("mode", MODES)
def test_sort_is_stable_and_ranges_match_brute_force(mode):
    p = small_params(4, 4, nu=512, nu_b=64)
    rng = np.random.default_rng(3)
    o = OracleFilter(p, mode)
    o.set_state(scene.random_state(p, rng, occupied_frac=0.4))
    g = scene.random_measurement_grid(4, 4, rng)
    o.set_measurement_grid(g["m_occ"], g["m_free"])
    o.step(0.1)
    im = o.intermediates()
    key, perm = im["key"], im["perm"]
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    for c in range(16):
        js = [j for j in range(p["nu"]) if key[perm[j]] == c]
        if js:
            assert im["cell_start"][c] == min(js) and im["cell_end"][c] == max(js) + 1
        else:
            assert im["cell_start"][c] == 0 and im["cell_end"][c] == 0


@pytest.mark.parametrize("mode", MODES)
def test_cell_index_matches_geometry(mode):
    p = small_params(12, 9, nu=6000, nu_b=100, cell_size=0.37)
    rng = np.random.default_rng(4)
    o = OracleFilter(p, mode)
    o.set_state(scene.random_state(p, rng))
    g = scene.random_measurement_grid(12, 9, rng)
    o.set_measurement_grid(g["m_occ"], g["m_free"])
    o.step(0.1)
    im = o.intermediates()
    x, y, key, w = (im[k] for k in ("pred_x", "pred_y", "key", "pred_w"))
    s = 0.37
    col, row = key % 12, key // 12
    inside = (x >= 0) & (x < 12 * s) & (y >= 0) & (y < 9 * s)
    eps = 1e-5
    xi, yi = x[inside] / s, y[inside] / s
    assert np.all(xi >= col[inside] - eps) and np.all(xi < col[inside] + 1 + eps)
    assert np.all(yi >= row[inside] - eps) and np.all(yi < row[inside] + 1 + eps)
    outside = (x < -eps) | (x > 12 * s + eps) | (y < -eps) | (y > 9 * s + eps)
    assert outside.any() and np.all(w[outside] == 0)


def test_zero_noise_prediction_is_constant_velocity():
    """Eq. process with xi = 0: x' = x + T v_x, v' = v; Eq. particle_persistence: w' = p_S w."""
    p = small_params(16, 16, nu=2048, nu_b=16, sigma_pos=0.0, sigma_vel=0.0, p_S=0.97)
    rng = np.random.default_rng(5)
    st = scene.random_state(p, rng)
    o = OracleFilter(p, "f32")
    o.set_state(st)
    g = scene.random_measurement_grid(16, 16, rng)
    o.set_measurement_grid(g["m_occ"], g["m_free"])
    T = np.float32(0.1)
    o.step(float(T))
    im = o.intermediates()
    assert np.array_equal(im["pred_x"], st["x"] + T * st["vx"])
    assert np.array_equal(im["pred_y"], st["y"] + T * st["vy"])
    assert np.array_equal(im["pred_vx"], st["vx"]) and np.array_equal(im["pred_vy"], st["vy"])
    inside = im["pred_w"] > 0
    assert np.array_equal(im["pred_w"][inside], (np.float32(0.97) * st["w"])[inside])


# --------------------------------------------------------------- normalisation / moments
@pytest.mark.parametrize("mode,radar", [("f32", False), ("f64", False), ("f32", True), ("f64", True)])
def test_normalised_weights_sum_to_persistent_mass(mode, radar):
    """Eq. DSnormalization with Eq. DSnormalizationfactor(2): in every cell the normalised
    persistent weights sum to rho_p (the radar likelihood only redistributes them)."""
    p = small_params(16, 16, nu=8192, nu_b=512)
    rng = np.random.default_rng(6)
    o = OracleFilter(p, mode)
    o.set_state(scene.random_state(p, rng, occupied_frac=0.3))
    g = scene.random_measurement_grid(16, 16, rng, radar=radar)
    o.set_measurement_grid(**g)
    o.step(0.1)
    im, c = o.intermediates(), o.cells()
    wn = im["w_norm"].astype(np.float64)
    eps = 1e-15 if mode == "f64" else 2.0 ** -22
    checked = 0
    for cell in range(p["width"] * p["height"]):
        a, b = im["cell_start"][cell], im["cell_end"][cell]
        if b > a and im["S"][cell] > 0:
            n, rp = int(b - a), float(c["rho_p"][cell])
            # the normaliser divides by the truncated fixed-point sum (n quanta at most)
            # and each weight carries one rounding of the mode's precision
            den = float(im["A"][cell] if radar and im["A"][cell] > 0 else im["S"][cell])
            tol = rp * n / den + 4 * eps * n * max(rp, 1e-30) + 1e-300
            if radar and im["A"][cell] > 0:
                tol += rp * n / float(im["S"][cell])
            assert abs(wn[a:b].sum() - rp) <= tol, (cell, n, wn[a:b].sum(), rp)
            checked += 1
    assert checked > 20
    if radar:  # the sum rule held in cells whose weights the likelihood redistributed
        assert sum(1 for cell in range(p["width"] * p["height"]) if im["A"][cell] > 0) > 5


def test_moments_are_textbook_weighted_mean_and_variance():
    """Eq. mean_x, var_x, covar_xy on hand-built cells (dt = 0, no noise, no births)."""
    W = H = 4
    p = small_params(W, H, nu=6, nu_b=4, cell_size=1.0, sigma_pos=0.0, sigma_vel=0.0, p_S=1.0,
                     p_B=0.0, flags=NO_RESAMPLE)
    # cell 5: one particle; cell 6: two; cell 9: three
    cells = np.array([5, 6, 6, 9, 9, 9])
    vx = np.array([3.0, 1.0, -2.0, 0.5, 1.5, 4.0], np.float32)
    vy = np.array([-2.0, 0.0, 2.0, 1.0, -1.0, 2.5], np.float32)
    w = np.array([0.4, 0.1, 0.3, 0.05, 0.2, 0.15], np.float32)
    st = dict(x=(cells % W) + 0.5, y=(cells // W) + 0.5, vx=vx, vy=vy, w=w, m_free=np.zeros(16), frame=0)
    for mode in MODES:
        o = OracleFilter(p, mode)
        o.set_state(st)
        zo = np.zeros(16, np.float32)
        zo[[5, 6, 9]] = 0.8
        o.set_measurement_grid(zo, np.zeros(16, np.float32))
        o.step(0.0)
        c = o.cells()
        for cell in (5, 6, 9):
            sel = cells == cell
            ww = w[sel].astype(np.float64) / w[sel].sum()
            mx, my = (ww * vx[sel]).sum(), (ww * vy[sel]).sum()
            varx = (ww * (vx[sel] - mx) ** 2).sum()
            vary = (ww * (vy[sel] - my) ** 2).sum()
            cov = (ww * (vx[sel] - mx) * (vy[sel] - my)).sum()
            got = [c[k][cell] for k in ("mean_vx", "mean_vy", "var_vx", "var_vy", "cov_vxy")]
            assert np.allclose(got, [mx, my, varx, vary, cov], atol=2e-5), (mode, cell, got)
        assert c["var_vx"][5] == pytest.approx(0.0, abs=1e-5)
        others = np.setdiff1d(np.arange(16), [5, 6, 9])
        assert np.all(c["mean_vx"][others] == 0) and np.all(c["var_vx"][others] == 0)


# --------------------------------------------------------------------- births / resample
def _run_random_frames(mode, radar=False, frames=3, seed=7, **kw):
    p = small_params(24, 20, nu=16384, nu_b=4096, **kw)
    rng = np.random.default_rng(seed)
    o = OracleFilter(p, mode)
    o.set_state(scene.random_state(p, rng, occupied_frac=0.2))
    for _ in range(frames):
        g = scene.random_measurement_grid(24, 20, rng, radar=radar)
        o.set_measurement_grid(**g)
        o.step(0.1)
    return o, p, g


@pytest.mark.parametrize("mode,radar", [("f32", False), ("f64", False), ("f32", True)])
def test_newborn_allocation_is_proportional_to_birth_mass(mode, radar):
    """Alg. 5: slot counts sum to nu_b; each cell gets floor or ceil of nu_b rho_b / sum;
    its newborn weights sum to rho_b (Eq. weights_associated / unassociated); births
    only in cells whose measurement reports occupied mass; positions inside the cell."""
    o, p, g = _run_random_frames(mode, radar)
    im, c = o.intermediates(), o.cells()
    C, nb = p["width"] * p["height"], p["nu_b"]
    qb = q40(c["rho_b"])
    R = int(qb.sum(dtype=np.uint64))
    assert R == im["R_total"] and R > 0
    cnt = np.bincount(im["birth_cell"], minlength=C)
    assert cnt.sum() == nb
    for cell in range(C):
        lo, hi = (nb * int(qb[cell])) // R, -((-nb * int(qb[cell])) // R)
        assert lo <= cnt[cell] <= hi
    assert np.all(np.asarray(g["m_occ"])[cnt > 0] > 0)
    bw = im["birth_w"].astype(np.float64)
    sums = np.bincount(im["birth_cell"], weights=bw, minlength=C)
    has = cnt > 0
    assert np.allclose(sums[has], c["rho_b"][has], rtol=2e-6 * max(1, cnt.max()), atol=1e-7)
    s = p["cell_size"]
    col, row = im["birth_cell"] % p["width"], im["birth_cell"] // p["width"]
    assert np.all(im["birth_x"] >= col * s - 1e-5) and np.all(im["birth_x"] <= (col + 1) * s + 1e-5)
    assert np.all(im["birth_y"] >= row * s - 1e-5) and np.all(im["birth_y"] <= (row + 1) * s + 1e-5)
    if radar:
        pa = np.asarray(g["p_A"])[im["birth_cell"]]
        assert np.all(im["birth_assoc"][pa == 0] == 0)
        assert im["birth_assoc"].sum() > 0


@pytest.mark.parametrize("mode", MODES)
def test_systematic_resampling_bounds(mode):
    """Alg. 7 with systematic draws: source j is copied floor or ceil of nu q_j / W times,
    sources stay in order, nu is conserved and the new equal weights sum to the posterior
    total (Eq. resampledParticleWeights)."""
    o, p, _ = _run_random_frames(mode)
    im = o.intermediates()
    nu, nb = p["nu"], p["nu_b"]
    q = np.concatenate([q40(im["w_norm"]), q40(im["birth_w"])])
    Wt = int(q.sum(dtype=np.uint64))
    assert Wt == im["W_total"] and Wt > 0
    src = im["resample_src"]
    assert src.size == nu and np.all(np.diff(src.astype(np.int64)) >= 0)
    copies = np.bincount(src, minlength=nu + nb)
    for j in np.flatnonzero((copies > 0) | (q > 0)):
        lo, hi = (nu * int(q[j])) // Wt, -((-nu * int(q[j])) // Wt)
        assert lo <= copies[j] <= hi
    st = o.get_state()
    assert st["w"].astype(np.float64).sum() == pytest.approx(Wt * 2.0 ** -40, rel=1e-6)


@pytest.mark.parametrize("mode", MODES)
def test_mass_invariants_over_frames(mode):
    """Masses are non-negative and m_O + m_F <= 1 (Eq. DS_freespace_pred and Dempster's
    rule); rho_b, rho_p >= 0; the pignistic probability lies in [0, 1]."""
    o, p, _ = _run_random_frames(mode, frames=6, seed=8)
    c = o.cells()
    assert np.all(c["m_occ"] >= 0) and np.all(c["m_free"] >= 0)
    assert np.all(c["m_occ"] + c["m_free"] <= 1 + 1e-6)
    assert np.all(c["rho_b"] >= 0) and np.all(c["rho_p"] >= 0)
    assert np.all((c["p_occ"] >= 0) & (c["p_occ"] <= 1 + 1e-6))


def test_no_birth_mass_edge_case():
    """An all-unknown measurement grid gives no birth mass: newborn slots get weight 0."""
    p = small_params(8, 8, nu=1024, nu_b=100)
    o = OracleFilter(p, "f32")
    o.set_measurement_grid(np.zeros(64, np.float32), np.zeros(64, np.float32))
    o.step(0.1)
    im = o.intermediates()
    assert im["R_total"] == 0 and np.all(im["birth_w"] == 0)
    assert np.array_equal(im["birth_cell"], np.arange(100) % 64)


# ----------------------------------------------------------------- end-to-end behaviour
def _observed_grid(W, H, occ_cells):
    m_occ = np.zeros(W * H, np.float32)
    m_free = np.full(W * H, 0.7, np.float32)
    m_occ[occ_cells] = 0.9
    m_free[occ_cells] = 0.0
    return m_occ, m_free


def test_static_cells_converge_to_zero_velocity():
    """Fully observed static scene: velocities of particles that leave their cell are
    penalised by the free evidence around it, so the cells' mean velocity shrinks toward
    zero (Sect. VIII-B: birth distribution zero-mean, constant velocity model)."""
    W = H = 32
    rng = np.random.default_rng(5)
    m_occ, m_free = _observed_grid(W, H, rng.choice(W * H, 40, replace=False))
    p = dict(small_params(W, H, nu=16384, nu_b=4096, sigma_pos=0.02, sigma_vel=0.1), seed=3)
    o = OracleFilter(p, "f32")
    hist = []
    for _ in range(20):
        o.set_measurement_grid(m_occ, m_free)
        o.step(0.1)
        c = o.cells()
        occ = c["m_occ"] > 0.5
        hist.append(np.hypot(c["mean_vx"], c["mean_vy"])[occ].mean())
    assert hist[-1] < 0.3 and hist[-1] < 0.4 * hist[1]


def _moving_block_bias(p_B, frames=24):
    W, H, s = 48, 48, 0.5
    p = dict(width=W, height=H, cell_size=s, nu=32768, nu_b=8192, p_S=0.99, p_B=p_B, alpha=0.9,
             sigma_pos=0.05, sigma_vel=0.5, sigma_birth_vel=4.0, sensor_x=12.0, sensor_y=12.0,
             seed=9, flags=0)
    o = OracleFilter(p, "f32")
    est = []
    for k in range(frames):
        g = np.zeros((H, W), bool)
        g[20:23, 5 + k:8 + k] = True  # 5 m/s to +x: one cell per 0.1 s frame
        m_occ, m_free = _observed_grid(W, H, np.flatnonzero(g.ravel()))
        o.set_measurement_grid(m_occ, m_free)
        o.step(0.1)
        c = o.cells()
        occ = c["m_occ"] > 0.5
        est.append((c["mean_vx"][occ].mean(), c["mean_vy"][occ].mean()))
    return np.array(est)


def test_moving_object_velocity_recovered_with_birth_bias():
    """Sect. VIII-B: the estimate converges to the true velocity; the zero-mean birth
    distribution biases it toward zero, more so for a larger birth probability."""
    lo = _moving_block_bias(0.005)
    hi = _moving_block_bias(0.1)
    assert abs(lo[-5:, 0].mean() - 5.0) < 0.3 and abs(lo[-5:, 1].mean()) < 0.2
    assert hi[-5:, 0].mean() < lo[-5:, 0].mean() - 0.05
