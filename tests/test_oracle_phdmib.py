"""Pins of the oracle's PHD/MIB filter (Sect. VI, flag 0x40) with the Bernoulli observation
of each cell (the single-object likelihood 1 over a measured cell, clutter density p_c):

  * the proposition relating the filter to the binary Bayes filter: with a static world
    (p_S = 1, no process noise, no births) and no resampling, each cell's posterior
    existence follows logit r_n = logit r_0 + sum_k log(p_TP / p_FP) over measured frames
    and log((1 - p_TP) / (1 - p_FP)) over unmeasured ones (g_A = 1: p_c = 1);
  * an unmeasured cell with p_TP = p_FP carries no information: r' = r_p + p_B (1 - r_p);
  * the posterior weights of a cell sum to its posterior existence r' (persistent part
    rho_p, newborn part rho_b), Eq. occupancyProbParticles.
"""
import numpy as np
import pytest

from oracle import OracleFilter

W, H, S = 24, 20, 0.5
FULL, NO_RESAMPLE = 0x40, 0x2


def _params(**kw):
    p = dict(width=W, height=H, cell_size=S, nu=6000, nu_b=1200, p_S=1.0, p_B=0.0, alpha=0.9,
             sigma_pos=0.0, sigma_vel=0.0, sigma_birth_vel=2.0, sensor_x=6.0, sensor_y=5.0,
             seed=9, flags=FULL | NO_RESAMPLE)
    p.update(kw)
    return p


def _state(rng, nu):
    """Particles at cell centres (they stay in their cells without noise); per-cell weight
    sums r_0 in (0.05, 0.9)."""
    C = W * H
    cell = rng.integers(0, C, nu)
    x = ((cell % W) + 0.5) * S
    y = ((cell // W) + 0.5) * S
    r0 = rng.uniform(0.05, 0.9, C)
    cnt = np.bincount(cell, minlength=C)
    w = r0[cell] / cnt[cell]
    return dict(x=x, y=y, vx=rng.normal(0, 1, nu), vy=rng.normal(0, 1, nu), w=w,
                m_free=np.zeros(C), frame=0), cell, cnt


def _bern(rng, informative=True):
    C = W * H
    z = (rng.uniform(0, 1, C) < 0.4).astype(np.float64)
    p_tp = rng.uniform(0.6, 0.95, C)
    p_fp = rng.uniform(0.05, 0.4, C) if informative else p_tp.copy()
    return dict(z=z, p_tp=p_tp, p_fp=p_fp, p_a=rng.uniform(0, 1, C), p_c=np.ones(C))


@pytest.mark.parametrize("mode,tol", [("f64", 1e-9), ("f32", 3e-5)])
def test_binary_bayes_filter_proposition(mode, tol):
    rng = np.random.default_rng(1)
    st, cell, cnt = _state(rng, 6000)
    o = OracleFilter(_params(), mode)
    o.set_state(st)
    C = W * H
    r0 = np.bincount(cell, weights=st["w"], minlength=C)
    occupied = cnt > 0
    L = np.zeros(C)
    for _ in range(6):
        g = _bern(rng)
        o.set_bernoulli_grid(**g)
        o.step(0.0)
        L += np.where(g["z"] == 1, np.log(g["p_tp"] / g["p_fp"]), np.log((1 - g["p_tp"]) / (1 - g["p_fp"])))
    r = o.cells()["m_occ"].astype(np.float64)
    expect = 1.0 / (1.0 + np.exp(-(np.log(r0 / (1 - r0)) + L)))
    assert np.allclose(r[occupied], expect[occupied], atol=tol, rtol=0)


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_uninformative_observation_keeps_the_prediction(mode):
    rng = np.random.default_rng(2)
    st, cell, cnt = _state(rng, 6000)
    o = OracleFilter(_params(p_B=0.05, flags=FULL), mode)
    o.set_state(st)
    g = _bern(rng, informative=False)
    g["z"][:] = 0.0
    o.set_bernoulli_grid(**g)
    o.step(0.0)
    c = o.cells()
    r0 = np.minimum(np.bincount(cell, weights=st["w"], minlength=W * H), 1.0)
    pB = float(np.float32(0.05))  # the parameters are binary32
    expect = r0 + pB * (1 - r0)
    # binary64: only the 2^-40 truncation of each weight in the cell sum (~1e-11)
    tol = 1e-10 if mode == "f64" else 2e-6
    assert np.allclose(c["m_occ"], expect, atol=tol, rtol=0)
    assert np.allclose(c["rho_p"], r0, atol=tol, rtol=0)


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_posterior_weights_sum_to_the_existence(mode):
    rng = np.random.default_rng(3)
    st, cell, cnt = _state(rng, 6000)
    st["w"] = st["w"] * 1.6  # some cells over 1: their weights are scaled to sum 1
    o = OracleFilter(_params(nu_b=9600, p_B=0.05, p_S=0.99, sigma_pos=0.05, sigma_vel=0.5, flags=FULL),
                     mode)
    o.set_state(st)
    o.set_bernoulli_grid(**_bern(rng))
    o.step(0.1)
    im, c = o.intermediates(), o.cells()
    keys = np.asarray(im["key"])[np.asarray(im["perm"])]
    pers = np.bincount(keys, weights=np.asarray(im["w_norm"], np.float64), minlength=W * H)
    born = np.bincount(np.asarray(im["birth_cell"]), weights=np.asarray(im["birth_w"], np.float64),
                       minlength=W * H)
    nslots = np.bincount(np.asarray(im["birth_cell"]), minlength=W * H)
    tol = 1e-9 if mode == "f64" else 2e-5
    assert np.allclose(pers, c["rho_p"], atol=tol, rtol=0)
    # slots are shared out in proportion to the newborn existence, so a cell without a slot
    # holds less than one slot's worth of it (cells over 1 have r_p = 1, r_b = 0, no slot);
    # where a cell has slots they carry its newborn existence exactly
    has = nslots > 0
    slot = c["rho_b"].sum() / 9600
    assert (c["rho_b"][~has] < 2 * slot).all()
    assert np.allclose(born[has], c["rho_b"][has], atol=tol, rtol=0)
    assert np.allclose((c["rho_p"] + c["rho_b"]), c["m_occ"], atol=tol, rtol=0)
