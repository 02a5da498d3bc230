"""Pins of the oracle's radar likelihood and associated newborn particles (no GPU needed).

The radar model (the paper defers it to another paper; the reading taken: a detection's
cell carries p_A, the measured radial velocity z_vr and its SD sigma_vr, and a particle's
spatial likelihood is g = exp(-1/2 ((v_r - z_vr) / sigma_vr)^2) with v_r its velocity
projected on the line from the sensor to the particle) is pinned here against closed forms
computed independently in binary64 from the geometry:
  * g = 1 exactly when v_r = z_vr, g = e^-1/2 at one sigma_vr (sigma_vr != 1, so a sigma
    squared twice fails), v_r = +|v| moving straight away from the sensor, -|v| towards it
    and 0 moving across (a sign error in v_r fails), and random cases within a bound derived
    from the binary32 operations;
  * the normalised persistent weights of a radar cell follow Eq. DSnormalization with that
    g: w'_i = w_i (p_A rho_p g_i / sum_j g_j w_j + (1 - p_A) rho_p / sum_j w_j);
  * a radar grid with p_A = 0 everywhere gives the lidar filter's results bit for bit;
  * associated newborn particles (Eq. DSbirth_particle_samplingA reading) have radial
    velocity N(z_vr, sigma_vr^2) and tangential velocity N(0, sigma_B^2).
"""
import math

import numpy as np
import pytest

from oracle import OracleFilter, radar_likelihood

MODES = ["f32", "f64"]
NO_RESAMPLE = 0x2
U = 2.0 ** -24


def g_ref(sensor, x, y, vx, vy, z, sg):
    """Binary64 definition: radial velocity from the geometry, then the Gaussian."""
    dx, dy = x - sensor[0], y - sensor[1]
    r = math.hypot(dx, dy)
    vr = (dx * vx + dy * vy) / r if r > 0 else 0.0
    d = (vr - z) / sg
    return math.exp(-0.5 * d * d), vr, d


@pytest.mark.parametrize("mode", MODES)
def test_likelihood_is_one_at_the_measured_radial_velocity(mode):
    # particle at (3, 4) from the sensor, velocity (3, 4): v_r = 25 / 5 = 5 exactly
    for sensor in [(0.0, 0.0), (10.0, -2.0)]:
        x, y = sensor[0] + 3.0, sensor[1] + 4.0
        assert radar_likelihood(sensor, x, y, 3.0, 4.0, 5.0, 0.5, mode) == 1.0
        assert radar_likelihood(sensor, x, y, -3.0, -4.0, -5.0, 0.5, mode) == 1.0
        assert radar_likelihood(sensor, x, y, 4.0, -3.0, 0.0, 0.5, mode) == 1.0   # across: v_r = 0


@pytest.mark.parametrize("mode", MODES)
def test_likelihood_at_one_and_two_sigma(mode):
    tol = 8 * U if mode == "f32" else 1e-15
    x, y = 3.0, 4.0
    for sg in (0.5, 0.25, 2.0):
        g1 = radar_likelihood((0, 0), x, y, 3.0, 4.0, 5.0 - sg, sg, mode)   # d = 1
        g2 = radar_likelihood((0, 0), x, y, 3.0, 4.0, 5.0 + 2 * sg, sg, mode)  # d = -2
        assert abs(g1 - math.exp(-0.5)) <= tol * math.exp(-0.5), (sg, g1)
        assert abs(g2 - math.exp(-2.0)) <= tol * math.exp(-2.0), (sg, g2)


@pytest.mark.parametrize("mode", MODES)
def test_radial_velocity_sign_and_direction(mode):
    """Moving away from the sensor at speed s gives v_r = +s, towards it -s, across 0: each
    checked through g with z_vr = s (so only v_r = +s gives 1)."""
    rng = np.random.default_rng(1)
    sensor = (2.0, -1.0)
    sg, s = 0.7, 3.0
    for ang in rng.uniform(0, 2 * np.pi, 16):
        ex, ey = math.cos(ang), math.sin(ang)
        r = 6.0
        x, y = sensor[0] + r * ex, sensor[1] + r * ey
        for (vx, vy), vr in (((s * ex, s * ey), s), ((-s * ex, -s * ey), -s), ((-s * ey, s * ex), 0.0)):
            want = math.exp(-0.5 * ((vr - s) / sg) ** 2)
            got = radar_likelihood(sensor, x, y, vx, vy, s, sg, mode)
            tol = 1e-12 if mode == "f64" else 1e-5 + 64 * U * abs(vr - s) / sg * want
            assert abs(got - want) <= max(tol, 1e-300), (ang, vr, got, want)


@pytest.mark.parametrize("mode", MODES)
def test_likelihood_random_cases_within_rounding_bound(mode):
    rng = np.random.default_rng(2)
    for _ in range(2000):
        sensor = tuple(np.float32(rng.uniform(-20, 20, 2)).astype(float))
        x, y = (float(np.float32(v)) for v in rng.uniform(-50, 50, 2))
        vx, vy = (float(np.float32(v)) for v in rng.normal(0, 8, 2))
        z = float(np.float32(rng.normal(0, 8)))
        sg = float(np.float32(rng.uniform(0.1, 3.0)))
        want, vr, d = g_ref(sensor, x, y, vx, vy, z, sg)
        got = radar_likelihood(sensor, x, y, vx, vy, z, sg, mode)
        if mode == "f64":
            tol = 1e-12 * (1 + d * d) * want + 1e-300
        else:
            # binary32: v_r off by <= 8 u |v|; d by <= u (8 |v| + 2 |z_vr|) / sigma + u |d|;
            # g by g (|d| dd + 2 u d^2 + 4 u) (the series of exp adds a few units)
            v = math.hypot(vx, vy)
            dd = U * (8 * v + 2 * abs(z)) / sg + U * abs(d)
            tol = 2 * want * (abs(d) * dd + 2 * U * d * d + 4 * U) + 1e-30
        assert abs(got - want) <= tol, (sensor, x, y, vx, vy, z, sg, got, want)


def _radar_cell_frame(mode, pA=0.9, z_vr=4.0, sigma_vr=0.6):
    """One frame with hand-built persistent particles in one radar cell: no motion, no noise,
    no resampling, so the predicted particles are the given ones."""
    W = H = 8
    p = dict(width=W, height=H, cell_size=1.0, nu=7, nu_b=64, p_S=1.0, p_B=0.02, alpha=0.9,
             sigma_pos=0.0, sigma_vel=0.0, sigma_birth_vel=4.0, sensor_x=1.0, sensor_y=1.5,
             seed=3, flags=NO_RESAMPLE)
    cell = 5 * W + 6  # x in [6, 7), y in [5, 6)
    rng = np.random.default_rng(4)
    x = (6.0 + rng.uniform(0.1, 0.9, 7)).astype(np.float32)
    y = (5.0 + rng.uniform(0.1, 0.9, 7)).astype(np.float32)
    # velocities around the measured radial velocity: radial z_vr + sigma_vr t, |t| <= 2,
    # plus a tangential part, so that every g lies in [e^-2, 1]
    dx, dy = x - np.float32(1.0), y - np.float32(1.5)
    r = np.hypot(dx, dy)
    t = np.linspace(-2.0, 2.0, 7)
    vrad = z_vr + sigma_vr * t
    vtan = rng.normal(0, 3, 7)
    vx = ((vrad * dx - vtan * dy) / r).astype(np.float32)
    vy = ((vrad * dy + vtan * dx) / r).astype(np.float32)
    w = rng.uniform(0.02, 0.12, 7).astype(np.float32)
    st = dict(x=x, y=y, vx=vx, vy=vy, w=w, m_free=np.zeros(W * H), frame=0)
    C = W * H
    g = dict(m_occ=np.zeros(C), m_free=np.zeros(C), p_A=np.zeros(C), z_vr=np.zeros(C), sigma_vr=np.ones(C))
    g["m_occ"][cell] = 0.8
    g["p_A"][cell], g["z_vr"][cell], g["sigma_vr"][cell] = pA, z_vr, sigma_vr
    o = OracleFilter(p, mode)
    o.set_state(st)
    o.set_measurement_grid(**g)
    o.step(0.0)
    return o, p, st, g, cell


@pytest.mark.parametrize("mode", MODES)
def test_radar_normalisation_follows_the_likelihood(mode):
    """Eq. DSnormalization: w'_i = w_i (p_A rho_p g_i / sum g w + (1 - p_A) rho_p / sum w),
    with g_i from the binary64 geometry; the particle whose radial velocity matches z_vr
    gains weight relative to the others."""
    pA, z, sg = 0.9, 4.0, 0.6
    o, p, st, g, cell = _radar_cell_frame(mode, pA, z, sg)
    im, c = o.intermediates(), o.cells()
    perm = im["perm"]
    a, b = im["cell_start"][cell], im["cell_end"][cell]
    assert (a, b) == (0, 7)
    sensor = (p["sensor_x"], p["sensor_y"])
    w = st["w"].astype(np.float64)[perm]
    gi = np.array([g_ref(sensor, float(st["x"][i]), float(st["y"][i]), float(st["vx"][i]),
                         float(st["vy"][i]), z, sg)[0] for i in perm])
    rp = float(c["rho_p"][cell])
    want = w * (pA * rp * gi / (gi * w).sum() + (1 - pA) * rp / w.sum())
    got = im["w_norm"].astype(np.float64)
    assert gi.min() > 0.13 and gi.max() == pytest.approx(1.0, abs=1e-9)
    # the fixed-point sums truncate each of the 7 terms at 2^-40 (relative 7 2^-40 / sum);
    # binary32 weights carry a few roundings and g the bound of its radial velocity
    trunc = 7 * 2.0 ** -40 / (gi * w).sum() + 7 * 2.0 ** -40 / w.sum()
    tol = trunc + (1e-12 if mode == "f64" else 64 * U)
    assert np.allclose(got, want, rtol=tol, atol=0), (got, want)
    assert abs(got.sum() - rp) <= rp * tol
    # the weight each particle gains from the likelihood is g itself (a sign error in v_r or
    # a sigma squared twice changes it)
    ratio = (got / w - (1 - pA) * rp / w.sum()) / (pA * rp / (gi * w).sum())
    assert np.allclose(ratio, gi, rtol=20 * tol), (ratio, gi)


@pytest.mark.parametrize("mode", MODES)
def test_radar_grid_without_association_is_the_lidar_filter(mode):
    """p_A = 0 everywhere: the likelihood takes no part (Eq. DSnormalization reduces to
    mu_UA w) and every output equals the lidar filter's bit for bit."""
    W, H = 16, 12
    p = dict(width=W, height=H, cell_size=0.5, nu=4096, nu_b=1024, p_S=0.99, p_B=0.02, alpha=0.9,
             sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0, sensor_x=4.0, sensor_y=3.0,
             seed=11, flags=0)
    from paper_1605_02406_b300 import scene
    rng = np.random.default_rng(5)
    st = scene.random_state(p, rng, occupied_frac=0.3)
    grids = [scene.random_measurement_grid(W, H, rng) for _ in range(3)]
    lid, rad = OracleFilter(p, mode), OracleFilter(p, mode)
    lid.set_state(st)
    rad.set_state(st)
    C = W * H
    for gr in grids:
        lid.set_measurement_grid(gr["m_occ"], gr["m_free"])
        rad.set_measurement_grid(gr["m_occ"], gr["m_free"], np.zeros(C), rng.normal(0, 5, C),
                                 rng.uniform(0.1, 1, C))
        lid.step(0.1)
        rad.step(0.1)
        a, b = lid.cells(), rad.cells()
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        sa, sb = lid.get_state(), rad.get_state()
        for k in ("x", "y", "vx", "vy", "w"):
            assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("mode", MODES)
def test_associated_newborn_velocities(mode):
    """Newborns of a cell with p_A = 1 are all associated; their velocity's radial component
    (along sensor -> particle) is N(z_vr, sigma_vr^2) and its tangential component
    N(0, sigma_B^2)."""
    W = H = 16
    n = 20000
    z, sg, sB = 7.0, 0.2, 4.0
    p = dict(width=W, height=H, cell_size=1.0, nu=1024, nu_b=n, p_S=0.99, p_B=0.02, alpha=0.9,
             sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=sB, sensor_x=8.0, sensor_y=8.0,
             seed=21, flags=0)
    C = W * H
    cell = 3 * W + 12  # x in [12, 13), y in [3, 4): about 6.4 m from the sensor
    g = dict(m_occ=np.zeros(C), m_free=np.zeros(C), p_A=np.zeros(C), z_vr=np.zeros(C), sigma_vr=np.ones(C))
    g["m_occ"][cell], g["p_A"][cell], g["z_vr"][cell], g["sigma_vr"][cell] = 0.9, 1.0, z, sg
    o = OracleFilter(p, mode)
    o.set_measurement_grid(**g)
    o.step(0.1)  # the initial particles have weight 0: all newborn mass lies in this cell
    im = o.intermediates()
    assert np.all(im["birth_cell"] == cell) and np.all(im["birth_assoc"] == 1)
    bx, by = im["birth_x"].astype(np.float64), im["birth_y"].astype(np.float64)
    assert np.all((bx >= 12) & (bx <= 13) & (by >= 3) & (by <= 4))
    dx, dy = bx - p["sensor_x"], by - p["sensor_y"]
    r = np.hypot(dx, dy)
    vx, vy = im["birth_vx"].astype(np.float64), im["birth_vy"].astype(np.float64)
    vr = (dx * vx + dy * vy) / r
    vt = (-dy * vx + dx * vy) / r
    se = 5 / math.sqrt(n)
    assert abs(vr.mean() - z) < se * sg, vr.mean()
    assert abs(vr.std() / sg - 1) < 0.05, vr.std()
    assert abs(vt.mean()) < se * sB, vt.mean()
    assert abs(vt.std() / sB - 1) < 0.05, vt.std()
    assert abs(np.corrcoef(vr, vt)[0, 1]) < 0.05
