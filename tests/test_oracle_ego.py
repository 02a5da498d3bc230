"""Pins of the oracle's ego-motion compensation (the reading documented at
oracle_set_ego_motion: the grid moves with the vehicle, the sensor at q; after a motion d
and a turn theta a posterior particle enters the new grid at q + R(-theta)(p - q - d) with
velocity R(-theta) v, and each new cell takes the free mass of the old cell under its
centre).  The transform is isolated by a step that changes nothing else: no process noise
and dt = 0 (prediction is the identity on particles), a measurement with no information
(z_O = z_F = 0), alpha = 1 and no occupied mass (the posterior free mass is the warped one).
"""
import math

import numpy as np
import pytest

from oracle import OracleFilter

W, H, S = 48, 40, 0.5
QX, QY = 16.0, 12.0  # sensor position (dyadic, so translations by whole cells are exact)


def _params(**kw):
    p = dict(width=W, height=H, cell_size=S, nu=2000, nu_b=0, p_S=1.0, p_B=0.0, alpha=1.0,
             sigma_pos=0.0, sigma_vel=0.0, sigma_birth_vel=1.0, sensor_x=QX, sensor_y=QY,
             seed=3, flags=0)
    p.update(kw)
    return p


def _state(rng, nu, w=0.0):
    # positions on a 1/64 lattice inside the grid, velocities on a 1/8 lattice
    x = rng.integers(64, (W - 1) * S * 64, nu) / 64.0
    y = rng.integers(64, (H - 1) * S * 64, nu) / 64.0
    vx = rng.integers(-40, 40, nu) / 8.0
    vy = rng.integers(-40, 40, nu) / 8.0
    m_free = rng.integers(0, 64, W * H) / 64.0
    return dict(x=x, y=y, vx=vx, vy=vy, w=np.full(nu, w), m_free=m_free, frame=0)


def _quiet_grid():
    z = np.zeros(W * H)
    return dict(m_occ=z, m_free=z)


def _one_step(mode, st, motion):
    o = OracleFilter(_params(), mode)
    o.set_state(st)
    o.set_measurement_grid(**_quiet_grid())
    if motion is not None:
        o.set_ego_motion(*motion)
    o.step(0.0)
    im = o.intermediates()
    return o, im


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_zero_motion_is_the_identity(mode):
    rng = np.random.default_rng(1)
    st = _state(rng, 2000, w=0.01)
    o1 = OracleFilter(_params(sigma_pos=0.1, sigma_vel=1.0, p_S=0.99, p_B=0.02, alpha=0.9), mode)
    o2 = OracleFilter(_params(sigma_pos=0.1, sigma_vel=1.0, p_S=0.99, p_B=0.02, alpha=0.9), mode)
    for o in (o1, o2):
        o.set_state(st)
    g = dict(m_occ=rng.uniform(0, 0.5, W * H), m_free=rng.uniform(0, 0.4, W * H))
    for _ in range(3):
        for o in (o1, o2):
            o.set_measurement_grid(**g)
        o1.set_ego_motion(0.0, 0.0, 0.0)
        o1.step(0.1)
        o2.step(0.1)
    s1, s2 = o1.get_state(), o2.get_state()
    for k in ("x", "y", "vx", "vy", "w", "m_free"):
        assert np.array_equal(s1[k], s2[k]), k


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_translation_by_whole_cells_is_an_exact_shift(mode):
    rng = np.random.default_rng(2)
    st = _state(rng, 2000)
    k, j = 3, -2  # the vehicle moved 3 cells along x and -2 along y
    o, im = _one_step(mode, st, (k * S, j * S, 0.0))
    # particles: p' = p - d exactly (all values dyadic), velocities unchanged
    assert np.array_equal(im["pred_x"], st["x"] - k * S)
    assert np.array_equal(im["pred_y"], st["y"] - j * S)
    assert np.array_equal(im["pred_vx"], st["vx"]) and np.array_equal(im["pred_vy"], st["vy"])
    # free mass: new cell (r, c) holds old cell (r + j, c + k), 0 where that is outside
    old = st["m_free"].reshape(H, W)
    exp = np.zeros((H, W))
    rr, cc = np.mgrid[0:H, 0:W]
    inside = (rr + j >= 0) & (rr + j < H) & (cc + k >= 0) & (cc + k < W)
    exp[inside] = old[(rr + j)[inside], (cc + k)[inside]]
    assert np.array_equal(o.get_state()["m_free"].reshape(H, W), exp)


# the motion is passed in binary32 (as the C ABI takes it): pi/2 arrives as pi/2 + 4.4e-8,
# which moves a point 24 m from the sensor by 1e-6, so binary64 is held to 2e-6 here
@pytest.mark.parametrize("mode,tol", [("f32", 2e-5), ("f64", 2e-6)])
def test_quarter_turn(mode, tol):
    rng = np.random.default_rng(3)
    st = _state(rng, 2000)
    _, im = _one_step(mode, st, (0.0, 0.0, math.pi / 2))
    # R(-pi/2): (rx, ry) -> (ry, -rx) about the sensor; (vx, vy) -> (vy, -vx)
    assert np.allclose(im["pred_x"], QX + (st["y"] - QY), atol=tol, rtol=0)
    assert np.allclose(im["pred_y"], QY - (st["x"] - QX), atol=tol, rtol=0)
    assert np.allclose(im["pred_vx"], st["vy"], atol=tol, rtol=0)
    assert np.allclose(im["pred_vy"], -st["vx"], atol=tol, rtol=0)


# binary32 arguments: the inverse motion's displacement is rounded to binary32 (~1e-7)
@pytest.mark.parametrize("mode,tol", [("f32", 5e-5), ("f64", 1e-6)])
def test_motion_then_its_inverse_returns_the_particles(mode, tol):
    rng = np.random.default_rng(4)
    st = _state(rng, 2000)
    dx, dy, th = 1.3, -0.7, 0.21
    o = OracleFilter(_params(), mode)
    o.set_state(st)
    o.set_measurement_grid(**_quiet_grid())
    o.set_ego_motion(dx, dy, th)
    o.step(0.0)
    # back: in the new frame the vehicle moves by -R(-th) d and turns by -th
    c, s = math.cos(th), math.sin(th)
    bdx, bdy = -(c * dx + s * dy), -(-s * dx + c * dy)
    st2 = o.get_state()  # nothing was resampled away: all weights are 0 (no resampling)
    im = o.intermediates()
    o2 = OracleFilter(_params(), mode)
    o2.set_state(dict(x=im["pred_x"], y=im["pred_y"], vx=im["pred_vx"], vy=im["pred_vy"],
                      w=np.zeros(2000), m_free=st2["m_free"], frame=1))
    o2.set_measurement_grid(**_quiet_grid())
    o2.set_ego_motion(bdx, bdy, -th)
    o2.step(0.0)
    im2 = o2.intermediates()
    for a, b in (("pred_x", "x"), ("pred_y", "y"), ("pred_vx", "vx"), ("pred_vy", "vy")):
        assert np.allclose(im2[a], st[b], atol=tol, rtol=0), a


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_free_mass_warp_matches_nearest_cell_mapping(mode):
    rng = np.random.default_rng(5)
    st = _state(rng, 2000)
    dx, dy, th = 0.83, -1.37, 0.35
    o, _ = _one_step(mode, st, (dx, dy, th))
    got = o.get_state()["m_free"].reshape(H, W)
    old = st["m_free"].reshape(H, W)
    rr, cc = np.mgrid[0:H, 0:W].astype(np.float64)
    ux, uy = (cc + 0.5) * S - QX, (rr + 0.5) * S - QY
    c, s = math.cos(th), math.sin(th)
    fx = (QX + c * ux - s * uy + dx) / S
    fy = (QY + s * ux + c * uy + dy) / S
    # away from cell edges the binary32 and binary64 mappings agree on the cell
    clear = (np.abs(fx - np.round(fx)) > 1e-3) & (np.abs(fy - np.round(fy)) > 1e-3)
    inside = (fx >= 0) & (fx < W) & (fy >= 0) & (fy < H)
    exp = np.zeros((H, W))
    ix, iy = np.floor(fx).astype(int), np.floor(fy).astype(int)
    exp[inside] = old[iy[inside], ix[inside]]
    assert clear.mean() > 0.99
    assert np.array_equal(got[clear], exp[clear])
