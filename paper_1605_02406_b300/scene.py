"""Seeded synthetic workloads: scenes, lidar/radar measurement grids and particle states.

This module is the one input generator that both the CUDA path and the oracle are fed
from.  It holds none of the filter's arithmetic: it only produces the inputs the paper's
filter consumes -- a measurement grid with the same dimensions as the map (the paper's
meas_cell_array, Sect. VII) and, for single-frame tests, a posterior particle state.

The paper evaluates on recorded laser/radar logs that are not available; the workloads
here stand in for them with the shapes of the paper's setting (Table I: 0.1 m cells,
millions of particles, p_S = 0.99, sigma_B,v = 4 m/s) at the workload sizes below: a
small plain grid, the automotive-size grid and a lidar + radar fusion grid.

Measurement grid model (inverse sensor model of a 2D scanner at the grid centre):
beams at uniform angles are ray-cast against the scene (oriented rectangles plus a wall
border one cell thick); each hit range gets Gaussian noise; the cell containing the noisy
hit receives the occupancy BBA (0.9, 0), the cells the beam crosses before it (0, 0.7)
unless another beam marked them occupied ("occupied wins"), all other cells (0, 0).
Cells are traversed exactly with the Amanatides-Woo voxel walk.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------------------
# workload configurations
# --------------------------------------------------------------------------------------
COMMON = dict(p_S=0.99, p_B=0.02, alpha=0.9, sigma_pos=0.1, sigma_vel=2.0,
              sigma_birth_vel=4.0, occ_mass=0.9, free_mass=0.7, range_noise=0.1, dt=0.1)

CONFIGS = {
    "plain_128": dict(COMMON, name="plain 128x128 @0.5 m, 65,536 + 16,384 particles",
            width=128, height=128, cell_size=0.5, nu=65536, nu_b=16384, frames=20,
            n_moving=4, moving_size=(2.0, 4.5), moving_speed=(0.0, 15.0), n_static=0,
            beams=1080),
    "automotive_1024": dict(COMMON, name="automotive 1024x1024 @0.1 m, 4,194,304 + 1,048,576 particles",
            width=1024, height=1024, cell_size=0.1, nu=4194304, nu_b=1048576, frames=100,
            n_moving=30, moving_side=(1.0, 5.0), moving_speed=(0.0, 20.0), n_static=200,
            static_side=(0.5, 3.0), beams=2160),
    "fusion_2048": dict(COMMON, name="fusion 2048x2048 @0.1 m, 16,777,216 + 4,194,304 particles, lidar + radar",
            width=2048, height=2048, cell_size=0.1, nu=16777216, nu_b=4194304, frames=100,
            n_moving=30, moving_side=(1.0, 5.0), moving_speed=(0.0, 20.0), n_static=200,
            static_side=(0.5, 3.0), beams=4320, radar_detections=64, radar_sigma_r=0.3,
            radar_sigma_vr=0.2, radar_p_A=0.9, radar_occ_mass=0.6),
}


def filter_params(cfg: dict, seed: int = 42, flags: int = 0, **over) -> dict:
    """The filter's parameter set for a workload (sensor at the grid centre)."""
    p = dict(width=int(cfg["width"]), height=int(cfg["height"]), cell_size=float(cfg["cell_size"]),
             nu=int(cfg["nu"]), nu_b=int(cfg["nu_b"]), p_S=cfg["p_S"], p_B=cfg["p_B"],
             alpha=cfg["alpha"], sigma_pos=cfg["sigma_pos"], sigma_vel=cfg["sigma_vel"],
             sigma_birth_vel=cfg["sigma_birth_vel"],
             sensor_x=cfg["width"] * cfg["cell_size"] / 2.0,
             sensor_y=cfg["height"] * cfg["cell_size"] / 2.0, seed=int(seed), flags=int(flags))
    p.update(over)
    return p


def batched_configs(n_filters: int = 64, seed: int = 1003) -> list:
    """Batched workload: uneven grids (sides from {256,512,768,1024} at 0.1 m), particle
    counts 2^U[18,22] rounded to a multiple of 1024, newborn = count/4, 5-30 objects."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_filters):
        side = int(rng.choice([256, 512, 768, 1024]))
        nu = int(round(2.0 ** rng.uniform(18, 22) / 1024.0)) * 1024
        n_obj = int(rng.integers(5, 31))
        cfg = dict(COMMON, name=f"batched filter {k}", width=side, height=side, cell_size=0.1,
                   nu=nu, nu_b=nu // 4, frames=50, n_moving=max(1, n_obj // 2),
                   moving_side=(1.0, 5.0), moving_speed=(0.0, 20.0),
                   n_static=n_obj - max(1, n_obj // 2), static_side=(0.5, 3.0),
                   beams=max(360, 2160 * side // 1024))
        out.append(cfg)
    return out


def serving_stream_configs(n_streams: int = 256, seed: int = 1004) -> list:
    """Serving workload: grids 256^2/512^2/1024^2 w.p. 0.5/0.3/0.2 at 0.1 m, 16 particles
    per cell, newborn = count/4, Poisson arrivals at 10 Hz per stream."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_streams):
        side = int(rng.choice([256, 512, 1024], p=[0.5, 0.3, 0.2]))
        nu = 16 * side * side
        n_obj = int(rng.integers(5, 31))
        out.append(dict(COMMON, name=f"stream {k}", width=side, height=side, cell_size=0.1,
                        nu=nu, nu_b=nu // 4, rate_hz=10.0, n_moving=max(1, n_obj // 2),
                        moving_side=(1.0, 5.0), moving_speed=(0.0, 20.0),
                        n_static=n_obj - max(1, n_obj // 2), static_side=(0.5, 3.0),
                        beams=max(360, 2160 * side // 1024)))
    return out


# --------------------------------------------------------------------------------------
# scene
# --------------------------------------------------------------------------------------
@dataclass
class Box:
    cx: float
    cy: float
    hl: float       # half length (along heading)
    hw: float       # half width
    heading: float
    vx: float = 0.0
    vy: float = 0.0


@dataclass
class Scene:
    cfg: dict
    seed: int
    boxes: list = field(default_factory=list)
    t: float = 0.0

    @property
    def extent(self):
        return self.cfg["width"] * self.cfg["cell_size"], self.cfg["height"] * self.cfg["cell_size"]

    @property
    def origin(self):
        ex, ey = self.extent
        return ex / 2.0, ey / 2.0


def make_scene(cfg: dict, seed: int) -> Scene:
    """Moving rectangles (uniform position inside the walls, non-overlapping by rejection,
    uniform heading, uniform speed) and static boxes, none covering the sensor."""
    rng = np.random.default_rng(seed)
    sc = Scene(cfg=cfg, seed=seed)
    ex, ey = sc.extent
    s = cfg["cell_size"]
    ox, oy = sc.origin

    def place(hl, hw, moving):
        r = math.hypot(hl, hw)
        for _ in range(1000):
            cx = rng.uniform(2 * s + r, ex - 2 * s - r)
            cy = rng.uniform(2 * s + r, ey - 2 * s - r)
            if math.hypot(cx - ox, cy - oy) < r + 1.0:
                continue
            if any(math.hypot(cx - b.cx, cy - b.cy) < r + math.hypot(b.hl, b.hw) for b in sc.boxes):
                continue
            head = rng.uniform(0, 2 * math.pi)
            vx = vy = 0.0
            if moving:
                sp = rng.uniform(*cfg["moving_speed"])
                vx, vy = sp * math.cos(head), sp * math.sin(head)
            return Box(cx, cy, hl, hw, head, vx, vy)
        return None

    for _ in range(cfg.get("n_moving", 0)):
        if "moving_size" in cfg:
            w, l = cfg["moving_size"]
        else:
            w, l = sorted(rng.uniform(*cfg["moving_side"], size=2))
        b = place(l / 2, w / 2, True)
        if b is not None:
            sc.boxes.append(b)
    for _ in range(cfg.get("n_static", 0)):
        a, c = rng.uniform(*cfg["static_side"], size=2)
        b = place(max(a, c) / 2, min(a, c) / 2, False)
        if b is not None:
            sc.boxes.append(b)
    return sc


def advance(sc: Scene, dt: float) -> None:
    """Constant velocity; a rectangle whose circumcircle reaches the wall is reflected."""
    ex, ey = sc.extent
    s = sc.cfg["cell_size"]
    for b in sc.boxes:
        if b.vx == 0.0 and b.vy == 0.0:
            continue
        b.cx += b.vx * dt
        b.cy += b.vy * dt
        r = math.hypot(b.hl, b.hw)
        if b.cx - r < s or b.cx + r > ex - s:
            b.vx = -b.vx
        if b.cy - r < s or b.cy + r > ey - s:
            b.vy = -b.vy
        b.heading = math.atan2(b.vy, b.vx)
    sc.t += dt


def _ray_boxes(ox, oy, dx, dy, boxes):
    """Nearest entry distance of each beam into any oriented rectangle (inf if none)."""
    n = dx.shape[0]
    best = np.full(n, np.inf)
    best_k = np.full(n, -1, dtype=np.int64)
    for k, b in enumerate(boxes):
        c, s_ = math.cos(b.heading), math.sin(b.heading)
        px, py = ox - b.cx, oy - b.cy
        lx, ly = c * px + s_ * py, -s_ * px + c * py          # origin in box frame
        ldx, ldy = c * dx + s_ * dy, -s_ * dx + c * dy        # directions in box frame
        with np.errstate(divide="ignore", invalid="ignore"):
            t1x = (-b.hl - lx) / ldx
            t2x = (b.hl - lx) / ldx
            t1y = (-b.hw - ly) / ldy
            t2y = (b.hw - ly) / ldy
        tminx, tmaxx = np.minimum(t1x, t2x), np.maximum(t1x, t2x)
        tminy, tmaxy = np.minimum(t1y, t2y), np.maximum(t1y, t2y)
        tminx = np.where(ldx == 0, np.where(abs(lx) <= b.hl, -np.inf, np.inf), tminx)
        tmaxx = np.where(ldx == 0, np.where(abs(lx) <= b.hl, np.inf, -np.inf), tmaxx)
        tminy = np.where(ldy == 0, np.where(abs(ly) <= b.hw, -np.inf, np.inf), tminy)
        tmaxy = np.where(ldy == 0, np.where(abs(ly) <= b.hw, np.inf, -np.inf), tmaxy)
        tin = np.maximum(tminx, tminy)
        tout = np.minimum(tmaxx, tmaxy)
        hit = (tin <= tout) & (tout > 0)
        t = np.where(hit, np.maximum(tin, 0.0), np.inf)
        upd = t < best
        best = np.where(upd, t, best)
        best_k = np.where(upd, k, best_k)
    return best, best_k


def _walk_cells(ox, oy, dx, dy, r_hit, W, H, s):
    """Amanatides-Woo traversal.  Returns (free cell indices, hit cell indices)."""
    n = dx.shape[0]
    ix = np.floor(ox / s).astype(np.int64) * np.ones(n, np.int64)
    iy = np.floor(oy / s).astype(np.int64) * np.ones(n, np.int64)
    stx = np.where(dx > 0, 1, -1)
    sty = np.where(dy > 0, 1, -1)
    with np.errstate(divide="ignore"):
        nbx = np.where(dx > 0, (ix + 1) * s, ix * s)
        nby = np.where(dy > 0, (iy + 1) * s, iy * s)
        tmx = np.where(dx != 0, (nbx - ox) / dx, np.inf)
        tmy = np.where(dy != 0, (nby - oy) / dy, np.inf)
        tdx = np.where(dx != 0, s / np.abs(dx), np.inf)
        tdy = np.where(dy != 0, s / np.abs(dy), np.inf)
    active = np.ones(n, bool)
    free_l, hit_l = [], []
    for _ in range(2 * (W + H) + 4):
        if not active.any():
            break
        inside = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
        active &= inside
        texit = np.minimum(tmx, tmy)
        is_free = active & (texit <= r_hit)
        is_hit = active & (texit > r_hit)
        free_l.append((iy[is_free] * W + ix[is_free]))
        hit_l.append((iy[is_hit] * W + ix[is_hit]))
        active &= ~is_hit
        stepx = tmx < tmy
        ix = np.where(active & stepx, ix + stx, ix)
        tmx = np.where(active & stepx, tmx + tdx, tmx)
        iy = np.where(active & ~stepx, iy + sty, iy)
        tmy = np.where(active & ~stepx, tmy + tdy, tmy)
    free = np.concatenate(free_l) if free_l else np.zeros(0, np.int64)
    hit = np.concatenate(hit_l) if hit_l else np.zeros(0, np.int64)
    return free, hit


def measurement_grid(sc: Scene, rng: np.random.Generator) -> dict:
    """Lidar measurement grid (and, when configured, the radar layer) for the scene's
    current time.  Returns float32 arrays m_occ, m_free (and p_A, z_vr, sigma_vr)."""
    cfg = sc.cfg
    W, H, s = cfg["width"], cfg["height"], cfg["cell_size"]
    ex, ey = sc.extent
    ox, oy = sc.origin
    nb = cfg["beams"]
    ang = 2 * math.pi * (np.arange(nb) + 0.5) / nb
    dx, dy = np.cos(ang), np.sin(ang)
    # the wall border: inner boundary of the outermost ring of cells
    with np.errstate(divide="ignore", invalid="ignore"):
        tx = np.where(dx > 0, (ex - s - ox) / dx, np.where(dx < 0, (s - ox) / dx, np.inf))
        ty = np.where(dy > 0, (ey - s - oy) / dy, np.where(dy < 0, (s - oy) / dy, np.inf))
    t_wall = np.minimum(tx, ty)
    t_box, _ = _ray_boxes(ox, oy, dx, dy, sc.boxes)
    r = np.minimum(t_wall, t_box) + rng.normal(0.0, cfg["range_noise"], nb)
    r = np.maximum(r, 0.0)
    free, hit = _walk_cells(ox, oy, dx, dy, r, W, H, s)
    occ_mask = np.zeros(W * H, bool)
    free_mask = np.zeros(W * H, bool)
    occ_mask[hit] = True
    free_mask[free] = True
    free_mask &= ~occ_mask
    m_occ = np.where(occ_mask, np.float32(cfg["occ_mass"]), np.float32(0)).astype(np.float32)
    m_free = np.where(free_mask, np.float32(cfg["free_mass"]), np.float32(0)).astype(np.float32)
    out = dict(m_occ=m_occ, m_free=m_free)
    if cfg.get("radar_detections"):
        out.update(_radar_layer(sc, rng, m_occ, m_free))
    return out


def _radar_layer(sc: Scene, rng, m_occ, m_free) -> dict:
    """Radar detections on the boundaries of moving rectangles: range noise sigma_r along
    the line of sight, radial velocity with noise sigma_vr.  The detection cell carries
    p_A, the measured radial velocity and its standard deviation; its occupancy BBA
    becomes at least (radar_occ_mass, 0)."""
    cfg = sc.cfg
    W, H, s = cfg["width"], cfg["height"], cfg["cell_size"]
    ox, oy = sc.origin
    C = W * H
    p_A = np.zeros(C, np.float32)
    z_vr = np.zeros(C, np.float32)
    sig = np.ones(C, np.float32)
    movers = [b for b in sc.boxes if b.vx != 0.0 or b.vy != 0.0]
    if not movers:
        return dict(p_A=p_A, z_vr=z_vr, sigma_vr=sig)
    for _ in range(cfg["radar_detections"]):
        b = movers[int(rng.integers(len(movers)))]
        # a point on the rectangle's perimeter
        u = rng.uniform(0, 4)
        side = int(u)
        f = u - side
        lx = [-1 + 2 * f, 1, 1 - 2 * f, -1][side] * b.hl
        ly = [-1, -1 + 2 * f, 1, 1 - 2 * f][side] * b.hw
        c, s_ = math.cos(b.heading), math.sin(b.heading)
        px, py = b.cx + c * lx - s_ * ly, b.cy + s_ * lx + c * ly
        dxs, dys = px - ox, py - oy
        rr = math.hypot(dxs, dys)
        if rr <= 0:
            continue
        ex_, ey_ = dxs / rr, dys / rr
        rn = rr + rng.normal(0.0, cfg["radar_sigma_r"])
        hx, hy = ox + rn * ex_, oy + rn * ey_
        ix, iy = int(math.floor(hx / s)), int(math.floor(hy / s))
        if not (0 <= ix < W and 0 <= iy < H):
            continue
        k = iy * W + ix
        vr = b.vx * ex_ + b.vy * ey_ + rng.normal(0.0, cfg["radar_sigma_vr"])
        p_A[k] = cfg["radar_p_A"]
        z_vr[k] = vr
        sig[k] = cfg["radar_sigma_vr"]
        if m_occ[k] < cfg["radar_occ_mass"]:
            m_occ[k] = cfg["radar_occ_mass"]
            m_free[k] = 0.0
    return dict(p_A=p_A, z_vr=z_vr, sigma_vr=sig)


def frame_sequence(cfg: dict, n_frames: int, seed: int) -> list:
    """n_frames consecutive measurement grids of one seeded scene (scene seed = seed,
    noise seed = seed + 1)."""
    sc = make_scene(cfg, seed)
    rng = np.random.default_rng(seed + 1)
    grids = []
    for _ in range(n_frames):
        advance(sc, cfg["dt"])
        grids.append(measurement_grid(sc, rng))
    return grids


# --------------------------------------------------------------------------------------
# random states and grids for single-frame tests
# --------------------------------------------------------------------------------------
def random_measurement_grid(W: int, H: int, rng: np.random.Generator, radar: bool = False) -> dict:
    """Random BBAs: unknown, free, occupied and mixed cells, including the extremes
    (1, 0) and (0, 1)."""
    C = W * H
    kind = rng.choice(5, size=C, p=[0.45, 0.22, 0.2, 0.08, 0.05])
    m_occ = np.zeros(C, np.float32)
    m_free = np.zeros(C, np.float32)
    m_free[kind == 1] = rng.uniform(0.3, 0.8, (kind == 1).sum())
    m_occ[kind == 2] = rng.uniform(0.5, 0.95, (kind == 2).sum())
    a = rng.uniform(0, 1, (kind == 3).sum())
    b = rng.uniform(0, 1, (kind == 3).sum()) * (1 - a)
    m_occ[kind == 3] = a
    m_free[kind == 3] = b
    ext = np.flatnonzero(kind == 4)
    half = ext.size // 2
    m_occ[ext[:half]] = 1.0
    m_free[ext[half:]] = 1.0
    m_free = np.minimum(m_free, np.float32(1) - m_occ)
    out = dict(m_occ=m_occ, m_free=m_free)
    if radar:
        p_A = np.where((m_occ > 0) & (rng.uniform(0, 1, C) < 0.5), np.float32(0.9), np.float32(0))
        out.update(p_A=p_A.astype(np.float32),
                   z_vr=rng.normal(0, 5, C).astype(np.float32),
                   sigma_vr=rng.uniform(0.2, 2.0, C).astype(np.float32))
    return out


def bernoulli_grid(grid: dict, p_tp: float = 0.9, p_fp: float = 0.1, p_a: float = 0.9) -> dict:
    """Bernoulli observation per cell for the PHD/MIB filter from a lidar measurement grid of
    this module: a cell with a hit (m_occ > 0) is measured (z = 1); cells the beams saw (a hit
    or free space) get the sensor's true / false positive probabilities, unseen cells
    p_TP = p_FP = 0.5 (no information); p_c = 1 (clutter as likely as the object over the
    cell)."""
    occ = np.asarray(grid["m_occ"]) > 0
    seen = occ | (np.asarray(grid["m_free"]) > 0)
    f32 = np.float32
    return dict(z=occ.astype(f32), p_tp=np.where(seen, f32(p_tp), f32(0.5)).astype(f32),
                p_fp=np.where(seen, f32(p_fp), f32(0.5)).astype(f32),
                p_a=np.full(occ.size, f32(p_a)), p_c=np.ones(occ.size, f32))


def random_state(params: dict, rng: np.random.Generator, occupied_frac: float = 0.05,
                 frame: int = 7) -> dict:
    """A posterior-like particle state: most particles clustered in a few cells (per-cell
    weight sums spread over [0, 1.4] so that some exceed 1), a uniform remainder, a share
    of zero weights and some particles near or beyond the grid border."""
    W, H, s = params["width"], params["height"], params["cell_size"]
    nu, C = params["nu"], W * H
    k = max(1, int(C * occupied_frac))
    cells = rng.choice(C, size=k, replace=False)
    owner = rng.integers(0, k, nu)
    uniform = rng.uniform(0, 1, nu) < 0.15
    col = (cells[owner] % W).astype(np.float64)
    row = (cells[owner] // W).astype(np.float64)
    x = (col + rng.uniform(0, 1, nu)) * s
    y = (row + rng.uniform(0, 1, nu)) * s
    x[uniform] = rng.uniform(-0.02, 1.02, uniform.sum()) * W * s
    y[uniform] = rng.uniform(-0.02, 1.02, uniform.sum()) * H * s
    vx = rng.normal(0, 3, nu)
    vy = rng.normal(0, 3, nu)
    target = rng.uniform(0, 1.4, k)
    cnt = np.bincount(owner, minlength=k).astype(np.float64)
    w = target[owner] / np.maximum(cnt[owner], 1) * rng.uniform(0.5, 1.5, nu)
    w[uniform] = rng.uniform(0, 1e-3, uniform.sum())
    w[rng.uniform(0, 1, nu) < 0.05] = 0.0
    m_free = np.where(rng.uniform(0, 1, C) < 0.3, rng.uniform(0, 0.6, C), 0.0)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(x=f32(x), y=f32(y), vx=f32(vx), vy=f32(vy), w=f32(w), m_free=f32(m_free),
                frame=int(frame))


# --------------------------------------------------------------------------------------
# ground truth for the evaluation (object cells and velocities)
# --------------------------------------------------------------------------------------
def label_cells(sc: Scene) -> dict:
    """Cells whose centre lies inside an object at the scene's current time.

    Returns object (int32 [C]: 0 = no object, k = sc.boxes[k - 1]), dynamic (uint8 [C]:
    1 = a moving object, 2 = a static one, 0 = none) and the objects' true velocities
    (float64 [n, 2])."""
    W, H, s = int(sc.cfg["width"]), int(sc.cfg["height"]), float(sc.cfg["cell_size"])
    obj = np.zeros(W * H, np.int32)
    dyn = np.zeros(W * H, np.uint8)
    vel = np.zeros((len(sc.boxes), 2))
    for k, b in enumerate(sc.boxes):
        vel[k] = (b.vx, b.vy)
        r = math.hypot(b.hl, b.hw)
        c0, c1 = max(0, int((b.cx - r) / s)), min(W - 1, int((b.cx + r) / s))
        r0, r1 = max(0, int((b.cy - r) / s)), min(H - 1, int((b.cy + r) / s))
        if c0 > c1 or r0 > r1:
            continue
        cols = np.arange(c0, c1 + 1)
        rows = np.arange(r0, r1 + 1)
        X, Y = np.meshgrid((cols + 0.5) * s - b.cx, (rows + 0.5) * s - b.cy)
        c, sn = math.cos(b.heading), math.sin(b.heading)
        inside = (np.abs(c * X + sn * Y) <= b.hl) & (np.abs(-sn * X + c * Y) <= b.hw)
        idx = (rows[:, None] * W + cols[None, :])[inside]
        obj[idx] = k + 1
        dyn[idx] = 1 if (b.vx != 0.0 or b.vy != 0.0) else 2
    return dict(object=obj, dynamic=dyn, velocity=vel)


def frame_sequence_with_truth(cfg: dict, n_frames: int, seed: int) -> list:
    """As frame_sequence, each frame paired with its ground truth (label_cells)."""
    sc = make_scene(cfg, seed)
    rng = np.random.default_rng(seed + 1)
    out = []
    for _ in range(n_frames):
        advance(sc, cfg["dt"])
        out.append((measurement_grid(sc, rng), label_cells(sc)))
    return out
