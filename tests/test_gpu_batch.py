"""GPU tests of batched stepping (dog_batch_*): several independent filters of different
sizes advanced by one graph launch per frame must give, bit for bit, what stepping each
filter alone gives -- and hence what the oracle gives, which the parity tests establish for
single filters.  One filter switches from a lidar to a lidar + radar grid mid-run, which
re-captures the batch graph.
"""
import numpy as np
import pytest

from paper_1605_02406_b300 import scene

pytestmark = pytest.mark.gpu


def _params(W, H, nu, nu_b, seed, cell=0.5):
    return dict(width=W, height=H, cell_size=cell, nu=nu, nu_b=nu_b, p_S=0.99, p_B=0.02,
                alpha=0.9, sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0,
                sensor_x=W * cell * 0.5, sensor_y=H * cell * 0.4, seed=seed, flags=0)


CASES = [_params(64, 48, 3000, 600, 11), _params(96, 96, 8192, 2048, 12),
         _params(40, 40, 1000, 0, 13), _params(128, 80, 20000, 5000, 14, cell=0.25)]


def _setup(filters, rng_seed):
    rng = np.random.default_rng(rng_seed)
    grids = []
    for f, p in zip(filters, CASES):
        st = scene.random_state(p, rng, occupied_frac=0.1)
        f.set_state(st)
        gl = [scene.random_measurement_grid(p["width"], p["height"], rng) for _ in range(4)]
        gr = scene.random_measurement_grid(p["width"], p["height"], rng, radar=True)
        grids.append((gl, gr))
    return grids


def _snapshot(f):
    out = {k: v.copy() for k, v in f.cells().items()}
    out.update({"state." + k: np.asarray(v).copy() for k, v in f.get_state().items()})
    return out


@pytest.mark.parametrize("group_bytes", [0, 1 << 62, "pairs"])
def test_batch_equals_single_filters(group_bytes):
    """Every grouping: each filter its own branch, all four fused into one launch per phase,
    and two groups of two (fused phases in two concurrent branches)."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    shared = torch.cuda.Stream()
    batched = [DogFilter(p, stream=shared) for p in CASES]
    single = [DogFilter(p) for p in CASES]
    g_b = _setup(batched, 7)
    g_s = _setup(single, 7)
    batch = DogBatch(batched)
    if group_bytes == "pairs":
        w = [f.nbytes for f in batched]
        group_bytes = max(w[0] + w[1], w[2] + w[3])
        assert batch.set_group_bytes(group_bytes) == 2
    else:
        assert batch.set_group_bytes(group_bytes) == (4 if group_bytes == 0 else 1)
    dts = [0.1, 0.05, 0.1, 0.2]
    for frame in range(5):
        for i in range(len(CASES)):
            gl, gr = g_b[i]
            # filter 1 switches to a radar grid from frame 3 on (graph re-capture)
            grid = gr if (i == 1 and frame >= 3) else gl[frame % len(gl)]
            batched[i].set_measurement_grid(**grid)
            single[i].set_measurement_grid(**grid)
            single[i].step(dts[i])
        batch.step(dts)
        for i in range(len(CASES)):
            a, b = _snapshot(batched[i]), _snapshot(single[i])
            assert a.keys() == b.keys()
            for k in a:
                va, vb = np.asarray(a[k]), np.asarray(b[k])
                if va.dtype.kind == "f":
                    va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
                assert np.array_equal(va, vb), f"frame {frame}, filter {i}: {k} differs"
    batch.close()


def test_batch_rejects_mixed_streams_and_missing_grid():
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    a = DogFilter(CASES[0])
    b = DogFilter(CASES[2])  # its own stream
    with pytest.raises(N.DogError) as e:
        DogBatch([a, b])
    assert e.value.code == -1
    s = torch.cuda.Stream()
    c, d = DogFilter(CASES[0], stream=s), DogFilter(CASES[2], stream=s)
    batch = DogBatch([c, d])
    with pytest.raises(N.DogError) as e:
        batch.step([0.1, 0.1])  # no measurement grid yet
    assert e.value.code == -6
    rng = np.random.default_rng(3)
    for f, p in ((c, CASES[0]), (d, CASES[2])):
        f.set_measurement_grid(**scene.random_measurement_grid(p["width"], p["height"], rng))
    with pytest.raises(N.DogError) as e:
        batch.step([0.1, float("nan")])
    assert e.value.code == -1
    batch.step([0.1, 0.1])
    c.sync()
    batch.close()


def test_streams_in_a_mix_equal_streams_alone():
    """Filters stepped concurrently on their own CUDA streams, with their frames interleaved
    as the serving loop issues them, end in exactly the state each reaches alone."""
    import torch

    from paper_1605_02406_b300.filter import DogFilter
    mix = [DogFilter(p) for p in CASES]
    alone = [DogFilter(p) for p in CASES]
    g_m = _setup(mix, 9)
    g_a = _setup(alone, 9)
    order = [0, 2, 1, 3, 3, 0, 1, 2, 0, 3, 1, 1, 2, 0]  # an interleaving of requests
    seen = [0] * len(CASES)
    for i in order:  # issued back to back, no synchronisation in between
        mix[i].set_measurement_grid(**g_m[i][0][seen[i] % 4])
        mix[i].step(0.1)
        seen[i] += 1
    torch.cuda.synchronize()
    for i in range(len(CASES)):
        for t in range(order.count(i)):
            alone[i].set_measurement_grid(**g_a[i][0][t % 4])
            alone[i].step(0.1)
    for i in range(len(CASES)):
        a, b = _snapshot(mix[i]), _snapshot(alone[i])
        for k in a:
            va, vb = np.asarray(a[k]), np.asarray(b[k])
            if va.dtype.kind == "f":
                va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
            assert np.array_equal(va, vb), f"filter {i}: {k} differs"


def test_batch_with_ego_motion_equals_single_filters():
    """A filter with ego-motion compensation in a batch: the motion set before each batched
    step applies to that filter only, as when it is stepped alone."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    cases = [dict(CASES[0], flags=0x20), CASES[2]]
    shared = torch.cuda.Stream()
    batched = [DogFilter(p, stream=shared) for p in cases]
    single = [DogFilter(p) for p in cases]
    rng = np.random.default_rng(17)
    grids = []
    for fb, fs, p in zip(batched, single, cases):
        st = scene.random_state(p, rng, occupied_frac=0.1)
        fb.set_state(st)
        fs.set_state(st)
        grids.append([scene.random_measurement_grid(p["width"], p["height"], rng) for _ in range(3)])
    batch = DogBatch(batched)
    motions = [(0.5, 0.1, 0.03), None, (0.0, -0.4, -0.1)]
    for frame in range(3):
        for i in range(2):
            for f in (batched[i], single[i]):
                f.set_measurement_grid(**grids[i][frame])
                if i == 0 and motions[frame] is not None:
                    f.set_ego_motion(*motions[frame])
            single[i].step(0.1)
        batch.step([0.1, 0.1])
        for i in range(2):
            a, b = _snapshot(batched[i]), _snapshot(single[i])
            for k in a:
                va, vb = np.asarray(a[k]), np.asarray(b[k])
                if va.dtype.kind == "f":
                    va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
                assert np.array_equal(va, vb), f"frame {frame}, filter {i}: {k} differs"
    batch.close()


def test_batch_with_phdmib_filter_equals_single_filters():
    """A PHD/MIB filter (Sect. VI, Bernoulli observation) next to a DS filter in a batch."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    cases = [dict(CASES[1], flags=0x40), CASES[0]]
    shared = torch.cuda.Stream()
    batched = [DogFilter(p, stream=shared) for p in cases]
    single = [DogFilter(p) for p in cases]
    rng = np.random.default_rng(19)
    grids = []
    for fb, fs, p in zip(batched, single, cases):
        st = scene.random_state(p, rng, occupied_frac=0.1)
        fb.set_state(st)
        fs.set_state(st)
        grids.append([scene.random_measurement_grid(p["width"], p["height"], rng) for _ in range(3)])
    grids[0] = [scene.bernoulli_grid(g) for g in grids[0]]
    batch = DogBatch(batched)
    for frame in range(3):
        for i in range(2):
            for f in (batched[i], single[i]):
                if i == 0:
                    f.set_bernoulli_grid(**grids[i][frame])
                else:
                    f.set_measurement_grid(**grids[i][frame])
            single[i].step(0.1)
        batch.step([0.1, 0.1])
        for i in range(2):
            a, b = _snapshot(batched[i]), _snapshot(single[i])
            for k in a:
                va, vb = np.asarray(a[k]), np.asarray(b[k])
                if va.dtype.kind == "f":
                    va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
                assert np.array_equal(va, vb), f"frame {frame}, filter {i}: {k} differs"
    batch.close()


def test_sessions_admit_waiting_streams_and_match_streams_alone():
    """Streams that come and go (serve.run_sessions): with room for three at once, the later
    streams wait and are admitted as earlier ones leave; every served stream's cells equal,
    bit for bit, the same stream stepped alone for as many frames."""
    from paper_1605_02406_b300 import serve
    from paper_1605_02406_b300.filter import DogFilter

    base = scene.serving_stream_configs(12)
    cfgs = [dict(c, width=64 if k % 2 else 96, height=64, nu=16 * (64 if k % 2 else 96) * 64)
            for k, c in enumerate(base)]
    for c in cfgs:
        c["nu_b"] = c["nu"] // 4
    room = 3 * max(serve.stream_need(c) for c in cfgs)
    r = serve.run_sessions(seconds=1.0, budget_gb=room / 1e9, slots=3, mean_session_s=0.2,
                           connect_s=0.3, cfgs=cfgs, keep=True)
    assert r["most_streams_at_once"] <= 3
    assert r["streams_served"] + r["streams_never_admitted"] == len(cfgs)
    assert r["admitted_after_waiting"] >= 1 and r["streams_served"] >= 4
    checked = 0
    for k, s in r["served"].items():
        if s["frames"] == 0:
            continue
        g = DogFilter(scene.filter_params(cfgs[k], seed=500 + k))
        g.set_measurement_grid(**s["grid"])
        for _ in range(s["frames"]):
            g.step(0.1)
        alone = g.cells(["m_occ", "m_free", "p_occ"])
        g.close()
        for f in ("m_occ", "m_free", "p_occ"):
            assert np.array_equal(alone[f], s["cells"][f]), (k, f)
        checked += 1
    assert checked >= 4


def test_batch_captures_again_after_configuration_changes_and_across_batches():
    """Each filter's description lives in a slot of its workspace, written when a batch
    captures: a filter shared by two batches stepped in turn, and a filter whose sort
    configuration changes between batched frames, must still equal the same filters stepped
    alone, bit for bit."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    cases = CASES[:2] + [dict(CASES[3], flags=0x80)]  # the last one may take a third pass
    shared = torch.cuda.Stream()
    batched = [DogFilter(p, stream=shared) for p in cases]
    single = [DogFilter(p) for p in cases]
    rng = np.random.default_rng(3)
    grids = []
    for fb, fs, p in zip(batched, single, cases):
        st = scene.random_state(p, rng, occupied_frac=0.1)
        fb.set_state(st)
        fs.set_state(st)
        grids.append([scene.random_measurement_grid(p["width"], p["height"], rng) for _ in range(3)])
    one = DogBatch(batched)                   # all three
    two = DogBatch([batched[1], batched[2]])  # two of them again
    plan = [(one, [0, 1, 2]), (two, [1, 2]), (one, [0, 1, 2]), ("config", None), (one, [0, 1, 2]),
            (two, [1, 2]), ("config", None), (two, [1, 2]), (one, [0, 1, 2])]
    configs = iter([(3, 2), (2, 8)])
    for step, (batch, members) in enumerate(plan):
        if batch == "config":  # a new sort configuration for the shared filter with room for it
            passes, ct = next(configs)
            batched[2].set_sort_config(passes, ct)
            single[2].set_sort_config(passes, ct)
            continue
        for i in members:
            g = grids[i][step % 3]
            batched[i].set_measurement_grid(**g)
            single[i].set_measurement_grid(**g)
            single[i].step(0.1)
        batch.step([0.1] * len(members))
        for i in members:
            a, b = _snapshot(batched[i]), _snapshot(single[i])
            for k in a:
                va, vb = np.asarray(a[k]), np.asarray(b[k])
                if va.dtype.kind == "f":
                    va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
                assert np.array_equal(va, vb), f"step {step}, filter {i}: {k} differs"
    assert batched[2].sort_config()["passes"] == 2
    one.close()
    two.close()


def test_batch_limits():
    import torch

    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    s = torch.cuda.Stream()
    f = DogFilter(CASES[2], stream=s)
    with pytest.raises(N.DogError) as e:
        DogBatch([f, f])  # a filter listed twice
    assert e.value.code == -1
    with pytest.raises(N.DogError) as e:
        N.dog_batch_create([f.h] * 129)
    assert e.value.code in (-1, -7)


def test_batch_autotune_steps_real_frames():
    """dog_batch_autotune times groupings on real frames: afterwards every filter equals the
    same filter stepped alone as many times, and later batched frames stay equal."""
    import torch

    from paper_1605_02406_b300.filter import DogBatch, DogFilter
    shared = torch.cuda.Stream()
    batched = [DogFilter(p, stream=shared) for p in CASES]
    single = [DogFilter(p) for p in CASES]
    g_b = _setup(batched, 9)
    _setup(single, 9)
    for i in range(len(CASES)):
        batched[i].set_measurement_grid(**g_b[i][0][0])
        single[i].set_measurement_grid(**g_b[i][0][0])
    batch = DogBatch(batched)
    before = batched[0].get_state()["frame"]
    choice = batch.autotune(0.1, frames=1)
    assert choice["groups"] >= 1
    frames = batched[0].get_state()["frame"] - before
    assert frames >= 2  # at least one capture frame and one timed frame per grouping tried
    for i in range(len(CASES)):
        for _ in range(frames):
            single[i].step(0.1)
    batch.step(0.1)
    for i in range(len(CASES)):
        single[i].step(0.1)
        a, b = _snapshot(batched[i]), _snapshot(single[i])
        for k in a:
            va, vb = np.asarray(a[k]), np.asarray(b[k])
            if va.dtype.kind == "f":
                va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
            assert np.array_equal(va, vb), f"filter {i}: {k} differs"
    batch.close()
