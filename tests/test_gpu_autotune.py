"""GPU tests of the sort configuration and its autotuning: every configuration the workspace
holds (number of digit passes, sort tiles per counting block) sorts to the same order, so
the filter's results are the same bit for bit whatever is chosen; dog_autotune keeps the
outputs unchanged and its choice is cached for the size class."""
import numpy as np
import pytest

from paper_1605_02406_b300 import scene

pytestmark = pytest.mark.gpu

AUTOTUNE = 0x80


def _params(flags=AUTOTUNE, seed=21):
    # 64 x 64 cells: 12-bit keys, 2 passes by default (3 with the autotune buffers); 4 tiles
    return dict(width=64, height=64, cell_size=0.5, nu=3 * 4096 + 1234, nu_b=2048 + 77, p_S=0.99,
                p_B=0.02, alpha=0.9, sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0,
                sensor_x=16.0, sensor_y=12.0, seed=seed, flags=flags)


def _run(f, st, grids, frames):
    f.set_state(st)
    for k in range(frames):
        f.set_measurement_grid(**grids[k % len(grids)])
        f.step(0.1)
    out = {k: np.asarray(v).copy() for k, v in f.cells().items()}
    out.update({"state." + k: np.asarray(v).copy() for k, v in f.get_state().items()})
    out["perm"] = f.debug("PERM").copy()
    return out


def _same(a, b, what):
    for k in a:
        va, vb = np.asarray(a[k]), np.asarray(b[k])
        if va.dtype.kind == "f":
            va, vb = va.astype(np.float32).view(np.uint32), vb.astype(np.float32).view(np.uint32)
        assert np.array_equal(va, vb), f"{what}: {k} differs"


def _inputs(seed):
    rng = np.random.default_rng(seed)
    p = _params()
    st = scene.random_state(p, rng, occupied_frac=0.1)
    grids = [scene.random_measurement_grid(64, 64, rng) for _ in range(3)]
    return st, grids


def test_every_sort_configuration_gives_the_same_results():
    from paper_1605_02406_b300.filter import DogFilter
    st, grids = _inputs(4)
    ref = _run(DogFilter(_params(flags=0)), st, grids, 3)
    tried = 0
    for passes in (2, 3):
        for ct in (1, 2, 4, 8):
            f = DogFilter(_params())
            f.set_sort_config(passes, ct)
            assert f.sort_config() == {"passes": passes, "digit_bits": -(-12 // passes), "count_tiles": ct}
            _same(_run(f, st, grids, 3), ref, f"passes {passes}, {ct} tiles per block")
            tried += 1
    assert tried == 8


def test_autotune_keeps_results_and_caches_the_choice():
    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter
    st, grids = _inputs(5)
    ref = DogFilter(_params(flags=0, seed=22))
    f = DogFilter(_params(seed=22))
    with pytest.raises(N.DogError) as e:  # nothing to time before the first step
        f.autotune()
    assert e.value.code == -6
    for g in (ref, f):
        g.set_state(st)
        g.set_measurement_grid(**grids[0])
        g.step(0.1)
    cfg = f.autotune()
    assert cfg["passes"] in (2, 3) and cfg["count_tiles"] in (1, 2, 4, 8)
    for k in range(1, 4):
        for g in (ref, f):
            g.set_measurement_grid(**grids[k % 3])
            g.step(0.1)
    a, b = ({k: np.asarray(v).copy() for k, v in g.cells().items()} for g in (f, ref))
    _same(a, b, "after autotuning")
    # a filter of the same size class created later starts from the tuned configuration
    assert DogFilter(_params(seed=23)).sort_config() == cfg


def test_sort_configuration_errors():
    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter
    plain = DogFilter(_params(flags=0, seed=24))
    with pytest.raises(N.DogError) as e:  # one pass more needs the autotune buffers
        plain.set_sort_config(3, 1)
    assert e.value.code == -7
    with pytest.raises(N.DogError) as e:
        plain.set_sort_config(1, 1)  # 12-bit keys need two passes of at most 11 bits
    assert e.value.code == -7
    with pytest.raises(N.DogError) as e:
        plain.set_sort_config(2, 3)
    assert e.value.code == -7
    plain.set_sort_config(2, 4)
