"""The oracle's forced-decision mode (used to measure the binary32 path's arithmetic error
against binary64 on one and the same Monte Carlo run).  Pinned by two consistency checks:
forcing a run's own decisions on a twin run changes nothing, and a binary64 run forced with
the binary32 mirror's decisions reproduces every integer result of the mirror (cells, sort
order, newborn slots, resampled sources) while its real-valued results stay close."""
import numpy as np
import pytest

from oracle import OracleFilter
from paper_1605_02406_b300 import scene


def _params(**kw):
    p = dict(width=24, height=20, cell_size=0.5, nu=16384, nu_b=4096, p_S=0.99, p_B=0.02, alpha=0.9,
             sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0, sensor_x=6.0, sensor_y=5.0, seed=77, flags=0)
    p.update(kw)
    return p


@pytest.mark.parametrize("radar", [False, True])
def test_forcing_a_runs_own_decisions_changes_nothing(radar):
    p = _params()
    rng = np.random.default_rng(1)
    st = scene.random_state(p, rng, occupied_frac=0.2)
    grids = [scene.random_measurement_grid(24, 20, rng, radar=radar) for _ in range(4)]
    a, b = OracleFilter(p, "f32"), OracleFilter(p, "f32")
    a.set_state(st)
    b.set_state(st)
    for g in grids:
        a.set_measurement_grid(**g)
        a.step(0.1)
        b.set_measurement_grid(**g)
        b.force_decisions(a.decisions())
        b.step(0.1)
        ca, cb = a.cells(), b.cells()
        for k in ca:
            assert np.array_equal(ca[k], cb[k]), k
        sa, sb = a.get_state(), b.get_state()
        for k in ("x", "y", "vx", "vy", "w"):
            assert np.array_equal(sa[k], sb[k]), k


def test_binary64_run_with_the_mirrors_decisions():
    p = _params()
    rng = np.random.default_rng(2)
    st = scene.random_state(p, rng, occupied_frac=0.2)
    grids = [scene.random_measurement_grid(24, 20, rng) for _ in range(5)]
    o32, o64 = OracleFilter(p, "f32"), OracleFilter(p, "f64")
    o32.set_state(st)
    o64.set_state(st)
    for g in grids:
        o32.set_measurement_grid(**g)
        o32.step(0.1)
        d = o32.decisions()
        o64.set_measurement_grid(**g)
        o64.force_decisions(d)
        o64.step(0.1)
        i32, i64 = o32.intermediates(), o64.intermediates()
        for k in ("key", "perm", "cell_start", "cell_end", "birth_cell", "birth_assoc", "resample_src", "in_grid"):
            assert np.array_equal(i32[k], i64[k]), k
        c32, c64 = o32.cells(), o64.cells()
        for k in ("m_occ", "m_free", "rho_p", "rho_b"):
            assert np.abs(c32[k].astype(np.float64) - c64[k]).max() < 1e-4, k
