"""GPU test at the largest sizes the C ABI accepts: C = 4096 x 4095 cells (C < 2^24, keys of
24 bits, three sort passes), nu = 2^25 - 1 persistent and 2^23 newborn particles, two frames
from a random posterior (the first from weights as given, the second from a resampled
posterior).  The oracle would take minutes per frame here, so each frame is checked through
properties that hold at any size and fail on a wrong index, a lost particle or a wrong sum:

  * Alg. 2: PERM is a permutation, the keys in sorted order never decrease, and particles of
    one cell keep their index order (a stable sort);
  * Eq. DS_particle_sum_pred: every cell's 2^-40 fixed-point weight sum equals the exact
    integer sum of the truncated weights of the particles the sort put in it;
  * Alg. 3: masses in [0, 1] and m_O + m_F <= 1 (up to a few binary32 ulps), rho_p =
    m_O - rho_b in binary32;
  * Alg. 7: the resampling sources never decrease, stay below nu + nu_b, the total W equals
    the exact sum of the quantised joint weights, and systematic resampling gives source j
    floor or ceil of nu q_j / W outputs.
"""
import numpy as np
import pytest

from paper_1605_02406_b300 import scene

pytestmark = pytest.mark.gpu


def _q40(w):
    # the truncating 2^-40 quantisation (exact in binary64 for binary32 inputs)
    return np.floor(np.asarray(w, np.float64) * 2.0 ** 40).astype(np.uint64)


def test_maximum_sizes():
    from paper_1605_02406_b300.filter import DogFilter
    W, H = 4096, 4095
    p = dict(width=W, height=H, cell_size=0.1, nu=(1 << 25) - 1, nu_b=1 << 23, p_S=0.99, p_B=0.02,
             alpha=0.9, sigma_pos=0.1, sigma_vel=2.0, sigma_birth_vel=4.0, sensor_x=W * 0.05,
             sensor_y=H * 0.05, seed=31, flags=0)
    nu, nu_b = p["nu"], p["nu_b"]
    rng = np.random.default_rng(31)
    st = scene.random_state(p, rng, occupied_frac=0.002)
    grid = scene.random_measurement_grid(W, H, rng)
    g = DogFilter(p)
    g.set_state(st)
    for frame in range(2):
        g.set_measurement_grid(**grid)
        g.step(0.1)
        what = f"frame {frame}: "
        # sort
        key, perm = g.debug("KEY"), g.debug("PERM")
        assert perm.max() < nu and np.bincount(perm, minlength=nu).max() == 1, what + "PERM"
        ks = key[perm]
        assert (ks[1:] >= ks[:-1]).all(), what + "sorted keys"
        same = ks[1:] == ks[:-1]
        assert (perm[1:][same] > perm[:-1][same]).all(), what + "stability"
        # per-cell fixed-point sums
        q = _q40(g.debug("PRED_W"))[perm]
        starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
        S = g.debug("SUM_W")
        assert np.array_equal(S[ks[starts]], np.add.reduceat(q, starts)), what + "SUM_W"
        empty = np.ones(W * H, bool)
        empty[ks[starts]] = False
        assert not S[empty].any(), what + "SUM_W of empty cells"
        # masses
        c = g.cells(["m_occ", "m_free", "rho_p", "rho_b"])
        mO, mF, rp, rb = (c[k] for k in ("m_occ", "m_free", "rho_p", "rho_b"))
        # Dempster's rule evaluated in binary32 (as the oracle's mirror does) can land one ulp
        # above 1, e.g. m_O = 1 + 2^-23 for a measurement z_O = 1: a few ulps of slack
        top = 1.0 + 2.0 ** -21
        bad = ~((mO >= 0) & (mO <= top) & (mF >= 0) & (mF <= top))
        assert not bad.any(), (what + "mass range", int(bad.sum()), mO[bad][:5].tolist(), mF[bad][:5].tolist())
        assert (mO.astype(np.float64) + mF <= top).all(), what + "m_O + m_F"
        assert np.array_equal((mO - rb).view(np.uint32), rp.view(np.uint32)), what + "rho_p"
        # resampling
        src = g.debug("RESAMPLE_SRC")
        assert (src[1:] >= src[:-1]).all() and src.max() < nu + nu_b, what + "sources"
        qj = np.concatenate([_q40(g.debug("W_NORM")), _q40(g.debug("BIRTH_W"))])
        Wt = int(qj.sum(dtype=np.uint64))  # < 2^64: at most C masses of 1 at scale 2^40
        assert Wt == int(g.debug("SCALARS")[1]), what + "W_total"
        expect = qj.astype(np.float64) * (nu / Wt)
        cnt = np.bincount(src, minlength=nu + nu_b)
        assert (np.abs(cnt - expect) < 1.0 + 1e-6).all(), what + "output counts"
    g.close()
