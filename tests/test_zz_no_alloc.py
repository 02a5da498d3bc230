"""GPU test of dog_assign_cells_noalloc, the allocation-free particle-to-cell assignment.

That entry point exists for callers that cannot allocate device memory (code running
where cudaMalloc is forbidden or unavailable: host callbacks, real-time threads that must
not take the allocator's locks, processes whose device memory belongs to another
framework's pool).  Its scratch lives in one fixed array inside the library, shared by all
calls.  The test feeds it the cell indices that dog_step computed for a frame and checks
that it returns the same sort permutation and cell ranges that dog_step itself produced,
on two calls in a row of different sizes (the second must not see the first's leftovers).
Keys outside [0, num_cells) -- which the filter never produces but a caller may pass -- must
sort after every valid key, in input order, and belong to no cell's range; that case and the
largest accepted sizes are checked against numpy's stable argsort and a brute-force scan.
This file is collected last so that a failure here stops a `-x` run only after every other
test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1605_02406_b300 import scene

pytestmark = pytest.mark.gpu

RECORD = 0x4


def _frame_keys(params, seed):
    """Run one dog_step from a seeded random state; return its keys, perm and ranges."""
    from paper_1605_02406_b300.filter import DogFilter
    rng = np.random.default_rng(seed)
    g = DogFilter(dict(params, flags=RECORD))
    g.set_state(scene.random_state(params, rng, occupied_frac=0.2))
    grid = scene.random_measurement_grid(params["width"], params["height"], rng)
    g.set_measurement_grid(**grid)
    g.step(0.1)
    out = {k: g.debug(k) for k in ("KEY", "PERM", "CELL_START", "CELL_END")}
    g.close()
    return out


def _noalloc(keys_np, num_cells):
    import torch

    from paper_1605_02406_b300 import native as N
    stream = torch.cuda.current_stream()
    keys = torch.from_numpy(np.ascontiguousarray(keys_np, dtype=np.uint32).view(np.int32)).cuda()
    n = keys_np.size
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    start = torch.full((num_cells,), -1, dtype=torch.int32, device="cuda")
    end = torch.full((num_cells,), -1, dtype=torch.int32, device="cuda")
    N.dog_assign_cells_noalloc(keys.data_ptr(), n, num_cells, perm.data_ptr(), start.data_ptr(),
                               end.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    view = lambda t: t.cpu().numpy().view(np.uint32)
    return view(perm)[:n], view(start), view(end)


def test_noalloc_assignment_matches_dog_step_twice():
    cases = [
        dict(scene.filter_params(scene.CONFIGS["plain_128"])),                        # 65,536 particles, 128x128
        dict(scene.filter_params(scene.CONFIGS["plain_128"]), width=300, height=200,  # ragged, other size
             nu=3 * 4096 + 777, nu_b=1000, cell_size=0.3),
    ]
    for seed, p in enumerate(cases):
        ref = _frame_keys(p, seed)
        C = p["width"] * p["height"]
        perm, start, end = _noalloc(ref["KEY"], C)
        assert np.array_equal(perm, ref["PERM"]), f"call {seed}: permutation differs"
        assert np.array_equal(start, ref["CELL_START"]), f"call {seed}: cell starts differ"
        assert np.array_equal(end, ref["CELL_END"]), f"call {seed}: cell ends differ"


def _reference(keys, num_cells):
    """Stable order with every key >= num_cells treated as the sentinel num_cells, and the
    half-open range of each cell found by scanning the sorted keys."""
    sk = np.minimum(keys.astype(np.int64), num_cells)
    perm = np.argsort(sk, kind="stable").astype(np.uint32)
    ks = sk[perm]
    start = np.zeros(num_cells, np.uint32)
    end = np.zeros(num_cells, np.uint32)
    heads = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    tails = np.r_[heads[1:], ks.size]
    for h, t in zip(heads, tails):
        if ks[h] < num_cells:
            start[ks[h]], end[ks[h]] = h, t
    return perm, start, end


def _check_against_reference(keys, num_cells, what):
    perm, start, end = _noalloc(keys, num_cells)
    rp, rs, re_ = _reference(keys, num_cells)
    assert np.array_equal(perm, rp), f"{what}: permutation differs"
    assert np.array_equal(start, rs), f"{what}: cell starts differ"
    assert np.array_equal(end, re_), f"{what}: cell ends differ"
    # every particle with a valid key lies in its cell's range
    k = keys.astype(np.int64)
    pos = np.empty(keys.size, np.int64)
    pos[perm] = np.arange(keys.size)
    ok = k < num_cells
    assert np.all((rs[k[ok]] <= pos[ok]) & (pos[ok] < re_[k[ok]])), what


def test_noalloc_keys_beyond_the_grid_sort_last_in_no_range():
    rng = np.random.default_rng(11)
    num_cells, n = 1000, 3 * 4096 + 123
    keys = rng.integers(0, num_cells, n).astype(np.uint32)
    bad = rng.random(n) < 0.1
    keys[bad] = rng.choice(np.array([num_cells, num_cells + 33, 1 << 20, (1 << 31) | 5, 0xFFFFFFFF],
                                    dtype=np.uint32), int(bad.sum()))
    _check_against_reference(keys, num_cells, "1000 cells, 10 % of keys out of range")
    # a cell index just below the limit next to keys just above it (133 = 100 + 33 shares its
    # low bits with cell 5, which must keep its own range)
    keys2 = np.array([5, 133, 5, 99, 100, 0, 133, 5], np.uint32)
    _check_against_reference(keys2, 100, "100 cells, keys sharing low bits with cell 5")


def test_noalloc_at_its_largest_sizes():
    import torch

    from paper_1605_02406_b300 import native as N
    rng = np.random.default_rng(12)
    n, C = N.DOG_NOALLOC_MAX_PARTICLES, N.DOG_NOALLOC_MAX_CELLS
    keys = rng.integers(0, C + 64, n).astype(np.uint32)  # a few beyond the grid
    keys[: n // 8] = np.sort(keys[: n // 8])             # a nearly sorted stretch
    _check_against_reference(keys, C, "largest sizes")
    torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    from paper_1605_02406_b300 import native as N
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    p = buf.data_ptr()
    with pytest.raises(N.DogError) as e:
        N.dog_assign_cells_noalloc(p, N.DOG_NOALLOC_MAX_PARTICLES + 1, 4, p, p, p, s)
    assert e.value.code == -7
    with pytest.raises(N.DogError) as e:
        N.dog_assign_cells_noalloc(p, 4, N.DOG_NOALLOC_MAX_CELLS + 1, p, p, p, s)
    assert e.value.code == -7
