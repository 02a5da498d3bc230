"""GPU test of dog_assign_cells_noalloc, the allocation-free particle-to-cell assignment.

That entry point exists for callers that cannot allocate device memory (code running
where cudaMalloc is forbidden or unavailable: host callbacks, real-time threads that must
not take the allocator's locks, processes whose device memory belongs to another
framework's pool).  Its scratch lives in one fixed array inside the library, shared by all
calls.  The test feeds it the cell indices that dog_step computed for a frame and checks
that it returns the same sort permutation and cell ranges that dog_step itself produced,
on two calls in a row of different sizes (the second must not see the first's leftovers).
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
    keys = torch.from_numpy(keys_np.astype(np.int32).view(np.int32)).cuda()
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
