"""``DogFilter``: one DS-PHD/MIB filter on one GPU, a thin object over the C ABI.

PyTorch provides the device workspace and the CUDA stream; every step of the recursion
runs in ``libdog.so``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N


def _ptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


class DogFilter:
    def __init__(self, params: dict, device: str = "cuda:0", stream: torch.cuda.Stream | None = None):
        self.params = dict(params)
        self.device = torch.device(device)
        self.cparams = N.make_params(params)
        self.nbytes = N.dog_workspace_bytes(self.cparams)
        self.C = int(params["width"]) * int(params["height"])
        self.nu, self.nu_b = int(params["nu"]), int(params["nu_b"])
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self._ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self._ws_ptr = (_ptr(self._ws) + 255) // 256 * 256
            # the workspace allocation is ordered before the library's first use of it
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            self.h = N.dog_create(self.cparams, self._ws_ptr, self.nbytes, self.stream.cuda_stream)
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            N.dog_destroy(self.h)  # waits for the filter's stream first
            self.h = None
            self._ws = None  # the workspace goes back to torch's allocator
            self._keep = []  # and so do the grid buffers recorded on the filter's stream

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_measurement_grid(self, m_occ, m_free, p_A=None, z_vr=None, sigma_vr=None):
        """numpy arrays (host) or CUDA tensors (device) of C float32 values each."""
        arrs = dict(m_occ=m_occ, m_free=m_free, p_A=p_A, z_vr=z_vr, sigma_vr=sigma_vr)
        self._set_grid(arrs, N.dog_set_measurement_grid)

    def set_bernoulli_grid(self, z, p_tp, p_fp, p_a, p_c):
        """Bernoulli observation per cell (filters created with DOG_FULL): numpy arrays
        (host) or CUDA tensors (device) of C float32 values each."""
        self._set_grid(dict(z=z, p_tp=p_tp, p_fp=p_fp, p_a=p_a, p_c=p_c), N.dog_set_bernoulli_grid)

    def _set_grid(self, arrs, call):
        first = next(a for a in arrs.values() if a is not None)
        on_dev = isinstance(first, torch.Tensor) and first.is_cuda
        ptrs, keep = {}, []
        for k, a in arrs.items():
            if a is None:
                continue
            if on_dev:
                t = a.to(self.device, torch.float32).contiguous().view(-1)
                assert t.numel() == self.C
                keep.append(t)
                ptrs[k] = _ptr(t)
            else:
                h = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1))
                assert h.size == self.C
                keep.append(h)
                ptrs[k] = h.ctypes.data
        if on_dev:
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            for t in keep:
                t.record_stream(self.stream)
        call(self.h, ptrs, N.DOG_DEVICE if on_dev else N.DOG_HOST)
        self._keep = keep

    def autotune(self) -> dict:
        """Time the sort configurations on the last step's keys and keep the fastest."""
        N.dog_autotune(self.h)
        return self.sort_config()

    def sort_config(self) -> dict:
        return N.dog_sort_config(self.h)

    def set_sort_config(self, passes: int, count_tiles: int):
        N.dog_set_sort_config(self.h, passes, count_tiles)

    def set_ego_motion(self, dx: float, dy: float, dyaw: float):
        """Vehicle motion since the previous frame (filters created with DOG_EGO): moved by
        (dx, dy) m in the previous grid's axes, turned by dyaw rad about the sensor."""
        N.dog_set_ego_motion(self.h, dx, dy, dyaw)

    def step(self, dt: float):
        N.dog_step(self.h, dt)

    def sync(self):
        N.dog_sync(self.h)

    def cells(self, fields=None) -> dict:
        fields = fields or N.CELL_FIELDS
        out = {k: np.empty(self.C, np.float32) for k in fields}
        N.dog_get_cells(self.h, {k: v.ctypes.data for k, v in out.items()}, N.DOG_HOST)
        return out

    def cells_into(self, out: dict, device: bool):
        """Copy cell outputs into caller-owned buffers (CUDA tensors or pinned tensors)."""
        N.dog_get_cells(self.h, {k: _ptr(v) for k, v in out.items()},
                        N.DOG_DEVICE if device else N.DOG_HOST)

    def get_state(self) -> dict:
        st = {k: np.empty(self.nu, np.float32) for k in ("x", "y", "vx", "vy", "w")}
        st["m_free"] = np.empty(self.C, np.float32)
        fr = N.dog_get_state(self.h, {k: v.ctypes.data for k, v in st.items()}, N.DOG_HOST)
        st["frame"] = fr
        return st

    def set_state(self, st: dict):
        arrs = {k: np.ascontiguousarray(np.asarray(st[k], dtype=np.float32).reshape(-1))
                for k in ("x", "y", "vx", "vy", "w", "m_free")}
        N.dog_set_state(self.h, {k: v.ctypes.data for k, v in arrs.items()}, N.DOG_HOST,
                        int(st.get("frame", 0)))

    def debug(self, name: str) -> np.ndarray:
        which = N.DOG_DBG[name]
        if name == "SCALARS":
            out = np.empty(4, np.uint64)
        else:
            n = {"CELL_START": self.C, "CELL_END": self.C, "SUM_W": self.C, "SUM_GW": self.C,
                 "M_OCC_PRED": self.C, "MU_A": self.C, "MU_UA": self.C}.get(name)
            if n is None:
                n = self.nu_b if name.startswith("BIRTH") else self.nu
            dt = {"KEY": np.uint32, "PERM": np.uint32, "CELL_START": np.uint32, "CELL_END": np.uint32,
                  "SUM_W": np.uint64, "SUM_GW": np.uint64, "BIRTH_CELL": np.uint32,
                  "BIRTH_ASSOC": np.uint32, "RESAMPLE_SRC": np.uint32}.get(name, np.float32)
            out = np.empty(max(n, 1), dt)[:n]
        if out.size:
            N.dog_get_debug(self.h, which, out.ctypes.data, N.DOG_HOST)
        return out

    def profile(self):
        return N.dog_profile_read(self.h)

    def kernels_per_step(self) -> int:
        return N.dog_kernels_per_step(self.h)


class DogBatch:
    """Several ``DogFilter`` objects created on one stream, advanced together by one graph
    launch per frame (``dog_batch_step``)."""

    def __init__(self, filters: list):
        self.filters = list(filters)
        self.h = N.dog_batch_create([f.h for f in self.filters])

    def step(self, dts) -> None:
        if not hasattr(dts, "__len__"):
            dts = [dts] * len(self.filters)
        N.dog_batch_step(self.h, dts)

    def autotune(self, dts, frames: int = 2) -> dict:
        """Time the candidate groupings on real frames (each advances every filter) and keep
        the fastest; returns the choice."""
        if not hasattr(dts, "__len__"):
            dts = [dts] * len(self.filters)
        gb = N.dog_batch_autotune(self.h, dts, frames)
        return {"group_bytes": gb, "groups": N.dog_batch_groups(self.h)}

    def set_group_bytes(self, group_bytes: int) -> int:
        """Group consecutive filters up to group_bytes of workspace; returns the groups."""
        N.dog_batch_set_group_bytes(self.h, group_bytes)
        return N.dog_batch_groups(self.h)

    def close(self):
        if getattr(self, "h", None):
            N.dog_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _main():
    """Run one filter on a seeded synthetic workload for a few frames (CUDA-graph path): the
    program the profiler captures of single kernels run."""
    import argparse
    import time

    from . import scene

    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--workload", default="automotive_1024", choices=sorted(scene.CONFIGS))
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--sort", default=None, help="passes,count_tiles (default: the library's choice)")
    ap.add_argument("--seed", type=int, default=1002)
    a = ap.parse_args()
    cfg = scene.CONFIGS[a.workload]
    grids = scene.frame_sequence(cfg, a.frames, a.seed)
    dev = [{k: torch.tensor(v, device="cuda") for k, v in g.items()} for g in grids]
    f = DogFilter(scene.filter_params(cfg))
    if a.sort:
        passes, count_tiles = (int(x) for x in a.sort.split(","))
        f.set_sort_config(passes, count_tiles)
    t0 = time.perf_counter()
    for g in dev:
        f.set_measurement_grid(**g)
        f.step(cfg["dt"])
    f.sync()
    dt = time.perf_counter() - t0
    print(f"{a.workload}: {a.frames} frames in {dt * 1e3:.1f} ms (first frames include graph capture); "
          f"sort {f.sort_config()}")
    f.close()


if __name__ == "__main__":
    _main()
