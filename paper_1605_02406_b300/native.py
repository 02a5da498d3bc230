"""ctypes binding of the C ABI in ``include/dog.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all computation happens in
``libdog.so``.  Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdog.so")

DOG_OK = 0
DOG_ERR = {-1: "DOG_ERR_INVALID_ARG", -2: "DOG_ERR_WORKSPACE_TOO_SMALL", -3: "DOG_ERR_CUDA",
           -4: "DOG_ERR_DEVICE", -5: "DOG_ERR_INPUT", -6: "DOG_ERR_BAD_STATE",
           -7: "DOG_ERR_UNSUPPORTED"}
DOG_NO_RESAMPLE, DOG_RECORD, DOG_NO_GRAPH, DOG_PROFILE = 0x2, 0x4, 0x8, 0x10
DOG_EGO, DOG_FULL, DOG_AUTOTUNE = 0x20, 0x40, 0x80
DOG_HOST, DOG_DEVICE, DOG_HOST_ASYNC = 0, 1, 2

DBG = ["PRED_X", "PRED_Y", "PRED_VX", "PRED_VY", "PRED_W", "KEY", "PERM", "CELL_START",
       "CELL_END", "SUM_W", "SUM_GW", "M_OCC_PRED", "MU_A", "MU_UA", "W_NORM", "BIRTH_X",
       "BIRTH_Y", "BIRTH_VX", "BIRTH_VY", "BIRTH_W", "BIRTH_CELL", "BIRTH_ASSOC",
       "RESAMPLE_SRC", "SCALARS"]
DOG_DBG = {n: k for k, n in enumerate(DBG)}

# entry points the header declares (checked by the CPU test suite)
SYMBOLS = ["dog_workspace_bytes", "dog_create", "dog_set_measurement_grid", "dog_step",
           "dog_get_cells", "dog_get_state", "dog_set_state", "dog_sync", "dog_get_debug",
           "dog_profile_read", "dog_kernels_per_step", "dog_destroy", "dog_error_string",
           "dog_assign_cells_noalloc", "dog_batch_create", "dog_batch_step", "dog_batch_destroy",
           "dog_last_cuda_error", "dog_eval_clusters", "dog_eval_mahalanobis",
           "dog_get_cells_async", "dog_wait_cells", "dog_set_ego_motion", "dog_set_bernoulli_grid",
           "dog_autotune", "dog_set_sort_config", "dog_sort_config", "dog_batch_set_group_bytes",
           "dog_batch_groups", "dog_batch_autotune"]
DOG_NOALLOC_MAX_PARTICLES, DOG_NOALLOC_MAX_CELLS = 1 << 19, (1 << 22) - 1


class dog_params(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("cell_size", C.c_float),
                ("num_particles", C.c_uint32), ("num_birth", C.c_uint32),
                ("p_S", C.c_float), ("p_B", C.c_float), ("alpha_free", C.c_float),
                ("sigma_pos", C.c_float), ("sigma_vel", C.c_float),
                ("sigma_birth_vel", C.c_float), ("sensor_x", C.c_float),
                ("sensor_y", C.c_float), ("seed", C.c_uint64), ("flags", C.c_uint32)]


class dog_meas_grid(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("m_occ", "m_free", "p_A", "z_vr", "sigma_vr")]


BERN_FIELDS = ("z", "p_tp", "p_fp", "p_a", "p_c")


class dog_bern_grid(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in BERN_FIELDS]


CELL_FIELDS = ["m_occ", "m_free", "rho_p", "rho_b", "p_occ", "mean_vx", "mean_vy", "var_vx",
               "var_vy", "cov_vxy"]


class dog_cells(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in CELL_FIELDS]


STATE_FIELDS = ["x", "y", "vx", "vy", "w", "m_free"]


class dog_state(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in STATE_FIELDS]


_lib = None


class DogError(RuntimeError):
    def __init__(self, fn: str, code: int):
        detail = ""
        if code == -3 and _lib is not None:
            detail = f" ({_lib.dog_last_cuda_error().decode()})"
        super().__init__(f"{fn} failed: {DOG_ERR.get(code, code)}{detail}")
        self.code = code


def lib() -> C.CDLL:
    """Load libdog.so (built by paper_1605_02406_b300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1605_02406_b300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.c_size_t
        L.dog_workspace_bytes.argtypes = [C.POINTER(dog_params), C.POINTER(sz)]
        L.dog_create.argtypes = [C.POINTER(dog_params), vp, sz, vp, C.POINTER(vp)]
        L.dog_set_measurement_grid.argtypes = [vp, C.POINTER(dog_meas_grid), C.c_int]
        L.dog_set_bernoulli_grid.argtypes = [vp, C.POINTER(dog_bern_grid), C.c_int]
        L.dog_autotune.argtypes = [vp]
        L.dog_set_sort_config.argtypes = [vp, C.c_int, C.c_int]
        L.dog_sort_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dog_step.argtypes = [vp, C.c_float]
        L.dog_get_cells.argtypes = [vp, C.POINTER(dog_cells), C.c_int]
        L.dog_get_state.argtypes = [vp, C.POINTER(dog_state), C.c_int, C.POINTER(C.c_uint32)]
        L.dog_set_state.argtypes = [vp, C.POINTER(dog_state), C.c_int, C.c_uint32]
        L.dog_sync.argtypes = [vp]
        L.dog_get_debug.argtypes = [vp, C.c_int, vp, C.c_int]
        L.dog_profile_read.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_char_p), C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dog_kernels_per_step.argtypes = [vp]
        L.dog_destroy.argtypes = [vp]
        L.dog_destroy.restype = None
        L.dog_assign_cells_noalloc.argtypes = [vp, C.c_uint32, C.c_uint32, vp, vp, vp, vp]
        L.dog_error_string.argtypes = [C.c_int]
        L.dog_error_string.restype = C.c_char_p
        L.dog_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
        L.dog_batch_step.argtypes = [vp, C.POINTER(C.c_float)]
        L.dog_batch_destroy.argtypes = [vp]
        L.dog_batch_set_group_bytes.argtypes = [vp, C.c_size_t]
        L.dog_batch_groups.argtypes = [vp, C.POINTER(C.c_int)]
        L.dog_batch_autotune.argtypes = [vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_size_t)]
        L.dog_batch_destroy.restype = None
        L.dog_last_cuda_error.argtypes = []
        L.dog_eval_clusters.argtypes = [vp, vp, C.c_uint32, vp, vp]
        L.dog_get_cells_async.argtypes = [vp, C.POINTER(dog_cells)]
        L.dog_wait_cells.argtypes = [vp]
        L.dog_set_ego_motion.argtypes = [vp, C.c_float, C.c_float, C.c_float]
        L.dog_eval_mahalanobis.argtypes = [vp, vp, C.c_float, vp, C.c_uint32, vp, vp]
        L.dog_last_cuda_error.restype = C.c_char_p
        for n in SYMBOLS:
            if n not in ("dog_destroy", "dog_error_string", "dog_batch_destroy", "dog_last_cuda_error"):
                getattr(L, n).restype = C.c_int
        _lib = L
    return _lib


def check(fn: str, rc: int) -> None:
    if rc != DOG_OK:
        raise DogError(fn, rc)


def make_params(p: dict) -> dog_params:
    return dog_params(width=int(p["width"]), height=int(p["height"]),
                      cell_size=float(p["cell_size"]), num_particles=int(p["nu"]),
                      num_birth=int(p["nu_b"]), p_S=float(p["p_S"]), p_B=float(p["p_B"]),
                      alpha_free=float(p["alpha"]), sigma_pos=float(p["sigma_pos"]),
                      sigma_vel=float(p["sigma_vel"]),
                      sigma_birth_vel=float(p["sigma_birth_vel"]),
                      sensor_x=float(p["sensor_x"]), sensor_y=float(p["sensor_y"]),
                      seed=int(p["seed"]), flags=int(p.get("flags", 0)))


# thin wrappers with the C names ---------------------------------------------------------
def dog_workspace_bytes(params: dog_params) -> int:
    n = C.c_size_t()
    check("dog_workspace_bytes", lib().dog_workspace_bytes(C.byref(params), C.byref(n)))
    return n.value


def dog_create(params: dog_params, workspace_ptr: int, nbytes: int, stream_ptr: int) -> int:
    h = C.c_void_p()
    check("dog_create", lib().dog_create(C.byref(params), C.c_void_p(workspace_ptr), nbytes,
                                         C.c_void_p(stream_ptr), C.byref(h)))
    return h.value


def dog_set_measurement_grid(h: int, ptrs: dict, mem_kind: int) -> None:
    g = dog_meas_grid(**{k: ptrs.get(k) for k in ("m_occ", "m_free", "p_A", "z_vr", "sigma_vr")})
    check("dog_set_measurement_grid", lib().dog_set_measurement_grid(h, C.byref(g), mem_kind))


def dog_set_bernoulli_grid(h: int, ptrs: dict, mem_kind: int) -> None:
    g = dog_bern_grid(**{k: ptrs.get(k) for k in BERN_FIELDS})
    check("dog_set_bernoulli_grid", lib().dog_set_bernoulli_grid(h, C.byref(g), mem_kind))


def dog_autotune(h: int) -> None:
    check("dog_autotune", lib().dog_autotune(h))


def dog_set_sort_config(h: int, passes: int, count_tiles: int) -> None:
    check("dog_set_sort_config", lib().dog_set_sort_config(h, int(passes), int(count_tiles)))


def dog_sort_config(h: int) -> dict:
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    check("dog_sort_config", lib().dog_sort_config(h, C.byref(a), C.byref(b), C.byref(c)))
    return {"passes": a.value, "digit_bits": b.value, "count_tiles": c.value}


def dog_step(h: int, dt: float) -> None:
    check("dog_step", lib().dog_step(h, float(dt)))


def dog_set_ego_motion(h: int, dx: float, dy: float, dyaw: float) -> None:
    check("dog_set_ego_motion", lib().dog_set_ego_motion(h, float(dx), float(dy), float(dyaw)))


def dog_get_cells(h: int, ptrs: dict, mem_kind: int) -> None:
    c = dog_cells(**{k: ptrs.get(k) for k in CELL_FIELDS})
    check("dog_get_cells", lib().dog_get_cells(h, C.byref(c), mem_kind))


def dog_get_state(h: int, ptrs: dict, mem_kind: int) -> int:
    s = dog_state(**{k: ptrs.get(k) for k in STATE_FIELDS})
    fr = C.c_uint32()
    check("dog_get_state", lib().dog_get_state(h, C.byref(s), mem_kind, C.byref(fr)))
    return fr.value


def dog_set_state(h: int, ptrs: dict, mem_kind: int, frame: int) -> None:
    s = dog_state(**{k: ptrs.get(k) for k in STATE_FIELDS})
    check("dog_set_state", lib().dog_set_state(h, C.byref(s), mem_kind, int(frame)))


def dog_sync(h: int) -> None:
    check("dog_sync", lib().dog_sync(h))


def dog_get_debug(h: int, which: int, ptr: int, mem_kind: int) -> None:
    check("dog_get_debug", lib().dog_get_debug(h, which, C.c_void_p(ptr), mem_kind))


def dog_profile_read(h: int, max_kernels: int = 16):
    """(per-kernel ms summed over the steps since the last read, number of steps)"""
    ms = (C.c_float * max_kernels)()
    names = (C.c_char_p * max_kernels)()
    n, steps = C.c_int(), C.c_int()
    check("dog_profile_read", lib().dog_profile_read(h, ms, names, max_kernels, C.byref(n),
                                                     C.byref(steps)))
    return {names[k].decode(): float(ms[k]) for k in range(n.value)}, steps.value


def dog_kernels_per_step(h: int) -> int:
    return int(lib().dog_kernels_per_step(h))


def dog_destroy(h: int) -> None:
    lib().dog_destroy(h)


def dog_assign_cells_noalloc(keys_ptr: int, n: int, num_cells: int, perm_ptr: int,
                             start_ptr: int, end_ptr: int, stream_ptr: int) -> None:
    """Stable sort of cell indices and per-cell ranges with no allocation (device pointers)."""
    check("dog_assign_cells_noalloc",
          lib().dog_assign_cells_noalloc(C.c_void_p(keys_ptr), n, num_cells, C.c_void_p(perm_ptr),
                                         C.c_void_p(start_ptr), C.c_void_p(end_ptr),
                                         C.c_void_p(stream_ptr)))


def dog_error_string(code: int) -> str:
    return lib().dog_error_string(code).decode()


def dog_batch_create(handles: list) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    b = C.c_void_p()
    check("dog_batch_create", lib().dog_batch_create(arr, len(handles), C.byref(b)))
    return b.value


def dog_batch_step(b: int, dts) -> None:
    arr = (C.c_float * len(dts))(*[float(x) for x in dts])
    check("dog_batch_step", lib().dog_batch_step(b, arr))


def dog_batch_set_group_bytes(b: int, group_bytes: int) -> None:
    check("dog_batch_set_group_bytes", lib().dog_batch_set_group_bytes(b, int(group_bytes)))


def dog_batch_groups(b: int) -> int:
    n = C.c_int()
    check("dog_batch_groups", lib().dog_batch_groups(b, C.byref(n)))
    return n.value


def dog_batch_autotune(b: int, dts, frames: int) -> int:
    arr = (C.c_float * len(dts))(*[float(x) for x in dts])
    chosen = C.c_size_t()
    check("dog_batch_autotune", lib().dog_batch_autotune(b, arr, int(frames), C.byref(chosen)))
    return chosen.value


def dog_batch_destroy(b: int) -> None:
    lib().dog_batch_destroy(b)


def dog_eval_clusters(h: int, d_cell_object: int, n_objects: int, d_scratch: int, d_stats: int) -> None:
    check("dog_eval_clusters", lib().dog_eval_clusters(h, C.c_void_p(d_cell_object), n_objects,
                                                       C.c_void_p(d_scratch), C.c_void_p(d_stats)))


def dog_eval_mahalanobis(h: int, d_label: int, min_occ: float, d_thresholds: int, n_thresholds: int,
                         d_counts: int, d_m: int | None) -> None:
    check("dog_eval_mahalanobis", lib().dog_eval_mahalanobis(
        h, C.c_void_p(d_label), float(min_occ), C.c_void_p(d_thresholds), n_thresholds,
        C.c_void_p(d_counts), C.c_void_p(d_m)))


def dog_get_cells_async(h: int, ptrs: dict) -> None:
    c = dog_cells(**{k: ptrs.get(k) for k in CELL_FIELDS})
    check("dog_get_cells_async", lib().dog_get_cells_async(h, C.byref(c)))


def dog_wait_cells(h: int) -> None:
    check("dog_wait_cells", lib().dog_wait_cells(h))
