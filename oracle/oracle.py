"""ctypes binding of the C oracle (test infrastructure only; see package docstring)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build

_LIBS: dict = {}


class _OrParams(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("cell_size", C.c_float),
        ("nu", C.c_uint32), ("nu_b", C.c_uint32),
        ("p_S", C.c_float), ("p_B", C.c_float), ("alpha", C.c_float),
        ("sigma_pos", C.c_float), ("sigma_vel", C.c_float), ("sigma_birth_vel", C.c_float),
        ("sensor_x", C.c_float), ("sensor_y", C.c_float),
        ("seed", C.c_uint64), ("flags", C.c_uint32),
    ]


def _lib(mode: str):
    if mode not in _LIBS:
        paths = build()
        lib = C.CDLL(paths[mode])
        fp = C.POINTER(C.c_float)
        u32p = C.POINTER(C.c_uint32)
        u64p = C.POINTER(C.c_uint64)
        lib.oracle_create.restype = C.c_void_p
        lib.oracle_create.argtypes = [C.POINTER(_OrParams)]
        lib.oracle_destroy.argtypes = [C.c_void_p]
        dp = C.POINTER(C.c_double)
        lib.oracle_set_measurement_grid.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.oracle_step.argtypes = [C.c_void_p, C.c_float]
        lib.oracle_set_ego_motion.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float]
        lib.oracle_set_bernoulli_grid.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.oracle_set_ego_motion.restype = None
        lib.oracle_get_cell_array.argtypes = [C.c_void_p, C.c_int, dp]
        lib.oracle_get_particle_array.argtypes = [C.c_void_p, C.c_int, dp]
        lib.oracle_get_index_array.argtypes = [C.c_void_p, C.c_int, u32p]
        lib.oracle_get_fixed_array.argtypes = [C.c_void_p, C.c_int, u64p]
        lib.oracle_get_scalars.argtypes = [C.c_void_p, u64p]
        lib.oracle_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, u32p]
        lib.oracle_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, C.c_uint32]
        lib.oracle_cell_update.argtypes = [C.c_double] * 6 + [C.POINTER(C.c_double)]
        lib.oracle_box_muller.argtypes = [C.c_uint32, C.c_uint32, fp]
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        u8p = C.POINTER(C.c_uint8)
        lib.oracle_force_decisions.argtypes = [C.c_void_p, u32p, u8p, u32p, u8p, C.c_int, C.c_int, u32p]
        lib.oracle_force_decisions.restype = None
        lib.oracle_radar_likelihood.restype = C.c_double
        lib.oracle_radar_likelihood.argtypes = [C.c_double] * 8
        if mode == "f32":
            lib.oracle_ln_f32.restype = C.c_float
            lib.oracle_ln_f32.argtypes = [C.c_float]
            lib.oracle_exp_f32.restype = C.c_float
            lib.oracle_exp_f32.argtypes = [C.c_float]
            lib.oracle_sincos2pi_f32.argtypes = [C.c_float, fp, fp]
        _LIBS[mode] = lib
    return _LIBS[mode]


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _u32(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _u64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _cf64(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    assert a.size == n
    return a


CELL_FIELDS = ["m_occ", "m_free", "rho_p", "rho_b", "p_occ", "mean_vx", "mean_vy",
               "var_vx", "var_vy", "cov_vxy", "m_occ_pred", "mu_A", "mu_UA"]
PARTICLE_FIELDS = ["pred_x", "pred_y", "pred_vx", "pred_vy", "pred_w", "w_norm",
                   "birth_x", "birth_y", "birth_vx", "birth_vy", "birth_w"]
INDEX_FIELDS = ["key", "perm", "cell_start", "cell_end", "birth_cell", "birth_assoc",
                "resample_src", "in_grid"]


class OracleFilter:
    """Plain CPU DS-PHD/MIB filter.  ``mode`` is ``"f32"`` (FP32 mirror) or ``"f64"``."""

    def __init__(self, params: dict, mode: str = "f32"):
        self.mode = mode
        self.lib = _lib(mode)
        p = _OrParams()
        for name, _ in _OrParams._fields_:
            setattr(p, name, params.get(name, 0))
        self.params = dict(params)
        self.nu = int(p.nu)
        self.nu_b = int(p.nu_b)
        self.C = int(p.width) * int(p.height)
        self._h = self.lib.oracle_create(C.byref(p))
        if not self._h:
            raise ValueError("oracle_create rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.oracle_destroy(h)
            self._h = None

    def set_measurement_grid(self, m_occ, m_free, p_A=None, z_vr=None, sigma_vr=None):
        n = self.C
        a, b = _cf64(m_occ, n), _cf64(m_free, n)
        if p_A is None:
            rc = self.lib.oracle_set_measurement_grid(self._h, _d(a), _d(b), None, None, None)
        else:
            pa, zv, sg = _cf64(p_A, n), _cf64(z_vr, n), _cf64(sigma_vr, n)
            rc = self.lib.oracle_set_measurement_grid(self._h, _d(a), _d(b), _d(pa), _d(zv), _d(sg))
        if rc != 0:
            raise ValueError(f"oracle_set_measurement_grid: invalid input ({rc})")

    def set_bernoulli_grid(self, z, p_tp, p_fp, p_a, p_c):
        """Bernoulli observation per cell (PHD/MIB filter, flag 0x40)."""
        arrs = [_cf64(a, self.C) for a in (z, p_tp, p_fp, p_a, p_c)]
        rc = self.lib.oracle_set_bernoulli_grid(self._h, *[_d(a) for a in arrs])
        if rc != 0:
            raise ValueError(f"oracle_set_bernoulli_grid: {rc}")

    def set_ego_motion(self, dx: float, dy: float, dyaw: float):
        """Vehicle motion since the previous frame, applied at the start of the next step."""
        self.lib.oracle_set_ego_motion(self._h, float(dx), float(dy), float(dyaw))

    def step(self, dt: float):
        rc = self.lib.oracle_step(self._h, float(dt))
        if rc != 0:
            raise RuntimeError(f"oracle_step failed ({rc})")

    def _out_dtype(self):
        return np.float32 if self.mode == "f32" else np.float64

    def cells(self) -> dict:
        """Per-cell outputs (float32 for the FP32 mirror, float64 for FP64 mode)."""
        out = {}
        for k, name in enumerate(CELL_FIELDS):
            a = np.empty(self.C, np.float64)
            self.lib.oracle_get_cell_array(self._h, k, _d(a))
            out[name] = a.astype(self._out_dtype())
        return out

    def intermediates(self) -> dict:
        out = {}
        for k, name in enumerate(PARTICLE_FIELDS):
            n = self.nu if k < 6 else self.nu_b
            a = np.empty(n, np.float64)
            self.lib.oracle_get_particle_array(self._h, k, _d(a))
            out[name] = a.astype(self._out_dtype())
        sizes = [self.nu, self.nu, self.C, self.C, self.nu_b, self.nu_b, self.nu, self.nu]
        for k, name in enumerate(INDEX_FIELDS):
            a = np.empty(sizes[k], np.uint32)
            self.lib.oracle_get_index_array(self._h, k, _u32(a))
            out[name] = a
        for k, name in enumerate(["S", "A"]):
            a = np.empty(self.C, np.uint64)
            self.lib.oracle_get_fixed_array(self._h, k, _u64(a))
            out[name] = a
        sc = np.empty(4, np.uint64)
        self.lib.oracle_get_scalars(self._h, _u64(sc))
        out["frame"], out["W_total"], out["R_total"], out["u_offset"] = (int(v) for v in sc)
        return out

    def decisions(self) -> dict:
        """The integer decisions of the last step (see force_decisions)."""
        im = self.intermediates()
        return {"key": im["key"], "in_grid": im["in_grid"].astype(np.uint8),
                "birth_cell": im["birth_cell"], "birth_assoc": im["birth_assoc"].astype(np.uint8),
                "birth_mass": int(im["R_total"] > 0),
                # resampling ran unless switched off or no weight was left (Alg. 7 reading)
                "resampled": int(im["W_total"] > 0 and not (self.params.get("flags", 0) & 0x2)),
                "resample_src": im["resample_src"]}

    def force_decisions(self, d: dict):
        """Take the next step's integer decisions (cells, in-grid flags, newborn slots,
        resampling) from another run, e.g. the binary32 mirror's, so that the difference
        between the two runs is arithmetic only."""
        arr = {k: np.ascontiguousarray(d[k], dtype=np.uint8 if k in ("in_grid", "birth_assoc") else np.uint32)
               for k in ("key", "in_grid", "birth_cell", "birth_assoc", "resample_src")}
        u8 = lambda a: a.ctypes.data_as(C.POINTER(C.c_uint8))
        self.lib.oracle_force_decisions(self._h, _u32(arr["key"]), u8(arr["in_grid"]), _u32(arr["birth_cell"]),
                                        u8(arr["birth_assoc"]), int(d["birth_mass"]), int(d["resampled"]),
                                        _u32(arr["resample_src"]))
        self._forced = arr  # kept alive until the step has copied them (it copies at once)

    def get_state(self) -> dict:
        st = {k: np.empty(self.nu, np.float64) for k in ("x", "y", "vx", "vy", "w")}
        st["m_free"] = np.empty(self.C, np.float64)
        fr = np.zeros(1, np.uint32)
        self.lib.oracle_get_state(self._h, _d(st["x"]), _d(st["y"]), _d(st["vx"]), _d(st["vy"]),
                                  _d(st["w"]), _d(st["m_free"]), _u32(fr))
        st = {k: v.astype(self._out_dtype()) for k, v in st.items()}
        st["frame"] = int(fr[0])
        return st

    def set_state(self, st: dict):
        arrs = [_cf64(st[k], self.nu) for k in ("x", "y", "vx", "vy", "w")]
        mf = _cf64(st["m_free"], self.C)
        self.lib.oracle_set_state(self._h, *[_d(a) for a in arrs], _d(mf), int(st.get("frame", 0)))


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _lib("f32")
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_u32(c), _u32(k), _u32(out))
    return out


def box_muller(ra: int, rb: int, mode: str = "f32"):
    out = np.zeros(2, np.float32)
    _lib(mode).oracle_box_muller(int(ra), int(rb), _f(out))
    return float(out[0]), float(out[1])


def ln_f32(u: float) -> float:
    return _lib("f32").oracle_ln_f32(float(u))


def exp_f32(x: float) -> float:
    return _lib("f32").oracle_exp_f32(float(x))


def sincos2pi_f32(u: float):
    s, c = C.c_float(), C.c_float()
    _lib("f32").oracle_sincos2pi_f32(float(u), C.byref(s), C.byref(c))
    return s.value, c.value


def radar_likelihood(sensor, x, y, vx, vy, z_vr, sigma_vr, mode: str = "f32") -> float:
    """The radar spatial likelihood g of one particle (constant factor dropped)."""
    return _lib(mode).oracle_radar_likelihood(float(sensor[0]), float(sensor[1]), float(x), float(y),
                                              float(vx), float(vy), float(z_vr), float(sigma_vr))


def cell_update(m_pred, m_free_prev, zO, zF, alpha, p_B, mode: str = "f32") -> dict:
    out = np.zeros(5, np.float64)
    _lib(mode).oracle_cell_update(float(m_pred), float(m_free_prev), float(zO), float(zF),
                                  float(alpha), float(p_B), out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(zip(["m_occ", "m_free", "rho_b", "rho_p", "m_free_pred"], (float(v) for v in out)))
