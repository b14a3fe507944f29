"""GB300 (sm_103a) buoyancy-driven-cavity step of Xue & Roy (arXiv 2006.02602).

Thin ctypes binding of the C ABI declared in ``include/cavity.h``: every
function below has the name of the C entry point it marshals arguments for,
and every step of the computation runs in the CUDA kernels of
``libbdc_cavity.so``.  There is no CPU fallback: importing the binding without
the built library raises, and so does every call that returns an error code.

Build the library with ``python -m paper_2006_02602_gb300.build`` (nvcc,
``-gencode arch=compute_103a,code=sm_103a``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbdc_cavity.so")

CAVITY_OK = 0
CAVITY_ERR_INVALID_ARG = -1
CAVITY_ERR_OOM = -2
CAVITY_ERR_CUDA = -3
CAVITY_ERR_NONFINITE = -4
CAVITY_ERR_TIMEOUT = -5
CAVITY_ERR_UNSUPPORTED = -6

CAVITY_FP64 = 0
CAVITY_FP32_MIXED = 1

CAVITY_DT_GLOBAL = 0
CAVITY_DT_LOCAL = 1

CAVITY_FIELD_P, CAVITY_FIELD_U, CAVITY_FIELD_V, CAVITY_FIELD_W, CAVITY_FIELD_T = 1, 2, 4, 8, 16
CAVITY_FIELD_ALL = 31

EXPORTED = (
    "cavity_default_params", "cavity_create", "cavity_set_params", "cavity_set_wall_temperature",
    "cavity_step", "cavity_residual", "cavity_nusselt", "cavity_get_fields", "cavity_get_fields_box",
    "cavity_set_fields",
    "cavity_get_time", "cavity_num_blocks", "cavity_get_block_array", "cavity_get_face_buffer",
    "cavity_exchange", "cavity_time_kernels", "cavity_step_block_noalloc", "cavity_sync", "cavity_destroy",
    "cavity_strerror", "cavity_last_error", "cavity_create_batch", "cavity_batch_size", "cavity_batch_state",
    "cavity_batch_get_fields", "cavity_autotune", "cavity_adjoint_forward", "cavity_adjoint_backward",
    "cavity_set_time_stepping", "cavity_set_overlap", "cavity_check_sqrt", "cavity_check_div3", "cavity_test_wait_timeout",
    "cavity_measure_fp64_peak", "cavity_adjoint_kernel_ms", "cavity_set_step_log", "cavity_step_log_alloc",
    "cavity_step_log_free",
)


class CavityError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__(f"{code}: {msg}")


class cavity_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int),
                ("precision", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("noise_amp", ctypes.c_double), ("device", ctypes.c_int), ("stream", ctypes.c_void_p)]


class cavity_params(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("Pr", ctypes.c_double), ("cfl", ctypes.c_double),
                ("kappa", ctypes.c_double), ("c4", ctypes.c_double), ("u_ref", ctypes.c_double),
                ("t_inf", ctypes.c_double), ("t_hot", ctypes.c_double), ("t_cold", ctypes.c_double),
                ("gravity_axis", ctypes.c_int)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbdc_cavity.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library missing: {path} (build it with python -m paper_2006_02602_gb300.build)")
    L = ctypes.CDLL(path)
    sig = {
        "cavity_default_params": ([ctypes.POINTER(cavity_params)], ctypes.c_int),
        "cavity_create": ([ctypes.POINTER(cavity_desc), ctypes.POINTER(_H)], ctypes.c_int),
        "cavity_set_params": ([_H, ctypes.POINTER(cavity_params)], ctypes.c_int),
        "cavity_set_wall_temperature": ([_H, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_step": ([_H, ctypes.c_int], ctypes.c_int),
        "cavity_residual": ([_H, _dp], ctypes.c_int),
        "cavity_nusselt": ([_H, _dp, _dp], ctypes.c_int),
        "cavity_get_fields": ([_H, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_get_fields_box": ([_H, ctypes.c_int] + [ctypes.c_int] * 6 + [_dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_set_fields": ([_H, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_get_time": ([_H, ctypes.POINTER(ctypes.c_longlong), _dp, _dp], ctypes.c_int),
        "cavity_num_blocks": ([_H], ctypes.c_int),
        "cavity_get_block_array": ([_H, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cavity_get_face_buffer": ([_H, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_exchange": ([_H], ctypes.c_int),
        "cavity_time_kernels": ([_H, ctypes.c_int, _dp], ctypes.c_int),
        "cavity_check_sqrt": ([_dp, ctypes.c_longlong, _dp, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "cavity_check_div3": ([_dp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "cavity_set_time_stepping": ([_H, ctypes.c_int], ctypes.c_int),
        "cavity_set_overlap": ([_H, ctypes.c_int], ctypes.c_int),
        "cavity_create_batch": ([ctypes.POINTER(cavity_desc), ctypes.POINTER(cavity_params), ctypes.c_int,
                                 ctypes.POINTER(_H)], ctypes.c_int),
        "cavity_batch_size": ([_H], ctypes.c_int),
        "cavity_batch_state": ([_H, ctypes.c_int, _dp], ctypes.c_int),
        "cavity_batch_get_fields": ([_H, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t], ctypes.c_int),
        "cavity_autotune": ([_H, ctypes.c_int, _dp], ctypes.c_int),
        "cavity_adjoint_forward": ([_H, ctypes.c_int, ctypes.c_int, _dp], ctypes.c_int),
        "cavity_adjoint_backward": ([_H, _dp, ctypes.c_size_t, _dp], ctypes.c_int),
        "cavity_step_block_noalloc": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(cavity_params), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "cavity_test_wait_timeout": ([_H, ctypes.c_longlong, ctypes.c_int], ctypes.c_int),
        "cavity_measure_fp64_peak": ([ctypes.c_int, _dp], ctypes.c_int),
        "cavity_adjoint_kernel_ms": ([_H, _dp], ctypes.c_int),
        "cavity_set_step_log": ([_H, ctypes.c_void_p, ctypes.c_longlong], ctypes.c_int),
        "cavity_step_log_alloc": ([ctypes.c_longlong, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "cavity_step_log_free": ([ctypes.c_void_p], ctypes.c_int),
        "cavity_sync": ([_H], ctypes.c_int),
        "cavity_destroy": ([_H], ctypes.c_int),
        "cavity_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "cavity_last_error": ([_H], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc: int, h=None) -> int:
    if rc < 0:
        L = load_library()
        msg = L.cavity_strerror(rc).decode()
        if h is not None:
            extra = L.cavity_last_error(h).decode()
            if extra:
                msg += f" ({extra})"
        raise CavityError(rc, msg)
    return rc


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# -- C-ABI mirrors --------------------------------------------------------------

def cavity_default_params(**overrides) -> cavity_params:
    p = cavity_params()
    _check(load_library().cavity_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    # defaults left to the library: u_ref = max(1, sqrt(Ra Pr)) (and it then
    # follows Ra in derivatives), t_inf = (t_hot + t_cold) / 2
    if "u_ref" not in overrides:
        p.u_ref = -1.0
    if "t_inf" not in overrides:
        p.t_inf = math.nan
    return p


def cavity_create(nx, ny, nz, blocks=(1, 1, 1), precision=CAVITY_FP64, seed=0, noise_amp=0.0,
                  device=0, stream=None):
    d = cavity_desc(int(nx), int(ny), int(nz), int(blocks[0]), int(blocks[1]), int(blocks[2]),
                    int(precision), int(seed), float(noise_amp), int(device), stream)
    h = _H()
    _check(load_library().cavity_create(ctypes.byref(d), ctypes.byref(h)))
    return h


def cavity_set_params(h, params: cavity_params) -> None:
    _check(load_library().cavity_set_params(h, ctypes.byref(params)), h)


def cavity_set_wall_temperature(h, wall: int, values) -> None:
    v = _f64(values).reshape(-1)
    _check(load_library().cavity_set_wall_temperature(h, int(wall), v.ctypes.data_as(_dp), v.size), h)


def cavity_step(h, nsteps: int = 1) -> None:
    _check(load_library().cavity_step(h, int(nsteps)), h)


def cavity_residual(h) -> np.ndarray:
    out = np.zeros(5)
    _check(load_library().cavity_residual(h, out.ctypes.data_as(_dp)), h)
    return out


def cavity_nusselt(h) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().cavity_nusselt(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def _nfields(mask: int) -> int:
    return bin(mask & CAVITY_FIELD_ALL).count("1")


def cavity_get_fields(h, shape: tuple[int, int, int], mask: int = CAVITY_FIELD_ALL, out=None) -> np.ndarray:
    """Interior fields as an array [nf, nz, ny, nx] (shape = (nx, ny, nz)); `out`: a C-contiguous
    float64 array of that shape to fill (page-locked memory copies at the full link rate)."""
    nx, ny, nz = shape
    want = (_nfields(mask), nz, ny, nx)
    if out is None:
        out = np.empty(want)
    elif out.shape != want or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a C-contiguous float64 array of shape %s" % (want,))
    _check(load_library().cavity_get_fields(h, int(mask), out.ctypes.data_as(_dp), out.size), h)
    return out


def cavity_get_fields_box(h, lo: tuple[int, int, int], size: tuple[int, int, int],
                          mask: int = CAVITY_FIELD_ALL) -> np.ndarray:
    """Fields on the global 1-based node box lo .. lo+size-1 as [nf, nk, nj, ni]."""
    (i0, j0, k0), (ni, nj, nk) = lo, size
    out = np.empty((_nfields(mask), nk, nj, ni))
    _check(load_library().cavity_get_fields_box(h, int(mask), int(i0), int(j0), int(k0), int(ni), int(nj), int(nk),
                                                out.ctypes.data_as(_dp), out.size), h)
    return out


def cavity_set_fields(h, values, mask: int = CAVITY_FIELD_ALL) -> None:
    v = _f64(values)
    _check(load_library().cavity_set_fields(h, int(mask), v.ctypes.data_as(_dp), v.size), h)


def cavity_get_time(h) -> tuple[int, float, float]:
    s, t, dt = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().cavity_get_time(h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(dt)), h)
    return s.value, t.value, dt.value


def cavity_num_blocks(h) -> int:
    return _check(load_library().cavity_num_blocks(h), h)


def cavity_get_block_array(h, block: int, field: int):
    """(array [nz+4, ny+4, nx+4] of the block incl. walls/ghosts, (nx, ny, nz, ox, oy, oz))."""
    dims = (ctypes.c_int * 6)()
    L = load_library()
    _check(L.cavity_get_block_array(h, int(block), int(field), None, 0, dims), h)
    nx, ny, nz = dims[0], dims[1], dims[2]
    out = np.empty((nz + 4, ny + 4, nx + 4))
    _check(L.cavity_get_block_array(h, int(block), int(field), out.ctypes.data_as(_dp), out.size, dims), h)
    return out, tuple(dims)


def cavity_get_face_buffer(h, block: int, face: int, nb: int, nc: int) -> np.ndarray:
    out = np.empty(6 * nb * nc)
    _check(load_library().cavity_get_face_buffer(h, int(block), int(face), out.ctypes.data_as(_dp), out.size), h)
    return out


def cavity_exchange(h) -> None:
    _check(load_library().cavity_exchange(h), h)


def cavity_set_overlap(h, on: bool) -> None:
    _check(load_library().cavity_set_overlap(h, int(bool(on))), h)


def cavity_set_time_stepping(h, mode: int) -> None:
    _check(load_library().cavity_set_time_stepping(h, int(mode)), h)


def cavity_time_kernels(h, nsteps: int) -> np.ndarray:
    """Mean ms per launch of [step, wall/finalise, pack, unpack] over nsteps real steps."""
    out = np.zeros(4)
    _check(load_library().cavity_time_kernels(h, int(nsteps), out.ctypes.data_as(_dp)), h)
    return out


def cavity_check_sqrt(x) -> tuple:
    """(largest relative difference, count of differing values) of the FP64
    step's Newton square root from CUDA's sqrt over the positive, normal,
    finite values x, evaluated on the current CUDA device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = ctypes.c_double(0.0)
    nd = ctypes.c_longlong(0)
    _check(load_library().cavity_check_sqrt(x.ctypes.data_as(_dp), x.size, ctypes.byref(m), ctypes.byref(nd)))
    return m.value, nd.value


def cavity_check_div3(x) -> int:
    """Count of the finite values x (|x| >= 4 DBL_MIN) where the FP64 wall
    kernel's division by 3 differs from CUDA's correctly rounded x / 3,
    evaluated on the current CUDA device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nd = ctypes.c_longlong(0)
    _check(load_library().cavity_check_div3(x.ctypes.data_as(_dp), x.size, ctypes.byref(nd)))
    return nd.value


def cavity_step_block_noalloc(q_in_ptr: int, q_out_ptr: int, shape, params: cavity_params, dt: float,
                              pshift: float, out6_ptr: int, stream=None) -> None:
    """Allocation-free fused step of one caller-held block (device pointers
    given as integers, e.g. tensor.data_ptr()); for callers that must not
    allocate device memory.  See include/cavity.h."""
    nx, ny, nz = shape
    _check(load_library().cavity_step_block_noalloc(q_in_ptr, q_out_ptr, int(nx), int(ny), int(nz),
                                                    ctypes.byref(params), float(dt), float(pshift),
                                                    out6_ptr, stream))


def cavity_measure_fp64_peak(device: int = 0) -> float:
    out = ctypes.c_double()
    _check(load_library().cavity_measure_fp64_peak(int(device), ctypes.byref(out)))
    return out.value


def cavity_test_wait_timeout(h, wait_cycles: int, withhold_plane: int = -1) -> None:
    _check(load_library().cavity_test_wait_timeout(h, int(wait_cycles), int(withhold_plane)), h)


def cavity_sync(h) -> int:
    return load_library().cavity_sync(h)


def cavity_destroy(h) -> None:
    _check(load_library().cavity_destroy(h))


def cavity_create_batch(sizes, params_list=None, precision=CAVITY_FP32_MIXED, seeds=None, noise_amp=0.0,
                        device=0, stream=None):
    """Batch handle of len(sizes) single-block cavities; sizes = [(nx, ny, nz), ...]."""
    n = len(sizes)
    seeds = list(range(n)) if seeds is None else list(seeds)
    noise = [noise_amp] * n if np.isscalar(noise_amp) else list(noise_amp)
    descs = (cavity_desc * n)(*[cavity_desc(int(s[0]), int(s[1]), int(s[2]), 1, 1, 1, int(precision),
                                            int(seeds[c]), float(noise[c]), int(device), stream)
                                for c, s in enumerate(sizes)])
    prm = None
    if params_list is not None:
        prm = (cavity_params * n)(*params_list)
    h = _H()
    _check(load_library().cavity_create_batch(descs, prm, n, ctypes.byref(h)))
    return h


def cavity_batch_size(h) -> int:
    return _check(load_library().cavity_batch_size(h), h)


def cavity_batch_state(h, cav: int) -> dict:
    out = np.zeros(10)
    _check(load_library().cavity_batch_state(h, int(cav), out.ctypes.data_as(_dp)), h)
    return {"step": int(out[0]), "t": out[1], "dt": out[2], "residual": out[3:8].copy(),
            "nusselt": (out[8], out[9])}


def cavity_batch_get_fields(h, cav: int, shape, mask: int = CAVITY_FIELD_ALL) -> np.ndarray:
    nx, ny, nz = shape
    out = np.empty((_nfields(mask), nz, ny, nx))
    _check(load_library().cavity_batch_get_fields(h, int(cav), int(mask), out.ctypes.data_as(_dp), out.size), h)
    return out


def cavity_autotune(h, steps: int = 20) -> dict:
    out = np.zeros(5)
    _check(load_library().cavity_autotune(h, int(steps), out.ctypes.data_as(_dp)), h)
    return {"tile_y": int(out[0]), "kc": int(out[1]), "ring": int(out[2]), "kernel_form": int(out[3]),
            "us_per_step": out[4]}


def cavity_adjoint_forward(h, nsteps: int, ckpt: int) -> float:
    """J = mean Nu_hot over the next nsteps steps; checkpoints every ckpt steps."""
    J = ctypes.c_double()
    _check(load_library().cavity_adjoint_forward(h, int(nsteps), int(ckpt), ctypes.byref(J)), h)
    return J.value


def cavity_adjoint_backward(h, ny: int, nz: int) -> tuple[np.ndarray, float]:
    """(dJ/d hot-wall temperature [ny*nz], dJ/dRa) of the last adjoint forward run."""
    g = np.zeros(ny * nz)
    gra = ctypes.c_double()
    _check(load_library().cavity_adjoint_backward(h, g.ctypes.data_as(_dp), g.size, ctypes.byref(gra)), h)
    return g, gra.value


def cavity_adjoint_kernel_ms(h) -> float:
    out = ctypes.c_double()
    _check(load_library().cavity_adjoint_kernel_ms(h, ctypes.byref(out)), h)
    return out.value


def cavity_strerror(code: int) -> str:
    return load_library().cavity_strerror(int(code)).decode()


def cavity_last_error(h) -> str:
    return load_library().cavity_last_error(h).decode()


# the C ABI's cavity_step_record
STEP_RECORD = np.dtype([("step", np.int64), ("t", np.float64), ("dt", np.float64), ("res", np.float64, (5,)),
                        ("nu_hot", np.float64), ("nu_cold", np.float64), ("flags", np.int64)])


class StepLog:
    """Page-locked host memory for `records` step records (cavity_step_log_alloc),
    viewed as a numpy structured array of STEP_RECORD; freed by close()."""

    def __init__(self, records: int):
        self.records = int(records)
        ptr = ctypes.c_void_p()
        _check(load_library().cavity_step_log_alloc(self.records, ctypes.byref(ptr)))
        self.ptr = ptr.value
        buf = (ctypes.c_char * (self.records * STEP_RECORD.itemsize)).from_address(self.ptr)
        self.array = np.frombuffer(buf, dtype=STEP_RECORD)

    def close(self) -> None:
        if getattr(self, "ptr", None):
            self.array = None
            load_library().cavity_step_log_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cavity_step_log_alloc(records: int) -> StepLog:
    return StepLog(records)


def cavity_step_log_free(log: StepLog) -> None:
    log.close()


def cavity_set_step_log(h, log: "StepLog | None", capacity: int | None = None) -> None:
    """Attach `log` (a StepLog; capacity records per cavity, default all of them) or detach (None)."""
    if log is None:
        _check(load_library().cavity_set_step_log(h, None, 0), h)
    else:
        cap = log.records if capacity is None else int(capacity)
        _check(load_library().cavity_set_step_log(h, ctypes.c_void_p(log.ptr), cap), h)


# -- convenience object -------------------------------------------------------

class Cavity:
    """Owning wrapper: ``Cavity(32, 32, 32, Ra=1e4, noise_amp=1e-3).step(200)``."""

    def __init__(self, nx, ny, nz, blocks=(1, 1, 1), precision=CAVITY_FP64, seed=0, noise_amp=0.0,
                 device=0, stream=None, **params):
        self.shape = (int(nx), int(ny), int(nz))
        self.h = cavity_create(nx, ny, nz, blocks, precision, seed, noise_amp, device, stream)
        self.params = cavity_default_params(**params)
        cavity_set_params(self.h, self.params)

    def step(self, n: int = 1):
        cavity_step(self.h, n)
        return self

    def fields(self, mask: int = CAVITY_FIELD_ALL, out=None) -> np.ndarray:
        return cavity_get_fields(self.h, self.shape, mask, out)

    def set_fields(self, values, mask: int = CAVITY_FIELD_ALL) -> None:
        cavity_set_fields(self.h, values, mask)

    @property
    def residual(self) -> np.ndarray:
        return cavity_residual(self.h)

    @property
    def nusselt(self) -> tuple[float, float]:
        return cavity_nusselt(self.h)

    @property
    def time(self) -> tuple[int, float, float]:
        return cavity_get_time(self.h)

    def sync(self) -> int:
        return cavity_sync(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            cavity_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
