"""ctypes binding of the C ABI in ``include/lbm_sw.h`` (argument marshalling only).

The functions keep the C names (``lbm_sw_create``, ``lbm_sw_set_state``,
``lbm_sw_step``, ``lbm_sw_get_moments``, ``lbm_sw_destroy`` ...) and raise
``LbmSwError`` on a negative status.  Every compute step runs in the CUDA library;
loading fails loudly if ``liblbm_sw.so`` has not been built: there is no fallback.

``Simulation`` is a convenience owner of one handle that moves numpy arrays or
torch CUDA tensors across the boundary.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PERIODIC, WALL, OUTFLOW, INFLOW = 0, 1, 2, 3
XM, XP, YM, YP = 0, 1, 2, 3
FP32, FP64 = 0, 1
POST_COLLISION, PRE_COLLISION = 0, 1
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_VEC, KERNEL_CLUSTER, KERNEL_TEMPORAL = 0, 1, 2, 3, 4

OK, E_ARG, E_CUDA, E_UNSTABLE, E_STATE, E_NOMEM = 0, -1, -2, -3, -5, -6


class LbmSwError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class lbm_sw_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("g", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("s", ctypes.c_double),
        ("a", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("inflow", (ctypes.c_double * 3) * 4),
        ("stream", ctypes.c_void_p),
        ("kernel", ctypes.c_int),
        ("graph_chunk", ctypes.c_int),
        ("temporal_steps", ctypes.c_int),
        ("reserved", ctypes.c_int * 5),
    ]


class lbm_sw_info(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("pitch", ctypes.c_size_t),
        ("population_bytes", ctypes.c_size_t),
        ("bytes_per_update", ctypes.c_double),
        ("steps_done", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("steps_per_launch", ctypes.c_int),
    ]


class lbm_sw_batch_params(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int),
        ("nx", ctypes.POINTER(ctypes.c_int)),
        ("ny", ctypes.POINTER(ctypes.c_int)),
        ("precision", ctypes.c_int),
        ("g", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("s", ctypes.c_double),
        ("a", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("inflow", (ctypes.c_double * 3) * 4),
        ("stream", ctypes.c_void_p),
        ("tile_rows", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("graph_chunk", ctypes.c_int),
        ("temporal_steps", ctypes.c_int),
        ("reserved", ctypes.c_int * 4),
    ]


class lbm_sw_batch_tuning(ctypes.Structure):
    _fields_ = [
        ("tile_rows", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("candidates", ctypes.c_int),
        ("ms_per_step", ctypes.c_double),
        ("tiles", ctypes.c_longlong),
        ("cells", ctypes.c_longlong),
        ("temporal_steps", ctypes.c_int),
    ]


class lbm_sw_tape_info(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int),
        ("interval", ctypes.c_int),
        ("checkpoints", ctypes.c_int),
        ("recorded", ctypes.c_int),
        ("checkpoint_bytes", ctypes.c_size_t),
        ("replay_bytes", ctypes.c_size_t),
    ]


_lib = None

# name -> (restype, argtypes); the complete list of entry points of include/lbm_sw.h
_H = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "lbm_sw_params_init": (ctypes.c_int, [ctypes.POINTER(lbm_sw_params)]),
    "lbm_sw_create": (ctypes.c_int, [ctypes.POINTER(lbm_sw_params), ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_sw_destroy": (None, [_H]),
    "lbm_sw_set_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "lbm_sw_step_plan": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "lbm_sw_set_relaxation": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "lbm_sw_set_obstacle": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_get_moments": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_diagnostics": (ctypes.c_int, [_H, _DP]),
    "lbm_sw_get_populations": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_set_populations": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "lbm_sw_get_rows": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_set_rows": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_diagnostics_rows": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _DP]),
    "lbm_sw_synchronize": (ctypes.c_int, [_H]),
    "lbm_sw_get_info": (ctypes.c_int, [_H, ctypes.POINTER(lbm_sw_info)]),
    "lbm_sw_last_error": (ctypes.c_char_p, [_H]),
    "lbm_sw_create_error": (ctypes.c_char_p, []),
    "lbm_sw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_sw_abi_version": (ctypes.c_int, []),
    "lbm_sw_batch_params_init": (ctypes.c_int, [ctypes.POINTER(lbm_sw_batch_params)]),
    "lbm_sw_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_sw_batch_params), ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_sw_batch_destroy": (None, [_H]),
    "lbm_sw_batch_set_state": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int]),
    "lbm_sw_batch_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "lbm_sw_batch_get_moments": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int]),
    "lbm_sw_batch_get_populations": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "lbm_sw_batch_diagnostics": (ctypes.c_int, [_H, ctypes.c_int, _DP]),
    "lbm_sw_batch_autotune": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(lbm_sw_batch_tuning)]),
    "lbm_sw_batch_get_tuning": (ctypes.c_int, [_H, ctypes.POINTER(lbm_sw_batch_tuning)]),
    "lbm_sw_batch_last_error": (ctypes.c_char_p, [_H]),
    "lbm_sw_tape_create": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_sw_tape_destroy": (None, [_H]),
    "lbm_sw_forward_record": (ctypes.c_int, [_H, _H]),
    "lbm_sw_adjoint": (ctypes.c_int, [_H, _H] + [ctypes.c_void_p] * 6 + [ctypes.c_int]),
    "lbm_sw_tape_get_info": (ctypes.c_int, [_H, ctypes.POINTER(lbm_sw_tape_info)]),
    "lbm_sw_tape_last_error": (ctypes.c_char_p, [_H]),
    "lbm_sw_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                                                  ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblbm_sw.so (built by ``__graft_entry__.build()`` / ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build()); "
                          "the lattice Boltzmann path has no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, handle=None, what: str = "") -> int:
    if status < 0:
        lib = load()
        msg = lib.lbm_sw_last_error(handle).decode() if handle else ""
        if not msg:
            msg = lib.lbm_sw_status_string(status).decode()
        raise LbmSwError(status, f"{what}: {msg}" if what else msg)
    return status


# ---------------------------------------------------------------- C entry points
def lbm_sw_params_init() -> lbm_sw_params:
    p = lbm_sw_params()
    _check(load().lbm_sw_params_init(ctypes.byref(p)))
    return p


def lbm_sw_create(p: lbm_sw_params) -> int:
    lib = load()
    h = ctypes.c_void_p()
    st = lib.lbm_sw_create(ctypes.byref(p), ctypes.byref(h))
    if st < 0:
        raise LbmSwError(st, "lbm_sw_create: " + (lib.lbm_sw_create_error().decode() or lib.lbm_sw_status_string(st).decode()))
    return h.value


def lbm_sw_destroy(h: int) -> None:
    load().lbm_sw_destroy(h)


def lbm_sw_set_state(h: int, depth: int, hu: int, hv: int | None, on_device: bool) -> None:
    _check(load().lbm_sw_set_state(h, depth, hu, hv, int(on_device)), h, "lbm_sw_set_state")


def lbm_sw_step(h: int, n: int) -> None:
    _check(load().lbm_sw_step(h, int(n)), h, "lbm_sw_step")


def lbm_sw_step_plan(h: int, n: int) -> list[int]:
    """Steps advanced by each kernel launch that lbm_sw_step(h, n) would make, in order."""
    lib = load()
    count = _check(lib.lbm_sw_step_plan(h, int(n), None, 0), h, "lbm_sw_step_plan")
    sizes = (ctypes.c_int * max(count, 1))()
    _check(lib.lbm_sw_step_plan(h, int(n), sizes, count), h, "lbm_sw_step_plan")
    return list(sizes[:count])


def lbm_sw_set_relaxation(h: int, rates=None) -> None:
    """MRT rates in the paper's moment order (13 in 2D, 5 in 1D), or None for BGK."""
    if rates is None:
        _check(load().lbm_sw_set_relaxation(h, None, 0), h, "lbm_sw_set_relaxation")
        return
    arr = (ctypes.c_double * len(rates))(*[float(r) for r in rates])
    _check(load().lbm_sw_set_relaxation(h, arr, len(rates)), h, "lbm_sw_set_relaxation")


def lbm_sw_set_obstacle(h: int, solid: int | None, on_device: bool) -> None:
    """Solid-cell mask ([ny][nx] bytes, nonzero = solid) at address ``solid``, or None."""
    _check(load().lbm_sw_set_obstacle(h, solid, int(on_device)), h, "lbm_sw_set_obstacle")


def lbm_sw_get_moments(h: int, depth: int, hu: int, hv: int | None, on_device: bool) -> None:
    _check(load().lbm_sw_get_moments(h, depth, hu, hv, int(on_device)), h, "lbm_sw_get_moments")


def lbm_sw_diagnostics(h: int, raise_unstable: bool = True):
    """Returns (sum h, sum hu, sum hv, min h, status)."""
    out = (ctypes.c_double * 4)()
    st = load().lbm_sw_diagnostics(h, out)
    if st != E_UNSTABLE or raise_unstable:
        _check(st, h, "lbm_sw_diagnostics")
    return out[0], out[1], out[2], out[3], st


def lbm_sw_get_populations(h: int, dst: int, on_device: bool) -> None:
    _check(load().lbm_sw_get_populations(h, dst, int(on_device)), h, "lbm_sw_get_populations")


def lbm_sw_set_populations(h: int, src: int, on_device: bool, form: int) -> None:
    _check(load().lbm_sw_set_populations(h, src, int(on_device), int(form)), h, "lbm_sw_set_populations")


def lbm_sw_get_rows(h: int, y0: int, nrows: int, dst: int, on_device: bool) -> None:
    _check(load().lbm_sw_get_rows(h, int(y0), int(nrows), dst, int(on_device)), h, "lbm_sw_get_rows")


def lbm_sw_set_rows(h: int, y0: int, nrows: int, src: int, on_device: bool) -> None:
    _check(load().lbm_sw_set_rows(h, int(y0), int(nrows), src, int(on_device)), h, "lbm_sw_set_rows")


def lbm_sw_diagnostics_rows(h: int, y0: int, nrows: int, raise_unstable: bool = True):
    """Returns (sum h, sum hu, sum hv, min h, status) over rows [y0, y0 + nrows)."""
    out = (ctypes.c_double * 4)()
    st = load().lbm_sw_diagnostics_rows(h, int(y0), int(nrows), out)
    if st != E_UNSTABLE or raise_unstable:
        _check(st, h, "lbm_sw_diagnostics_rows")
    return out[0], out[1], out[2], out[3], st


def lbm_sw_synchronize(h: int) -> None:
    _check(load().lbm_sw_synchronize(h), h, "lbm_sw_synchronize")


def lbm_sw_get_info(h: int) -> lbm_sw_info:
    info = lbm_sw_info()
    _check(load().lbm_sw_get_info(h, ctypes.byref(info)), h, "lbm_sw_get_info")
    return info


def lbm_sw_abi_version() -> int:
    return load().lbm_sw_abi_version()


NOALLOC_MAX_ROWS = 8192  # LBM_SW_NOALLOC_MAX_ROWS


def lbm_sw_diagnostics_noalloc(populations: int, dim: int, precision: int, nx: int, ny: int, row_pitch: int,
                               plane_pitch: int, out: int, stream: int | None) -> None:
    """Allocation-free diagnostics for callers that may not allocate device memory when
    they check a state (see include/lbm_sw.h).  ``populations`` and ``out`` (5 doubles)
    are device addresses; the result is written asynchronously on ``stream``."""
    st = load().lbm_sw_diagnostics_noalloc(populations, int(dim), int(precision), int(nx), int(ny),
                                           int(row_pitch), int(plane_pitch), out, stream)
    if st == E_ARG and ny > NOALLOC_MAX_ROWS:
        raise LbmSwError(st, f"lbm_sw_diagnostics_noalloc: ny = {ny} rows exceeds the static scratch "
                             f"capacity of {NOALLOC_MAX_ROWS} rows")
    _check(st, None, "lbm_sw_diagnostics_noalloc")


def _bcheck(status: int, b, what: str) -> int:
    if status < 0:
        lib = load()
        msg = lib.lbm_sw_batch_last_error(b).decode() if b else ""
        raise LbmSwError(status, f"{what}: {msg or lib.lbm_sw_status_string(status).decode()}")
    return status


def lbm_sw_batch_params_init() -> lbm_sw_batch_params:
    p = lbm_sw_batch_params()
    _check(load().lbm_sw_batch_params_init(ctypes.byref(p)))
    return p


def lbm_sw_batch_create(p: lbm_sw_batch_params) -> int:
    lib = load()
    b = ctypes.c_void_p()
    st = lib.lbm_sw_batch_create(ctypes.byref(p), ctypes.byref(b))
    if st < 0:
        raise LbmSwError(st, "lbm_sw_batch_create: " + (lib.lbm_sw_create_error().decode() or
                                                        lib.lbm_sw_status_string(st).decode()))
    return b.value


def lbm_sw_batch_destroy(b: int) -> None:
    load().lbm_sw_batch_destroy(b)


def lbm_sw_batch_set_state(b: int, i: int, depth: int, hu: int, hv: int | None, on_device: bool) -> None:
    _bcheck(load().lbm_sw_batch_set_state(b, int(i), depth, hu, hv, int(on_device)), b, "lbm_sw_batch_set_state")


def lbm_sw_batch_step(b: int, n: int) -> None:
    _bcheck(load().lbm_sw_batch_step(b, int(n)), b, "lbm_sw_batch_step")


def lbm_sw_batch_get_moments(b: int, i: int, depth: int, hu: int, hv: int | None, on_device: bool) -> None:
    _bcheck(load().lbm_sw_batch_get_moments(b, int(i), depth, hu, hv, int(on_device)), b, "lbm_sw_batch_get_moments")


def lbm_sw_batch_get_populations(b: int, i: int, dst: int, on_device: bool) -> None:
    _bcheck(load().lbm_sw_batch_get_populations(b, int(i), dst, int(on_device)), b, "lbm_sw_batch_get_populations")


def lbm_sw_batch_diagnostics(b: int, i: int, raise_unstable: bool = True):
    out = (ctypes.c_double * 4)()
    st = load().lbm_sw_batch_diagnostics(b, int(i), out)
    if st != E_UNSTABLE or raise_unstable:
        _bcheck(st, b, "lbm_sw_batch_diagnostics")
    return out[0], out[1], out[2], out[3], st


def lbm_sw_batch_autotune(b: int, trial_steps: int) -> lbm_sw_batch_tuning:
    t = lbm_sw_batch_tuning()
    _bcheck(load().lbm_sw_batch_autotune(b, int(trial_steps), ctypes.byref(t)), b, "lbm_sw_batch_autotune")
    return t


def lbm_sw_batch_get_tuning(b: int) -> lbm_sw_batch_tuning:
    t = lbm_sw_batch_tuning()
    _bcheck(load().lbm_sw_batch_get_tuning(b, ctypes.byref(t)), b, "lbm_sw_batch_get_tuning")
    return t


def _tcheck(status: int, t, h, what: str) -> int:
    if status < 0:
        lib = load()
        msg = (lib.lbm_sw_tape_last_error(t).decode() if t else "") or (lib.lbm_sw_last_error(h).decode() if h else "")
        raise LbmSwError(status, f"{what}: {msg or lib.lbm_sw_status_string(status).decode()}")
    return status


def lbm_sw_tape_create(h: int, steps: int, interval: int = 0) -> int:
    t = ctypes.c_void_p()
    _tcheck(load().lbm_sw_tape_create(h, int(steps), int(interval), ctypes.byref(t)), None, h, "lbm_sw_tape_create")
    return t.value


def lbm_sw_tape_destroy(t: int) -> None:
    load().lbm_sw_tape_destroy(t)


def lbm_sw_forward_record(h: int, t: int) -> None:
    _tcheck(load().lbm_sw_forward_record(h, t), t, h, "lbm_sw_forward_record")


def lbm_sw_adjoint(h: int, t: int, g_h: int, g_hu: int | None, g_hv: int | None, d_h: int, d_hu: int | None,
                   d_hv: int | None, on_device: bool) -> None:
    _tcheck(load().lbm_sw_adjoint(h, t, g_h, g_hu, g_hv, d_h, d_hu, d_hv, int(on_device)), t, h, "lbm_sw_adjoint")


def lbm_sw_tape_get_info(t: int) -> lbm_sw_tape_info:
    info = lbm_sw_tape_info()
    _tcheck(load().lbm_sw_tape_get_info(t, ctypes.byref(info)), t, None, "lbm_sw_tape_get_info")
    return info


# ---------------------------------------------------------------- convenience
def make_params(nx: int, ny: int = 1, *, dim: int | None = None, precision: int = FP32, g: float = 1.0,
                lam: float = 8.0, s: float = 1.8, a: float | None = None, bc=(PERIODIC,) * 4, inflow=None,
                stream: int | None = None, kernel: int = KERNEL_AUTO, graph_chunk: int = 0,
                temporal_steps: int = 0) -> lbm_sw_params:
    dim = 2 if dim is None else int(dim)
    p = lbm_sw_params_init()
    p.dim, p.nx, p.ny, p.precision = dim, int(nx), int(ny), int(precision)
    p.g, p.lambda_, p.s = float(g), float(lam), float(s)
    p.a = float(a if a is not None else (0.15 if dim == 1 else 0.05))
    bc = list(bc) + [PERIODIC] * (4 - len(bc))
    for k in range(4):
        p.bc[k] = int(bc[k])
    if inflow is not None:
        for k in range(min(4, len(inflow))):
            if inflow[k] is not None:
                for c, v in enumerate(inflow[k]):
                    p.inflow[k][c] = float(v)
    p.stream = stream
    p.kernel = int(kernel)
    p.graph_chunk = int(graph_chunk)
    p.temporal_steps = int(temporal_steps)
    return p


def _ptr(x, on_device: bool, dtype: str | None = None, count: int | None = None, what: str = "buffer"):
    """Address of a contiguous numpy array or torch tensor (and whether it is on the GPU).

    With ``dtype`` ("float64", "float32", "uint8") and ``count`` the buffer is checked first:
    the C library reads or writes exactly ``count`` elements of that type through the pointer,
    so a buffer of another type or size is refused here, before any copy."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        name, n = str(x.dtype).replace("torch.", ""), x.numel()
    else:
        if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
            raise ValueError(f"{what}: expected a C-contiguous numpy array or a torch tensor")
        name, n = x.dtype.name, x.size
    if dtype is not None and name != dtype:
        raise ValueError(f"{what}: dtype {name}, expected {dtype}")
    if count is not None and n != count:
        raise ValueError(f"{what}: {n} elements, expected {count}")
    return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data


class Simulation:
    """Owner of one lbm_sw handle.  Moment arrays are FP64 [ny][nx]; populations
    [q][ny][nx] in the handle's precision.  numpy arrays cross as host memory,
    torch CUDA tensors as device memory."""

    def __init__(self, nx: int, ny: int = 1, **kw):
        self.params = make_params(nx, ny, **kw)
        self.handle = lbm_sw_create(self.params)
        self.nx, self.ny, self.dim = self.params.nx, self.params.ny, self.params.dim
        self.q = 5 if self.dim == 1 else 13
        self.dtype = np.float64 if self.params.precision == FP64 else np.float32

    def close(self):
        if self.handle:
            lbm_sw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _on_device(x) -> bool:
        return hasattr(x, "is_cuda") and bool(x.is_cuda)

    def set_state(self, h, hu, hv=None):
        dev = self._on_device(h)
        if not dev:
            h, hu = (np.ascontiguousarray(x, dtype=np.float64) for x in (h, hu))
            hv = None if hv is None else np.ascontiguousarray(hv, dtype=np.float64)
        n = self.nx * self.ny
        lbm_sw_set_state(self.handle, _ptr(h, dev, "float64", n, "h"), _ptr(hu, dev, "float64", n, "hu"),
                         _ptr(hv, dev, "float64", n, "hv"), dev)

    def step(self, n: int = 1):
        lbm_sw_step(self.handle, n)

    def step_plan(self, n: int) -> list[int]:
        """Steps per kernel launch of ``step(n)``, in order (nothing is launched)."""
        return lbm_sw_step_plan(self.handle, n)

    def set_relaxation(self, rates=None):
        lbm_sw_set_relaxation(self.handle, rates)

    def set_obstacle(self, solid=None):
        """Solid cells: a [ny][nx] array (numpy, or a uint8 CUDA tensor), nonzero = solid;
        None removes the obstacles."""
        if solid is None:
            lbm_sw_set_obstacle(self.handle, None, False)
            return
        dev = self._on_device(solid)
        if not dev:
            solid = np.ascontiguousarray(np.asarray(solid) != 0, dtype=np.uint8)
        if tuple(solid.shape) != (self.ny, self.nx):
            raise ValueError(f"solid must have shape ({self.ny}, {self.nx})")
        lbm_sw_set_obstacle(self.handle, _ptr(solid, dev, "uint8", self.nx * self.ny, "solid"), dev)

    def moments(self):
        h = np.empty((self.ny, self.nx))
        hu = np.empty_like(h)
        hv = np.empty_like(h) if self.dim == 2 else None
        lbm_sw_get_moments(self.handle, _ptr(h, False), _ptr(hu, False), _ptr(hv, False), False)
        return (h, hu, hv) if self.dim == 2 else (h[0], hu[0])

    def moments_into(self, h, hu, hv=None):
        dev = self._on_device(h)
        n = self.nx * self.ny
        lbm_sw_get_moments(self.handle, _ptr(h, dev, "float64", n, "h"), _ptr(hu, dev, "float64", n, "hu"),
                           _ptr(hv, dev, "float64", n, "hv"), dev)

    def populations(self) -> np.ndarray:
        out = np.empty((self.q, self.ny, self.nx), dtype=self.dtype)
        lbm_sw_get_populations(self.handle, _ptr(out, False), False)
        return out

    def populations_into(self, out):
        dev = self._on_device(out)
        lbm_sw_get_populations(self.handle, _ptr(out, dev, np.dtype(self.dtype).name, self.q * self.nx * self.ny,
                                                 "populations"), dev)

    def set_populations(self, F, form: int = POST_COLLISION):
        dev = self._on_device(F)
        if not dev:
            F = np.ascontiguousarray(F, dtype=self.dtype).reshape(self.q, self.ny, self.nx)
        lbm_sw_set_populations(self.handle, _ptr(F, dev, np.dtype(self.dtype).name, self.q * self.nx * self.ny,
                                                 "populations"), dev, form)

    def diagnostics(self, raise_unstable: bool = True):
        return lbm_sw_diagnostics(self.handle, raise_unstable)

    def diagnostics_rows(self, y0: int, nrows: int, raise_unstable: bool = True):
        return lbm_sw_diagnostics_rows(self.handle, y0, nrows, raise_unstable)

    def get_rows_into(self, y0: int, nrows: int, out):
        """Rows [y0, y0 + nrows) of every plane into ``out`` ([q][nrows][nx], numpy or CUDA tensor)."""
        dev = self._on_device(out)
        lbm_sw_get_rows(self.handle, y0, nrows, _ptr(out, dev, np.dtype(self.dtype).name, self.q * nrows * self.nx,
                                                     "rows"), dev)

    def set_rows(self, y0: int, nrows: int, src):
        """Rows [y0, y0 + nrows) of every plane from ``src`` ([q][nrows][nx])."""
        dev = self._on_device(src)
        if not dev:
            src = np.ascontiguousarray(src, dtype=self.dtype)
        lbm_sw_set_rows(self.handle, y0, nrows, _ptr(src, dev, np.dtype(self.dtype).name, self.q * nrows * self.nx,
                                                     "rows"), dev)

    def synchronize(self):
        lbm_sw_synchronize(self.handle)

    def info(self) -> lbm_sw_info:
        return lbm_sw_get_info(self.handle)


class Batch:
    """Owner of one lbm_sw_batch: many independent 2D grids advanced by one launch per step."""

    def __init__(self, sizes, *, precision: int = FP32, g: float = 1.0, lam: float = 8.0, s: float = 1.8,
                 a: float = 0.05, bc=(PERIODIC,) * 4, inflow=None, stream: int | None = None, tile_rows: int = 0,
                 ctas_per_sm: int = 0, graph_chunk: int = 0, temporal_steps: int = 0):
        self.sizes = [(int(nx), int(ny)) for nx, ny in sizes]
        self._nx = (ctypes.c_int * len(self.sizes))(*[nx for nx, _ in self.sizes])
        self._ny = (ctypes.c_int * len(self.sizes))(*[ny for _, ny in self.sizes])
        p = lbm_sw_batch_params_init()
        p.count, p.nx, p.ny, p.precision = len(self.sizes), self._nx, self._ny, int(precision)
        p.g, p.lambda_, p.s, p.a = float(g), float(lam), float(s), float(a)
        for k in range(4):
            p.bc[k] = int(bc[k])
        if inflow is not None:
            for k in range(4):
                if inflow[k] is not None:
                    for c, v in enumerate(inflow[k]):
                        p.inflow[k][c] = float(v)
        p.stream = stream
        p.tile_rows, p.ctas_per_sm, p.graph_chunk = int(tile_rows), int(ctas_per_sm), int(graph_chunk)
        p.temporal_steps = int(temporal_steps)
        self.params = p
        self.handle = lbm_sw_batch_create(p)
        self.dtype = np.float64 if precision == FP64 else np.float32

    def close(self):
        if self.handle:
            lbm_sw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, i: int, h, hu, hv=None):
        dev = Simulation._on_device(h)
        if not dev:
            h, hu = (np.ascontiguousarray(x, dtype=np.float64) for x in (h, hu))
            hv = None if hv is None else np.ascontiguousarray(hv, dtype=np.float64)
        # an index out of range is the library's to refuse (LBM_SW_E_ARG)
        n = self.sizes[i][0] * self.sizes[i][1] if 0 <= i < len(self.sizes) else None
        lbm_sw_batch_set_state(self.handle, i, _ptr(h, dev, "float64", n, "h"), _ptr(hu, dev, "float64", n, "hu"),
                               _ptr(hv, dev, "float64", n, "hv"), dev)

    def step(self, n: int = 1):
        lbm_sw_batch_step(self.handle, n)

    def moments(self, i: int):
        nx, ny = self.sizes[i]
        out = [np.empty((ny, nx)) for _ in range(3)]
        lbm_sw_batch_get_moments(self.handle, i, *[_ptr(o, False) for o in out], False)
        return tuple(out)

    def populations(self, i: int) -> np.ndarray:
        nx, ny = self.sizes[i]
        out = np.empty((13, ny, nx), dtype=self.dtype)
        lbm_sw_batch_get_populations(self.handle, i, _ptr(out, False), False)
        return out

    def diagnostics(self, i: int, raise_unstable: bool = True):
        return lbm_sw_batch_diagnostics(self.handle, i, raise_unstable)

    def autotune(self, trial_steps: int = 5) -> lbm_sw_batch_tuning:
        return lbm_sw_batch_autotune(self.handle, trial_steps)

    def tuning(self) -> lbm_sw_batch_tuning:
        return lbm_sw_batch_get_tuning(self.handle)


class Tape:
    """Checkpoint tape of a forward run of a 2D Simulation, for the discrete adjoint."""

    def __init__(self, sim: Simulation, steps: int, interval: int = 0):
        self.sim = sim
        self.handle = lbm_sw_tape_create(sim.handle, steps, interval)

    def close(self):
        if self.handle:
            lbm_sw_tape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def record(self):
        lbm_sw_forward_record(self.sim.handle, self.handle)

    def adjoint(self, g_h, g_hu=None, g_hv=None, want_momentum: bool = False):
        """dL/dW^0 from dL/dW^T.  numpy in, numpy out (host), or torch CUDA in, torch out."""
        dev = Simulation._on_device(g_h)
        ny, nx = self.sim.ny, self.sim.nx
        if dev:
            import torch

            outs = [torch.empty((ny, nx), dtype=torch.float64, device=g_h.device)
                    for _ in range(3 if want_momentum else 1)]
        else:
            g_h = np.ascontiguousarray(g_h, dtype=np.float64)
            g_hu = None if g_hu is None else np.ascontiguousarray(g_hu, dtype=np.float64)
            g_hv = None if g_hv is None else np.ascontiguousarray(g_hv, dtype=np.float64)
            outs = [np.empty((ny, nx)) for _ in range(3 if want_momentum else 1)]
        d = [outs[0], outs[1] if want_momentum else None, outs[2] if want_momentum else None]
        n = nx * ny
        g = [_ptr(x, dev, "float64", n, w) for x, w in ((g_h, "g_h"), (g_hu, "g_hu"), (g_hv, "g_hv"))]
        lbm_sw_adjoint(self.sim.handle, self.handle, *g, _ptr(d[0], dev), _ptr(d[1], dev), _ptr(d[2], dev), dev)
        return tuple(outs) if want_momentum else outs[0]

    def info(self) -> lbm_sw_tape_info:
        return lbm_sw_tape_get_info(self.handle)
