"""FP64 CPU oracle for the D1Q3Q2 and D2Q5Q4Q4 vectorial lattice Boltzmann schemes.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
(``paper_1401_0427_gb300``) never does, and it shares no code with it.

The arithmetic lives in ``lbm_oracle.cpp`` (plain loops, FP64, the paper's
steps in the paper's order: moments, entropy variables, equilibria from the
potentials, relaxation, streaming with explicit ghost cells).  This module only
compiles it with g++ and marshals numpy arrays through ctypes.

Population order: 1D ``f0 f+ f- g+ g-``; 2D ``f0 f1 f2 f3 f4 gx1 gx2 gx3 gx4
gy1 gy2 gy3 gy4`` with v1 = (lam, 0), v2 = (0, lam), v3 = (-lam, 0),
v4 = (0, -lam) (section 3, Eq. 3-stencil-d2q5).  Arrays are ``[q][ny][nx]``
(x fastest), pre-collision populations unless a function says otherwise.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")

PERIODIC, WALL, OUTFLOW, INFLOW = 0, 1, 2, 3
XM, XP, YM, YP = 0, 1, 2, 3


class OracleParams(ctypes.Structure):
    """Field-for-field mirror of ``struct oracle_params`` in lbm_oracle.cpp."""

    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("g", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("s", ctypes.c_double),
        ("a", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("inflow", (ctypes.c_double * 3) * 4),
        ("mrt", ctypes.c_int),
        ("s_moments", ctypes.c_double * 13),
        ("solid", ctypes.c_void_p),
    ]


def params(nx, ny=1, *, g=1.0, lam=8.0, s=1.8, a=0.05, bc=(PERIODIC,) * 4,
           inflow=None, s_moments=None, solid=None) -> OracleParams:
    """Build an ``OracleParams``; ``s_moments`` (13 or 5 rates) switches on MRT; ``solid``
    (2D, ``[ny][nx]``, nonzero = solid) places obstacles with mirror walls on their faces."""
    p = OracleParams()
    p.nx, p.ny = int(nx), int(ny)
    p.g, p.lam, p.s, p.a = float(g), float(lam), float(s), float(a)
    bc = list(bc) + [PERIODIC] * (4 - len(bc))
    for k in range(4):
        p.bc[k] = int(bc[k])
    if inflow is not None:
        for k in range(4):
            w = inflow[k] if inflow[k] is not None else (1.0, 0.0, 0.0)
            for c in range(len(w)):
                p.inflow[k][c] = float(w[c])
    p.mrt = 0
    if s_moments is not None:
        p.mrt = 1
        for k, v in enumerate(s_moments):
            p.s_moments[k] = float(v)
    p.solid = None
    if solid is not None:
        mask = np.ascontiguousarray(np.asarray(solid) != 0, dtype=np.uint8)
        if mask.shape != (int(ny), int(nx)):
            raise ValueError(f"solid must have shape ({ny}, {nx})")
        p._solid_keep = mask  # the struct holds a raw pointer: keep the array alive with it
        p.solid = mask.ctypes.data
    return p


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liblbm_oracle.so`` (g++, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """The compiled oracle; ``LBM_ORACLE_LIB`` names another build of this source to load
    instead (the planted-mistake tests point the pins at mutated copies this way)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("LBM_ORACLE_LIB") or build()
            _lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(OracleParams)
            sigs = {
                "oracle_equilibrium_1d": [dp, dp, dp, pp],
                "oracle_moments_1d": [dp, dp, dp, pp],
                "oracle_collide_1d": [dp, pp],
                "oracle_stream_1d": [dp, dp, pp],
                "oracle_run_1d": [dp, ctypes.c_int, pp],
                "oracle_equilibrium_2d": [dp, dp, dp, dp, pp],
                "oracle_moments_2d": [dp, dp, dp, dp, pp],
                "oracle_collide_2d": [dp, pp],
                "oracle_stream_2d": [dp, dp, pp],
                "oracle_run_2d": [dp, ctypes.c_int, pp],
                "oracle_equilibrium_2d_cplx": [dp] * 8 + [pp],
                "oracle_run_2d_cplx": [dp, dp, ctypes.c_int, pp],
                "oracle_equilibrium_1d_cplx": [dp] * 6 + [pp],
                "oracle_run_1d_cplx": [dp, dp, ctypes.c_int, pp],
            }
            for name, args in sigs.items():
                fn = getattr(_lib, name)
                fn.argtypes = args
                fn.restype = None
            _lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib.oracle_set_threads.restype = ctypes.c_int
        return _lib


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (n <= 0: every core this process may run on); returns the
    count in use."""
    if n <= 0:
        n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return lib().oracle_set_threads(int(n))


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- 1D (D1Q3Q2)
def equilibrium_1d(rho, q, p: OracleParams) -> np.ndarray:
    rho, q = _f64(rho).reshape(-1), _f64(q).reshape(-1)
    assert rho.size == q.size == p.nx
    F = np.empty((5, p.nx))
    lib().oracle_equilibrium_1d(_d(rho), _d(q), _d(F), ctypes.byref(p))
    return F


def moments_1d(F, p: OracleParams):
    F = _f64(F)
    rho, q = np.empty(p.nx), np.empty(p.nx)
    lib().oracle_moments_1d(_d(F), _d(rho), _d(q), ctypes.byref(p))
    return rho, q


def collide_1d(F, p: OracleParams) -> np.ndarray:
    F = _f64(F).copy()
    lib().oracle_collide_1d(_d(F), ctypes.byref(p))
    return F


def stream_1d(Fs, p: OracleParams) -> np.ndarray:
    Fs = _f64(Fs)
    F = np.empty_like(Fs)
    lib().oracle_stream_1d(_d(Fs), _d(F), ctypes.byref(p))
    return F


def run_1d(F, nsteps: int, p: OracleParams) -> np.ndarray:
    """``nsteps`` of (collide, stream) from pre-collision ``F``; returns pre-collision."""
    F = _f64(F).copy()
    assert F.shape == (5, p.nx)
    lib().oracle_run_1d(_d(F), int(nsteps), ctypes.byref(p))
    return F


def run_1d_cplx(F: np.ndarray, nsteps: int, p: OracleParams) -> np.ndarray:
    re, im = _f64(F.real).copy(), _f64(F.imag).copy()
    lib().oracle_run_1d_cplx(_d(re), _d(im), int(nsteps), ctypes.byref(p))
    return re + 1j * im


def equilibrium_1d_cplx(rho, q, p: OracleParams) -> np.ndarray:
    rho, q = np.asarray(rho, complex).reshape(-1), np.asarray(q, complex).reshape(-1)
    a = [_f64(x) for x in (rho.real, rho.imag, q.real, q.imag)]
    re, im = np.empty((5, p.nx)), np.empty((5, p.nx))
    lib().oracle_equilibrium_1d_cplx(*[_d(x) for x in a], _d(re), _d(im), ctypes.byref(p))
    return re + 1j * im


# ------------------------------------------------------------- 2D (D2Q5Q4Q4)
def equilibrium_2d(rho, qx, qy, p: OracleParams) -> np.ndarray:
    rho, qx, qy = (_f64(x).reshape(-1) for x in (rho, qx, qy))
    n = p.nx * p.ny
    assert rho.size == qx.size == qy.size == n
    F = np.empty((13, p.ny, p.nx))
    lib().oracle_equilibrium_2d(_d(rho), _d(qx), _d(qy), _d(F), ctypes.byref(p))
    return F


def moments_2d(F, p: OracleParams):
    F = _f64(F)
    out = [np.empty((p.ny, p.nx)) for _ in range(3)]
    lib().oracle_moments_2d(_d(F), *[_d(o) for o in out], ctypes.byref(p))
    return tuple(out)


def collide_2d(F, p: OracleParams) -> np.ndarray:
    F = _f64(F).copy()
    lib().oracle_collide_2d(_d(F), ctypes.byref(p))
    return F


def stream_2d(Fs, p: OracleParams) -> np.ndarray:
    Fs = _f64(Fs)
    F = np.empty_like(Fs)
    lib().oracle_stream_2d(_d(Fs), _d(F), ctypes.byref(p))
    return F


def run_2d(F, nsteps: int, p: OracleParams) -> np.ndarray:
    """``nsteps`` of (collide, stream) from pre-collision ``F``; returns pre-collision."""
    F = _f64(F).copy()
    assert F.shape == (13, p.ny, p.nx)
    lib().oracle_run_2d(_d(F), int(nsteps), ctypes.byref(p))
    return F


def equilibrium_2d_cplx(rho, qx, qy, p: OracleParams) -> np.ndarray:
    arrs = [np.asarray(x, complex).reshape(-1) for x in (rho, qx, qy)]
    parts = []
    for x in arrs:
        parts += [_f64(x.real), _f64(x.imag)]
    re, im = np.empty((13, p.ny, p.nx)), np.empty((13, p.ny, p.nx))
    lib().oracle_equilibrium_2d_cplx(*[_d(x) for x in parts], _d(re), _d(im), ctypes.byref(p))
    return re + 1j * im


def run_2d_cplx(F: np.ndarray, nsteps: int, p: OracleParams) -> np.ndarray:
    re, im = _f64(F.real).copy(), _f64(F.imag).copy()
    lib().oracle_run_2d_cplx(_d(re), _d(im), int(nsteps), ctypes.byref(p))
    return re + 1j * im
