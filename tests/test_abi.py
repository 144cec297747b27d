"""The C ABI library loads without a GPU, exports every entry point that
include/lbm_sw.h declares, and its host-side argument checks reject bad input.
No test here launches a kernel."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1401_0427_gb300 import build as libbuild
from paper_1401_0427_gb300 import lbm_sw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_entry_points():
    names = []
    for hdr in HEADERS:
        text = open(hdr).read()
        names += re.findall(r"^LBM_SW_API\s+[\w\s\*]+?\b(lbm_sw\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return lbm_sw.load()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["lbm_sw_create", "lbm_sw_set_state", "lbm_sw_step", "lbm_sw_get_moments", "lbm_sw_destroy",
                     "lbm_sw_diagnostics", "lbm_sw_get_populations", "lbm_sw_set_populations"]:
        assert required in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_entry_points()
    assert len(names) == len(set(names))
    for name in names:
        assert hasattr(lib, name), name
        assert name in lbm_sw.SIGNATURES, f"{name} has no binding"
    assert set(lbm_sw.SIGNATURES) <= set(names)


def test_exports_are_only_the_declared_ones(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lbm_sw.library_path()], capture_output=True, text=True).stdout
    exported = {m for m in re.findall(r" T (lbm_sw\w+)", out)}
    assert exported == set(declared_entry_points())


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lbm_sw.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_sw_params), offsetof(lbm_sw_params, g),\n'
        "   offsetof(lbm_sw_params, bc), offsetof(lbm_sw_params, inflow), offsetof(lbm_sw_params, stream),\n"
        "   offsetof(lbm_sw_params, kernel), offsetof(lbm_sw_params, reserved));\n"
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(lbm_sw_info), offsetof(lbm_sw_info, pitch),\n'
        "   offsetof(lbm_sw_info, bytes_per_update), offsetof(lbm_sw_info, kernel_launches),\n"
        "   offsetof(lbm_sw_info, steps_per_launch));\n"
        ' printf("%zu %zu %zu %zu %zu\\n", sizeof(lbm_sw_batch_params), offsetof(lbm_sw_batch_params, stream),\n'
        "   offsetof(lbm_sw_batch_params, temporal_steps), sizeof(lbm_sw_batch_tuning),\n"
        "   offsetof(lbm_sw_batch_tuning, temporal_steps));\n"
        " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_params, c_info, c_batch = subprocess.run([str(exe)], capture_output=True, text=True,
                                               check=True).stdout.split("\n")[:3]
    P, I = lbm_sw.lbm_sw_params, lbm_sw.lbm_sw_info
    py_params = [ctypes.sizeof(P), P.g.offset, P.bc.offset, P.inflow.offset, P.stream.offset, P.kernel.offset,
                 P.reserved.offset]
    py_info = [ctypes.sizeof(I), I.pitch.offset, I.bytes_per_update.offset, I.kernel_launches.offset,
               I.steps_per_launch.offset]
    assert [int(v) for v in c_params.split()] == py_params
    assert [int(v) for v in c_info.split()] == py_info
    B, BT = lbm_sw.lbm_sw_batch_params, lbm_sw.lbm_sw_batch_tuning
    py_batch = [ctypes.sizeof(B), B.stream.offset, B.temporal_steps.offset, ctypes.sizeof(BT), BT.temporal_steps.offset]
    assert [int(v) for v in c_batch.split()] == py_batch


def test_params_defaults(lib):
    p = lbm_sw.lbm_sw_params_init()
    assert (p.dim, p.precision, p.g, p.lambda_, p.s, p.a) == (2, lbm_sw.FP32, 1.0, 8.0, 1.8, 0.05)
    assert list(p.bc) == [lbm_sw.PERIODIC] * 4 and p.stream is None and list(p.reserved) == [0] * 5
    assert lib.lbm_sw_abi_version() == 1
    assert lib.lbm_sw_params_init(None) == lbm_sw.E_ARG


def _bad(**changes):
    p = lbm_sw.make_params(16, 16)
    for k, v in changes.items():
        if k == "bc":
            for i, b in enumerate(v):
                p.bc[i] = b
        elif k == "reserved":
            p.reserved[0] = v
        elif k == "inflow_h":
            p.inflow[0][0] = v
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("changes,needle", [
    (dict(dim=3), "dim"),
    (dict(nx=0), "nx"),
    (dict(dim=1, ny=2), "ny must be 1"),
    (dict(precision=2), "precision"),
    (dict(g=-1.0), "g must"),
    (dict(lambda_=0.0), "lambda"),
    (dict(s=2.0), "s must"),
    (dict(s=float("nan")), "s must"),
    (dict(a=-0.1), "a must"),
    (dict(bc=[7, 0, 0, 0]), "bc[0]"),
    (dict(bc=[lbm_sw.PERIODIC, lbm_sw.WALL, 0, 0]), "pairs"),
    (dict(bc=[lbm_sw.INFLOW, lbm_sw.WALL, 0, 0], inflow_h=0.0), "inflow[0]"),
    (dict(kernel=9), "kernel"),
    (dict(kernel=3), "CLUSTER is for 1D"),
    (dict(temporal_steps=9), "temporal_steps"),
    (dict(reserved=1), "reserved"),
])
def test_create_rejects_bad_parameters_before_touching_the_gpu(lib, changes, needle):
    with pytest.raises(lbm_sw.LbmSwError) as ei:
        lbm_sw.lbm_sw_create(_bad(**changes))
    assert ei.value.status == lbm_sw.E_ARG
    assert needle in str(ei.value)


def test_null_arguments(lib):
    assert lib.lbm_sw_create(None, None) == lbm_sw.E_ARG
    out = ctypes.c_void_p()
    assert lib.lbm_sw_create(None, ctypes.byref(out)) == lbm_sw.E_ARG and not out.value
    assert lib.lbm_sw_step(None, 1) == lbm_sw.E_ARG
    assert lib.lbm_sw_set_state(None, None, None, None, 0) == lbm_sw.E_ARG
    assert lib.lbm_sw_get_moments(None, None, None, None, 0) == lbm_sw.E_ARG
    assert lib.lbm_sw_diagnostics(None, None) == lbm_sw.E_ARG
    assert lib.lbm_sw_synchronize(None) == lbm_sw.E_ARG
    assert lib.lbm_sw_get_info(None, None) == lbm_sw.E_ARG
    assert lib.lbm_sw_step_plan(None, 4, None, 0) == lbm_sw.E_ARG
    assert lib.lbm_sw_get_rows(None, 0, 1, None, 0) == lbm_sw.E_ARG
    assert lib.lbm_sw_set_rows(None, 0, 1, None, 0) == lbm_sw.E_ARG
    assert lib.lbm_sw_diagnostics_rows(None, 0, 1, None) == lbm_sw.E_ARG
    lib.lbm_sw_destroy(None)  # NULL-safe
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert lib.lbm_sw_status_string(code)


def _batch_params(**changes):
    nx = (ctypes.c_int * 2)(8, 16)
    ny = (ctypes.c_int * 2)(8, 4)
    p = lbm_sw.lbm_sw_batch_params_init()
    p.count, p.nx, p.ny = 2, nx, ny
    for k, v in changes.items():
        setattr(p, k, v)
    return p, (nx, ny)


@pytest.mark.parametrize("changes,needle", [
    (dict(count=0), "count"),
    (dict(nx=None), "arrays"),
    (dict(tile_rows=3), "tile_rows"),
    (dict(ctas_per_sm=40), "ctas_per_sm"),
    (dict(s=-0.1), "s must"),
    (dict(precision=5), "precision"),
])
def test_batch_create_rejects_bad_parameters(lib, changes, needle):
    p, keep = _batch_params(**changes)
    with pytest.raises(lbm_sw.LbmSwError) as ei:
        lbm_sw.lbm_sw_batch_create(p)
    assert ei.value.status == lbm_sw.E_ARG and needle in str(ei.value)


def test_batch_rejects_a_zero_width_instance(lib):
    p, keep = _batch_params()
    keep[0][1] = 0
    with pytest.raises(lbm_sw.LbmSwError) as ei:
        lbm_sw.lbm_sw_batch_create(p)
    assert "instance 1" in str(ei.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the compiled CUDA library the binding raises: there is no CPU fallback."""
    monkeypatch.setattr(lbm_sw, "_lib", None)
    with pytest.raises(ImportError, match="no CPU fallback"):
        lbm_sw.load(str(tmp_path / "liblbm_sw.so"))


def test_no_gpu_means_an_error_not_a_fallback(lib):
    """On a machine without a GPU, creating a handle fails with the CUDA status instead of
    computing anywhere else."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm_sw.LbmSwError) as err:
        lbm_sw.Simulation(16, 16)
    assert err.value.status == lbm_sw.E_CUDA


def _handleless(nx, ny, precision=lbm_sw.FP32, dim=2):
    """A Simulation object without a handle: enough to exercise the binding's own checks,
    which run before any call into the library."""
    sim = object.__new__(lbm_sw.Simulation)
    sim.handle, sim.nx, sim.ny, sim.dim = None, nx, ny, dim
    sim.q = 13 if dim == 2 else 5
    sim.dtype = np.float64 if precision == lbm_sw.FP64 else np.float32
    return sim


def test_binding_refuses_buffers_of_another_type_or_size():
    """The C library reads or writes a fixed number of elements of a fixed type through each
    pointer: the binding refuses any other buffer before the call."""
    sim = _handleless(6, 4)
    ok = [np.empty((4, 6)) for _ in range(3)]
    with pytest.raises(ValueError, match="dtype float32, expected float64"):
        sim.moments_into(np.empty((4, 6), np.float32), *ok[1:])
    with pytest.raises(ValueError, match="23 elements, expected 24"):
        sim.moments_into(ok[0], np.empty(23), ok[2])
    with pytest.raises(ValueError, match="contiguous"):
        sim.moments_into(np.empty((4, 12))[:, ::2], *ok[1:])
    with pytest.raises(ValueError, match="dtype float64, expected float32"):
        sim.populations_into(np.empty((13, 4, 6)))
    with pytest.raises(ValueError, match="expected 312"):
        sim.populations_into(np.empty((13, 4, 5), np.float32))
    with pytest.raises(ValueError, match="expected 24"):
        sim.set_state(np.ones((4, 5)), np.zeros((4, 6)), np.zeros((4, 6)))
    with pytest.raises(ValueError, match="solid must have shape"):
        sim.set_obstacle(np.zeros((4, 5), np.uint8))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="dtype float32, expected float64"):
        sim.moments_into(torch.empty((4, 6), dtype=torch.float32), *ok[1:])
    with pytest.raises(ValueError, match="dtype float64, expected float32"):
        sim.populations_into(torch.empty((13, 4, 6), dtype=torch.float64))
    one_d = _handleless(10, 1, lbm_sw.FP64, dim=1)
    with pytest.raises(ValueError, match="expected 50"):
        one_d.populations_into(np.empty((5, 9)))
