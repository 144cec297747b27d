"""The allocation-free diagnostics entry point, lbm_sw_diagnostics_noalloc, against the
allocating lbm_sw_diagnostics, through the C ABI.

Callers that may not allocate device memory when they check a state (a memory manager
that owns the device, a fixed budget, an out-of-memory path) use the allocation-free
entry point; it must give the same totals (FP64, different summation tree: within the
1e-12 tolerance of the parity tests), the same minimum depth and the same bad-cell count.
Two calls in a row check that the shared static scratch carries nothing over.  This file
is collected last so that a stop at the first failure has already run every other test.
"""

import numpy as np
import pytest

from paper_1401_0427_gb300 import build as libbuild
from paper_1401_0427_gb300 import inputs, lbm_sw

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _library():
    libbuild.build()
    lbm_sw.load()


def _noalloc(F, dim, precision, nx, ny, row_pitch, plane_pitch):
    import torch

    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    lbm_sw.lbm_sw_diagnostics_noalloc(F.data_ptr(), dim, precision, nx, ny, row_pitch, plane_pitch,
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare(got, want):
    scale = abs(want[0])
    assert abs(got[0] - want[0]) <= TOL * scale
    assert abs(got[1] - want[1]) <= TOL * scale and abs(got[2] - want[2]) <= TOL * scale
    assert got[3] == want[3]
    assert got[4] == 0.0


@pytest.mark.parametrize("dim,precision,nx,ny", [(2, lbm_sw.FP32, 300, 211), (2, lbm_sw.FP64, 257, 19),
                                                 (2, lbm_sw.FP32, 4096, 4096), (1, lbm_sw.FP64, 1000, 1),
                                                 (1, lbm_sw.FP32, 129, 1)])
def test_noalloc_matches_allocating_diagnostics_twice_in_a_row(dim, precision, nx, ny):
    import torch

    q = 13 if dim == 2 else 5
    tdt = torch.float64 if precision == lbm_sw.FP64 else torch.float32
    h, hu, hv = (x.reshape(ny, nx) for x in inputs.random_states(nx * ny, seed=99 + nx))
    stream = torch.cuda.current_stream().cuda_stream
    bc = (lbm_sw.WALL,) * (4 if dim == 2 else 2)
    with lbm_sw.Simulation(nx, ny, dim=dim, precision=precision, bc=bc, stream=stream) as sim:
        sim.set_state(h, hu, hv) if dim == 2 else sim.set_state(h[0], hu[0])
        for call in range(2):
            sim.step(3)
            want = sim.diagnostics()
            F = torch.empty((q, ny, nx), dtype=tdt, device="cuda")
            sim.populations_into(F)
            _compare(_noalloc(F, dim, precision, nx, ny, nx, nx * ny), want)
            # the same planes with padded rows
            pad = 7
            Fp = torch.zeros((q, ny, nx + pad), dtype=tdt, device="cuda")
            Fp[:, :, :nx] = F
            _compare(_noalloc(Fp, dim, precision, nx, ny, nx + pad, ny * (nx + pad)), want)


def test_noalloc_rejects_more_rows_than_its_scratch_holds():
    import torch

    F = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm_sw.LbmSwError) as ei:
        lbm_sw.lbm_sw_diagnostics_noalloc(F.data_ptr(), 2, lbm_sw.FP32, 1, lbm_sw.NOALLOC_MAX_ROWS + 1, 1,
                                          lbm_sw.NOALLOC_MAX_ROWS + 1, out.data_ptr(), None)
    assert ei.value.status == lbm_sw.E_ARG and "exceeds the static scratch" in str(ei.value)
    with pytest.raises(lbm_sw.LbmSwError):
        lbm_sw.lbm_sw_diagnostics_noalloc(F.data_ptr(), 2, lbm_sw.FP32, 8, 2, 4, 16, out.data_ptr(), None)
