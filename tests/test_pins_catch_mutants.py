"""Planted mistakes in the oracle, each of which one of its pins must catch.

Each case copies ``oracle/lbm_oracle.cpp``, makes one plausible mistake in it (a sign,
a dropped term, a wrong index or partner, a transposed operand), compiles the copy
with the oracle's own flags and runs the oracle's pin suite (``tests/test_oracle_*.py``)
against it through ``LBM_ORACLE_LIB``. The suite has to fail. The mistakes are planted
in the oracle on the CPU only; nothing here touches the CUDA library.
"""

from __future__ import annotations

import glob
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.cpp")
PINS = sorted(glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")))

# (name, text in the oracle, replacement): each text occurs exactly once.
MUTANTS = [
    # section 2, D1Q3Q2
    ("1d_f_minus_sign", "feq[2] = K * w * (1.0 - beta / pr.lam)", "feq[2] = K * w * (1.0 + beta / pr.lam)"),
    ("1d_pressure_flux_dropped", "feq[3] = K * w * beta * (1.0 + beta / pr.lam) + K / 2.0 * w * w / pr.lam;",
     "feq[3] = K * w * beta * (1.0 + beta / pr.lam);"),
    ("1d_rho_without_f0", "rho = f[0] + (f[1] + f[2]);  // rho", "rho = (f[1] + f[2]);  // rho"),
    ("1d_g_velocities_swapped", "const int kEx1[5] = {0, 1, -1, 1, -1};", "const int kEx1[5] = {0, 1, -1, -1, 1};"),
    ("1d_wall_without_partner", "const int kMirror1[5] = {0, 2, 1, 4, 3};", "const int kMirror1[5] = {0, 1, 2, 3, 4};"),
    ("1d_wall_keeps_momentum_sign", "const double kMirrorSign1[5] = {1, 1, 1, -1, -1};",
     "const double kMirrorSign1[5] = {1, 1, 1, 1, 1};"),
    ("1d_mrt_eps_without_lambda2", "m[2] = lam * lam * (f[1] + f[2] - 2.0 * f[0]);",
     "m[2] = lam * (f[1] + f[2] - 2.0 * f[0]);"),
    ("1d_inflow_discharge_sign", "equilibrium_1d<T>(pr.inflow[side][0], pr.inflow[side][1], pr, win)",
     "equilibrium_1d<T>(pr.inflow[side][0], -pr.inflow[side][1], pr, win)"),
    ("1d_periodic_copies_own_edge", "case BC_PERIODIC: g(j, ghost) = g(j, opposite); break;",
     "case BC_PERIODIC: g(j, ghost) = g(j, edge); break;"),
    ("1d_outflow_copies_far_side", "case BC_OUTFLOW: g(j, ghost) = g(j, edge); break;",
     "case BC_OUTFLOW: g(j, ghost) = g(j, opposite); break;"),
    ("1d_mrt_inverse_f0_sign", "f[0] = m[0] - sum_pm;", "f[0] = m[0] + sum_pm;"),
    ("1d_mrt_skips_j_q_not_q", "if (l != 0 && l != 3) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);",
     "if (l != 0 && l != 4) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);"),
    # section 3, D2Q5Q4Q4
    ("2d_theta_half_dropped", "const T theta = pr.g * rho - uu / 2.0;", "const T theta = pr.g * rho - uu;"),
    ("2d_rest_potential_without_K", "const T h0_t = pr.a * K * theta;", "const T h0_t = pr.a * theta;"),
    ("2d_f3_sign", "feq[3] = quarter - p_t * u * c;", "feq[3] = quarter + p_t * u * c;"),
    ("2d_gy_pressure_dropped", "feq[10] = p_v / 4.0 + (p_v * v + p) * c;", "feq[10] = p_v / 4.0 + (p_v * v) * c;"),
    ("2d_gy1_u_for_v", "feq[9] = p_v / 4.0 + p_v * u * c;", "feq[9] = p_v / 4.0 + p_v * v * c;"),
    ("2d_gx2_transposed", "feq[6] = p_u / 4.0 + p_u * v * c;", "feq[6] = p_v / 4.0 + p_u * v * c;"),
    ("2d_rho_without_f0", "rho = f[0] + ((f[1] + f[3]) + (f[2] + f[4]));", "rho = ((f[1] + f[3]) + (f[2] + f[4]));"),
    ("2d_relaxation_sign", "for (int j = 0; j < 13; ++j) f[j] = f[j] + pr.s * (feq[j] - f[j]);",
     "for (int j = 0; j < 13; ++j) f[j] = f[j] + pr.s * (f[j] - feq[j]);"),
    ("2d_mrt_inverse_sign", "f[2] = (s24 + m[2] / lam) / 2.0;", "f[2] = (s24 - m[2] / lam) / 2.0;"),
    ("2d_gx_moves_along_y", "const int kEx2[13] = {0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1, 0};",
     "const int kEx2[13] = {0, 1, 0, -1, 0, 0, 1, 0, -1, 1, 0, -1, 0};"),
    ("2d_gy_directions_swapped", "const int kEy2[13] = {0, 0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1};",
     "const int kEy2[13] = {0, 0, 1, 0, -1, 0, 1, 0, -1, 0, -1, 0, 1};"),
    ("2d_x_wall_keeps_normal_momentum", "const double kSignX[13] = {1, 1, 1, 1, 1, -1, -1, -1, -1, 1, 1, 1, 1};",
     "const double kSignX[13] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};"),
    ("2d_y_wall_f_not_mirrored", "const int kMirrorY[13] = {0, 1, 4, 3, 2, 5, 8, 7, 6, 9, 12, 11, 10};",
     "const int kMirrorY[13] = {0, 1, 2, 3, 4, 5, 8, 7, 6, 9, 12, 11, 10};"),
    ("2d_outflow_copies_far_side", "case BC_OUTFLOW: g(p, gi, gj) = g(p, ei, ej); break;",
     "case BC_OUTFLOW: g(p, gi, gj) = g(p, oi, oj); break;"),
    ("2d_periodic_copies_own_edge", "case BC_PERIODIC: g(p, gi, gj) = g(p, oi, oj); break;",
     "case BC_PERIODIC: g(p, gi, gj) = g(p, ei, ej); break;"),
    ("2d_inflow_velocity_transposed",
     "equilibrium_2d<T>(pr.inflow[side][0], pr.inflow[side][1], pr.inflow[side][2], pr, win);",
     "equilibrium_2d<T>(pr.inflow[side][0], pr.inflow[side][2], pr.inflow[side][1], pr, win);"),
    ("2d_pressure_linear_in_w", "const T p = K * w * w;", "const T p = K * w;"),
    ("2d_mrt_relaxes_qy", "if (l != 0 && l != 5 && l != 9) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);",
     "if (l != 0 && l != 5 && l != 10) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);"),
    ("2d_mrt_xx_rho_basis", "m[4] = f[1] - f[2] + f[3] - f[4];", "m[4] = f[1] + f[2] - f[3] - f[4];"),
    ("2d_x_wall_gy_not_mirrored", "const int kMirrorX[13] = {0, 3, 2, 1, 4, 7, 6, 5, 8, 11, 10, 9, 12};",
     "const int kMirrorX[13] = {0, 3, 2, 1, 4, 7, 6, 5, 8, 9, 10, 11, 12};"),
    ("2d_solid_cells_collide", "if (pr.solid && pr.solid[c]) continue;  // no fluid to relax",
     "if (false) continue;  // no fluid to relax"),
    # stand-alone entry points
    ("2d_moments_entry_transposed", "moments_2d(f, rho[c], qx[c], qy[c]);", "moments_2d(f, rho[c], qy[c], qx[c]);"),
    ("1d_moments_entry_swapped", "moments_1d(f, rho[i], q[i]);", "moments_1d(f, q[i], rho[i]);"),
    ("2d_stream_entry_skips_ghosts", "stream_2d<double>(Fs, F, *pr, ghosts);",
     "{ oracle_params open = *pr; for (int k = 0; k < 4; ++k) open.bc[k] = BC_OUTFLOW; "
     "stream_2d<double>(Fs, F, open, ghosts); }"),
    # complex-step entry points
    ("1d_cplx_run_one_step_short", "run_1d<cplx>(z.data(), nsteps, *pr);",
     "run_1d<cplx>(z.data(), nsteps > 0 ? nsteps - 1 : 0, *pr);"),
    ("1d_cplx_equilibrium_drops_q_im",
     "equilibrium_1d<cplx>(cplx(rho_re[i], rho_im[i]), cplx(q_re[i], q_im[i]), *pr, f);",
     "equilibrium_1d<cplx>(cplx(rho_re[i], rho_im[i]), cplx(q_re[i], 0.0), *pr, f);"),
    ("2d_cplx_equilibrium_qx_im_from_qy", "cplx(qx_re[c], qx_im[c])", "cplx(qx_re[c], qy_im[c])"),
    ("2d_obstacle_face_without_sign",
     "f[p * plane + c] = kEx2[p] != 0 ? kSignX[p] * g(kMirrorX[p], i, j) : kSignY[p] * g(kMirrorY[p], i, j);",
     "f[p * plane + c] = kEx2[p] != 0 ? g(kMirrorX[p], i, j) : g(kMirrorY[p], i, j);"),
]


def _compile(text: str, out_dir: str, name: str) -> str:
    src = os.path.join(out_dir, f"{name}.cpp")
    lib = os.path.join(out_dir, f"lib{name}.so")
    with open(src, "w") as fh:
        fh.write(text)
    # the flags of oracle.build()
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", src, "-o", lib], check=True, capture_output=True)
    return lib


def _pins(lib: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, LBM_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *PINS]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _first_failure(out: str) -> str:
    for line in out.splitlines():
        if line.startswith("FAILED") or line.startswith("ERROR"):
            return line
    return out.strip().splitlines()[-1] if out.strip() else ""


def test_each_mutant_text_occurs_once():
    text = open(SRC).read()
    for name, old, new in MUTANTS:
        assert text.count(old) == 1, name
        assert old != new, name


def test_pins_pass_on_the_unmutated_copy():
    with tempfile.TemporaryDirectory() as d:
        lib = _compile(open(SRC).read(), d, "unmutated")
        r = _pins(lib)
    assert r.returncode == 0, r.stdout[-2000:]


def test_pins_catch_every_planted_mistake():
    text = open(SRC).read()
    with tempfile.TemporaryDirectory() as d:
        def run(m):
            name, old, new = m
            lib = _compile(text.replace(old, new), d, name)
            r = _pins(lib)
            return name, r.returncode, _first_failure(r.stdout)

        workers = max(1, min(8, (os.cpu_count() or 2) // 2))
        with ThreadPoolExecutor(workers) as pool:
            results = list(pool.map(run, MUTANTS))
    survivors = [(name, last) for name, rc, last in results if rc == 0]
    assert not survivors, f"mistakes no pin caught: {survivors}"
    for name, rc, first in results:  # each run stops at its first failing pin
        assert rc == 1, (name, rc, first)


if __name__ == "__main__":  # list which pin catches each mistake
    text = open(SRC).read()
    with tempfile.TemporaryDirectory() as d:
        for name, old, new in MUTANTS:
            r = _pins(_compile(text.replace(old, new), d, name))
            print(f"{name:36s} rc={r.returncode}  {_first_failure(r.stdout)}")
