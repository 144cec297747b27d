"""The paper's test cases run on the GPU, with their exact solutions, as numeric profiles.

* Section 2, Figure 1: the shock tube with the D1Q3Q2 scheme (80 mesh points,
  rho_l/rho_0 = 2, rho_r/rho_0 = 0.5, q = 0, lambda/c0 = 8, a = 0.15, s_j = 1.8) against the
  exact Riemann solution (Stoker's wet dam-break).
* The same Riemann problem with the D2Q5Q4Q4 scheme on a grid that is uniform in y.
* Section 4, first test case: the stationary reflection of an oblique shock by a wall,
  with the three states printed in the paper, on the 35 x 20, 70 x 40 and 140 x 80 meshes,
  run to a steady state and compared with the exact piecewise-constant solution.
* Section 4, second test case: Emery's forward-facing step, a flow at Froude number 3 in a
  channel of height 1 meeting a step of height 0.2 at x = 0.6, on the paper's meshes
  120 x 40, 240 x 80 and 480 x 120 with lambda = 80, a = 0.05, s = 1.8, at t = 1/2 and 4
  (the paper shows density maps only; no exact solution).

Every lattice Boltzmann step runs in the CUDA library through lbm_sw; this module only
sets up inputs, drives the runs and evaluates the exact solutions (which are not part of
the scheme).  ``python -m paper_1401_0427_gb300.experiments --out DIR`` writes the profiles
as CSV files.
"""

from __future__ import annotations

import argparse
import csv
import math
import os

import numpy as np

from . import inputs, lbm_sw

G = 1.0

# Section 4, first test case: states printed to 15 digits (rho, u, v).
REFLECTION_LEFT = (1.0, 1.59497132403753, 0.0)
REFLECTION_TOP = (1.17150636388320, 1.47822089880855, -0.116750425228984)
REFLECTION_RIGHT = (1.38196199044604, 1.33228286727232, 0.0)
INCIDENT_ANGLE = -math.pi / 4  # incident shock line, from the x axis


# ----------------------------------------------------------------- exact solutions
def stoker(h_left: float, h_right: float, g: float = G):
    """Middle depth and velocity of the wet dam-break and its wave speeds (fan head,
    fan tail, shock), by Newton's method on
    2 (sqrt(g h_l) - sqrt(g h)) = (h - h_r) sqrt(g (h + h_r) / (2 h h_r))."""
    cl = math.sqrt(g * h_left)

    def f(h):
        return 2.0 * (cl - math.sqrt(g * h)) - (h - h_right) * math.sqrt(g * (h + h_right) / (2.0 * h * h_right))

    h = 0.5 * (h_left + h_right)
    for _ in range(100):
        d = 1e-7 * h
        step = f(h) / ((f(h + d) - f(h - d)) / (2 * d))
        h -= step
        if abs(step) < 1e-15 * h:
            break
    u = 2.0 * (cl - math.sqrt(g * h))
    return h, u, -cl, u - math.sqrt(g * h), h * u / (h - h_right)


def stoker_profile(x, t, h_left, h_right, x0=0.5, g=G):
    hs, us, head, tail, shock = stoker(h_left, h_right, g)
    cl = math.sqrt(g * h_left)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.where(xi < head, h_left, np.where(xi < tail, (2 * cl - xi) ** 2 / (9 * g),
                                             np.where(xi < shock, hs, h_right)))
    u = np.where(xi < head, 0.0, np.where(xi < tail, 2.0 / 3.0 * (cl + xi), np.where(xi < shock, us, 0.0)))
    return h, u


def reflected_shock_angle(top=REFLECTION_TOP, right=REFLECTION_RIGHT) -> float:
    """Angle of the stationary reflected shock: its normal is parallel to the velocity jump
    (the tangential velocity is continuous across it)."""
    du = (right[1] - top[1], right[2] - top[2])
    ang = math.atan2(du[0], -du[1])
    return ang + math.pi if ang <= -math.pi / 2 else (ang - math.pi if ang > math.pi / 2 else ang)


def reflection_exact(xc, yc, height: float = 1.0, x_top: float = 0.0):
    """Exact steady solution (h, hu, hv) at cell centres: the incident shock enters at
    (x_top, height) at -pi/4, reaches the wall at x_w = x_top + height, and the reflected
    shock leaves the wall there at the angle of reflected_shock_angle()."""
    X, Y = np.meshgrid(xc, yc)
    xw = x_top + height
    ang = reflected_shock_angle()
    below_incident = Y < height - (X - x_top)
    below_reflected = (X > xw) & (Y < math.tan(ang) * (X - xw))
    out = []
    for k, f in enumerate((lambda s: s[0], lambda s: s[0] * s[1], lambda s: s[0] * s[2])):
        field = np.full(X.shape, f(REFLECTION_TOP))
        field[below_incident] = f(REFLECTION_LEFT)
        field[below_reflected] = f(REFLECTION_RIGHT)
        out.append(field)
    return tuple(out)


# ----------------------------------------------------------------- runs on the GPU
def shock_tube(n: int = 80, h_right: float = 0.5, t_end: float = 0.25, lam: float = 8.0, a: float = 0.15,
               s: float = 1.8, precision: int = lbm_sw.FP64, stream=None):
    """Section 2 shock tube on [0, 1] with walls; t_end = steps dt, dt = 1/(n lam)."""
    steps = int(round(t_end * n * lam))
    h0, q0 = inputs.dam_break_1d(n, 2.0, h_right)
    with lbm_sw.Simulation(n, 1, dim=1, precision=precision, lam=lam, a=a, s=s, bc=(lbm_sw.WALL, lbm_sw.WALL),
                           stream=stream) as sim:
        sim.set_state(h0, q0)
        sim.step(steps)
        h, q = sim.moments()
    x = inputs.cell_centres(n)
    t = steps / (n * lam)
    he, ue = stoker_profile(x, t, 2.0, h_right)
    return {"x": x, "h": h, "u": q / h, "h_exact": he, "u_exact": ue, "t": t, "steps": steps,
            "l1_h": float(np.abs(h - he).mean()), "l1_u": float(np.abs(q / h - ue).mean())}


def dam_break_y_invariant(n: int = 400, ny: int = 4, h_right: float = 1.0, t_end: float = 0.0625, lam: float = 8.0,
                          a: float = 0.05, s: float = 1.8, precision: int = lbm_sw.FP64, stream=None):
    """The Riemann problem with the D2Q5Q4Q4 scheme on an n x ny grid, walls in x,
    periodic in y (every row equal)."""
    steps = int(round(t_end * n * lam))
    h1, q1 = inputs.dam_break_1d(n, 2.0, h_right)
    W0 = (np.tile(h1, (ny, 1)), np.tile(q1, (ny, 1)), np.zeros((ny, n)))
    with lbm_sw.Simulation(n, ny, precision=precision, lam=lam, a=a, s=s,
                           bc=(lbm_sw.WALL, lbm_sw.WALL, lbm_sw.PERIODIC, lbm_sw.PERIODIC), stream=stream) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        h, hu, hv = sim.moments()
    x = inputs.cell_centres(n)
    t = steps / (n * lam)
    he, ue = stoker_profile(x, t, 2.0, h_right)
    return {"x": x, "h": h, "hu": hu, "hv": hv, "h_exact": he, "u_exact": ue, "t": t, "steps": steps,
            "l1_h": float(np.abs(h[0] - he).mean())}


def oblique_shock_reflection(nx: int = 140, ny: int = 80, lam: float = 8.0, a: float = 0.05, s: float = 1.8,
                             max_steps: int = 40000, check_every: int = 200, tol: float = 1e-10,
                             precision: int = lbm_sw.FP64, stream=None):
    """Section 4 stationary shock reflection on [0, nx/ny] x [0, 1] (square cells): inflow
    of the left state on x-, of the top state on y+, wall on y-, outflow on x+; started
    from the exact solution's upstream states (left state below the incident shock, top
    state above) and run until the largest change of h over `check_every` steps falls below
    tol (relative).  Returns the steady fields, the exact solution and the residual history."""
    length = nx / ny
    xc = (np.arange(nx) + 0.5) / ny
    yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc)
    left, top = REFLECTION_LEFT, REFLECTION_TOP
    upstream = Y < 1.0 - X
    h0 = np.where(upstream, left[0], top[0])
    hu0 = np.where(upstream, left[0] * left[1], top[0] * top[1])
    hv0 = np.where(upstream, left[0] * left[2], top[0] * top[2])
    inflow = [(left[0], left[0] * left[1], left[0] * left[2]), None, None,
              (top[0], top[0] * top[1], top[0] * top[2])]
    history = []
    with lbm_sw.Simulation(nx, ny, precision=precision, lam=lam, a=a, s=s,
                           bc=(lbm_sw.INFLOW, lbm_sw.OUTFLOW, lbm_sw.WALL, lbm_sw.INFLOW), inflow=inflow,
                           stream=stream) as sim:
        sim.set_state(h0, hu0, hv0)
        prev = sim.moments()[0]
        steps = 0
        while steps < max_steps:
            sim.step(check_every)
            steps += check_every
            cur = sim.moments()[0]
            res = float(np.abs(cur - prev).max() / np.abs(cur).max())
            history.append((steps, res))
            prev = cur
            if res < tol:
                break
        h, hu, hv = sim.moments()
    he, hue, hve = reflection_exact(xc, yc)
    return {"x": xc, "y": yc, "h": h, "hu": hu, "hv": hv, "h_exact": he, "hu_exact": hue, "hv_exact": hve,
            "steps": steps, "residuals": history, "length": length,
            "l1_h": float(np.abs(h - he).mean()), "reflected_angle": reflected_shock_angle()}


def emery_step(nx: int = 120, ny: int = 40, t_end: float = 0.5, lam: float = 80.0, a: float = 0.05,
               s: float = 1.8, froude: float = 3.0, precision: int = lbm_sw.FP64, stream=None):
    """Section 4 forward-facing step: channel [0, nx/ny] x [0, 1] (square cells of side
    1/ny), inflow of (h, u, v) = (1, froude, 0) on x-, outflow on x+, walls on y-+ and on the
    faces of the step (solid cells, inputs.emery_step); started filled with the inflow
    state; t_end = steps dt, dt = 1/(ny lam)."""
    solid, W0, win = inputs.emery_step(nx, ny, froude=froude)
    steps = int(round(t_end * ny * lam))
    with lbm_sw.Simulation(nx, ny, precision=precision, lam=lam, a=a, s=s,
                           bc=(lbm_sw.INFLOW, lbm_sw.OUTFLOW, lbm_sw.WALL, lbm_sw.WALL),
                           inflow=[win, None, None, None], stream=stream) as sim:
        sim.set_obstacle(solid)
        sim.set_state(*W0)
        sim.step(steps)
        h, hu, hv = sim.moments()
    fluid = solid == 0
    return {"x": (np.arange(nx) + 0.5) / ny, "y": (np.arange(ny) + 0.5) / ny, "h": h, "hu": hu, "hv": hv,
            "solid": solid, "steps": steps, "t": steps / (ny * lam), "inflow": win,
            "min_h": float(h[fluid].min()), "max_h": float(h[fluid].max())}


# ----------------------------------------------------------------- output
def _write_csv(path, header, rows):
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(header)
        w.writerows(rows)


def main():
    ap = argparse.ArgumentParser(description="run the paper's test cases on the GPU and write CSV profiles")
    ap.add_argument("--out", default="experiments_out")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    r = shock_tube()
    _write_csv(os.path.join(args.out, "figure1_shock_tube_80.csv"), ["x", "h", "u", "h_exact", "u_exact"],
               zip(r["x"], r["h"], r["u"], r["h_exact"], r["u_exact"]))
    print(f"shock tube (80 points, t = {r['t']:.4f}): L1(h) = {r['l1_h']:.4e}, L1(u) = {r['l1_u']:.4e}")
    for nx, ny in ((35, 20), (70, 40), (140, 80)):
        e = oblique_shock_reflection(nx, ny)
        rows = [(e["x"][i], e["y"][j], e["h"][j, i], e["h_exact"][j, i]) for j in range(ny) for i in range(nx)]
        _write_csv(os.path.join(args.out, f"figure2_shock_reflection_{nx}x{ny}.csv"), ["x", "y", "h", "h_exact"], rows)
        print(f"shock reflection {nx}x{ny}: {e['steps']} steps, residual {e['residuals'][-1][1]:.2e}, "
              f"L1(h) = {e['l1_h']:.4e}")
    for nx, ny in ((120, 40), (240, 80), (480, 120)):
        for t_end in (0.5, 4.0):
            e = emery_step(nx, ny, t_end)
            rows = [(e["x"][i], e["y"][j], int(e["solid"][j, i]), e["h"][j, i]) for j in range(ny) for i in range(nx)]
            _write_csv(os.path.join(args.out, f"figure{3 if t_end < 1 else 4}_emery_{nx}x{ny}_t{t_end:g}.csv"),
                       ["x", "y", "solid", "h"], rows)
            print(f"Emery step {nx}x{ny}, t = {e['t']:g} ({e['steps']} steps): h in [{e['min_h']:.4f}, "
                  f"{e['max_h']:.4f}]")


if __name__ == "__main__":
    main()
