// Plain FP64 CPU oracle for the vectorial lattice Boltzmann schemes of
// F. Dubois, "Simulation of strong nonlinear waves with vectorial lattice
// Boltzmann schemes" (DSFD 2013): the D1Q3Q2 scheme of section 2 and the
// D2Q5Q4Q4 scheme of section 3, applied to the shallow-water equations.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this
// file: only the tests, the smoke check and the CPU-baseline leg of the
// benchmark use it.  It shares no code, header or constant with the CUDA
// library; the two sides agree only through the written definition of the
// population order below.
//
// Method, in the paper's order and notation (one time step):
//   1. conserved moments W^k = sum_j f_j^k                          (Eq. 1-hyp-N-vconserv)
//   2. entropy variables phi = (theta, beta) from W, with gamma = 2:
//        theta = c^2/(gamma-1) - |u|^2/2 = g h - |u|^2/2, beta = u   (section 2, section 3)
//   3. equilibria f_j^eq = d h_j^* / d phi_k from the potentials h_j^*  (section 1)
//        1D: Eq. (2-potentiels-st-venant-1d) and (2-potentiels-st-venant-1d-suite)
//        2D: h_0^* = (a/2) K theta^2 plus the constraints (3-st-venant-contraintes-2),
//            (3-st-venant-enplus)
//   4. relaxation f* = f + s (f^eq - f) (BGK: every s_l equal, Eq. 2-relaxation),
//      or the MRT form m* = m + s_l (m^eq - m) on the moment bases of sections 2 and 3
//   5. streaming f_j(x + v_j dt, t + dt) = f_j*(x, t), lambda = dx/dt, with one layer of
//      explicit ghost cells filled by the boundary rule of each side.
//
// Shallow water as the gamma = 2 system: rho = h, q = h u, p = g h^2 / 2, so
// p0/rho0^2 = g/2, c0^2 = g rho0 and K = p0/c0^4 = rho0/(2 c0^2) = 1/(2g).
//
// Population order (both dimensions, a plane of nx*ny values per population,
// x fastest):
//   1D: f0, f+, f-, g+, g-                         (velocities 0, +lam, -lam, +lam, -lam)
//   2D: f0 f1 f2 f3 f4 gx1 gx2 gx3 gx4 gy1 gy2 gy3 gy4, with v_1 = (lam,0),
//       v_2 = (0,lam), v_3 = (-lam,0), v_4 = (0,-lam)   (Eq. 3-stencil-d2q5)
//
// Boundary rules (the paper only names bounce-back and anti-bounce-back,
// section 3, last paragraph); the ghost cell beyond each side holds
//   PERIODIC: the cell on the opposite side;
//   WALL:     the mirror image of the boundary cell (populations of the
//             reflected velocity, normal momentum family negated);
//   OUTFLOW:  a copy of the boundary cell (zero gradient);
//   INFLOW:   the equilibrium of a prescribed state W_in.
// Obstacles (2D, optional): a mask of solid cells inside the domain.  A face between a
// fluid cell and a solid cell is a wall with the same mirror rule: the population that
// would arrive from the solid cell takes the value of the reflected population of the
// fluid cell itself, normal momentum family negated (exactly what the WALL ghost gives
// at a domain side).  Solid cells hold no fluid: they are neither collided nor streamed,
// and keep the populations they hold.
//
// Templated on the scalar so that std::complex<double> gives complex-step
// derivatives of a whole run (the scheme is analytic in its inputs).

#include <cmath>
#include <complex>
#include <cstddef>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_OUTFLOW = 2, BC_INFLOW = 3 };
enum { SIDE_XM = 0, SIDE_XP = 1, SIDE_YM = 2, SIDE_YP = 3 };

}  // namespace

extern "C" {
// Mirrored field by field by the ctypes structure in oracle/__init__.py.
struct oracle_params {
  int nx, ny;             // cells; ny = 1 in 1D
  double g;               // gravity
  double lam;             // lattice velocity lambda = dx/dt
  double s;               // BGK relaxation rate (all s_l equal)
  double a;               // weight of the rest potential h_0^* = (a/2) K theta^2
  int bc[4];              // x-, x+, y-, y+
  double inflow[4][3];    // W_in = (h, h u, h v) per side for INFLOW
  int mrt;                // 0: BGK with s; 1: MRT with s_moments
  double s_moments[13];   // relaxation rate per moment (MRT only; conserved ones unused)
  const unsigned char* solid;  // 2D: nx*ny flags, x fastest, nonzero = solid; NULL = none
};
}

namespace {

using P = oracle_params;
using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// Section 2: D1Q3Q2.  f on D1Q3 (0, +lam, -lam); g on D1Q2 (+lam, -lam).
// ---------------------------------------------------------------------------

// Equilibrium of the five populations for W = (rho, q).
// Potentials: h_0^* = (a/2) K theta^2,
//             h_pm^* = (K/2) w^2 (1 pm beta/lam) - (aK/4) theta^2,  w = theta + beta^2/2,
// and f_j = d h_j^*/d theta, g_j = d h_j^*/d beta (dw/dtheta = 1, dw/dbeta = beta).
// h_0^* does not depend on beta, so there is no g_0.
template <class T>
void equilibrium_1d(T rho, T q, const P& pr, T feq[5]) {
  const double K = 1.0 / (2.0 * pr.g);
  const T beta = q / rho;
  const T theta = pr.g * rho - beta * beta / 2.0;
  const T w = theta + beta * beta / 2.0;
  feq[0] = pr.a * K * theta;
  feq[1] = K * w * (1.0 + beta / pr.lam) - pr.a * K / 2.0 * theta;
  feq[2] = K * w * (1.0 - beta / pr.lam) - pr.a * K / 2.0 * theta;
  feq[3] = K * w * beta * (1.0 + beta / pr.lam) + K / 2.0 * w * w / pr.lam;
  feq[4] = K * w * beta * (1.0 - beta / pr.lam) - K / 2.0 * w * w / pr.lam;
}

template <class T>
void moments_1d(const T f[5], T& rho, T& q) {
  rho = f[0] + (f[1] + f[2]);  // rho = f0 + f+ + f-
  q = f[3] + f[4];             // q = g+ + g-
}

// MRT moments of section 2: rho, J_rho = lam (f+ - f-), eps_rho = lam^2 (f+ + f- - 2 f0),
// q, J_q = lam (g+ - g-).
template <class T>
void to_moments_1d(const T f[5], double lam, T m[5]) {
  m[0] = f[0] + f[1] + f[2];
  m[1] = lam * (f[1] - f[2]);
  m[2] = lam * lam * (f[1] + f[2] - 2.0 * f[0]);
  m[3] = f[3] + f[4];
  m[4] = lam * (f[3] - f[4]);
}

template <class T>
void from_moments_1d(const T m[5], double lam, T f[5]) {
  // Inverse of to_moments_1d.
  const T sum_pm = (m[2] / (lam * lam) + 2.0 * m[0]) / 3.0;  // f+ + f-
  f[0] = m[0] - sum_pm;
  f[1] = (sum_pm + m[1] / lam) / 2.0;
  f[2] = (sum_pm - m[1] / lam) / 2.0;
  f[3] = (m[3] + m[4] / lam) / 2.0;
  f[4] = (m[3] - m[4] / lam) / 2.0;
}

template <class T>
void collide_cell_1d(T f[5], const P& pr) {
  T rho, q;
  moments_1d(f, rho, q);
  T feq[5];
  equilibrium_1d(rho, q, pr, feq);
  if (!pr.mrt) {
    for (int j = 0; j < 5; ++j) f[j] = f[j] + pr.s * (feq[j] - f[j]);
    return;
  }
  T m[5], meq[5];
  to_moments_1d(f, pr.lam, m);
  to_moments_1d(feq, pr.lam, meq);
  for (int l = 0; l < 5; ++l)
    if (l != 0 && l != 3) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);
  from_moments_1d(m, pr.lam, f);
}

// Velocity of each 1D population in lattice units, and its mirror partner.
const int kEx1[5] = {0, 1, -1, 1, -1};
const int kMirror1[5] = {0, 2, 1, 4, 3};
const double kMirrorSign1[5] = {1, 1, 1, -1, -1};

template <class T>
void stream_1d(const T* fs, T* f, const P& pr, std::vector<T>& G) {
  // Ghost-padded copy: index i + 1 for cell i, 0 and n + 1 are the ghosts.
  const int n = pr.nx;
  G.assign(5 * static_cast<size_t>(n + 2), T(0.0));
  auto g = [&](int j, int i) -> T& { return G[static_cast<size_t>(j) * (n + 2) + i + 1]; };
  for (int j = 0; j < 5; ++j)
    for (int i = 0; i < n; ++i) g(j, i) = fs[static_cast<size_t>(j) * n + i];
  for (int side = 0; side < 2; ++side) {
    const int ghost = side == SIDE_XM ? -1 : n;
    const int edge = side == SIDE_XM ? 0 : n - 1;
    const int opposite = side == SIDE_XM ? n - 1 : 0;
    T win[5];
    if (pr.bc[side] == BC_INFLOW) equilibrium_1d<T>(pr.inflow[side][0], pr.inflow[side][1], pr, win);
    for (int j = 0; j < 5; ++j) {
      switch (pr.bc[side]) {
        case BC_PERIODIC: g(j, ghost) = g(j, opposite); break;
        case BC_WALL: g(j, ghost) = kMirrorSign1[j] * g(kMirror1[j], edge); break;
        case BC_OUTFLOW: g(j, ghost) = g(j, edge); break;
        default: g(j, ghost) = win[j]; break;
      }
    }
  }
  for (int j = 0; j < 5; ++j)
    for (int i = 0; i < n; ++i) f[static_cast<size_t>(j) * n + i] = g(j, i - kEx1[j]);
}

template <class T>
void collide_1d(T* F, const P& pr) {
  const size_t n = pr.nx;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < static_cast<long>(n); ++i) {
    T f[5];
    for (int j = 0; j < 5; ++j) f[j] = F[j * n + i];
    collide_cell_1d(f, pr);
    for (int j = 0; j < 5; ++j) F[j * n + i] = f[j];
  }
}

template <class T>
void run_1d(T* F, int nsteps, const P& pr) {
  std::vector<T> fs(F, F + 5 * static_cast<size_t>(pr.nx));
  std::vector<T> ghosts;
  for (int n = 0; n < nsteps; ++n) {
    std::memcpy(static_cast<void*>(fs.data()), F, sizeof(T) * fs.size());
    collide_1d(fs.data(), pr);
    stream_1d(fs.data(), F, pr, ghosts);
  }
}

// ---------------------------------------------------------------------------
// Section 3: D2Q5Q4Q4.  f on D2Q5, gx and gy on D2Q4 (no rest population).
// ---------------------------------------------------------------------------

// Equilibrium of the 13 populations for W = (rho, qx, qy), phi = (theta, u, v).
// eta* = p = K w^2 with w = theta + (u^2 + v^2)/2.  Potentials:
//   h_0^* = (a/2) K theta^2
//   h_1^* = (p - h_0^*)/4 + p u/(2 lam),   h_3^* = (p - h_0^*)/4 - p u/(2 lam)
//   h_2^* = (p - h_0^*)/4 + p v/(2 lam),   h_4^* = (p - h_0^*)/4 - p v/(2 lam)
// which solve sum_j h_j^* = p, lam (h_1^* - h_3^*) = p u, lam (h_2^* - h_4^*) = p v and the
// split h_1^* + h_3^* = h_2^* + h_4^* = (p - h_0^*)/2.  Then f_j = dh_j^*/dtheta,
// gx_j = dh_j^*/du, gy_j = dh_j^*/dv, with dp/dtheta = 2Kw, dp/du = 2Kw u, dp/dv = 2Kw v.
template <class T>
void equilibrium_2d(T rho, T qx, T qy, const P& pr, T feq[13]) {
  const double K = 1.0 / (2.0 * pr.g);
  const double c = 1.0 / (2.0 * pr.lam);
  const T u = qx / rho;
  const T v = qy / rho;
  const T uu = u * u + v * v;
  const T theta = pr.g * rho - uu / 2.0;
  const T w = theta + uu / 2.0;
  const T p = K * w * w;
  const T p_t = 2.0 * K * w;
  const T p_u = p_t * u;
  const T p_v = p_t * v;
  const T h0_t = pr.a * K * theta;  // d h_0^* / d theta
  const T quarter = (p_t - h0_t) / 4.0;
  feq[0] = h0_t;
  feq[1] = quarter + p_t * u * c;
  feq[2] = quarter + p_t * v * c;
  feq[3] = quarter - p_t * u * c;
  feq[4] = quarter - p_t * v * c;
  feq[5] = p_u / 4.0 + (p_u * u + p) * c;   // d/du of h_1^*
  feq[6] = p_u / 4.0 + p_u * v * c;         // d/du of h_2^*
  feq[7] = p_u / 4.0 - (p_u * u + p) * c;   // d/du of h_3^*
  feq[8] = p_u / 4.0 - p_u * v * c;         // d/du of h_4^*
  feq[9] = p_v / 4.0 + p_v * u * c;         // d/dv of h_1^*
  feq[10] = p_v / 4.0 + (p_v * v + p) * c;  // d/dv of h_2^*
  feq[11] = p_v / 4.0 - p_v * u * c;        // d/dv of h_3^*
  feq[12] = p_v / 4.0 - (p_v * v + p) * c;  // d/dv of h_4^*
}

// Sums are taken in mirror-symmetric pairs so that mirror images round alike.
template <class T>
void moments_2d(const T f[13], T& rho, T& qx, T& qy) {
  rho = f[0] + ((f[1] + f[3]) + (f[2] + f[4]));
  qx = (f[5] + f[7]) + (f[6] + f[8]);
  qy = (f[9] + f[11]) + (f[10] + f[12]);
}

// The 13 moments of section 3, in the order
//   rho, J_x, J_y, eps, XX_rho, q_x, f_xx, f_xy, XX_u, q_y, f_yx, f_yy, XX_v.
template <class T>
void to_moments_2d(const T f[13], double lam, T m[13]) {
  m[0] = f[0] + f[1] + f[2] + f[3] + f[4];
  m[1] = lam * (f[1] - f[3]);
  m[2] = lam * (f[2] - f[4]);
  m[3] = f[1] + f[2] + f[3] + f[4] - 4.0 * f[0];
  m[4] = f[1] - f[2] + f[3] - f[4];
  for (int k = 0; k < 2; ++k) {
    const T* g = f + 5 + 4 * k;
    T* mm = m + 5 + 4 * k;
    mm[0] = g[0] + g[1] + g[2] + g[3];
    mm[1] = lam * (g[0] - g[2]);
    mm[2] = lam * (g[1] - g[3]);
    mm[3] = g[0] - g[1] + g[2] - g[3];
  }
}

template <class T>
void from_moments_2d(const T m[13], double lam, T f[13]) {
  // Inverse of to_moments_2d.
  const T sum4 = (m[3] + 4.0 * m[0]) / 5.0;  // f1 + f2 + f3 + f4
  f[0] = m[0] - sum4;
  const T s13 = (sum4 + m[4]) / 2.0;
  const T s24 = (sum4 - m[4]) / 2.0;
  f[1] = (s13 + m[1] / lam) / 2.0;
  f[3] = (s13 - m[1] / lam) / 2.0;
  f[2] = (s24 + m[2] / lam) / 2.0;
  f[4] = (s24 - m[2] / lam) / 2.0;
  for (int k = 0; k < 2; ++k) {
    const T* mm = m + 5 + 4 * k;
    T* g = f + 5 + 4 * k;
    const T g13 = (mm[0] + mm[3]) / 2.0;
    const T g24 = (mm[0] - mm[3]) / 2.0;
    g[0] = (g13 + mm[1] / lam) / 2.0;
    g[2] = (g13 - mm[1] / lam) / 2.0;
    g[1] = (g24 + mm[2] / lam) / 2.0;
    g[3] = (g24 - mm[2] / lam) / 2.0;
  }
}

template <class T>
void collide_cell_2d(T f[13], const P& pr) {
  T rho, qx, qy;
  moments_2d(f, rho, qx, qy);
  T feq[13];
  equilibrium_2d(rho, qx, qy, pr, feq);
  if (!pr.mrt) {
    for (int j = 0; j < 13; ++j) f[j] = f[j] + pr.s * (feq[j] - f[j]);
    return;
  }
  T m[13], meq[13];
  to_moments_2d(f, pr.lam, m);
  to_moments_2d(feq, pr.lam, meq);
  for (int l = 0; l < 13; ++l)
    if (l != 0 && l != 5 && l != 9) m[l] = m[l] + pr.s_moments[l] * (meq[l] - m[l]);
  from_moments_2d(m, pr.lam, f);
}

// Lattice velocity of each 2D population (units of lam), and its mirror
// partners across an x-wall and a y-wall.
const int kEx2[13] = {0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1, 0};
const int kEy2[13] = {0, 0, 1, 0, -1, 0, 1, 0, -1, 0, 1, 0, -1};
const int kMirrorX[13] = {0, 3, 2, 1, 4, 7, 6, 5, 8, 11, 10, 9, 12};
const double kSignX[13] = {1, 1, 1, 1, 1, -1, -1, -1, -1, 1, 1, 1, 1};
const int kMirrorY[13] = {0, 1, 4, 3, 2, 5, 8, 7, 6, 9, 12, 11, 10};
const double kSignY[13] = {1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1};

template <class T>
void collide_2d(T* F, const P& pr) {
  const size_t plane = static_cast<size_t>(pr.nx) * pr.ny;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < static_cast<long>(plane); ++c) {
    if (pr.solid && pr.solid[c]) continue;  // no fluid to relax
    T f[13];
    for (int j = 0; j < 13; ++j) f[j] = F[j * plane + c];
    collide_cell_2d(f, pr);
    for (int j = 0; j < 13; ++j) F[j * plane + c] = f[j];
  }
}

template <class T>
void stream_2d(const T* fs, T* f, const P& pr, std::vector<T>& G) {
  const int nx = pr.nx, ny = pr.ny;
  const size_t px = nx + 2, py = ny + 2, plane = static_cast<size_t>(nx) * ny;
  // Ghost-padded post-collision field: cell (i, j) sits at (i + 1, j + 1).  The
  // four corner ghosts are never read (no population moves diagonally).
  G.resize(13 * px * py);
  auto g = [&](int p, int i, int j) -> T& { return G[(p * py + (j + 1)) * px + (i + 1)]; };
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int p = 0; p < 13; ++p)
      for (int i = 0; i < nx; ++i) g(p, i, j) = fs[p * plane + static_cast<size_t>(j) * nx + i];

  for (int side = 0; side < 4; ++side) {
    const bool xside = side == SIDE_XM || side == SIDE_XP;
    const int len = xside ? ny : nx;
    T win[13];
    if (pr.bc[side] == BC_INFLOW)
      equilibrium_2d<T>(pr.inflow[side][0], pr.inflow[side][1], pr.inflow[side][2], pr, win);
    for (int t = 0; t < len; ++t) {
      int gi, gj, ei, ej, oi, oj;  // ghost, boundary (edge) cell, opposite-side cell
      if (side == SIDE_XM) { gi = -1; ei = 0; oi = nx - 1; gj = ej = oj = t; }
      else if (side == SIDE_XP) { gi = nx; ei = nx - 1; oi = 0; gj = ej = oj = t; }
      else if (side == SIDE_YM) { gj = -1; ej = 0; oj = ny - 1; gi = ei = oi = t; }
      else { gj = ny; ej = ny - 1; oj = 0; gi = ei = oi = t; }
      for (int p = 0; p < 13; ++p) {
        switch (pr.bc[side]) {
          case BC_PERIODIC: g(p, gi, gj) = g(p, oi, oj); break;
          case BC_WALL:
            g(p, gi, gj) = xside ? kSignX[p] * g(kMirrorX[p], ei, ej)
                                 : kSignY[p] * g(kMirrorY[p], ei, ej);
            break;
          case BC_OUTFLOW: g(p, gi, gj) = g(p, ei, ej); break;
          default: g(p, gi, gj) = win[p]; break;
        }
      }
    }
  }

  // Pull: the population moving with v_p arrives at (i, j) from (i - ex, j - ey).
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int p = 0; p < 13; ++p)
      for (int i = 0; i < nx; ++i)
        f[p * plane + static_cast<size_t>(j) * nx + i] = g(p, i - kEx2[p], j - kEy2[p]);

  if (!pr.solid) return;
  // Obstacles: solid cells keep their populations; a fluid cell whose source cell is
  // solid takes the mirror image of its own population instead.
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t c = static_cast<size_t>(j) * nx + i;
      if (pr.solid[c]) {
        for (int p = 0; p < 13; ++p) f[p * plane + c] = fs[p * plane + c];
        continue;
      }
      for (int p = 1; p < 13; ++p) {
        int si = i - kEx2[p], sj = j - kEy2[p];
        // beyond a periodic side the source is the cell on the opposite side; beyond any
        // other side the side's own rule above applies
        if (si < 0 || si >= nx) {
          if (pr.bc[si < 0 ? SIDE_XM : SIDE_XP] != BC_PERIODIC) continue;
          si = (si + nx) % nx;
        }
        if (sj < 0 || sj >= ny) {
          if (pr.bc[sj < 0 ? SIDE_YM : SIDE_YP] != BC_PERIODIC) continue;
          sj = (sj + ny) % ny;
        }
        if (!pr.solid[static_cast<size_t>(sj) * nx + si]) continue;
        f[p * plane + c] = kEx2[p] != 0 ? kSignX[p] * g(kMirrorX[p], i, j) : kSignY[p] * g(kMirrorY[p], i, j);
      }
    }
}

template <class T>
void run_2d(T* F, int nsteps, const P& pr) {
  const size_t count = 13 * static_cast<size_t>(pr.nx) * pr.ny;
  std::vector<T> fs(count);
  std::vector<T> ghosts;
  for (int n = 0; n < nsteps; ++n) {
    std::memcpy(static_cast<void*>(fs.data()), F, sizeof(T) * count);
    collide_2d(fs.data(), pr);
    stream_2d(fs.data(), F, pr, ghosts);
  }
}

void split(const double* re, const double* im, size_t n, std::vector<cplx>& z) {
  z.resize(n);
  for (size_t k = 0; k < n; ++k) z[k] = cplx(re[k], im[k]);
}

void join(const std::vector<cplx>& z, double* re, double* im) {
  for (size_t k = 0; k < z.size(); ++k) { re[k] = z[k].real(); im[k] = z[k].imag(); }
}

}  // namespace

extern "C" {

int oracle_version(void) { return 1; }

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// ---- 1D (F holds 5 planes of nx values, pre-collision) ----
void oracle_equilibrium_1d(const double* rho, const double* q, double* F, const oracle_params* pr) {
  const size_t n = pr->nx;
  for (size_t i = 0; i < n; ++i) {
    double f[5];
    equilibrium_1d<double>(rho[i], q[i], *pr, f);
    for (int j = 0; j < 5; ++j) F[j * n + i] = f[j];
  }
}
void oracle_moments_1d(const double* F, double* rho, double* q, const oracle_params* pr) {
  const size_t n = pr->nx;
  for (size_t i = 0; i < n; ++i) {
    double f[5];
    for (int j = 0; j < 5; ++j) f[j] = F[j * n + i];
    moments_1d(f, rho[i], q[i]);
  }
}
void oracle_collide_1d(double* F, const oracle_params* pr) { collide_1d<double>(F, *pr); }
void oracle_stream_1d(const double* Fs, double* F, const oracle_params* pr) {
  std::vector<double> ghosts;
  stream_1d<double>(Fs, F, *pr, ghosts);
}
void oracle_run_1d(double* F, int nsteps, const oracle_params* pr) { run_1d<double>(F, nsteps, *pr); }

// ---- 2D (F holds 13 planes of nx*ny values, x fastest, pre-collision) ----
void oracle_equilibrium_2d(const double* rho, const double* qx, const double* qy, double* F,
                           const oracle_params* pr) {
  const size_t n = static_cast<size_t>(pr->nx) * pr->ny;
  for (size_t c = 0; c < n; ++c) {
    double f[13];
    equilibrium_2d<double>(rho[c], qx[c], qy[c], *pr, f);
    for (int j = 0; j < 13; ++j) F[j * n + c] = f[j];
  }
}
void oracle_moments_2d(const double* F, double* rho, double* qx, double* qy, const oracle_params* pr) {
  const size_t n = static_cast<size_t>(pr->nx) * pr->ny;
  for (size_t c = 0; c < n; ++c) {
    double f[13];
    for (int j = 0; j < 13; ++j) f[j] = F[j * n + c];
    moments_2d(f, rho[c], qx[c], qy[c]);
  }
}
void oracle_collide_2d(double* F, const oracle_params* pr) { collide_2d<double>(F, *pr); }
void oracle_stream_2d(const double* Fs, double* F, const oracle_params* pr) {
  std::vector<double> ghosts;
  stream_2d<double>(Fs, F, *pr, ghosts);
}
void oracle_run_2d(double* F, int nsteps, const oracle_params* pr) { run_2d<double>(F, nsteps, *pr); }

// ---- complex-step variants (real and imaginary parts in separate arrays) ----
void oracle_equilibrium_2d_cplx(const double* rho_re, const double* rho_im, const double* qx_re,
                                const double* qx_im, const double* qy_re, const double* qy_im,
                                double* F_re, double* F_im, const oracle_params* pr) {
  const size_t n = static_cast<size_t>(pr->nx) * pr->ny;
  for (size_t c = 0; c < n; ++c) {
    cplx f[13];
    equilibrium_2d<cplx>(cplx(rho_re[c], rho_im[c]), cplx(qx_re[c], qx_im[c]),
                         cplx(qy_re[c], qy_im[c]), *pr, f);
    for (int j = 0; j < 13; ++j) { F_re[j * n + c] = f[j].real(); F_im[j * n + c] = f[j].imag(); }
  }
}
void oracle_run_2d_cplx(double* F_re, double* F_im, int nsteps, const oracle_params* pr) {
  const size_t count = 13 * static_cast<size_t>(pr->nx) * pr->ny;
  std::vector<cplx> z;
  split(F_re, F_im, count, z);
  run_2d<cplx>(z.data(), nsteps, *pr);
  join(z, F_re, F_im);
}
void oracle_equilibrium_1d_cplx(const double* rho_re, const double* rho_im, const double* q_re,
                                const double* q_im, double* F_re, double* F_im, const oracle_params* pr) {
  const size_t n = pr->nx;
  for (size_t i = 0; i < n; ++i) {
    cplx f[5];
    equilibrium_1d<cplx>(cplx(rho_re[i], rho_im[i]), cplx(q_re[i], q_im[i]), *pr, f);
    for (int j = 0; j < 5; ++j) { F_re[j * n + i] = f[j].real(); F_im[j * n + i] = f[j].imag(); }
  }
}
void oracle_run_1d_cplx(double* F_re, double* F_im, int nsteps, const oracle_params* pr) {
  const size_t count = 5 * static_cast<size_t>(pr->nx);
  std::vector<cplx> z;
  split(F_re, F_im, count, z);
  run_1d<cplx>(z.data(), nsteps, *pr);
  join(z, F_re, F_im);
}

}  // extern "C"
