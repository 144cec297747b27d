// Device arithmetic of the D1Q3Q2 (section 2) and D2Q5Q4Q4 (section 3) schemes of
// Dubois' vectorial lattice Boltzmann method for the shallow-water equations.
//
// The equilibria are the derivatives of the potentials h_j^* of the dual entropy
// (f_j = dh_j^*/dtheta, g_j = dh_j^*/du ...), written here in closed form in the
// conserved variables W = (h, qx = h u, qy = h v).  With gamma = 2, p = g h^2/2,
// K = 1/(2g) and kappa = K theta = h/2 - (u^2 + v^2)/(4g):
//
//   2D  f0 = a kappa,  r = (h - f0)/4,
//       f1,3 = r +- qx/(2 lambda),            f2,4 = r +- qy/(2 lambda)
//       gx1,3 = qx/4 +- (qx u + p)/(2 lambda), gx2,4 = qx/4 +- qx qy/(h 2 lambda)
//       gy1,3 = qy/4 +- qx qy/(h 2 lambda),    gy2,4 = qy/4 +- (qy v + p)/(2 lambda)
//   1D  f0 = a kappa,  f+- = h/2 - a kappa/2 +- q/(2 lambda),
//       g+- = q/2 +- (q u + p)/(2 lambda)
//
// and the collision is the BGK form of Eq. 2-relaxation, f* = f + s (f^eq - f).
//
// Every operation is an explicitly rounded intrinsic (no compiler contraction), laid
// out so that mirror-image cells see mirror-image operations: a field with a
// symmetry of the square keeps it bit for bit, in FP32 and FP64.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float recip(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double recip(double a) { return __drcp_rn(a); }

// Scheme constants in the storage precision.
template <class T>
struct Consts {
  T s;       // relaxation rate
  T a;       // rest-potential weight
  T c;       // 1 / (2 lambda)
  T half_g;  // g / 2
  T inv4g;   // 1 / (4 g)
};

template <class T>
__host__ Consts<T> make_consts(double g, double lambda, double s, double a) {
  Consts<T> k;
  k.s = static_cast<T>(s);
  k.a = static_cast<T>(a);
  k.c = static_cast<T>(1.0 / (2.0 * lambda));
  k.half_g = static_cast<T>(g / 2.0);
  k.inv4g = static_cast<T>(1.0 / (4.0 * g));
  return k;
}

// Conserved moments, summed in mirror-symmetric pairs.
template <class T>
__device__ __forceinline__ void moments13(const T f[13], T& h, T& qx, T& qy) {
  h = add(f[0], add(add(f[1], f[3]), add(f[2], f[4])));
  qx = add(add(f[5], f[7]), add(f[6], f[8]));
  qy = add(add(f[9], f[11]), add(f[10], f[12]));
}

template <class T>
__device__ __forceinline__ void equilibrium13(T h, T qx, T qy, const Consts<T>& k, T e[13]) {
  const T rh = recip(h);
  const T u = mul(qx, rh);
  const T v = mul(qy, rh);
  const T uu = add(mul(u, u), mul(v, v));
  const T kap = fmad(-uu, k.inv4g, mul(T(0.5), h));
  const T f0 = mul(k.a, kap);
  const T r = mul(sub(h, f0), T(0.25));
  const T p = mul(mul(k.half_g, h), h);
  const T ax = mul(qx, k.c);
  const T ay = mul(qy, k.c);
  const T x4 = mul(qx, T(0.25));
  const T y4 = mul(qy, T(0.25));
  const T pxx = mul(fmad(qx, u, p), k.c);
  const T pyy = mul(fmad(qy, v, p), k.c);
  const T pxy = mul(mul(mul(qx, qy), rh), k.c);
  e[0] = f0;
  e[1] = add(r, ax);
  e[2] = add(r, ay);
  e[3] = sub(r, ax);
  e[4] = sub(r, ay);
  e[5] = add(x4, pxx);
  e[6] = add(x4, pxy);
  e[7] = sub(x4, pxx);
  e[8] = sub(x4, pxy);
  e[9] = add(y4, pxy);
  e[10] = add(y4, pyy);
  e[11] = sub(y4, pxy);
  e[12] = sub(y4, pyy);
}

// Moments -> equilibria -> BGK relaxation, in place; the moments (h, qx, qy) are
// returned too (the collision conserves them).
template <class T>
__device__ __forceinline__ void collide13(T f[13], const Consts<T>& k, T& h, T& qx, T& qy) {
  moments13(f, h, qx, qy);
  T e[13];
  equilibrium13(h, qx, qy, k, e);
#pragma unroll
  for (int j = 0; j < 13; ++j) f[j] = fmad(k.s, sub(e[j], f[j]), f[j]);
}

template <class T>
__device__ __forceinline__ void collide13(T f[13], const Consts<T>& k) {
  T h, qx, qy;
  collide13(f, k, h, qx, qy);
}

// ---- 1D: populations f0, f+, f-, g+, g- ----
template <class T>
__device__ __forceinline__ void moments5(const T f[5], T& h, T& q) {
  h = add(f[0], add(f[1], f[2]));
  q = add(f[3], f[4]);
}

template <class T>
__device__ __forceinline__ void equilibrium5(T h, T q, const Consts<T>& k, T e[5]) {
  const T rh = recip(h);
  const T u = mul(q, rh);
  const T kap = fmad(-mul(u, u), k.inv4g, mul(T(0.5), h));
  const T f0 = mul(k.a, kap);
  const T half = mul(sub(h, f0), T(0.5));
  const T aq = mul(q, k.c);
  const T p = mul(mul(k.half_g, h), h);
  const T q2 = mul(q, T(0.5));
  const T pq = mul(fmad(q, u, p), k.c);
  e[0] = f0;
  e[1] = add(half, aq);
  e[2] = sub(half, aq);
  e[3] = add(q2, pq);
  e[4] = sub(q2, pq);
}

template <class T>
__device__ __forceinline__ void collide5(T f[5], const Consts<T>& k) {
  T h, q;
  moments5(f, h, q);
  T e[5];
  equilibrium5(h, q, k, e);
#pragma unroll
  for (int j = 0; j < 5; ++j) f[j] = fmad(k.s, sub(e[j], f[j]), f[j]);
}

}  // namespace lbm
