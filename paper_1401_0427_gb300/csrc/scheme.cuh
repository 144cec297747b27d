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
// and the collision is the BGK form of Eq. 2-relaxation, f* = f + s (f^eq - f), evaluated
// as f* = (1 - s) f + s f^eq with s folded into the constants of each equilibrium term
// (collide13: two operations per population instead of three).
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
// FP32: the fast reciprocal intrinsic (at most 2 ulp; the FP32 path is compared with the
// FP64 oracle at 1e-5).  FP64: Newton-Raphson for 1/a, two iterations of r <- r + r (1 - a r)
// (each residual and update one fused multiply-add) from the PTX approximation
// rcp.approx.ftz.f64; for positive normal depths it equals the IEEE round-to-nearest
// reciprocal (0 ulp on 2.7e8 sampled inputs in [1e-3, 1e3)) at fewer FP64 operations, the
// resource that bounds the FP64 kernels on GB300.  Either is a fixed function of h, so
// mirror-image cells still round alike.
__device__ __forceinline__ float recip(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double recip(double a) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
  double e = __fma_rn(-a, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-a, r, 1.0);
  return __fma_rn(r, e, r);
}

// Scheme constants in the storage precision.
template <class T>
struct Consts {
  T s;       // relaxation rate
  T a;       // rest-potential weight
  T c;       // 1 / (2 lambda)
  T half_g;  // g / 2
  T inv4g;   // 1 / (4 g)
  T nz;      // -0, a value the compiler cannot see (products of the paired path, below)
  // Rates of the non-conserved moments for the MRT collision (Eq. 2-relaxation with
  // distinct s_l), in the order of the paper's moment bases:
  //   2D: J_x, J_y, eps, XX_rho | f_xx, f_xy, XX_u | f_yx, f_yy, XX_v   (r[0..9])
  //   1D: J_rho, eps_rho, J_q                                            (r[0..2])
  T r[10];
  // 2D: the same rates with the exact power-of-two factors of the moment transforms folded
  // in (collide13_mrt): J_x / 2, J_y / 2, eps, XX_rho | f_xx / 2, f_xy / 2, XX_u / 4 | f_yx / 2,
  // f_yy / 2, XX_v / 4.  Scaling by a power of two commutes with rounding, so each product
  // is exactly half (a quarter) of the unscaled one and the halvings that follow it vanish.
  T m[10];
  // BGK with the rate folded in (collide13): f* = om f + s f^eq, s f^eq built from
  //   z = -(s f0) / 4 = s_a2 h + s_a4g (u^2 + v^2)  (s_a2, s_a4g carry the -1/4),
  //   s f0 = -4 z,  s r = s (h - f0) / 4 = s_4 h + z  (one rounding),
  //   s c p = (s_p h) h,  s c q and s q / 4 = q s_c and q s_4.
  // om and s_4 are formed from s as stored (om = 1 - s and s_4 = s / 4 exactly for s in
  // [1/2, 2]), so om + 4 s_4 = 1 and the masses and momenta of om f and s f^eq add up to those
  // of f with no bias from the rounding of the constants.
  T om;     // 1 - s
  T s_a2;   // -s a / 8
  T s_a4g;  // s a / (16 g)
  T s_p;    // s c g / 2
  T s_c;    // s c
  T s_4;    // s / 4
};

template <class T>
__host__ void set_mrt_folded(Consts<T>& k) {
  constexpr double scale[10] = {0.5, 0.5, 1.0, 1.0, 0.5, 0.5, 0.25, 0.5, 0.5, 0.25};
  for (int i = 0; i < 10; ++i) k.m[i] = static_cast<T>(static_cast<double>(k.r[i]) * scale[i]);
}

template <class T>
__host__ Consts<T> make_consts(double g, double lambda, double s, double a) {
  Consts<T> k;
  k.s = static_cast<T>(s);
  k.a = static_cast<T>(a);
  k.c = static_cast<T>(1.0 / (2.0 * lambda));
  k.half_g = static_cast<T>(g / 2.0);
  k.inv4g = static_cast<T>(1.0 / (4.0 * g));
  k.nz = static_cast<T>(-0.0);
  const double c = 1.0 / (2.0 * lambda), st = static_cast<double>(k.s);  // s as stored
  k.om = static_cast<T>(1.0 - st);
  k.s_a2 = static_cast<T>(-st * a / 8.0);
  k.s_a4g = static_cast<T>(st * a / (16.0 * g));
  k.s_p = static_cast<T>(st * c * g / 2.0);
  k.s_c = static_cast<T>(st * c);
  k.s_4 = static_cast<T>(st / 4.0);
  for (int i = 0; i < 10; ++i) k.r[i] = k.s;
  set_mrt_folded(k);
  return k;
}

// Constants with MRT rates (10 in 2D, 3 in 1D, in the order documented on Consts::r).
template <class T>
__host__ Consts<T> make_consts_mrt(double g, double lambda, double s, double a, const double* rates, int n) {
  Consts<T> k = make_consts<T>(g, lambda, s, a);
  for (int i = 0; i < n && i < 10; ++i) k.r[i] = static_cast<T>(rates[i]);
  set_mrt_folded(k);
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
  const T hf = sub(h, f0);  // r = hf / 4
  const T p = mul(mul(k.half_g, h), h);
  const T ax = mul(qx, k.c);
  const T ay = mul(qy, k.c);
  const T pxx = mul(fmad(qx, u, p), k.c);
  const T pyy = mul(fmad(qy, v, p), k.c);
  const T pxy = mul(mul(mul(qx, qy), rh), k.c);
  // r +- a and q/4 +- b as one fused multiply-add each: the quarter is exact, so each is the
  // rounded sum of the exact quarter and the other term, as add(mul(., 1/4), +-b) would give
  const T q4 = T(0.25);
  e[0] = f0;
  e[1] = fmad(hf, q4, ax);
  e[2] = fmad(hf, q4, ay);
  e[3] = fmad(hf, q4, -ax);
  e[4] = fmad(hf, q4, -ay);
  e[5] = fmad(qx, q4, pxx);
  e[6] = fmad(qx, q4, pxy);
  e[7] = fmad(qx, q4, -pxx);
  e[8] = fmad(qx, q4, -pxy);
  e[9] = fmad(qy, q4, pxy);
  e[10] = fmad(qy, q4, pyy);
  e[11] = fmad(qy, q4, -pxy);
  e[12] = fmad(qy, q4, -pyy);
}

// Moments -> BGK relaxation, in place: f* = (1 - s) f + s f^eq, where s f^eq is formed from
// the terms of equilibrium13 each scaled by s through its constant (s f0 = s a kappa, s r,
// s q / 4, s c q, s c (q u + p), s c qx qy / h), so each population takes one add and one
// fused multiply-add.  s r is one fused multiply-add of h and -s f0 / 4: with s r rounded
// twice (s h / 4, then minus s f0 / 4) the FP32 depth drifted about 5 times as fast as with
// f + s (f^eq - f) on the 4096^2 dam-break; rounded once it drifts about as fast (+9e-7
// against +7e-7 relative over 1000 steps).  The moments (h, qx, qy) are returned too (the collision conserves
// them).  The operations stay mirror-symmetric: x -> -x flips the signs of qx, u, s c qx
// and s c qx qy / h exactly and leaves s c (qx u + p) unchanged.
template <class T>
__device__ __forceinline__ void collide13(T f[13], const Consts<T>& k, T& h, T& qx, T& qy) {
  moments13(f, h, qx, qy);
  const T rh = recip(h);
  const T u = mul(qx, rh);
  const T v = mul(qy, rh);
  const T uu = add(mul(u, u), mul(v, v));
  const T z = fmad(uu, k.s_a4g, mul(k.s_a2, h));  // -s f0^eq / 4
  const T f0 = mul(z, T(-4));                      // s f0^eq (exact)
  const T r = fmad(h, k.s_4, z);                   // s (h - f0^eq) / 4
  const T p = mul(mul(k.s_p, h), h);               // s c p
  const T ax = mul(qx, k.s_c);
  const T ay = mul(qy, k.s_c);
  const T x4 = mul(qx, k.s_4);
  const T y4 = mul(qy, k.s_4);
  const T pxx = fmad(ax, u, p);
  const T pyy = fmad(ay, v, p);
  const T pxy = mul(mul(mul(qx, qy), rh), k.s_c);
  const T om = k.om;
  f[0] = fmad(om, f[0], f0);
  f[1] = fmad(om, f[1], add(r, ax));
  f[2] = fmad(om, f[2], add(r, ay));
  f[3] = fmad(om, f[3], sub(r, ax));
  f[4] = fmad(om, f[4], sub(r, ay));
  f[5] = fmad(om, f[5], add(x4, pxx));
  f[6] = fmad(om, f[6], add(x4, pxy));
  f[7] = fmad(om, f[7], sub(x4, pxx));
  f[8] = fmad(om, f[8], sub(x4, pxy));
  f[9] = fmad(om, f[9], add(y4, pxy));
  f[10] = fmad(om, f[10], add(y4, pyy));
  f[11] = fmad(om, f[11], sub(y4, pxy));
  f[12] = fmad(om, f[12], sub(y4, pyy));
}

template <class T>
__device__ __forceinline__ void collide13(T f[13], const Consts<T>& k) {
  T h, qx, qy;
  collide13(f, k, h, qx, qy);
}

// MRT form: f* = f + M^-1 S M (f^eq - f), with M the 13 moments of section 3 (rho, J_x,
// J_y, eps, XX_rho; q_x, f_xx, f_xy, XX_u; q_y, f_yx, f_yy, XX_v), S = diag of the rates
// (0 on the conserved rho, q_x, q_y).  Family by family, with d = f^eq - f:
//   f:  dJx/lam = r0 (d1 - d3), dJy/lam = r1 (d2 - d4), deps = r2 (d1 + d2 + d3 + d4 - 4 d0),
//       dXX = r3 (d1 - d2 + d3 - d4); back: df0 = -deps/5, s13 = (deps/5 + dXX)/2,
//       s24 = (deps/5 - dXX)/2, df1,3 = (s13 +- dJx/lam)/2, df2,4 = (s24 +- dJy/lam)/2;
//   gx: dfxx/lam = r4 (g1 - g3), dfxy/lam = r5 (g2 - g4), dXX_u = r6 (g1 - g2 + g3 - g4);
//       back: dg1,3 = (dXX_u/2 +- dfxx/lam)/2, dg2,4 = (-dXX_u/2 +- dfxy/lam)/2;  gy alike (r7..r9).
// The halvings are folded into the rates (Consts::m) and into the quarter that forms s13/2
// and s24/2, which gives the same rounded values with 14 operations fewer per cell; the
// last correction of each momentum family is subtracted instead of negated and added.
template <class T>
__device__ __forceinline__ void mrt_family4(const T d[4], T ra2, T rb2, T rx4, T& g0, T& g1, T& g2, T& g3n) {
  const T ah = mul(ra2, sub(d[0], d[2]));  // (dfxx/lam) / 2
  const T bh = mul(rb2, sub(d[1], d[3]));  // (dfxy/lam) / 2
  const T xh = mul(rx4, sub(add(d[0], d[2]), add(d[1], d[3])));  // dXX_u / 4
  g0 = add(xh, ah);
  g2 = sub(xh, ah);
  g1 = sub(bh, xh);
  g3n = add(xh, bh);  // -dg4
}

template <class T>
__device__ __forceinline__ void collide13_mrt(T f[13], const Consts<T>& k, T& h, T& qx, T& qy) {
  moments13(f, h, qx, qy);
  T e[13];
  equilibrium13(h, qx, qy, k, e);
  T d[13];
#pragma unroll
  for (int j = 0; j < 13; ++j) d[j] = sub(e[j], f[j]);
  const T jxh = mul(k.m[0], sub(d[1], d[3]));
  const T jyh = mul(k.m[1], sub(d[2], d[4]));
  const T e5 = mul(mul(k.m[2], sub(add(add(d[1], d[2]), add(d[3], d[4])), mul(T(4), d[0]))), T(0.2));
  const T xx = mul(k.m[3], sub(add(d[1], d[3]), add(d[2], d[4])));
  const T s13q = mul(T(0.25), add(e5, xx)), s24q = mul(T(0.25), sub(e5, xx));
  f[0] = sub(f[0], e5);
  f[1] = add(f[1], add(s13q, jxh));
  f[3] = add(f[3], sub(s13q, jxh));
  f[2] = add(f[2], add(s24q, jyh));
  f[4] = add(f[4], sub(s24q, jyh));
  T g0, g1, g2, g3n;
  mrt_family4(d + 5, k.m[4], k.m[5], k.m[6], g0, g1, g2, g3n);
  f[5] = add(f[5], g0);
  f[6] = add(f[6], g1);
  f[7] = add(f[7], g2);
  f[8] = sub(f[8], g3n);
  mrt_family4(d + 9, k.m[7], k.m[8], k.m[9], g0, g1, g2, g3n);
  f[9] = add(f[9], g0);
  f[10] = add(f[10], g1);
  f[11] = add(f[11], g2);
  f[12] = sub(f[12], g3n);
}

// Relaxation of either form.
template <class T, bool MRT>
__device__ __forceinline__ void collide13_any(T f[13], const Consts<T>& k, T& h, T& qx, T& qy) {
  if (MRT)
    collide13_mrt(f, k, h, qx, qy);
  else
    collide13(f, k, h, qx, qy);
}

// z = D(W)^T psi: vector-Jacobian product of the equilibria (closed forms of section 3
// in W = (h, qx, qy); kappa = h/2 - (qx^2 + qy^2)/(4 g h^2), c = 1/(2 lambda)).
template <class T>
__device__ __forceinline__ void equilibrium_vjp(T h, T qx, T qy, const T psi[13], const Consts<T>& K, T& zh,
                                                T& zx, T& zy) {
  const T rh = recip(h);
  const T u = qx * rh, v = qy * rh;
  const T gh = T(2) * K.half_g * h;
  const T inv2gh = T(2) * K.inv4g * rh;
  const T kh = T(0.5) + (u * u + v * v) * inv2gh;  // dkappa/dh
  const T kx = -u * inv2gh;                        // dkappa/dqx
  const T ky = -v * inv2gh;                        // dkappa/dqy
  const T Sf = (psi[1] + psi[3]) + (psi[2] + psi[4]);
  const T Af = psi[0] - T(0.25) * Sf;
  const T Df13 = psi[1] - psi[3], Df24 = psi[2] - psi[4];
  const T Sx = (psi[5] + psi[7]) + (psi[6] + psi[8]);
  const T Dx13 = psi[5] - psi[7], Dx24 = psi[6] - psi[8];
  const T Sy = (psi[9] + psi[11]) + (psi[10] + psi[12]);
  const T Dy13 = psi[9] - psi[11], Dy24 = psi[10] - psi[12];
  const T X = Dx24 + Dy13;
  const T c = K.c;
  zh = K.a * kh * Af + T(0.25) * Sf + c * (Dx13 * (gh - u * u) - X * u * v + Dy24 * (gh - v * v));
  zx = K.a * kx * Af + c * Df13 + T(0.25) * Sx + c * (T(2) * Dx13 * u + X * v);
  zy = K.a * ky * Af + c * Df24 + T(0.25) * Sy + c * (X * u + T(2) * Dy24 * v);
}

// ---- Two FP32 cells at once (the paired FP32 instructions of sm_100 and later) ----
// The same operations as collide13, in the same order, on (cell a, cell b) pairs, so each
// lane rounds exactly like the scalar code and the results are equal bit for bit.  The code
// generator contracts a paired multiply feeding a paired add into one fused multiply-add
// even when both carry an explicit rounding mode, which would change the rounding (and
// break the mirror symmetry of u u + v v).  So every paired product is formed as
// fma(a, b, nz) with nz = -0 read from the kernel's constants: exactly the rounded product
// a b (also for a zero product of either sign), in one instruction, and not a product
// the code generator can merge into the add that follows.
__device__ __forceinline__ unsigned long long pack2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(c)));
  return unpack2(r);
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Moments and equilibria of two cells, as moments13 and equilibrium13.
__device__ __forceinline__ void moments_equilibrium13x2(const float2 f[13], const Consts<float>& k, float2& h,
                                                        float2& qx, float2& qy, float2 e[13]) {
  const float2 nz = dup2(k.nz);
  auto mul2 = [&](float2 a, float2 b) { return fma2(a, b, nz); };  // the rounded product a b
  h = add2(f[0], add2(add2(f[1], f[3]), add2(f[2], f[4])));
  qx = add2(add2(f[5], f[7]), add2(f[6], f[8]));
  qy = add2(add2(f[9], f[11]), add2(f[10], f[12]));
  const float2 rh = make_float2(recip(h.x), recip(h.y));
  const float2 u = mul2(qx, rh);
  const float2 v = mul2(qy, rh);
  const float2 uu = add2(mul2(u, u), mul2(v, v));
  // the sign on the constant instead of on uu: the same exact product, no negation per pair
  const float2 kap = fma2(uu, dup2(-k.inv4g), mul2(dup2(0.5f), h));
  const float2 f0 = mul2(dup2(k.a), kap);
  const float2 r = mul2(sub2(h, f0), dup2(0.25f));
  const float2 p = mul2(mul2(dup2(k.half_g), h), h);
  const float2 c = dup2(k.c);
  const float2 ax = mul2(qx, c);
  const float2 ay = mul2(qy, c);
  const float2 x4 = mul2(qx, dup2(0.25f));
  const float2 y4 = mul2(qy, dup2(0.25f));
  const float2 pxx = mul2(fma2(qx, u, p), c);
  const float2 pyy = mul2(fma2(qy, v, p), c);
  const float2 pxy = mul2(mul2(mul2(qx, qy), rh), c);
  e[0] = f0;
  e[1] = add2(r, ax);
  e[2] = add2(r, ay);
  e[3] = sub2(r, ax);
  e[4] = sub2(r, ay);
  e[5] = add2(x4, pxx);
  e[6] = add2(x4, pxy);
  e[7] = sub2(x4, pxx);
  e[8] = sub2(x4, pxy);
  e[9] = add2(y4, pxy);
  e[10] = add2(y4, pyy);
  e[11] = sub2(y4, pxy);
  e[12] = sub2(y4, pyy);
}

// collide13 on two cells, operation for operation; (h, qx, qy) receive the conserved
// moments of the pulled populations (as collide13's).
__device__ __forceinline__ void collide13x2(float2 f[13], const Consts<float>& k, float2& h, float2& qx, float2& qy) {
  const float2 nz = dup2(k.nz);
  auto mul2 = [&](float2 a, float2 b) { return fma2(a, b, nz); };  // the rounded product a b
  h = add2(f[0], add2(add2(f[1], f[3]), add2(f[2], f[4])));
  qx = add2(add2(f[5], f[7]), add2(f[6], f[8]));
  qy = add2(add2(f[9], f[11]), add2(f[10], f[12]));
  const float2 rh = make_float2(recip(h.x), recip(h.y));
  const float2 u = mul2(qx, rh);
  const float2 v = mul2(qy, rh);
  const float2 uu = add2(mul2(u, u), mul2(v, v));
  const float2 sc = dup2(k.s_c), s4 = dup2(k.s_4);
  const float2 z = fma2(uu, dup2(k.s_a4g), mul2(dup2(k.s_a2), h));
  const float2 f0 = mul2(z, dup2(-4.0f));
  const float2 r = fma2(h, s4, z);
  const float2 p = mul2(mul2(dup2(k.s_p), h), h);
  const float2 ax = mul2(qx, sc);
  const float2 ay = mul2(qy, sc);
  const float2 x4 = mul2(qx, s4);
  const float2 y4 = mul2(qy, s4);
  const float2 pxx = fma2(ax, u, p);
  const float2 pyy = fma2(ay, v, p);
  const float2 pxy = mul2(mul2(mul2(qx, qy), rh), sc);
  const float2 om = dup2(k.om);
  f[0] = fma2(om, f[0], f0);
  f[1] = fma2(om, f[1], add2(r, ax));
  f[2] = fma2(om, f[2], add2(r, ay));
  f[3] = fma2(om, f[3], sub2(r, ax));
  f[4] = fma2(om, f[4], sub2(r, ay));
  f[5] = fma2(om, f[5], add2(x4, pxx));
  f[6] = fma2(om, f[6], add2(x4, pxy));
  f[7] = fma2(om, f[7], sub2(x4, pxx));
  f[8] = fma2(om, f[8], sub2(x4, pxy));
  f[9] = fma2(om, f[9], add2(y4, pxy));
  f[10] = fma2(om, f[10], add2(y4, pyy));
  f[11] = fma2(om, f[11], sub2(y4, pxy));
  f[12] = fma2(om, f[12], sub2(y4, pyy));
}

__device__ __forceinline__ void collide13x2(float2 f[13], const Consts<float>& k) {
  float2 h, qx, qy;
  collide13x2(f, k, h, qx, qy);
}

// The MRT form of collide13_mrt on (cell a, cell b) pairs, operation for operation.
__device__ __forceinline__ void mrt_family4x2(const float2 d[4], float ra2, float rb2, float rx4, float2 nz,
                                              float2& g0, float2& g1, float2& g2, float2& g3n) {
  auto mul2 = [&](float2 a, float2 b) { return fma2(a, b, nz); };
  const float2 ah = mul2(dup2(ra2), sub2(d[0], d[2]));
  const float2 bh = mul2(dup2(rb2), sub2(d[1], d[3]));
  const float2 xh = mul2(dup2(rx4), sub2(add2(d[0], d[2]), add2(d[1], d[3])));
  g0 = add2(xh, ah);
  g2 = sub2(xh, ah);
  g1 = sub2(bh, xh);
  g3n = add2(xh, bh);
}

__device__ __forceinline__ void collide13x2_mrt(float2 f[13], const Consts<float>& k, float2& h, float2& qx,
                                                float2& qy) {
  const float2 nz = dup2(k.nz);
  auto mul2 = [&](float2 a, float2 b) { return fma2(a, b, nz); };
  float2 e[13];
  moments_equilibrium13x2(f, k, h, qx, qy, e);
  float2 d[13];
#pragma unroll
  for (int j = 0; j < 13; ++j) d[j] = sub2(e[j], f[j]);
  const float2 quarter = dup2(0.25f);
  const float2 jxh = mul2(dup2(k.m[0]), sub2(d[1], d[3]));
  const float2 jyh = mul2(dup2(k.m[1]), sub2(d[2], d[4]));
  const float2 e5 =
      mul2(mul2(dup2(k.m[2]), sub2(add2(add2(d[1], d[2]), add2(d[3], d[4])), mul2(dup2(4.0f), d[0]))), dup2(0.2f));
  const float2 xx = mul2(dup2(k.m[3]), sub2(add2(d[1], d[3]), add2(d[2], d[4])));
  const float2 s13q = mul2(quarter, add2(e5, xx)), s24q = mul2(quarter, sub2(e5, xx));
  f[0] = sub2(f[0], e5);
  f[1] = add2(f[1], add2(s13q, jxh));
  f[3] = add2(f[3], sub2(s13q, jxh));
  f[2] = add2(f[2], add2(s24q, jyh));
  f[4] = add2(f[4], sub2(s24q, jyh));
  float2 g0, g1, g2, g3n;
  mrt_family4x2(d + 5, k.m[4], k.m[5], k.m[6], nz, g0, g1, g2, g3n);
  f[5] = add2(f[5], g0);
  f[6] = add2(f[6], g1);
  f[7] = add2(f[7], g2);
  f[8] = sub2(f[8], g3n);
  mrt_family4x2(d + 9, k.m[7], k.m[8], k.m[9], nz, g0, g1, g2, g3n);
  f[9] = add2(f[9], g0);
  f[10] = add2(f[10], g1);
  f[11] = add2(f[11], g2);
  f[12] = sub2(f[12], g3n);
}

template <bool MRT>
__device__ __forceinline__ void collide13x2_any(float2 f[13], const Consts<float>& k, float2& h, float2& qx,
                                                float2& qy) {
  if constexpr (MRT)
    collide13x2_mrt(f, k, h, qx, qy);
  else
    collide13x2(f, k, h, qx, qy);
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
  const T hf = sub(h, f0);  // half = hf / 2
  const T aq = mul(q, k.c);
  const T p = mul(mul(k.half_g, h), h);
  const T pq = mul(fmad(q, u, p), k.c);
  // exact halves folded into fused multiply-adds, as in equilibrium13
  e[0] = f0;
  e[1] = fmad(hf, T(0.5), aq);
  e[2] = fmad(hf, T(0.5), -aq);
  e[3] = fmad(q, T(0.5), pq);
  e[4] = fmad(q, T(0.5), -pq);
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

// MRT form in 1D on the moments of section 2 (rho, J_rho = lam (f+ - f-),
// eps_rho = lam^2 (f+ + f- - 2 f0), q, J_q = lam (g+ - g-)); with d = f^eq - f:
// dJ/lam = r0 (d+ - d-), deps/lam^2 = r1 (d+ + d- - 2 d0), dJq/lam = r2 (dg+ - dg-);
// back: sum = deps/(3 lam^2), df0 = -sum, df+- = (sum +- dJ/lam)/2, dg+- = +- dJq/(2 lam).
template <class T>
__device__ __forceinline__ void collide5_mrt(T f[5], const Consts<T>& k) {
  T h, q;
  moments5(f, h, q);
  T e[5];
  equilibrium5(h, q, k, e);
  T d[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) d[j] = e[j] - f[j];
  const T j1 = k.r[0] * (d[1] - d[2]);
  const T sm = k.r[1] * ((d[1] + d[2]) - T(2) * d[0]) * T(1.0 / 3.0);
  const T jq = k.r[2] * (d[3] - d[4]) * T(0.5);
  f[0] = f[0] - sm;
  f[1] = f[1] + T(0.5) * (sm + j1);
  f[2] = f[2] + T(0.5) * (sm - j1);
  f[3] = f[3] + jq;
  f[4] = f[4] - jq;
}

template <class T, bool MRT>
__device__ __forceinline__ void collide5_any(T f[5], const Consts<T>& k) {
  if (MRT)
    collide5_mrt(f, k);
  else
    collide5(f, k);
}

}  // namespace lbm
