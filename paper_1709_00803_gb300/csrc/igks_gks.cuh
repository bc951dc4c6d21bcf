// igks_gks.cuh -- the gas-kinetic interface flux of one face (Eq. 4-14, 33-34) as device
// functions: Maxwellian moment tables, the closed-form 4x4 moment solves (Eq. 101, 11, 12),
// the time weights of Eq. 13 and the time-integrated flux with the Prandtl-number fix.
//
// The kernel is bound by the GB300 FP64 pipe, so the algebra is arranged to issue few
// FP64 instructions:
//  - every Maxwellian is set up with one reciprocal of the density and one reciprocal
//    square root (1/(2 lambda) = 2 e / ((K+2) rho); sqrt(lambda) = rsqrt(2 / (2 lambda)));
//  - a moment of a slope polynomial, <u^A v^B (a . psi) psi_k>, is assembled from the
//    products U_a V_b of the tables and five-term dot products (mv below), instead of
//    expanding every product psi_j psi_k;
//  - the two half-space tables of the interface Maxwellian share one erfc and one exp,
//    and e^(-dt/tau) is taken as 1 - (1 - e^(-dt/tau)) from the one expm1.
#pragma once
#include "igks_dev.h"

namespace igks {
namespace gks {

constexpr double RSQRT_PI = 0.56418958354775628695;   // 1/sqrt(pi)
constexpr double HK = 2.0 / (KDOF + 2);               // 1/(2 lambda) = HK * e_int / rho

// A Maxwellian of Eq. 2 in the face frame: density, velocity (U normal, V tangential),
// h = 1/(2 lambda) (the variance of each velocity component) and lambda itself.
struct Maxw {
  double r, U, V, h, lam, sl;   // sl = sqrt(lambda)
};

__device__ __forceinline__ Maxw maxw_of(const double* W) {
  Maxw g;
  g.r = W[0];
  const double ir = 1.0 / W[0];
  g.U = W[1] * ir;
  g.V = W[2] * ir;
  const double e = W[3] - 0.5 * (W[1] * g.U + W[2] * g.V);    // internal energy per volume
  g.h = HK * e * ir;
  g.sl = rsqrt(2.0 * g.h);
  g.lam = g.sl * g.sl;
  return g;
}

// <u^n>, n = 0..N-1, over the whole line: recurrence U_{n+2} = U U_{n+1} + (n+1) h U_n
template <int N>
__device__ __forceinline__ void table_full(double U, double h, double* m) {
  m[0] = 1.0;
  m[1] = U;
#pragma unroll
  for (int k = 0; k + 2 < N; k++) m[k + 2] = U * m[k + 1] + (k + 1) * h * m[k];
}

template <int N>
__device__ __forceinline__ void table_rec(double U, double h, double* m) {
#pragma unroll
  for (int k = 0; k + 2 < N; k++) m[k + 2] = U * m[k + 1] + (k + 1) * h * m[k];
}

// <u^n> over u >= 0 (sgn = +1) or u < 0 (sgn = -1):
// <u^0> = erfc(-sgn sqrt(lambda) U) / 2, <u^1> = U <u^0> + sgn e^{-lambda U^2} / (2 sqrt(pi lambda))
template <int N>
__device__ __forceinline__ void table_half(const Maxw& g, double sgn, double* m) {
  const double isl = 2.0 * g.h * g.sl;   // 1/sqrt(lambda)
  m[0] = 0.5 * erfc(-sgn * g.sl * g.U);
  m[1] = g.U * m[0] + sgn * (0.5 * RSQRT_PI) * isl * exp(-g.lam * g.U * g.U);
  table_rec<N>(g.U, g.h, m);
}

// both half-space tables from one erfc and one exp: <u^0>_{u<0} = 1 - <u^0>_{u>=0}
template <int N>
__device__ __forceinline__ void table_half_pair(const Maxw& g, double* mp, double* mn) {
  const double isl = 2.0 * g.h * g.sl;
  const double e = (0.5 * RSQRT_PI) * isl * exp(-g.lam * g.U * g.U);
  mp[0] = 0.5 * erfc(-g.sl * g.U);
  mn[0] = 1.0 - mp[0];
  mp[1] = g.U * mp[0] + e;
  mn[1] = g.U * mn[0] - e;
  table_rec<N>(g.U, g.h, mp);
  table_rec<N>(g.U, g.h, mn);
}

// moments of the internal degrees of freedom: <xi^2> = K h, <xi^4> = K (K+2) h^2
struct Xi {
  double x1, x2;
};
__device__ __forceinline__ Xi xi_of(double h) { return Xi{KDOF * h, KDOF * (KDOF + 2) * h * h}; }

// <u^A v^B psi>, psi = (1, u, v, (u^2 + v^2 + xi^2)/2)
template <int A, int B>
__device__ __forceinline__ void mpsi(const double* u, const double* v, const Xi& x, double* o) {
  const double p = u[A] * v[B];
  o[0] = p;
  o[1] = u[A + 1] * v[B];
  o[2] = u[A] * v[B + 1];
  o[3] = 0.5 * (u[A + 2] * v[B] + u[A] * v[B + 2] + x.x1 * p);
}

// slope polynomial a . psi = a0 + a1 u + a2 v + ha (u^2 + v^2 + xi^2), ha = a3 / 2
struct Slope {
  double a0, a1, a2, ha, c0, hx2;   // c0 = a0 + ha <xi^2>, hx2 = ha <xi^4>
};
__device__ __forceinline__ Slope slope_of(const double* a, const Xi& x) {
  Slope s;
  s.a0 = a[0]; s.a1 = a[1]; s.a2 = a[2]; s.ha = 0.5 * a[3];
  s.c0 = s.a0 + s.ha * x.x1;
  s.hx2 = s.ha * x.x2;
  return s;
}

// <u^I v^J (a . psi)> without the xi^2 part of the slope (t) and with it (returned)
template <int I, int J>
__device__ __forceinline__ double mq(const double* u, const double* v, const Slope& s, double* t) {
  const double q = s.a1 * (u[I + 1] * v[J]) + s.a2 * (u[I] * v[J + 1]) + s.ha * (u[I + 2] * v[J] + u[I] * v[J + 2]);
  const double p = u[I] * v[J];
  if (t) *t = q + s.a0 * p;
  return q + s.c0 * p;
}

// acc[k] += w * <u^A v^B (a . psi) psi_k>, k = 0..3
template <int A, int B>
__device__ __forceinline__ void mv(const double* u, const double* v, const Xi& x, const Slope& s, double w,
                                   double* acc) {
  double t;
  const double r0 = mq<A, B>(u, v, s, &t);
  const double r1 = mq<A + 1, B>(u, v, s, nullptr);
  const double r2 = mq<A, B + 1>(u, v, s, nullptr);
  // (u^2 + v^2 + xi^2)/2 times the slope: the u^2 and v^2 parts shift the table, the xi^2
  // part multiplies the slope's own terms by <xi^2> and its xi^2 term by <xi^4>
  const double r3 = 0.5 * (mq<A + 2, B>(u, v, s, nullptr) + mq<A, B + 2>(u, v, s, nullptr) + x.x1 * t +
                           s.hx2 * (u[A] * v[B]));
  acc[0] += w * r0;
  acc[1] += w * r1;
  acc[2] += w * r2;
  acc[3] += w * r3;
}

// Constants of the closed-form solve of <a psi>_g = b about one Maxwellian
struct MSolve {
  double U, V, E2, l2, c4;   // E2 = U^2 + V^2 + (K+2) h, l2 = 2 lambda, c4 = 4 lambda^2 / (K+2)
};
__device__ __forceinline__ MSolve msolve_of(const Maxw& g) {
  MSolve m;
  m.U = g.U; m.V = g.V;
  m.E2 = g.U * g.U + g.V * g.V + (KDOF + 2) * g.h;
  m.l2 = 2.0 * g.lam;
  m.c4 = (4.0 / (KDOF + 2)) * g.lam * g.lam;
  return m;
}

// closed-form solution of the 4x4 Maxwellian moment system <a psi>_g = b
__device__ __forceinline__ void solve(const MSolve& m, const double* b, double* a) {
  const double R4 = 2.0 * b[3] - m.E2 * b[0];
  const double R2 = b[1] - m.U * b[0];
  const double R3 = b[2] - m.V * b[0];
  a[3] = m.c4 * (R4 - 2.0 * m.U * R2 - 2.0 * m.V * R3);
  a[2] = m.l2 * R3 - m.V * a[3];
  a[1] = m.l2 * R2 - m.U * a[3];
  a[0] = b[0] - m.U * a[1] - m.V * a[2] - 0.5 * a[3] * m.E2;
}

// Running sums over the two sides of the interface: the equilibrium state W0 (Eq. 5's
// g0 is the Maxwellian of it), the non-equilibrium lines 4-6 of Eq. 13 (T3..T5) and the
// same integrals without the factor u (S4, S5) used by the heat flux.
struct SideSums {
  double W0[4], T3[4], T4[4], T5[4], S4[4], S5[4];
};

// One side of the interface: sgn = +1 for the left state with H[u], -1 for the right with
// 1 - H[u]. W, sn, st: conserved state and its normal / tangential slopes in the face frame.
// Returns the pressure of the side.
__device__ __forceinline__ double side_terms(const double* W, const double* sn, const double* st, double sgn,
                                             SideSums& acc) {
  const Maxw g = maxw_of(W);
  const Xi x = xi_of(g.h);
  double u[7], v[6];
  table_full<7>(g.U, g.h, u);
  table_full<6>(g.V, g.h, v);
  const MSolve ms = msolve_of(g);
  // slopes of Eq. 101 and the time slope of Eq. 11: <(a_n u + a_t v + A) psi>_g = 0
  double an[4], at[4], A[4], b[4];
  const double ir = 1.0 / g.r;
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = sn[k] * ir;
  solve(ms, b, an);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = st[k] * ir;
  solve(ms, b, at);
  const Slope sn_ = slope_of(an, x), st_ = slope_of(at, x);
  double m[4] = {0, 0, 0, 0};
  mv<1, 0>(u, v, x, sn_, 1.0, m);
  mv<0, 1>(u, v, x, st_, 1.0, m);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = -m[k];
  solve(ms, b, A);
  const Slope sA = slope_of(A, x);
  // half-space moments of this side
  table_half<7>(g, sgn, u);
  double t[4];
  mpsi<0, 0>(u, v, x, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.W0[k] += g.r * t[k];
  mpsi<1, 0>(u, v, x, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.T3[k] += g.r * t[k];
  mv<2, 0>(u, v, x, sn_, g.r, acc.T4);
  mv<1, 1>(u, v, x, st_, g.r, acc.T4);
  mv<1, 0>(u, v, x, sA, g.r, acc.T5);
  mv<1, 0>(u, v, x, sn_, g.r, acc.S4);
  mv<0, 1>(u, v, x, st_, g.r, acc.S4);
  mv<0, 0>(u, v, x, sA, g.r, acc.S5);
  return g.r * g.h;   // p = rho / (2 lambda)
}

// The time-integrated flux of one face in the face frame (Eq. 13-14) with the Prandtl
// fix. WL, WR: reconstructed face states; SLn.. their normal and tangential slopes;
// WcL, WcR: the centre states of the two cells (rotated); idL, idR: reciprocal normal
// distances centre to face; mu_face: laminar viscosity of the interface state is computed
// here from the free-stream Sutherland law via visc(lambda0); mut: face eddy viscosity.
template <class Visc>
__device__ __forceinline__ void face_flux(const double* WL, const double* WR, const double* SLn, const double* SLt,
                                          const double* SRn, const double* SRt, const double* WcL,
                                          const double* WcR, double idL, double idR, double mut, double dt,
                                          double c_num, double pr_fix, Visc visc, double* Fn) {
  SideSums acc;
#pragma unroll
  for (int k = 0; k < 4; k++) acc.W0[k] = acc.T3[k] = acc.T4[k] = acc.T5[k] = acc.S4[k] = acc.S5[k] = 0.0;
  const double pL = side_terms(WL, SLn, SLt, 1.0, acc);
  const double pR = side_terms(WR, SRn, SRt, -1.0, acc);

  // interface equilibrium g0 (Eq. 5) and its slopes
  const Maxw g0 = maxw_of(acc.W0);
  const Xi x = xi_of(g0.h);
  double up[7], un[7], uf[7], v0[6];
  table_full<7>(g0.U, g0.h, uf);
  table_full<6>(g0.V, g0.h, v0);
  table_half_pair<7>(g0, up, un);
  const MSolve ms0 = msolve_of(g0);
  const double ir0 = 1.0 / g0.r;
  double abl[4], abr[4], abt[4], Ab[4];
  {
    double b[4];
    const double sl = ir0 * idL, sr = ir0 * idR;
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = (acc.W0[k] - WcL[k]) * sl;
    solve(ms0, b, abl);
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = (WcR[k] - acc.W0[k]) * sr;
    solve(ms0, b, abr);
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = 0.5 * (SLt[k] + SRt[k]) * ir0;
    solve(ms0, b, abt);
  }
  const Slope sl_ = slope_of(abl, x), sr_ = slope_of(abr, x), st_ = slope_of(abt, x);
  // Eq. 12 (reduced): <(abar_l u H + abar_r u (1-H) + abar_t v + Abar) psi>_g0 = 0
  double sq1[4] = {0, 0, 0, 0};
  mv<1, 0>(up, v0, x, sl_, 1.0, sq1);
  mv<1, 0>(un, v0, x, sr_, 1.0, sq1);
  mv<0, 1>(uf, v0, x, st_, 1.0, sq1);
  {
    double b[4];
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = -sq1[k];
    solve(ms0, b, Ab);
  }
  const Slope sA = slope_of(Ab, x);

  // collision time (Eq. 33-34 with the pressure-jump term) and the time weights of Eq. 13
  const double p0 = g0.r * g0.h;
  const double tau = (visc(g0.lam) + mut) / p0 + c_num * fabs(pL - pR) / (pL + pR) * dt;
  const double xr = dt / tau;
  const double ome = -expm1(-xr);   // 1 - e^{-dt/tau}
  const double e = 1.0 - ome;
  const double q0 = dt - tau * ome;
  const double q1 = 2.0 * tau * tau * ome - tau * dt * (1.0 + e);
  const double q2 = 0.5 * dt * dt - tau * dt + tau * tau * ome;
  const double q3 = tau * ome;
  const double q4 = -2.0 * tau * tau * ome + tau * dt * e;
  const double q5 = -tau * tau * ome;

  // Eq. 14, and the state integrals for the heat flux
  double t[4], eq1[4] = {0, 0, 0, 0}, eq2[4] = {0, 0, 0, 0}, sq2[4] = {0, 0, 0, 0};
  mpsi<1, 0>(uf, v0, x, t);
  mv<2, 0>(up, v0, x, sl_, 1.0, eq1);
  mv<2, 0>(un, v0, x, sr_, 1.0, eq1);
  mv<1, 1>(uf, v0, x, st_, 1.0, eq1);
  mv<1, 0>(uf, v0, x, sA, 1.0, eq2);
  mv<0, 0>(uf, v0, x, sA, 1.0, sq2);
  double Ws[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    Fn[k] = q0 * g0.r * t[k] + q1 * g0.r * eq1[k] + q2 * g0.r * eq2[k] + q3 * acc.T3[k] + q4 * acc.T4[k] +
            q5 * acc.T5[k];
    Ws[k] = q0 * acc.W0[k] + q1 * g0.r * sq1[k] + q2 * g0.r * sq2[k] + q3 * acc.W0[k] + q4 * acc.S4[k] +
            q5 * acc.S5[k];
  }
  // heat flux about (U0, V0) and the Prandtl-number fix
  const double U0 = g0.U, V0 = g0.V;
  const double e0 = U0 * U0 + V0 * V0;
  const double heat = Fn[3] - U0 * Fn[1] - V0 * Fn[2] + 0.5 * e0 * Fn[0] - U0 * Ws[3] + U0 * U0 * Fn[0] +
                      U0 * V0 * Ws[2] - 0.5 * U0 * e0 * Ws[0];
  Fn[3] += pr_fix * heat;
}

}  // namespace gks
}  // namespace igks
