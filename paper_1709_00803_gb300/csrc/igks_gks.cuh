// igks_gks.cuh -- the gas-kinetic interface flux of one face (Eq. 4-14, 33-34) as device
// functions: Maxwellian moment tables, the closed-form 4x4 moment solves (Eq. 101, 11, 12),
// the time weights of Eq. 13 and the time-integrated flux with the Prandtl-number fix.
//
// The kernel is bound by the GB300 FP64 pipe, so the algebra is arranged to issue few
// FP64 instructions:
//  - every Maxwellian is set up with one reciprocal of the density and one reciprocal
//    square root (1/(2 lambda) = 2 e / ((K+2) rho); sqrt(lambda) = rsqrt(2 / (2 lambda)));
//  - a moment of a slope polynomial, <u^A v^B (a . psi) psi_k>, is taken in the frame
//    centred on the tangential velocity, where the odd moments of v - V vanish: the v and
//    xi integrals reduce the slope to a quadratic in u, contracted with the u-table by
//    three-term dot products (mv0 / mv1 below);
//  - erfc(x) is taken as e^(-x^2) erfcx(x) (x >= 0) or 2 - e^(-x^2) erfcx(-x) (x < 0),
//    with the e^(-lambda U^2) the first half-space moment needs anyway (erfcx costs two
//    thirds of erfc on GB300); the two half-space tables of the interface Maxwellian share
//    one erfcx and one exp; e^(-dt/tau) is taken as 1 - (1 - e^(-dt/tau)) from one expm1;
//  - reciprocals are __drcp_rn (the correctly rounded 1/x, bitwise 1.0 / x, about a
//    third cheaper than the division on GB300).
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
  const double ir = __drcp_rn(W[0]);
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

// erfc(x) / 2 from e2 = e^(-x^2): x >= 0 gives e2 erfcx(x) / 2, x < 0 gives
// 1 - e2 erfcx(-x) / 2 (erfc(x) + erfc(-x) = 2)
__device__ __forceinline__ double half_erfc(double x, double e2) {
  const double t = 0.5 * e2 * erfcx(fabs(x));
  return x >= 0.0 ? t : 1.0 - t;
}

// <u^n> over u >= 0 (sgn = +1) or u < 0 (sgn = -1):
// <u^0> = erfc(-sgn sqrt(lambda) U) / 2, <u^1> = U <u^0> + sgn e^{-lambda U^2} / (2 sqrt(pi lambda))
template <int N>
__device__ __forceinline__ void table_half(const Maxw& g, double sgn, double* m) {
  const double isl = 2.0 * g.h * g.sl;   // 1/sqrt(lambda)
  const double x = g.sl * g.U;
  const double e2 = exp(-x * x);
  m[0] = half_erfc(-sgn * x, e2);
  m[1] = g.U * m[0] + sgn * (0.5 * RSQRT_PI) * isl * e2;
  table_rec<N>(g.U, g.h, m);
}

// both half-space tables from one erfcx and one exp: <u^0>_{u<0} = 1 - <u^0>_{u>=0}
template <int N>
__device__ __forceinline__ void table_half_pair(const Maxw& g, double* mp, double* mn) {
  const double isl = 2.0 * g.h * g.sl;
  const double x = g.sl * g.U;
  const double e2 = exp(-x * x);
  const double e = (0.5 * RSQRT_PI) * isl * e2;
  mp[0] = half_erfc(-x, e2);
  mn[0] = 1.0 - mp[0];
  mp[1] = g.U * mp[0] + e;
  mn[1] = g.U * mn[0] - e;
  table_rec<N>(g.U, g.h, mp);
  table_rec<N>(g.U, g.h, mn);
}

// The tangential velocity v is always integrated over the whole line, so the moments are
// taken in the frame centred on it: v = V + c, where the odd moments of c vanish and
// <c^2> = h, <c^4> = 3 h^2; the internal energy has <xi^2> = X1 = K h, <xi^4> = X2 =
// K (K+2) h^2. Integrating c and xi out leaves polynomials of u, which are contracted with
// the u-table (whole line or half line) of the Maxwellian.
struct Frame {
  double V, h, X1, K1, Vh, c1, c2;
  // K1 = (h + X1 + V^2)/2, Vh = V^2 + h, c1 = h^2 + (X2 - X1^2)/2, c2 = (3h + X1 + V^2)/2
};
__device__ __forceinline__ Frame frame_of(const Maxw& g) {
  Frame f;
  f.V = g.V;
  f.h = g.h;
  f.X1 = KDOF * g.h;
  const double X2 = KDOF * (KDOF + 2) * g.h * g.h;
  f.Vh = g.V * g.V + g.h;
  f.K1 = 0.5 * (f.Vh + f.X1);
  f.c1 = g.h * g.h + 0.5 * (X2 - f.X1 * f.X1);
  f.c2 = 0.5 * (3.0 * g.h + f.X1 + g.V * g.V);
  return f;
}

// A slope polynomial a . psi = a0 + a1 u + a2 v + ha (u^2 + v^2 + xi^2), ha = a3/2, in the
// centred frame: al0 + a1 u + al2 c + ha (u^2 + c^2 + xi^2) with al0 = a0 + a2 V + ha V^2,
// al2 = a2 + 2 ha V. Integrated over c and xi it is S0(u) = s0 + a1 u + ha u^2 with
// s0 = al0 + ha (h + X1); times c, c^2, c^3 or xi^2 (see mv0 / mv1) it gives multiples of
// the same u-polynomial and of 1.
struct Slope {
  double s0, a1, ha, a2h, ka, kb2, kb3;
  // a2h = al2 h; ka = ha c1 + V al2 h (the u^0 term of the energy output, weight 1);
  // kb2 = 2 (V al2 h + ha h^2), kb3 = al2 h c2 + 2 V ha h^2 (the same for the weight v)
};
__device__ __forceinline__ Slope slope_of(const double* a, const Frame& f) {
  Slope s;
  s.ha = 0.5 * a[3];
  s.a1 = a[1];
  const double al0 = a[0] + f.V * (a[2] + s.ha * f.V);
  const double al2 = a[2] + 2.0 * s.ha * f.V;
  s.s0 = al0 + s.ha * (f.h + f.X1);
  s.a2h = al2 * f.h;
  const double hah2 = s.ha * f.h * f.h;
  s.ka = s.ha * f.c1 + f.V * s.a2h;
  s.kb2 = 2.0 * (f.V * s.a2h + hah2);
  s.kb3 = s.a2h * f.c2 + 2.0 * f.V * hah2;
  return s;
}

// P_j = <u^j S0(u)> over the u-table
template <int J>
__device__ __forceinline__ double pj(const double* u, const Slope& s) {
  return s.s0 * u[J] + s.a1 * u[J + 1] + s.ha * u[J + 2];
}

// acc[k] += w * <u^A (a . psi) psi_k>, psi = (1, u, v, (u^2 + v^2 + xi^2)/2)
template <int A>
__device__ __forceinline__ void mv0(const double* u, const Frame& f, const Slope& s, double w, double* acc) {
  const double P0 = pj<A>(u, s), P1 = pj<A + 1>(u, s), P2 = pj<A + 2>(u, s);
  acc[0] += w * P0;
  acc[1] += w * P1;
  acc[2] += w * (f.V * P0 + s.a2h * u[A]);
  acc[3] += w * (0.5 * P2 + f.K1 * P0 + s.ka * u[A]);
}

// acc[k] += w * <u^A v (a . psi) psi_k>
template <int A>
__device__ __forceinline__ void mv1(const double* u, const Frame& f, const Slope& s, double w, double* acc) {
  const double P0 = pj<A>(u, s), P1 = pj<A + 1>(u, s), P2 = pj<A + 2>(u, s);
  const double r3 = 0.5 * P2 + f.K1 * P0 + s.ka * u[A];   // the energy output with weight 1
  acc[0] += w * (f.V * P0 + s.a2h * u[A]);
  acc[1] += w * (f.V * P1 + s.a2h * u[A + 1]);
  acc[2] += w * (f.Vh * P0 + s.kb2 * u[A]);
  acc[3] += w * (f.V * r3 + 0.5 * s.a2h * u[A + 2] + s.kb3 * u[A] + f.V * f.h * P0);
}

// <u^A psi> (no slope)
template <int A>
__device__ __forceinline__ void mpsi(const double* u, const Frame& f, double* o) {
  o[0] = u[A];
  o[1] = u[A + 1];
  o[2] = f.V * u[A];
  o[3] = 0.5 * u[A + 2] + f.K1 * u[A];
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
  const Frame fr = frame_of(g);
  double u[7];
  table_full<7>(g.U, g.h, u);
  const MSolve ms = msolve_of(g);
  // slopes of Eq. 101 and the time slope of Eq. 11: <(a_n u + a_t v + A) psi>_g = 0
  double an[4], at[4], A[4], b[4];
  const double ir = __drcp_rn(g.r);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = sn[k] * ir;
  solve(ms, b, an);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = st[k] * ir;
  solve(ms, b, at);
  const Slope sn_ = slope_of(an, fr), st_ = slope_of(at, fr);
  double m[4] = {0, 0, 0, 0};
  mv0<1>(u, fr, sn_, 1.0, m);
  mv1<0>(u, fr, st_, 1.0, m);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = -m[k];
  solve(ms, b, A);
  const Slope sA = slope_of(A, fr);
  // half-space moments of this side
  table_half<7>(g, sgn, u);
  double t[4];
  mpsi<0>(u, fr, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.W0[k] += g.r * t[k];
  mpsi<1>(u, fr, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.T3[k] += g.r * t[k];
  mv0<2>(u, fr, sn_, g.r, acc.T4);
  mv1<1>(u, fr, st_, g.r, acc.T4);
  mv0<1>(u, fr, sA, g.r, acc.T5);
  mv0<1>(u, fr, sn_, g.r, acc.S4);
  mv1<0>(u, fr, st_, g.r, acc.S4);
  mv0<0>(u, fr, sA, g.r, acc.S5);
  return g.r * g.h;   // p = rho / (2 lambda)
}

// The time-integrated flux of one face in the face frame (Eq. 13-14) with the Prandtl
// fix. WL, WR: reconstructed face states; SLn.. their normal and tangential slopes;
// WcL, WcR: the centre states of the two cells (rotated); idL, idR: reciprocal normal
// distances centre to face; visc(h0) gives the laminar viscosity of the interface state
// from h0 = 1/(2 lambda0) (Sutherland's law); mut: face eddy viscosity.
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
  const Frame fr = frame_of(g0);
  double up[7], un[7], uf[7];
  table_full<7>(g0.U, g0.h, uf);
  table_half_pair<7>(g0, up, un);
  const MSolve ms0 = msolve_of(g0);
  const double ir0 = __drcp_rn(g0.r);
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
  const Slope sl_ = slope_of(abl, fr), sr_ = slope_of(abr, fr), st_ = slope_of(abt, fr);
  // Eq. 12 (reduced): <(abar_l u H + abar_r u (1-H) + abar_t v + Abar) psi>_g0 = 0
  double sq1[4] = {0, 0, 0, 0};
  mv0<1>(up, fr, sl_, 1.0, sq1);
  mv0<1>(un, fr, sr_, 1.0, sq1);
  mv1<0>(uf, fr, st_, 1.0, sq1);
  {
    double b[4];
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = -sq1[k];
    solve(ms0, b, Ab);
  }
  const Slope sA = slope_of(Ab, fr);

  // collision time (Eq. 33-34 with the pressure-jump term) and the time weights of Eq. 13
  // 1/p0 = 2 lambda0 / rho0 from the reciprocal already at hand
  const double ip0 = 2.0 * g0.lam * ir0;
  double tau = (visc(g0.h) + mut) * ip0;
  if (c_num != 0.0) tau += c_num * fabs(pL - pR) / (pL + pR) * dt;
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
  mpsi<1>(uf, fr, t);
  mv0<2>(up, fr, sl_, 1.0, eq1);
  mv0<2>(un, fr, sr_, 1.0, eq1);
  mv1<1>(uf, fr, st_, 1.0, eq1);
  mv0<1>(uf, fr, sA, 1.0, eq2);
  mv0<0>(uf, fr, sA, 1.0, sq2);
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
