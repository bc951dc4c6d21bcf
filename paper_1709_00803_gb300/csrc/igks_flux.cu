// igks_flux.cu -- BGK-NS gas-kinetic interface flux (Eq. 1-14, 33-34) and the
// Spalart-Allmaras face terms (Eq. 28-30) on sm_103a, one thread per face.
//
// Per face: reconstruct both sides at the face midpoint from the limited least-squares
// gradients (Eq. 10), rotate into the face frame, build the half-space Maxwellian moment
// tables (erfc/exp closed forms), solve the ten 4x4 moment systems of Eq. 101, 11 and 12
// in closed form, take the six time weights of Eq. 13 integrated over [0, dt], assemble
// the time-integrated flux of Eq. 14 with the Prandtl-number fix, rotate back and scale
// by the face length. The two sides are processed one after the other and folded into
// running sums so that only one side's moment tables are live at a time.
//
// The kernel is bound by FP64 arithmetic (erfc/exp and ~2 kflop of moment algebra per
// face), not by HBM: it reads ~250 B and writes ~80 B per face.
#include "igks_dev.h"
#include "igks_phys.cuh"

namespace igks {

namespace {

constexpr double RSQRT_PI = 0.56418958354775628695;   // 1/sqrt(pi)

// u-moments <u^n>, n = 0..N-1, of a Maxwellian over the whole line
template <int N>
__device__ __forceinline__ void moments_full(double U, double h, double* m) {   // h = 1/(2 lambda)
  m[0] = 1.0;
  m[1] = U;
#pragma unroll
  for (int k = 0; k + 2 < N; k++) m[k + 2] = U * m[k + 1] + (k + 1) * h * m[k];
}

// the recurrence of the u-moments from <u^0> and <u^1>
template <int N>
__device__ __forceinline__ void moments_rec(double U, double h, double* m) {
#pragma unroll
  for (int k = 0; k + 2 < N; k++) m[k + 2] = U * m[k + 1] + (k + 1) * h * m[k];
}

// u-moments over u >= 0 (sgn = +1) or u < 0 (sgn = -1)
template <int N>
__device__ __forceinline__ void moments_half(double U, double lam, double h, double sgn, double* m) {
  const double isl = rsqrt(lam);
  m[0] = 0.5 * erfc(-sgn * (lam * isl) * U);
  m[1] = U * m[0] + sgn * 0.5 * exp(-lam * U * U) * RSQRT_PI * isl;
  moments_rec<N>(U, h, m);
}

// both half-space u-moment tables of one Maxwellian: <u^0>_{u<0} = 1 - <u^0>_{u>=0}
// (erfc(x) + erfc(-x) = 2), and the exponential term is shared
template <int N>
__device__ __forceinline__ void moments_half_pair(double U, double lam, double h, double* mp, double* mn) {
  const double isl = rsqrt(lam);
  const double e = 0.5 * exp(-lam * U * U) * RSQRT_PI * isl;
  mp[0] = 0.5 * erfc(-(lam * isl) * U);
  mn[0] = 1.0 - mp[0];
  mp[1] = U * mp[0] + e;
  mn[1] = U * mn[0] - e;
  moments_rec<N>(U, h, mp);
  moments_rec<N>(U, h, mn);
}

// <u^A v^B psi>, psi = (1, u, v, (u^2+v^2+xi^2)/2)
template <int A, int B>
__device__ __forceinline__ void muv(const double* u, const double* v, double x2, double* o) {
  double ub = u[A] * v[B];
  o[0] = ub;
  o[1] = u[A + 1] * v[B];
  o[2] = u[A] * v[B + 1];
  o[3] = 0.5 * (u[A + 2] * v[B] + u[A] * v[B + 2] + ub * x2);
}

// acc += s * <u^A v^B (a . psi) psi>
template <int A, int B>
__device__ __forceinline__ void mauv(const double* u, const double* v, double x2, double x4,
                                     const double* a, double s, double* acc) {
  double t[4], r[4], h[4];
  muv<A, B>(u, v, x2, t);
#pragma unroll
  for (int k = 0; k < 4; k++) r[k] = a[0] * t[k];
  muv<A + 1, B>(u, v, x2, t);
#pragma unroll
  for (int k = 0; k < 4; k++) r[k] += a[1] * t[k];
  muv<A, B + 1>(u, v, x2, t);
#pragma unroll
  for (int k = 0; k < 4; k++) r[k] += a[2] * t[k];
  muv<A + 2, B>(u, v, x2, h);
  muv<A, B + 2>(u, v, x2, t);
  double ub = u[A] * v[B];
  h[0] += t[0] + x2 * ub;
  h[1] += t[1] + x2 * u[A + 1] * v[B];
  h[2] += t[2] + x2 * u[A] * v[B + 1];
  h[3] += t[3] + 0.5 * (x2 * u[A + 2] * v[B] + x2 * u[A] * v[B + 2] + x4 * ub);
#pragma unroll
  for (int k = 0; k < 4; k++) acc[k] += s * (r[k] + 0.5 * a[3] * h[k]);
}

// the constants of the closed-form moment solve of one Maxwellian (U, V, lambda), computed
// once and shared by all the solves about it (no division inside a solve)
struct MSolve {
  double U, V, E2, l2, c4;   // E2 = U^2 + V^2 + (K+2)/(2 lambda), l2 = 2 lambda, c4 = 4 lambda^2/(K+2)
};

__device__ __forceinline__ MSolve msolve(double U, double V, double lam, double h) {   // h = 1/(2 lambda)
  MSolve m;
  m.U = U; m.V = V;
  m.E2 = U * U + V * V + (KDOF + 2) * h;
  m.l2 = 2.0 * lam;
  m.c4 = (4.0 / (KDOF + 2)) * lam * lam;
  return m;
}

// closed-form solution of <a psi>_g = b for the Maxwellian of m, K internal dof
__device__ __forceinline__ void solve_moment(const MSolve& m, const double* b, double* a) {
  double R4 = 2.0 * b[3] - m.E2 * b[0];
  double R2 = b[1] - m.U * b[0];
  double R3 = b[2] - m.V * b[0];
  a[3] = m.c4 * (R4 - 2.0 * m.U * R2 - 2.0 * m.V * R3);
  a[2] = m.l2 * R3 - m.V * a[3];
  a[1] = m.l2 * R2 - m.U * a[3];
  a[0] = b[0] - m.U * a[1] - m.V * a[2] - 0.5 * a[3] * m.E2;
}

__device__ __forceinline__ void prim(const double* W, double* r, double* U, double* V, double* lam) {
  *r = W[0];
  double ir = 1.0 / W[0];
  *U = W[1] * ir;
  *V = W[2] * ir;
  *lam = (KDOF + 2) * W[0] / (4.0 * (W[3] - 0.5 * W[0] * ((*U) * (*U) + (*V) * (*V))));
}

__device__ __forceinline__ void rot(const double* g, double nx, double ny, double* o) {
  o[0] = g[0];
  o[1] = g[1] * nx + g[2] * ny;
  o[2] = -g[1] * ny + g[2] * nx;
  o[3] = g[3];
}

// running sums over the two sides of Eq. 13's non-equilibrium lines (4-6), the interface
// equilibrium state W0 and the matching state integrals used by the heat flux
struct SideSums {
  double W0[4], T3[4], T4[4], T5[4], S4[4], S5[4];
};

// One side (sgn = +1: left with H[u], -1: right with 1 - H[u]) of the interface.
__device__ __forceinline__ void side_terms(const double* Wf, const double* sn, const double* st,
                                           double sgn, SideSums& acc, double* p_out) {
  double r, U, V, lam;
  prim(Wf, &r, &U, &V, &lam);
  const double h = 0.5 / lam;
  double u[7], v[6];
  moments_full<7>(U, h, u);
  moments_full<6>(V, h, v);
  const double x2 = KDOF * h, x4 = KDOF * (KDOF + 2) * h * h;
  // spatial slopes of Eq. 101 and the time slope of Eq. 11
  double an[4], at[4], A[4], b[4];
  const double ir = 1.0 / r;
  const MSolve ms = msolve(U, V, lam, h);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = sn[k] * ir;
  solve_moment(ms, b, an);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = st[k] * ir;
  solve_moment(ms, b, at);
  double m[4] = {0, 0, 0, 0};
  mauv<1, 0>(u, v, x2, x4, an, 1.0, m);
  mauv<0, 1>(u, v, x2, x4, at, 1.0, m);
#pragma unroll
  for (int k = 0; k < 4; k++) b[k] = -m[k];
  solve_moment(ms, b, A);
  // half-space moments of this side
  moments_half<7>(U, lam, h, sgn, u);
  double t[4];
  muv<0, 0>(u, v, x2, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.W0[k] += r * t[k];
  muv<1, 0>(u, v, x2, t);
#pragma unroll
  for (int k = 0; k < 4; k++) acc.T3[k] += r * t[k];
  mauv<2, 0>(u, v, x2, x4, an, r, acc.T4);
  mauv<1, 1>(u, v, x2, x4, at, r, acc.T4);
  mauv<1, 0>(u, v, x2, x4, A, r, acc.T5);
  mauv<1, 0>(u, v, x2, x4, an, r, acc.S4);
  mauv<0, 1>(u, v, x2, x4, at, r, acc.S4);
  mauv<0, 0>(u, v, x2, x4, A, r, acc.S5);
  *p_out = r * h;   // p = rho / (2 lambda)
}

}  // namespace

__global__ void __launch_bounds__(128) k_flux(Dev d) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nf) return;
  const int s = d.fsolve[f];
  if (d.st[s].state != 0) return;
  const DevFlow& fl = d.flow[s];
  const int n = d.nc_pad, nf = d.nf;
  const int L = d.fL[f], R = d.fR[f], bc = d.fbc[f];
  const double nx = d.fnx[f], ny = d.fny[f], tx = -ny, ty = nx;
  const double S = d.fS[f], mxf = d.fmx[f], myf = d.fmy[f];
  const double dL = d.fdL[f], dR = d.fdR[f];
  const double dt = __longlong_as_double((long long)d.dt_bits[s]);

  // ---- left side: centre state, reconstruction (Eq. 10), slopes, rotation ----
  double WcLg[5], WcL[4], WL[4], SLn[4], SLt[4];
  {
    double g[4], sn[4], stt[4];
    const double ox = mxf - d.cx[L], oy = myf - d.cy[L];
#pragma unroll
    for (int v = 0; v < 5; v++) WcLg[v] = d.W[v * n + L];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      double ph = d.phi[v * n + L];
      double gx = ph * d.grad[(2 * v) * n + L], gy = ph * d.grad[(2 * v + 1) * n + L];
      g[v] = WcLg[v] + gx * ox + gy * oy;
      sn[v] = gx * nx + gy * ny;
      stt[v] = gx * tx + gy * ty;
    }
    rot(g, nx, ny, WL);
    rot(sn, nx, ny, SLn);
    rot(stt, nx, ny, SLt);
    rot(WcLg, nx, ny, WcL);
  }
  // ---- right side: interior cell, mirrored ghost (wall, symmetry, moving wall) or the
  //      free-stream / outflow ghost state without slopes ----
  double WcRg[5], WcR[4], WR[4], SRn[4], SRt[4];
  double muR, mtR;
  if (R >= 0) {
    double g[4], sn[4], stt[4];
    const double ox = mxf - d.cx[R], oy = myf - d.cy[R];
#pragma unroll
    for (int v = 0; v < 5; v++) WcRg[v] = d.W[v * n + R];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      double ph = d.phi[v * n + R];
      double gx = ph * d.grad[(2 * v) * n + R], gy = ph * d.grad[(2 * v + 1) * n + R];
      g[v] = WcRg[v] + gx * ox + gy * oy;
      sn[v] = gx * nx + gy * ny;
      stt[v] = gx * tx + gy * ty;
    }
    rot(g, nx, ny, WR);
    rot(sn, nx, ny, SRn);
    rot(stt, nx, ny, SRt);
    muR = d.mu_l[R];
    mtR = d.mu_t[R];
  } else {
#pragma unroll
    for (int v = 0; v < 5; v++) WcRg[v] = d.G[v * nf + f];
    muR = d.Gmu[f];
    mtR = d.Gmu[nf + f];
    if (bc == 2 || bc == 3 || bc == 5) {
      const double st2 = (bc == 2) ? 1.0 : -1.0;
      WR[0] = WL[0]; WR[1] = -WL[1]; WR[2] = st2 * WL[2]; WR[3] = WL[3];
      if (bc == 5) {   // moving wall: tangential velocity mirrored about the wall velocity
        const double uw = (fl.Winf[1] * tx + fl.Winf[2] * ty) / fl.Winf[0];
        const double ut = WL[2] / WL[0], utg = 2.0 * uw - ut;
        WR[2] = WL[0] * utg;
        WR[3] = WL[3] - 0.5 * WL[0] * ut * ut + 0.5 * WL[0] * utg * utg;
      }
      SRn[0] = -SLn[0]; SRn[1] = SLn[1]; SRn[2] = -st2 * SLn[2]; SRn[3] = -SLn[3];
      SRt[0] = SLt[0]; SRt[1] = -SLt[1]; SRt[2] = st2 * SLt[2]; SRt[3] = SLt[3];
    } else {
      rot(WcRg, nx, ny, WR);
#pragma unroll
      for (int v = 0; v < 4; v++) { SRn[v] = 0.0; SRt[v] = 0.0; }
    }
  }
  rot(WcRg, nx, ny, WcR);
  const double mut_face = 0.5 * (d.mu_t[L] + mtR);

  // ---- Eq. 4 and 11: non-equilibrium slopes of both sides, folded into sums ----
  SideSums acc;
#pragma unroll
  for (int k = 0; k < 4; k++) acc.W0[k] = acc.T3[k] = acc.T4[k] = acc.T5[k] = acc.S4[k] = acc.S5[k] = 0.0;
  double pL, pR;
  side_terms(WL, SLn, SLt, 1.0, acc, &pL);
  side_terms(WR, SRn, SRt, -1.0, acc, &pR);

  // ---- interface equilibrium g0 (Eq. 5) and its slopes ----
  double r0, U0, V0, lam0;
  prim(acc.W0, &r0, &U0, &V0, &lam0);
  const double h0 = 0.5 / lam0;
  double up[7], un[7], uf[7], v0[6];
  moments_full<7>(U0, h0, uf);
  moments_full<6>(V0, h0, v0);
  moments_half_pair<7>(U0, lam0, h0, up, un);
  const MSolve ms0 = msolve(U0, V0, lam0, h0);
  const double x2 = KDOF * h0, x4 = KDOF * (KDOF + 2) * h0 * h0;
  double abl[4], abr[4], abt[4], Ab[4];
  {
    double b[4];
    const double ir0 = 1.0 / r0;
    const double sl = ir0 / dL, sr = ir0 / dR;
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = (acc.W0[k] - WcL[k]) * sl;
    solve_moment(ms0, b, abl);
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = (WcR[k] - acc.W0[k]) * sr;
    solve_moment(ms0, b, abr);
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = 0.5 * (SLt[k] + SRt[k]) * ir0;
    solve_moment(ms0, b, abt);
  }
  // Eq. 12 (reduced): <(abar_l u H + abar_r u (1-H) + abar_t v + Abar) psi>_g0 = 0
  double sq1[4] = {0, 0, 0, 0};
  mauv<1, 0>(up, v0, x2, x4, abl, 1.0, sq1);
  mauv<1, 0>(un, v0, x2, x4, abr, 1.0, sq1);
  mauv<0, 1>(uf, v0, x2, x4, abt, 1.0, sq1);
  {
    double b[4];
#pragma unroll
    for (int k = 0; k < 4; k++) b[k] = -sq1[k];
    solve_moment(ms0, b, Ab);
  }

  // ---- collision time (Eq. 33-34 + pressure-jump term) and time weights ----
  const double p0 = r0 * h0;
  const double tau = (viscosity(fl, lam0) + mut_face) / p0 + fl.c_num * fabs(pL - pR) / (pL + pR) * dt;
  const double x = dt / tau;
  const double ome = -expm1(-x);   // 1 - e^{-dt/tau}
  const double e = exp(-x);
  const double q0 = dt - tau * ome;
  const double q1 = 2.0 * tau * tau * ome - tau * dt * (1.0 + e);
  const double q2 = 0.5 * dt * dt - tau * dt + tau * tau * ome;
  const double q3 = tau * ome;
  const double q4 = -2.0 * tau * tau * ome + tau * dt * e;
  const double q5 = -tau * tau * ome;

  // ---- Eq. 14: time-integrated flux, and the state integrals for the heat flux ----
  double Fn[4], eq1[4] = {0, 0, 0, 0}, eq2[4] = {0, 0, 0, 0}, sq2[4] = {0, 0, 0, 0}, t[4];
  muv<1, 0>(uf, v0, x2, t);
  mauv<2, 0>(up, v0, x2, x4, abl, 1.0, eq1);
  mauv<2, 0>(un, v0, x2, x4, abr, 1.0, eq1);
  mauv<1, 1>(uf, v0, x2, x4, abt, 1.0, eq1);
  mauv<1, 0>(uf, v0, x2, x4, Ab, 1.0, eq2);
  mauv<0, 0>(uf, v0, x2, x4, Ab, 1.0, sq2);
  double Ws[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    Fn[k] = q0 * r0 * t[k] + q1 * r0 * eq1[k] + q2 * r0 * eq2[k] + q3 * acc.T3[k] + q4 * acc.T4[k] + q5 * acc.T5[k];
    Ws[k] = q0 * acc.W0[k] + q1 * r0 * sq1[k] + q2 * r0 * sq2[k] + q3 * acc.W0[k] + q4 * acc.S4[k] + q5 * acc.S5[k];
  }
  // heat flux about (U0, V0) and the Prandtl-number fix
  const double e0 = U0 * U0 + V0 * V0;
  const double heat = Fn[3] - U0 * Fn[1] - V0 * Fn[2] + 0.5 * e0 * Fn[0] - U0 * Ws[3] + U0 * U0 * Fn[0]
                    + U0 * V0 * Ws[2] - 0.5 * U0 * e0 * Ws[0];
  Fn[3] += fl.pr_fix * heat;

  // ---- back to the global frame, times the face length ----
  d.F[f] = Fn[0] * S;
  d.F[nf + f] = (Fn[1] * nx - Fn[2] * ny) * S;
  d.F[2 * nf + f] = (Fn[1] * ny + Fn[2] * nx) * S;
  d.F[3 * nf + f] = Fn[3] * S;

  // ---- SA face terms (Eq. 28-30) and the coefficients of its implicit system ----
  double o4 = 0.0, o5 = 0.0, aLR = 0.0, aRL = 0.0, dgl = 0.0, dgr = 0.0;
  if (fl.sa_on) {
    const double idn = 1.0 / d.fdn[f];
    const double irl = 1.0 / WcLg[0], irr = 1.0 / WcRg[0];
    const double vni = (WcLg[1] * nx + WcLg[2] * ny) * irl;
    const double vnj = (WcRg[1] * nx + WcRg[2] * ny) * irr;
    const double nui = d.mu_l[L] * irl, nuj = muR * irr;
    const double gradn = (WcRg[4] - WcLg[4]) * idn;
    const double finv = fmax(vni, 0.0) * WcLg[4] + fmin(vnj, 0.0) * WcRg[4];
    const double kap = 1.0 / (2.0 * SA_SIGMA) * ((nui + nuj) + (1.0 + SA_CB2) * (WcLg[4] + WcRg[4]));
    const double fvis = kap * gradn;
    const double fadl = SA_CB2 / SA_SIGMA * WcLg[4] * gradn;
    const double fadr = SA_CB2 / SA_SIGMA * WcRg[4] * (-gradn);
    o4 = (-finv + fvis - fadl) * S;
    o5 = (finv - fvis - fadr) * S;
    const double kd = kap * idn;
    aLR = S * (fmin(vnj, 0.0) - kd);
    aRL = S * (fmin(-vni, 0.0) - kd);
    dgl = S * (fmax(vni, 0.0) + kd);
    dgr = S * (fmax(-vnj, 0.0) + kd);
  }
  d.F[4 * nf + f] = o4;
  d.F[5 * nf + f] = o5;
  d.sa_a[f] = aLR;
  d.sa_a[nf + f] = aRL;
  d.sa_a[2 * nf + f] = dgl;
  d.sa_a[3 * nf + f] = dgr;
}

void launch_flux(const Dev& d, cudaStream_t s) {
  const int b = d.flux_block > 0 ? d.flux_block : 128;
  if (d.nf) k_flux<<<(d.nf + b - 1) / b, b, 0, s>>>(d);
}

}  // namespace igks
