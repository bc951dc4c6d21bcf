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
#include "igks_gks.cuh"
#include "igks_phys.cuh"

namespace igks {

// momentum of a conserved 4-vector (or of its slope) into the face frame (n, t)
__device__ __forceinline__ void rot(const double* g, double nx, double ny, double* o) {
  o[0] = g[0];
  o[1] = g[1] * nx + g[2] * ny;
  o[2] = -g[1] * ny + g[2] * nx;
  o[3] = g[3];
}

#ifndef IGKS_FLUX_MINB
#define IGKS_FLUX_MINB 1   // resident blocks per SM the register budget is cut for
#endif

__global__ void __launch_bounds__(128, IGKS_FLUX_MINB) k_flux(Dev d) {
  const int f = d.g_face0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.g_face0 + d.g_nface) return;
  const int s = d.fsolve[f];
  if (d.st[s].state != 0) return;
  const DevFlow& fl = d.flow[s];
  const int n = d.nc_pad, nf = d.nf;
  const int L = d.fL[f], R = d.fR[f], bc = d.fbc[f];
  const double nx = d.fnx[f], ny = d.fny[f], tx = -ny, ty = nx;
  const double S = d.fS[f], mxf = d.fmx[f], myf = d.fmy[f];
  const double idL = d.fidL[f], idR = d.fidR[f];
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

  // ---- Eq. 4-14: the time-integrated flux in the face frame ----
  double Fn[4];
  gks::face_flux(WL, WR, SLn, SLt, SRn, SRt, WcL, WcR, idL, idR, mut_face, dt, fl.c_num, fl.pr_fix,
                 [&](double h) { return viscosity_h(fl, h); }, Fn);

  // ---- back to the global frame, times the face length ----
  d.F[f] = Fn[0] * S;
  d.F[nf + f] = (Fn[1] * nx - Fn[2] * ny) * S;
  d.F[2 * nf + f] = (Fn[1] * ny + Fn[2] * nx) * S;
  d.F[3 * nf + f] = Fn[3] * S;

  // ---- SA face terms (Eq. 28-30) and the coefficients of its implicit system ----
  double o4 = 0.0, o5 = 0.0, aLR = 0.0, aRL = 0.0, dgl = 0.0, dgr = 0.0;
  if (fl.sa_on) {
    const double idn = __drcp_rn(d.fdn[f]);
    const double irl = __drcp_rn(WcLg[0]), irr = __drcp_rn(WcRg[0]);
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
  if (d.g_nface) k_flux<<<(d.g_nface + b - 1) / b, b, 0, s>>>(d);
}

}  // namespace igks
