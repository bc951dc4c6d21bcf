// igks_phys.cuh -- small device functions shared by the kernels of libigks: gas state,
// viscosity, eddy viscosity and the ghost-cell boundary states of Section II.E.
#pragma once
#include "igks_dev.h"

namespace igks {

__device__ __forceinline__ double pressure_of(double r, double mx, double my, double E) {
  return (GAMMA - 1.0) * (E - 0.5 * (mx * mx + my * my) / r);
}

// lambda = rho / (2 p) of Eq. 2
__device__ __forceinline__ double lambda_of(double r, double mx, double my, double E) {
  return r / (2.0 * pressure_of(r, mx, my, E));
}

// Sutherland's law relative to the free stream, T/T_inf = lambda_inf / lambda
__device__ __forceinline__ double viscosity(const DevFlow& fl, double lam) {
  double tr = fl.lam_inf / lam;
  return fl.mu_inf * tr * sqrt(tr) * (1.0 + fl.s_star) / (tr + fl.s_star);
}

// the same law from h = 1/(2 lambda): T/T_inf = 2 h lambda_inf, no division by lambda
__device__ __forceinline__ double viscosity_h(const DevFlow& fl, double h) {
  double tr = 2.0 * h * fl.lam_inf;
  return fl.mu_inf * tr * sqrt(tr) * (1.0 + fl.s_star) / (tr + fl.s_star);
}

// eddy viscosity mu_t = rho nu_tilde fv1 (Eq. 34); zero for non-positive nu_tilde
__device__ __forceinline__ double eddy_viscosity(const DevFlow& fl, double r, double nut, double mu) {
  if (!fl.sa_on || !(nut > 0.0)) return 0.0;
  double chi = nut * r / mu;
  double c3 = chi * chi * chi;
  return r * nut * c3 / (c3 + SA_CV1 * SA_CV1 * SA_CV1);
}

// ghost state of a boundary face from the interior centre state Wi (global frame)
__device__ inline void ghost_state(const DevFlow& fl, int bc, double nx, double ny,
                                   const double* Wi, double* Wg) {
  if (bc == 3) {          // non-slip wall: momentum and nu_tilde reversed
    Wg[0] = Wi[0]; Wg[1] = -Wi[1]; Wg[2] = -Wi[2]; Wg[3] = Wi[3]; Wg[4] = -Wi[4];
    return;
  }
  if (bc == 5) {          // moving wall: velocity mirrored about the wall velocity
    const double* Wf = fl.Winf;
    const double tx = -ny, ty = nx;
    const double uw = (Wf[1] * tx + Wf[2] * ty) / Wf[0];
    const double r = Wi[0], u = Wi[1] / r, v = Wi[2] / r;
    const double ug = 2.0 * uw * tx - u, vg = 2.0 * uw * ty - v;
    Wg[0] = r; Wg[1] = r * ug; Wg[2] = r * vg;
    Wg[3] = Wi[3] - 0.5 * r * (u * u + v * v) + 0.5 * r * (ug * ug + vg * vg);
    Wg[4] = -Wi[4];
    return;
  }
  if (bc == 2) {          // symmetry: normal momentum reversed
    double mn = Wi[1] * nx + Wi[2] * ny;
    Wg[0] = Wi[0]; Wg[1] = Wi[1] - 2.0 * mn * nx; Wg[2] = Wi[2] - 2.0 * mn * ny;
    Wg[3] = Wi[3]; Wg[4] = Wi[4];
    return;
  }
  const double g = GAMMA;
  const double* Wf = fl.Winf;
  if (bc == 4) {
    // outflow (Section II.E): boundary-normal velocity from the Riemann invariants R+
    // (inside) and R- (free stream); density, tangential velocity, internal energy per
    // unit volume (the temperature, lambda) and nu_tilde from inside
    double ri = Wi[0], ui = Wi[1] / ri, vi = Wi[2] / ri;
    double ei = Wi[3] - 0.5 * ri * (ui * ui + vi * vi);
    double ci = sqrt(g * (g - 1.0) * ei / ri);
    double po = pressure_of(Wf[0], Wf[1], Wf[2], Wf[3]);
    double co = sqrt(g * po / Wf[0]);
    double uni = ui * nx + vi * ny, uno = (Wf[1] * nx + Wf[2] * ny) / Wf[0];
    double ub = 0.5 * ((uni + 2.0 * ci / (g - 1.0)) + (uno - 2.0 * co / (g - 1.0)));
    double bx = ub * nx + (ui - uni * nx), by = ub * ny + (vi - uni * ny);
    Wg[0] = ri; Wg[1] = ri * bx; Wg[2] = ri * by;
    Wg[3] = ei + 0.5 * ri * (bx * bx + by * by);
    Wg[4] = Wi[4];
    return;
  }
  // free stream (Section II.E)
  for (int v = 0; v < 5; v++) Wg[v] = Wf[v];
}

}  // namespace igks
