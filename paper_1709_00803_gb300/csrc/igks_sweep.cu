// igks_sweep.cu -- matrix-free LU-SGS forward and backward sweeps (Eq. 19-22 for the
// mean flow, Eq. 31-32 for the SA variable) with the FP64 state update, in FP64 or FP32.
#include <float.h>

#include "igks_dev.h"
#include "igks_phys.cuh"

namespace igks {

// ===================================================================================
// LU-SGS sweeps (Eq. 19-22 mean flow, Eq. 31-32 SA), level-scheduled: one block per
// solve walks its levels in order; cells of one level are independent. The increment
// of the Euler flux of each processed cell, dF = F(W + dW) - F(W) in x and y, is formed
// once by that cell in an incremental (difference-free) form and read by its
// neighbours, which project it on their face normal.
// ===================================================================================

template <class T>
__device__ __forceinline__ void delta_flux(T r, T mx, T my, T E, T dr, T dmx, T dmy, T dE, T* o) {
  const T g1 = (T)(GAMMA - 1.0);
  T r1 = r + dr;
  T u = mx / r, v = my / r;
  T inv = (T)1 / (r * r1);
  T du = (dmx * r - mx * dr) * inv, dv = (dmy * r - my * dr) * inv;
  T dmxu = dmx * u + mx * du + dmx * du;
  T dmyv = dmy * v + my * dv + dmy * dv;
  T p = g1 * (E - (T)0.5 * (mx * u + my * v));
  T dp = g1 * (dE - (T)0.5 * (dmxu + dmyv));
  T H = E + p, dH = dE + dp;
  o[0] = dmx;                               // x: mass
  o[1] = dmy;                               // y: mass
  o[2] = dmxu + dp;                         // x: x-momentum
  o[3] = dmx * v + mx * dv + dmx * dv;      // y: x-momentum
  o[4] = dmy * u + my * du + dmy * du;      // x: y-momentum
  o[5] = dmyv + dp;                         // y: y-momentum
  o[6] = dH * u + H * du + dH * du;         // x: energy
  o[7] = dH * v + H * dv + dH * dv;         // y: energy
}

template <class T>
__global__ void k_sweep_fwd(Dev d) {
  const int s = blockIdx.x;
  const SolveState& st = d.st[s];
  if (st.state != 0) return;
  const DevFlow& fl = d.flow[s];
  const int n = d.nc_pad, nf = d.nf;
  const double cfl = st.cfl;
  T* dWs = (T*)d.dWs;
  T* dF = (T*)d.dF;
  const int l0 = d.lvl_solve_ptr[s], l1 = d.lvl_solve_ptr[s + 1] - 1;
  for (int l = l0; l < l1; l++) {
    int b = d.fwd_lvl[l], e = d.fwd_lvl[l + 1];
    for (int k = b + threadIdx.x; k < e; k += blockDim.x) {
      int i = d.fwd_order[k];
      T acc[5];
#pragma unroll
      for (int v = 0; v < 5; v++) acc[v] = (T)d.M[v * n + i];
      for (int q = d.cf_ptr[i]; q < d.cf_ptr[i + 1]; q++) {
        int f = d.cf_face[q];
        int L = d.fL[f], R = d.fR[f];
        if (R < 0) continue;                 // ghost increments are zero in this sweep
        bool own = (L == i);
        int j = own ? R : L;
        if (j >= i) continue;
        T sg = own ? (T)1 : (T)-1;
        T nx = sg * (T)d.fnx[f], ny = sg * (T)d.fny[f];
        T hS = (T)0.5 * (T)d.fS[f], lam = (T)d.lam_f[f];
#pragma unroll
        for (int v = 0; v < 4; v++) {
          T dfn = dF[(2 * v) * n + j] * nx + dF[(2 * v + 1) * n + j] * ny;
          acc[v] -= hS * (dfn - lam * dWs[v * n + j]);
        }
        if (fl.sa_on) acc[4] -= (T)d.sa_a[(own ? 0 : 1) * nf + f] * dWs[4 * n + j];
      }
      double Lam = d.Lam[i];
      T D = (T)(Lam / cfl + Lam);
      T dw[5];
#pragma unroll
      for (int v = 0; v < 4; v++) dw[v] = acc[v] / D;
      dw[4] = fl.sa_on ? acc[4] / (T)(Lam / cfl + d.sa_diag[i]) : (T)0;
#pragma unroll
      for (int v = 0; v < 5; v++) dWs[v * n + i] = dw[v];
      T o[8];
      delta_flux<T>((T)d.W[i], (T)d.W[n + i], (T)d.W[2 * n + i], (T)d.W[3 * n + i], dw[0], dw[1], dw[2], dw[3], o);
#pragma unroll
      for (int c = 0; c < 8; c++) dF[c * n + i] = o[c];
    }
    __syncthreads();
  }
}

template <class T>
__global__ void k_sweep_bwd(Dev d) {
  const int s = blockIdx.x;
  SolveState& st = d.st[s];
  if (st.state != 0) return;
  const DevFlow& fl = d.flow[s];
  const int n = d.nc_pad, nf = d.nf;
  const double cfl = st.cfl;
  T* dWs = (T*)d.dWs;
  T* dWo = (T*)d.dW;
  T* dF = (T*)d.dF;
  double eq40 = 0.0;
  int bad = 0;
  const int l0 = d.blvl_solve_ptr[s], l1 = d.blvl_solve_ptr[s + 1] - 1;
  for (int l = l0; l < l1; l++) {
    int b = d.bwd_lvl[l], e = d.bwd_lvl[l + 1];
    for (int k = b + threadIdx.x; k < e; k += blockDim.x) {
      int i = d.bwd_order[k];
      T ws[5];
#pragma unroll
      for (int v = 0; v < 5; v++) ws[v] = dWs[v * n + i];
      T acc[5] = {0, 0, 0, 0, 0};
      for (int q = d.cf_ptr[i]; q < d.cf_ptr[i + 1]; q++) {
        int f = d.cf_face[q];
        int L = d.fL[f], R = d.fR[f];
        bool own = (L == i);
        T sg = own ? (T)1 : (T)-1;
        T nx = sg * (T)d.fnx[f], ny = sg * (T)d.fny[f];
        T hS = (T)0.5 * (T)d.fS[f], lam = (T)d.lam_f[f];
        if (R < 0) {
          int bc = d.fbc[f];
          if (bc == 1) continue;             // far-field increments are zero
          // wall / symmetry ghost: boundary map of the cell's own forward increment
          T g[5];
          g[0] = ws[0]; g[3] = ws[3];
          if (bc == 3) { g[1] = -ws[1]; g[2] = -ws[2]; g[4] = -ws[4]; }
          else {
            T fnx = (T)d.fnx[f], fny = (T)d.fny[f];
            T mn = ws[1] * fnx + ws[2] * fny;
            g[1] = ws[1] - (T)2 * mn * fnx; g[2] = ws[2] - (T)2 * mn * fny; g[4] = ws[4];
          }
          T o[8];
          delta_flux<T>((T)d.G[f], (T)d.G[nf + f], (T)d.G[2 * nf + f], (T)d.G[3 * nf + f], g[0], g[1], g[2], g[3], o);
#pragma unroll
          for (int v = 0; v < 4; v++) acc[v] += hS * ((o[2 * v] * nx + o[2 * v + 1] * ny) - lam * g[v]);
          if (fl.sa_on) acc[4] += (T)d.sa_a[f] * g[4];
          continue;
        }
        int j = own ? R : L;
        if (j <= i) continue;
#pragma unroll
        for (int v = 0; v < 4; v++) {
          T dfn = dF[(2 * v) * n + j] * nx + dF[(2 * v + 1) * n + j] * ny;
          acc[v] += hS * (dfn - lam * dWo[v * n + j]);
        }
        if (fl.sa_on) acc[4] += (T)d.sa_a[(own ? 0 : 1) * nf + f] * dWo[4 * n + j];
      }
      double Lam = d.Lam[i];
      T D = (T)(Lam / cfl + Lam);
      T dw[5];
#pragma unroll
      for (int v = 0; v < 4; v++) dw[v] = ws[v] - acc[v] / D;
      dw[4] = fl.sa_on ? ws[4] - acc[4] / (T)(Lam / cfl + d.sa_diag[i]) : (T)0;
#pragma unroll
      for (int v = 0; v < 5; v++) dWo[v * n + i] = dw[v];
      double Wi[5];
#pragma unroll
      for (int v = 0; v < 5; v++) Wi[v] = d.W[v * n + i];
      T o[8];
      delta_flux<T>((T)Wi[0], (T)Wi[1], (T)Wi[2], (T)Wi[3], dw[0], dw[1], dw[2], dw[3], o);
#pragma unroll
      for (int c = 0; c < 8; c++) dF[c * n + i] = o[c];
      // update (FP64) and the Eq. 40 ratio
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int v = 0; v < 4; v++) {
        double dv = (double)dw[v];
        num += dv * dv;
        den += Wi[v] * Wi[v];
        Wi[v] += dv;
      }
      Wi[4] += (double)dw[4];
      if (Wi[4] < 0.0) Wi[4] = 0.0;
      eq40 = fmax(eq40, sqrt(num) / sqrt(den));
      double p = pressure_of(Wi[0], Wi[1], Wi[2], Wi[3]);
      if (!(Wi[0] > 0.0) || !(p > 0.0) || !isfinite(Wi[3]) || !isfinite(Wi[4])) bad = 1;
#pragma unroll
      for (int v = 0; v < 5; v++) d.W[v * n + i] = Wi[v];
    }
    __syncthreads();
  }
  // block reductions of the Eq. 40 ratio and the divergence flag
  __shared__ double sm[32];
  __shared__ int sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    eq40 = fmax(eq40, __shfl_xor_sync(0xffffffffu, eq40, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { sm[threadIdx.x >> 5] = eq40; sb[threadIdx.x >> 5] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    int bb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a = fmax(a, sm[w]); bb |= sb[w]; }
    st.eq40 = a;
    if (bb) st.pending = -5;
  }
}

void launch_sweep_fwd(const Dev& d, int precision, int threads, cudaStream_t s) {
  if (precision == 1) k_sweep_fwd<float><<<d.n_solves, threads, 0, s>>>(d);
  else k_sweep_fwd<double><<<d.n_solves, threads, 0, s>>>(d);
}

void launch_sweep_bwd(const Dev& d, int precision, int threads, cudaStream_t s) {
  if (precision == 1) k_sweep_bwd<float><<<d.n_solves, threads, 0, s>>>(d);
  else k_sweep_bwd<double><<<d.n_solves, threads, 0, s>>>(d);
}

}  // namespace igks
