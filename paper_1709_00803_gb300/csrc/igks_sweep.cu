// igks_sweep.cu -- matrix-free LU-SGS forward and backward sweeps (Eq. 19-22 for the
// mean flow, Eq. 31-32 for the SA variable) with the FP64 state update, in FP64 or FP32.
//
// Each sweep visits the cells in the dependency order of the sequential sweep of Eq. 20
// (cell i needs its lower neighbours j < i forward, its upper neighbours j > i backward),
// grouped into levels of mutually independent cells. Everything that does not depend on
// the unknowns is formed first by a parallel pre-pass (1/D, velocities, enthalpy, the
// signed face coefficients of every cell's stencil), so the dependency chain carries only
// the neighbour contributions, one multiply by 1/D and the incremental flux of the new
// increment. On GB300 each warp-wide FP64 instruction costs the same whatever the number
// of active lanes, so the chain's FP64 instruction count sets the time of a level.
//
// Two schedules:
//  - narrow: one block per solve walks its levels with a block barrier between them (for
//    orderings with hundreds of thin levels). The increments of the last RING cells it
//    produced stay in a shared-memory ring, so a cell usually reads its neighbours'
//    increments from shared memory; its stencil (neighbour, ring slot, coefficients) is
//    stored in sweep-position order so it is fetched without an indirection;
//  - wide: one launch per level covering that level's cells of every solve (for low-depth
//    orderings, e.g. multicolour, whose few levels hold thousands of cells each).
#include <cooperative_groups.h>
#include <float.h>

#include <type_traits>

#include "igks_df64.cuh"
#include "igks_dev.h"
#include "igks_phys.cuh"

namespace cg = cooperative_groups;

namespace igks {

// The sweeps' arithmetic is written with explicitly rounded operations (fma_x, mul_x,
// add_x: __fma_rn / __dmul_rn / __dadd_rn in FP64, the __f*_rn intrinsics in FP32, the
// double-float operators): the compiler may not fuse or split them, so every schedule (one
// thread per cell, a quad of threads per cell, one launch per level) and every inlining
// context gives the same bits for the same cell.
__device__ __forceinline__ double fma_x(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double mul_x(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_x(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double div_x(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mul_x(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_x(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float div_x(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ df64 fma_x(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64 mul_x(df64 a, df64 b) { return a * b; }
__device__ __forceinline__ df64 add_x(df64 a, df64 b) { return a + b; }
__device__ __forceinline__ df64 div_x(df64 a, df64 b) { return a / b; }

// Increment of the x and y Euler fluxes for the increment (dr, dmx, dmy, dE) of a state
// with density r, momenta mx, my, velocity u, v and total enthalpy density H = E + p,
// written without differences of large numbers. o = {x mass, y mass, x x-mom, y x-mom,
// x y-mom, y y-mom, x energy, y energy}.
template <class T>
__device__ __forceinline__ void delta_flux(T r, T mx, T my, T u, T v, T H, T dr, T dmx, T dmy, T dE, T* o) {
  const T g1 = (T)(GAMMA - 1.0);
  const T inv1 = div_x((T)1, add_x(r, dr));
  const T du = mul_x(fma_x(-u, dr, dmx), inv1);          // (dmx - u dr) / (r + dr)
  const T dv = mul_x(fma_x(-v, dr, dmy), inv1);
  const T u1 = add_x(u, du), v1 = add_x(v, dv);
  const T dmxu = fma_x(dmx, u1, mul_x(mx, du));          // increment of mx u
  const T dmyv = fma_x(dmy, v1, mul_x(my, dv));          // increment of my v
  const T dp = mul_x(g1, fma_x((T)(-0.5), add_x(dmxu, dmyv), dE));
  const T dH = add_x(dE, dp);
  o[0] = dmx;
  o[1] = dmy;
  o[2] = add_x(dmxu, dp);
  o[3] = fma_x(dmx, v1, mul_x(mx, dv));
  o[4] = fma_x(dmy, u1, mul_x(my, du));
  o[5] = add_x(dmyv, dp);
  o[6] = fma_x(dH, u1, mul_x(H, du));
  o[7] = fma_x(dH, v1, mul_x(H, dv));
}

// Contribution of one stencil entry to a cell's sweep sum: (1/2) S (dF . n - lambda dW)
// for the mean flow (sx, sy = signed S n / 2, sl = S lambda / 2) and a_ij dnu for SA,
// subtracted from (forward) or added to (backward) the cell's accumulator. Every schedule
// applies the entries of a cell with these helpers in the same order, so a solve gives
// the same bits whichever schedule runs it (alone or in a batch).
// One component v of an entry: f0, f1 = the x and y flux increments of component v, w its
// increment (fwd subtracts, bwd adds); the SA row has its scalar coefficient. The
// schedules that split a cell's components over threads call these per component, so
// every schedule does the same arithmetic.
template <class T>
__device__ __forceinline__ T entry_sum(T sx, T sy, T sl, T f0, T f1, T w) {   // sx f0 + sy f1 - sl w
  return fma_x(sx, f0, fma_x(sy, f1, -mul_x(sl, w)));
}
template <class T>
__device__ __forceinline__ void fwd_comp(T& a, T sx, T sy, T sl, T f0, T f1, T w) {
  a = add_x(a, -entry_sum(sx, sy, sl, f0, f1, w));
}
template <class T>
__device__ __forceinline__ void bwd_comp(T& a, T sx, T sy, T sl, T f0, T f1, T w) {
  a = add_x(a, entry_sum(sx, sy, sl, f0, f1, w));
}
template <class T>
__device__ __forceinline__ void fwd_sa(T& a, T sa, T w) { a = fma_x(-sa, w, a); }
template <class T>
__device__ __forceinline__ void bwd_sa(T& a, T sa, T w) { a = fma_x(sa, w, a); }

// A cell's increments from its accumulators: one rounded product (forward), one fused
// multiply-add (backward). Written with explicitly rounded operations so that the compiler
// cannot fuse the product into the arithmetic that consumes the increment (the flux
// increment of the same thread): a schedule that takes the increments from other threads
// by shuffles must get the same bits.
template <class T>
__device__ __forceinline__ T inc_fwd(T acc, T c);
template <>
__device__ __forceinline__ double inc_fwd<double>(double acc, double c) { return __dmul_rn(acc, c); }
template <>
__device__ __forceinline__ float inc_fwd<float>(float acc, float c) { return __fmul_rn(acc, c); }
template <>
__device__ __forceinline__ df64 inc_fwd<df64>(df64 acc, df64 c) { return acc * c; }
template <class T>
__device__ __forceinline__ T inc_bwd(T ws, T acc, T c);   // ws - acc c
template <>
__device__ __forceinline__ double inc_bwd<double>(double ws, double acc, double c) { return __fma_rn(-acc, c, ws); }
template <>
__device__ __forceinline__ float inc_bwd<float>(float ws, float acc, float c) { return __fmaf_rn(-acc, c, ws); }
template <>
__device__ __forceinline__ df64 inc_bwd<df64>(df64 ws, df64 acc, df64 c) { return ws - acc * c; }

template <class T>
__device__ __forceinline__ void fwd_acc(T* acc, T sx, T sy, T sl, T sa, const T* f, const T* w, bool sa_on) {
#pragma unroll
  for (int v = 0; v < 4; v++) fwd_comp<T>(acc[v], sx, sy, sl, f[2 * v], f[2 * v + 1], w[v]);
  if (sa_on) fwd_sa<T>(acc[4], sa, w[4]);
}

template <class T>
__device__ __forceinline__ void bwd_acc(T* acc, T sx, T sy, T sl, T sa, const T* f, const T* w, bool sa_on) {
#pragma unroll
  for (int v = 0; v < 4; v++) bwd_comp<T>(acc[v], sx, sy, sl, f[2 * v], f[2 * v + 1], w[v]);
  if (sa_on) bwd_sa<T>(acc[4], sa, w[4]);
}

// The same two for double-float: every product is accumulated exactly into the running
// high part (two-sum), its rounding errors and the product's low part into the running low
// part, without renormalising after each term (the multiply that uses the sum does).
__device__ __forceinline__ void df_mac(df64& acc, df64 a, df64 b) {   // acc += a b
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

template <>
__device__ __forceinline__ void fwd_comp<df64>(df64& a, df64 sx, df64 sy, df64 sl, df64 f0, df64 f1, df64 w) {
  df_mac(a, -sx, f0);
  df_mac(a, -sy, f1);
  df_mac(a, sl, w);
}
template <>
__device__ __forceinline__ void bwd_comp<df64>(df64& a, df64 sx, df64 sy, df64 sl, df64 f0, df64 f1, df64 w) {
  df_mac(a, sx, f0);
  df_mac(a, sy, f1);
  df_mac(a, -sl, w);
}
template <>
__device__ __forceinline__ void fwd_sa<df64>(df64& a, df64 sa, df64 w) { df_mac(a, -sa, w); }
template <>
__device__ __forceinline__ void bwd_sa<df64>(df64& a, df64 sa, df64 w) { df_mac(a, sa, w); }

// ---- pre-pass: per-cell constants and the signed stencil of every cell ----
template <class T>
__global__ void __launch_bounds__(CELL_BLOCK) k_sweep_prep(Dev d) {
  const int i = (d.g_blk0 + blockIdx.x) * CELL_BLOCK + threadIdx.x;
  if (i >= d.nc_pad) return;
  const int s = d.cell_solve[i];
  if (s < 0 || d.st[s].state != 0 || d.flow[s].scheme == 1) return;   // explicit solves: no sweeps
  const DevFlow& fl = d.flow[s];
  const int n = d.nc_pad, nf = d.nf;
  const double cfl = d.st[s].cfl;
  const double Lam = d.Lam[i];
  const double r = d.W[i], mx = d.W[n + i], my = d.W[2 * n + i], E = d.W[3 * n + i];
  const double u = d.pu[i], v = d.pv[i];          // mx / r, my / r (k_prep)
  const double p = (GAMMA - 1.0) * (E - 0.5 * (mx * u + my * v));
  T cc[5];
  const double lc = Lam * __drcp_rn(cfl);                                 // Omega / dt_imp (Eq. 24)
  cc[0] = (T)__drcp_rn(lc + Lam);                                        // 1/D (Eq. 20)
  cc[1] = fl.sa_on ? (T)__drcp_rn(lc + d.sa_diag[i]) : (T)0;             // 1/a_ii (Eq. 32)
  cc[2] = (T)u;
  cc[3] = (T)v;
  cc[4] = (T)(E + p);
  const bool wide = d.wide != 0;
  if (wide) {   // the one-launch-per-level sweeps read the cell constants in cell order
    T* c = (T*)d.sw_cell;
#pragma unroll
    for (int q = 0; q < 5; q++) c[q * n + i] = cc[q];
  }
  // position-ordered records of the narrow schedule
  const int P = d.npos, pf = d.pos_f[i], pb = d.pos_b[i];
  const bool csr_f = d.cnt_f[pf] < 0, csr_b = d.cnt_b[pb] < 0;   // more entries than a record holds
  if (!wide) {
    T* rf = (T*)d.rec_f;
    T* rb = (T*)d.rec_b;
#pragma unroll
    for (int q = 0; q < 5; q++) rf[q * P + pf] = (T)d.M[q * n + i];
    rf[5 * P + pf] = (T)r; rf[6 * P + pf] = (T)mx; rf[7 * P + pf] = (T)my;
#pragma unroll
    for (int q = 0; q < 5; q++) { rf[(8 + q) * P + pf] = cc[q]; rb[(5 + q) * P + pb] = cc[q]; }
#pragma unroll
    for (int q = 0; q < 5; q++) rb[q * P + pb] = (T)d.W[q * n + i];
  }
  T* sc = (T*)d.sw_st;
  const int nnz = d.nnz;
  for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
    const int f = d.cf_face[k];
    const bool own = (d.fL[f] == i);
    const int j = own ? d.fR[f] : d.fL[f];
    const double hS = 0.5 * d.fS[f];
    const double sg = own ? hS : -hS;
    const T e0 = (T)(sg * d.fnx[f]), e1 = (T)(sg * d.fny[f]), e2 = (T)(hS * d.lam_f[f]);
    const T e3 = (T)d.sa_a[(own ? 0 : 1) * nf + f];
    if (wide) {   // the cell-ordered stencil of the one-launch-per-level sweeps
      d.sw_j[k] = j;                                  // -1 on a boundary face
      sc[k] = e0; sc[nnz + k] = e1; sc[2 * nnz + k] = e2; sc[3 * nnz + k] = e3;
    } else {
      // the narrow schedule: up to PF_E entries per position in its record, the rest of a
      // larger stencil in the position-ordered CSR lists
      const int ef = d.cf_to_fs[k], eb = d.cf_to_bs[k];
      if (ef >= 0 && csr_f) {
        T* o = (T*)d.sc_f;
        o[ef] = e0; o[d.nfs + ef] = e1; o[2 * d.nfs + ef] = e2; o[3 * d.nfs + ef] = e3;
      }
      if (eb >= 0 && csr_b) {
        T* o = (T*)d.sc_b;
        o[eb] = e0; o[d.nbs + eb] = e1; o[2 * d.nbs + eb] = e2; o[3 * d.nbs + eb] = e3;
      }
      const size_t PE = (size_t)PF_E * d.npos;
      const int xf = d.cf_to_ef[k], xb = d.cf_to_eb[k];
      if (xf >= 0) {
        T* o = (T*)d.ec_f;
        o[xf] = e0; o[PE + xf] = e1; o[2 * PE + xf] = e2; o[3 * PE + xf] = e3;
      }
      if (xb >= 0) {
        T* o = (T*)d.ec_b;
        o[xb] = e0; o[PE + xb] = e1; o[2 * PE + xb] = e2; o[3 * PE + xb] = e3;
      }
    }
    // the ghost state of a wall or symmetry face in the form the backward sweep's flux
    // increment takes it (its only ghost entries), so the sweep itself does no FP64 work
    const int bc = d.fbc[f];
    if (j < 0 && (bc == 2 || bc == 3 || bc == 5)) {
      const double gr = d.G[f], gmx = d.G[nf + f], gmy = d.G[2 * nf + f], gE = d.G[3 * nf + f];
      const double gu = gmx / gr, gv = gmy / gr;
      const double gp = (GAMMA - 1.0) * (gE - 0.5 * (gmx * gu + gmy * gv));
      T* g = (T*)d.gprim;
      g[f] = (T)gr; g[nf + f] = (T)gmx; g[2 * nf + f] = (T)gmy;
      g[3 * nf + f] = (T)gu; g[4 * nf + f] = (T)gv; g[5 * nf + f] = (T)(gE + gp);
    }
  }
}

// ---- one cell of the forward sweep (wide schedule, stencil in cell-face order) ----
template <class T>
__device__ __forceinline__ void fwd_cell(const Dev& d, int i, bool sa_on) {
  const int n = d.nc_pad, nnz = d.nnz;
  T* dWs = (T*)d.dWs;
  T* dF = (T*)d.dF;
  const T* c = (const T*)d.sw_cell;
  const T* sc = (const T*)d.sw_st;
  T acc[5];
#pragma unroll
  for (int v = 0; v < 5; v++) acc[v] = (T)d.M[v * n + i];
  for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
    const int j = d.sw_j[k];
    if (j < 0 || j >= i) continue;                   // ghost increments are zero forward
    T f[8], w[5];
#pragma unroll
    for (int q = 0; q < 8; q++) f[q] = dF[q * n + j];
#pragma unroll
    for (int v = 0; v < 5; v++) w[v] = dWs[v * n + j];
    fwd_acc<T>(acc, sc[k], sc[nnz + k], sc[2 * nnz + k], sc[3 * nnz + k], f, w, sa_on);
  }
  T dw[5];
#pragma unroll
  for (int v = 0; v < 4; v++) dw[v] = inc_fwd<T>(acc[v], c[i]);
  dw[4] = sa_on ? inc_fwd<T>(acc[4], c[n + i]) : (T)0;
#pragma unroll
  for (int v = 0; v < 5; v++) dWs[v * n + i] = dw[v];
  T o[8];
  delta_flux<T>((T)d.W[i], (T)d.W[n + i], (T)d.W[2 * n + i], c[2 * n + i], c[3 * n + i], c[4 * n + i],
                dw[0], dw[1], dw[2], dw[3], o);
#pragma unroll
  for (int q = 0; q < 8; q++) dF[q * n + i] = o[q];
}

__device__ __forceinline__ void flush_eq40(const Dev& d, int s, double eq40, int bad);

template <class T, int C>
__device__ __forceinline__ void bwd_entry(const Dev& d, const T* ring, const T* dF, const T* dWo, int j, int slot,
                                          const T* ws, T sx, T sy, T sl, T sa, bool sa_on, T* acc);

// ---- one cell of the backward sweep (wide schedule, stencil in cell-face order) ----
template <class T>
__device__ __forceinline__ void bwd_cell(const Dev& d, int i, bool sa_on) {
  const int n = d.nc_pad, nnz = d.nnz;
  const T* dWs = (const T*)d.dWs;
  T* dWo = (T*)d.dW;
  T* dF = (T*)d.dF;
  const T* c = (const T*)d.sw_cell;
  const T* sc = (const T*)d.sw_st;
  T ws[5];
#pragma unroll
  for (int v = 0; v < 5; v++) ws[v] = dWs[v * n + i];
  T acc[5] = {0, 0, 0, 0, 0};
  for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
    int j = d.sw_j[k];
    if (j >= 0) {
      if (j <= i) continue;
    } else {
      const int f = d.cf_face[k];
      if (d.fbc[f] == 1 || d.fbc[f] == 4) continue;  // free-stream and outflow increments are zero
      j = -1 - f;
    }
    bwd_entry<T, 1>(d, nullptr, dF, dWo, j, -1, ws, sc[k], sc[nnz + k], sc[2 * nnz + k], sc[3 * nnz + k], sa_on, acc);
  }
  T dw[5];
#pragma unroll
  for (int v = 0; v < 4; v++) { dw[v] = inc_bwd<T>(ws[v], acc[v], c[i]); dWo[v * n + i] = dw[v]; }
  dw[4] = sa_on ? inc_bwd<T>(ws[4], acc[4], c[n + i]) : (T)0;
  dWo[4 * n + i] = dw[4];
  T o[8];
  delta_flux<T>((T)d.W[i], (T)d.W[n + i], (T)d.W[2 * n + i], c[2 * n + i], c[3 * n + i], c[4 * n + i],
                dw[0], dw[1], dw[2], dw[3], o);
#pragma unroll
  for (int q = 0; q < 8; q++) dF[q * n + i] = o[q];
}

// ---- state update W += dW (FP64), nu_tilde floor, Eq. 40 ratio, divergence check ----
// Runs after the backward sweep over all cells at once: it is off the sweeps' dependency
// chain, and its FP64 square roots and division are spread over the whole GPU.
template <class T>
__global__ void __launch_bounds__(CELL_BLOCK) k_update(Dev d) {
  const int blk = d.g_blk0 + blockIdx.x;
  const int i = blk * CELL_BLOCK + threadIdx.x;
  const int s = d.cell_solve[blk * CELL_BLOCK];   // every block lies in one solve
  double eq40 = 0.0;
  int bad = 0;
  const bool live = (i < d.nc_pad) && d.cell_solve[i] >= 0 && d.st[d.cell_solve[i]].state == 0;
  if (live) {
    const int n = d.nc_pad;
    const T* dWo = (const T*)d.dW;
    double Wi[5];
#pragma unroll
    for (int v = 0; v < 5; v++) Wi[v] = d.W[v * n + i];
    const int si = d.cell_solve[i];
    const bool expl = d.flow[si].scheme == 1;
    // explicit scheme (Eq. 15 as Eq. 16): dW = dt M / Omega, in FP64
    const double xf = expl ? __longlong_as_double((long long)d.dt_bits[si]) / d.area[i] : 0.0;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const double dv = expl ? xf * d.M[v * n + i] : to_double(dWo[v * n + i]);
      num += dv * dv;
      den += Wi[v] * Wi[v];
      Wi[v] += dv;
    }
    Wi[4] += expl ? (d.flow[si].sa_on ? xf * d.M[4 * n + i] : 0.0) : to_double(dWo[4 * n + i]);
    if (Wi[4] < 0.0) Wi[4] = 0.0;
    eq40 = sqrt(num) / sqrt(den);
    const double p = pressure_of(Wi[0], Wi[1], Wi[2], Wi[3]);
    if (!(Wi[0] > 0.0) || !(p > 0.0) || !isfinite(Wi[3]) || !isfinite(Wi[4])) bad = 1;
#pragma unroll
    for (int v = 0; v < 5; v++) d.W[v * n + i] = Wi[v];
  }
  flush_eq40(d, (s >= 0 && d.st[s].state == 0) ? s : -1, eq40, bad);
}

// block-wide max of the Eq. 40 ratio and OR of the divergence flag, one atomic each;
// positive doubles order like their bit patterns, so the per-solve maximum is exact
__device__ __forceinline__ void flush_eq40(const Dev& d, int s, double eq40, int bad) {
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
    int b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a = fmax(a, sm[w]); b |= sb[w]; }
    if (s >= 0) {
      if (a > 0.0) atomicMax(d.eq40_bits + s, (unsigned long long)__double_as_longlong(a));
      if (b) atomicOr(d.bad + s, 1);
    }
  }
}

// ---- narrow schedule: one block per solve, shared-memory ring of recent increments ----
// ring layout: [13][RING] of T: the 8 flux increments, then the 5 variable increments of
// the cell at sweep position p (local to the solve), stored at slot p % RING.
//
// Per-position records (written by the pre-pass, position-major SoA so one level's
// records are contiguous) are prefetched into registers one level ahead: the block
// issues the loads of level l+1 before it works on level l, so by the time level l+1
// starts only the neighbours' increments (shared-memory ring) sit on the dependency chain.
template <class T>
__device__ __forceinline__ void ring_put(T* ring, int slot, const T* o, const T* dw) {
#pragma unroll
  for (int q = 0; q < 8; q++) ring[q * RING + slot] = o[q];
#pragma unroll
  for (int v = 0; v < 5; v++) ring[(8 + v) * RING + slot] = dw[v];
}

// With a cluster of C blocks per solve (C > 1), position q of the solve belongs to block
// q % C and its increments sit in that block's ring, read through distributed shared
// memory; RING is a multiple of C, so the slot q % RING names the owner too.
template <class T, int C>
__device__ __forceinline__ const T* ring_of(const T* ring, int slot) {
  if constexpr (C == 1) {
    return ring;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned owner = (unsigned)(slot & (C - 1));
    return owner == cl.block_rank() ? ring : cl.map_shared_rank(ring, owner);
  }
}

template <class T, int C = 1>
__device__ __forceinline__ void neighbour(const Dev& d, const T* ring, const T* dF, const T* dWv, int j, int slot,
                                          T* f, T* w) {
  const int n = d.nc_pad;
  if (slot >= 0) {
    const T* rb = ring_of<T, C>(ring, slot);
#pragma unroll
    for (int k = 0; k < 8; k++) f[k] = rb[k * RING + slot];
#pragma unroll
    for (int v = 0; v < 5; v++) w[v] = rb[(8 + v) * RING + slot];
  } else {
#pragma unroll
    for (int k = 0; k < 8; k++) f[k] = dF[k * n + j];
#pragma unroll
    for (int v = 0; v < 5; v++) w[v] = dWv[v * n + j];
  }
}

// Each cell of a level is handled by one thread. Its record (per-iteration data and up
// to PF_E stencil entries) is staged into shared memory by cp.async one level ahead.

// asynchronous global -> shared copies (cp.async, 4 or 8 bytes): the copy proceeds in the
// background and never holds registers, so the next level's records are in flight while
// the current level is computed
template <class U>
__device__ __forceinline__ void cpa(U* dst_smem, const U* src) {
  static_assert(sizeof(U) == 4 || sizeof(U) == 8, "cp.async element size");
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
  if (sizeof(U) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// forward record of one position: residual, state (r, mx, my), 1/D, 1/a_ii, u, v, H, cell,
// entry count, backward position, and PF_E stencil entries
template <class T>
struct FwdRec {
  T m[5], w[3], c[5];
  T co[4][PF_E];
  int i, cnt, pb, pad;
  int j[PF_E], slot[PF_E];
};

template <class T>
__device__ __forceinline__ void fwd_stage(const Dev& d, int p, FwdRec<T>* st) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_f;
  const T* ec = (const T*)d.ec_f;
#pragma unroll
  for (int v = 0; v < 5; v++) cpa(&st->m[v], rec + v * P + p);
#pragma unroll
  for (int v = 0; v < 3; v++) cpa(&st->w[v], rec + (5 + v) * P + p);
#pragma unroll
  for (int v = 0; v < 5; v++) cpa(&st->c[v], rec + (8 + v) * P + p);
  cpa(&st->i, d.fwd_order + p);
  cpa(&st->cnt, d.cnt_f + p);
  cpa(&st->pb, d.pb_of_pf + p);
#pragma unroll
  for (int e = 0; e < PF_E; e++) {
    cpa(&st->j[e], d.ej_f + e * P + p);
    cpa(&st->slot[e], d.eslot_f + e * P + p);
#pragma unroll
    for (int k = 0; k < 4; k++) cpa(&st->co[k][e], ec + (k * PF_E + e) * P + p);
  }
  cpa_commit();
}

template <class T>
__device__ __forceinline__ void fwd_load_direct(const Dev& d, int p, FwdRec<T>* st) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_f;
  const T* ec = (const T*)d.ec_f;
#pragma unroll
  for (int v = 0; v < 5; v++) st->m[v] = rec[v * P + p];
#pragma unroll
  for (int v = 0; v < 3; v++) st->w[v] = rec[(5 + v) * P + p];
#pragma unroll
  for (int v = 0; v < 5; v++) st->c[v] = rec[(8 + v) * P + p];
  st->i = d.fwd_order[p];
  st->cnt = d.cnt_f[p];
  st->pb = d.pb_of_pf[p];
#pragma unroll
  for (int e = 0; e < PF_E; e++) {
    st->j[e] = d.ej_f[e * P + p];
    st->slot[e] = d.eslot_f[e * P + p];
#pragma unroll
    for (int k = 0; k < 4; k++) st->co[k][e] = ec[(k * PF_E + e) * P + p];
  }
}

template <class T, int C = 1>
__device__ __forceinline__ void fwd_process(const Dev& d, T* ring, int p, int pbase, const FwdRec<T>* r, bool sa_on) {
  const int n = d.nc_pad, P = d.npos;
  T* dWs = (T*)d.dWs;
  T* dF = (T*)d.dF;
  T acc[5];
#pragma unroll
  for (int v = 0; v < 5; v++) acc[v] = r->m[v];
  const int cnt = r->cnt;
  if (cnt >= 0) {
#pragma unroll
    for (int e = 0; e < PF_E; e++) {
      if (e >= cnt) break;
      T f[8], w[5];
      neighbour<T, C>(d, ring, dF, dWs, r->j[e], r->slot[e], f, w);
      fwd_acc<T>(acc, r->co[0][e], r->co[1][e], r->co[2][e], r->co[3][e], f, w, sa_on);
    }
  } else {
    // more entries than the record holds: the position-ordered CSR stencil
    const T* sc = (const T*)d.sc_f;
    const int nfs = d.nfs;
    for (int k = d.fs_ptr[p]; k < d.fs_ptr[p + 1]; k++) {
      T f[8], w[5];
      neighbour<T, C>(d, ring, dF, dWs, d.fs_j[k], d.fs_slot[k], f, w);
      fwd_acc<T>(acc, sc[k], sc[nfs + k], sc[2 * nfs + k], sc[3 * nfs + k], f, w, sa_on);
    }
  }
  T dw[5];
#pragma unroll
  for (int v = 0; v < 4; v++) dw[v] = inc_fwd<T>(acc[v], r->c[0]);
  dw[4] = sa_on ? inc_fwd<T>(acc[4], r->c[1]) : (T)0;
  T o[8];
  delta_flux<T>(r->w[0], r->w[1], r->w[2], r->c[2], r->c[3], r->c[4], dw[0], dw[1], dw[2], dw[3], o);
  const int slot = (p - pbase) % RING;
  ring_put<T>(ring, slot, o, dw);
  const int i = r->i, pb = r->pb;
  T* recb = (T*)d.rec_b;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    dWs[v * n + i] = dw[v];
    recb[(10 + v) * P + pb] = dw[v];          // the backward sweep's copy of dW*
  }
#pragma unroll
  for (int k = 0; k < 8; k++) dF[k * n + i] = o[k];
}

// the first position at or after b that belongs to cluster block r (positions q = p - pbase
// are dealt round the C blocks: q % C == r)
template <int C>
__device__ __forceinline__ int first_own(int b, int pbase, int r) {
  if constexpr (C == 1) return b;
  return b + (((r - (b - pbase)) % C) + C) % C;
}

template <int C>
__device__ __forceinline__ void level_barrier() {
  if constexpr (C == 1) __syncthreads();
  else cg::this_cluster().sync();   // release/acquire over the cluster's shared and global writes
}

template <class T, int C>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_fwd_narrow(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  FwdRec<T>* stage = (FwdRec<T>*)(smem_raw + (size_t)13 * RING * sizeof(T));
  FwdRec<T>* st = stage + threadIdx.x;               // staged record of this thread's next position
  const int s = d.g_solve0 + blockIdx.x / C, r = blockIdx.x % C;  // one cluster of C blocks per solve
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;   // uniform over the cluster
  if constexpr (C > 1) cg::this_cluster().sync();    // every block runs before any remote read
  const bool sa_on = d.flow[s].sa_on;
  const int l0 = d.lvl_solve_ptr[s], l1 = d.lvl_solve_ptr[s + 1] - 1;
  const int pbase = d.fwd_lvl[l0];
  const int step = C * (int)blockDim.x;
  // level bounds travel in registers: level l spans [b, e), the next one [e, en)
  int b = d.fwd_lvl[l0], e = d.fwd_lvl[l0 + 1];
  int pm = first_own<C>(b, pbase, r) + C * (int)threadIdx.x;    // this thread's position of the level
  if (l0 < l1 && pm < e) fwd_stage<T>(d, pm, st);
  for (int l = l0; l < l1; l++) {
    const int en = (l + 1 < l1) ? d.fwd_lvl[l + 2] : e;
    const bool mine = pm < e;
    FwdRec<T> cur;
    if (mine) {
      cpa_wait_all();
      cur = *st;                 // this level's record into registers, freeing the stage
    }
    // the next level's record is in flight while this level is computed
    const int pn = first_own<C>(e, pbase, r) + C * (int)threadIdx.x;
    if (pn < en) fwd_stage<T>(d, pn, st);
    if (mine) fwd_process<T, C>(d, ring, pm, pbase, &cur, sa_on);
    for (int p = pm + step; p < e; p += step) {   // levels wider than the cluster's threads
      FwdRec<T> xt;
      fwd_load_direct<T>(d, p, &xt);
      fwd_process<T, C>(d, ring, p, pbase, &xt, sa_on);
    }
    level_barrier<C>();
    b = e;
    e = en;
    pm = pn;
  }
}

// backward record: state (5), 1/D, 1/a_ii, u, v, H, the forward increment dW* (5), cell,
// entry count and PF_E entries (upper neighbours, wall/symmetry ghosts)
template <class T>
struct BwdRec {
  T w[5], c[5], ws[5];
  T co[4][PF_E];
  int i, cnt;
  int j[PF_E], slot[PF_E];
};

template <class T>
__device__ __forceinline__ void bwd_stage(const Dev& d, int p, BwdRec<T>* st) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_b;
  const T* ec = (const T*)d.ec_b;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    cpa(&st->w[v], rec + v * P + p);
    cpa(&st->c[v], rec + (5 + v) * P + p);
    cpa(&st->ws[v], rec + (10 + v) * P + p);
  }
  cpa(&st->i, d.bwd_order + p);
  cpa(&st->cnt, d.cnt_b + p);
#pragma unroll
  for (int e = 0; e < PF_E; e++) {
    cpa(&st->j[e], d.ej_b + e * P + p);
    cpa(&st->slot[e], d.eslot_b + e * P + p);
#pragma unroll
    for (int k = 0; k < 4; k++) cpa(&st->co[k][e], ec + (k * PF_E + e) * P + p);
  }
  cpa_commit();
}

template <class T>
__device__ __forceinline__ void bwd_load_direct(const Dev& d, int p, BwdRec<T>* st) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_b;
  const T* ec = (const T*)d.ec_b;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    st->w[v] = rec[v * P + p];
    st->c[v] = rec[(5 + v) * P + p];
    st->ws[v] = rec[(10 + v) * P + p];
  }
  st->i = d.bwd_order[p];
  st->cnt = d.cnt_b[p];
#pragma unroll
  for (int e = 0; e < PF_E; e++) {
    st->j[e] = d.ej_b[e * P + p];
    st->slot[e] = d.eslot_b[e * P + p];
#pragma unroll
    for (int k = 0; k < 4; k++) st->co[k][e] = ec[(k * PF_E + e) * P + p];
  }
}

// contribution of one backward entry: upper neighbour j (its increments from the ring or
// global memory), or a wall/symmetry ghost (j = -1 - face: boundary map of this cell's
// own forward increment ws, flux increment about the ghost state)
// the increments of a wall / symmetry ghost (face fc) in the backward sweep: the boundary
// map of the cell's own forward increment ws, and the flux increment about the ghost state
template <class T>
__device__ __forceinline__ T mn_x(T a, T fx, T b, T fy) { return fma_x(a, fx, mul_x(b, fy)); }

template <class T>
__device__ __forceinline__ void ghost_entry(const Dev& d, int fc, const T* ws, T* f, T* w) {
  const int nf = d.nf;
  w[0] = ws[0]; w[3] = ws[3];
  if (d.fbc[fc] == 3 || d.fbc[fc] == 5) { w[1] = -ws[1]; w[2] = -ws[2]; w[4] = -ws[4]; }
  else {
    const T fx = (T)d.fnx[fc], fy = (T)d.fny[fc];
    const T mn = mn_x(ws[1], fx, ws[2], fy);
    const T mn2 = add_x(mn, mn);                                      // 2 (dm . n), exact
    w[1] = fma_x(-mn2, fx, ws[1]); w[2] = fma_x(-mn2, fy, ws[2]); w[4] = ws[4];
  }
  const T* g = (const T*)d.gprim;   // ghost r, mx, my, u, v, H of this face (pre-pass)
  delta_flux<T>(g[fc], g[nf + fc], g[2 * nf + fc], g[3 * nf + fc], g[4 * nf + fc], g[5 * nf + fc],
                w[0], w[1], w[2], w[3], f);
}

template <class T, int C>
__device__ __forceinline__ void bwd_entry(const Dev& d, const T* ring, const T* dF, const T* dWo, int j, int slot,
                                          const T* ws, T sx, T sy, T sl, T sa, bool sa_on, T* acc) {
  T f[8], w[5];
  if (j >= 0) neighbour<T, C>(d, ring, dF, dWo, j, slot, f, w);
  else ghost_entry<T>(d, -1 - j, ws, f, w);
  bwd_acc<T>(acc, sx, sy, sl, sa, f, w, sa_on);
}

template <class T, int C = 1>
__device__ __forceinline__ void bwd_process(const Dev& d, T* ring, int p, int pbase, const BwdRec<T>* r, bool sa_on) {
  const int n = d.nc_pad;
  T* dWo = (T*)d.dW;
  T* dF = (T*)d.dF;
  T ws[5];
#pragma unroll
  for (int v = 0; v < 5; v++) ws[v] = r->ws[v];
  T acc[5] = {0, 0, 0, 0, 0};
  const int cnt = r->cnt;
  if (cnt >= 0) {
#pragma unroll
    for (int e = 0; e < PF_E; e++) {
      if (e >= cnt) break;
      bwd_entry<T, C>(d, ring, dF, dWo, r->j[e], r->slot[e], ws, r->co[0][e], r->co[1][e], r->co[2][e],
                      r->co[3][e], sa_on, acc);
    }
  } else {
    const T* sc = (const T*)d.sc_b;
    const int nbs = d.nbs;
    for (int k = d.bs_ptr[p]; k < d.bs_ptr[p + 1]; k++)
      bwd_entry<T, C>(d, ring, dF, dWo, d.bs_j[k], d.bs_slot[k], ws, sc[k], sc[nbs + k], sc[2 * nbs + k],
                      sc[3 * nbs + k], sa_on, acc);
  }
  T dw[5];
#pragma unroll
  for (int v = 0; v < 4; v++) dw[v] = inc_bwd<T>(ws[v], acc[v], r->c[0]);
  dw[4] = sa_on ? inc_bwd<T>(ws[4], acc[4], r->c[1]) : (T)0;
  T o[8];
  delta_flux<T>(r->w[0], r->w[1], r->w[2], r->c[2], r->c[3], r->c[4], dw[0], dw[1], dw[2], dw[3], o);
  ring_put<T>(ring, (p - pbase) % RING, o, dw);
  const int i = r->i;
#pragma unroll
  for (int v = 0; v < 5; v++) dWo[v * n + i] = dw[v];
#pragma unroll
  for (int k = 0; k < 8; k++) dF[k * n + i] = o[k];
}

template <class T, int C>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_bwd_narrow(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  BwdRec<T>* stage = (BwdRec<T>*)(smem_raw + (size_t)13 * RING * sizeof(T));
  BwdRec<T>* st = stage + threadIdx.x;
  const int s = d.g_solve0 + blockIdx.x / C, r = blockIdx.x % C;
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  if constexpr (C > 1) cg::this_cluster().sync();
  const bool sa_on = d.flow[s].sa_on;
  const int l0 = d.blvl_solve_ptr[s], l1 = d.blvl_solve_ptr[s + 1] - 1;
  const int pbase = d.bwd_lvl[l0];
  const int step = C * (int)blockDim.x;
  int b = d.bwd_lvl[l0], e = d.bwd_lvl[l0 + 1];
  int pm = first_own<C>(b, pbase, r) + C * (int)threadIdx.x;
  if (l0 < l1 && pm < e) bwd_stage<T>(d, pm, st);
  for (int l = l0; l < l1; l++) {
    const int en = (l + 1 < l1) ? d.bwd_lvl[l + 2] : e;
    const bool mine = pm < e;
    BwdRec<T> cur;
    if (mine) {
      cpa_wait_all();
      cur = *st;
    }
    const int pn = first_own<C>(e, pbase, r) + C * (int)threadIdx.x;
    if (pn < en) bwd_stage<T>(d, pn, st);
    if (mine) bwd_process<T, C>(d, ring, pm, pbase, &cur, sa_on);
    for (int p = pm + step; p < e; p += step) {
      BwdRec<T> xt;
      bwd_load_direct<T>(d, p, &xt);
      bwd_process<T, C>(d, ring, p, pbase, &xt, sa_on);
    }
    level_barrier<C>();
    b = e;
    e = en;
    pm = pn;
  }
}


// ---- narrow schedule with a quad of threads per cell (FP32 and double-float sweeps) ----
// The four threads of a quad share one cell: thread q accumulates component q (and q = 0
// the SA row too) over the cell's entries, reading only its own component's three values
// per neighbour from the ring; the quad then exchanges the four increments by shuffles and
// each thread forms the flux increment (all eight values, the same function as one thread
// per cell) and keeps its component's two. The arithmetic of every component is the
// per-component helpers' in the same entry order, so the iterates are bitwise those of one
// thread per cell. It shortens the dependent chain of a cell about fourfold where a level
// holds few cells; it does not pay for FP64, whose cost is the SM's count of FP64 warp
// instructions (one per ~19 cycles whatever the active lanes), so FP64 keeps one thread
// per cell.
constexpr int QUAD = 4;

template <class T>
__device__ __forceinline__ T shfl_q(T x, int k) { return __shfl_sync(0xffffffffu, x, k, QUAD); }
template <>
__device__ __forceinline__ df64 shfl_q<df64>(df64 x, int k) {
  return df64(__shfl_sync(0xffffffffu, x.hi, k, QUAD), __shfl_sync(0xffffffffu, x.lo, k, QUAD));
}

// the quad's lanes share the copies of one staged forward record
template <class T>
__device__ __forceinline__ void fwd_stage_q(const Dev& d, int p, FwdRec<T>* st, int q) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_f;
  const T* ec = (const T*)d.ec_f;
  if (q == 0) {
#pragma unroll
    for (int v = 0; v < 5; v++) cpa(&st->m[v], rec + v * P + p);
    cpa(&st->i, d.fwd_order + p);
    cpa(&st->cnt, d.cnt_f + p);
    cpa(&st->pb, d.pb_of_pf + p);
  } else if (q == 1) {
#pragma unroll
    for (int v = 0; v < 3; v++) cpa(&st->w[v], rec + (5 + v) * P + p);
#pragma unroll
    for (int v = 0; v < 5; v++) cpa(&st->c[v], rec + (8 + v) * P + p);
  } else if (q == 2) {
#pragma unroll
    for (int e = 0; e < PF_E; e++) {
      cpa(&st->j[e], d.ej_f + e * P + p);
      cpa(&st->slot[e], d.eslot_f + e * P + p);
      cpa(&st->co[0][e], ec + e * P + p);
    }
  } else {
#pragma unroll
    for (int k = 1; k < 4; k++)
#pragma unroll
      for (int e = 0; e < PF_E; e++) cpa(&st->co[k][e], ec + (k * PF_E + e) * P + p);
  }
  cpa_commit();
}

template <class T>
__device__ __forceinline__ void bwd_stage_q(const Dev& d, int p, BwdRec<T>* st, int q) {
  const int P = d.npos;
  const T* rec = (const T*)d.rec_b;
  const T* ec = (const T*)d.ec_b;
  if (q == 0) {
#pragma unroll
    for (int v = 0; v < 5; v++) cpa(&st->ws[v], rec + (10 + v) * P + p);
    cpa(&st->i, d.bwd_order + p);
    cpa(&st->cnt, d.cnt_b + p);
  } else if (q == 1) {
#pragma unroll
    for (int v = 0; v < 5; v++) {
      cpa(&st->w[v], rec + v * P + p);
      cpa(&st->c[v], rec + (5 + v) * P + p);
    }
  } else if (q == 2) {
#pragma unroll
    for (int e = 0; e < PF_E; e++) {
      cpa(&st->j[e], d.ej_b + e * P + p);
      cpa(&st->slot[e], d.eslot_b + e * P + p);
      cpa(&st->co[0][e], ec + e * P + p);
    }
  } else {
#pragma unroll
    for (int k = 1; k < 4; k++)
#pragma unroll
      for (int e = 0; e < PF_E; e++) cpa(&st->co[k][e], ec + (k * PF_E + e) * P + p);
  }
  cpa_commit();
}

// component q of a neighbour's increments: x and y flux increments and the increment (and
// for q = 0 the SA increment w4)
template <class T>
__device__ __forceinline__ void neighbour_q(const Dev& d, const T* ring, const T* dF, const T* dWv, int j, int slot,
                                            int q, T& f0, T& f1, T& w, T& w4) {
  const int n = d.nc_pad;
  if (slot >= 0) {
    f0 = ring[(2 * q) * RING + slot];
    f1 = ring[(2 * q + 1) * RING + slot];
    w = ring[(8 + q) * RING + slot];
    if (q == 0) w4 = ring[12 * RING + slot];
  } else {
    f0 = dF[(2 * q) * n + j];
    f1 = dF[(2 * q + 1) * n + j];
    w = dWv[q * n + j];
    if (q == 0) w4 = dWv[4 * n + j];
  }
}

template <class T>
__device__ __forceinline__ T pick(const T* a, int q) {   // a[q] without local-memory indexing
  return q == 0 ? a[0] : (q == 1 ? a[1] : (q == 2 ? a[2] : a[3]));
}

// one forward position processed by a quad; live = the quad holds a position this round
template <class T>
__device__ __forceinline__ void fwd_quad(const Dev& d, T* ring, int p, int pbase, const FwdRec<T>& r, int q,
                                         bool live, bool sa_on) {
  const int n = d.nc_pad, P = d.npos;
  T* dWs = (T*)d.dWs;
  T* dF = (T*)d.dF;
  T acc = (T)0, acc4 = (T)0;
  if (live) {
    acc = pick(r.m, q);
    acc4 = r.m[4];
    const int cnt = r.cnt;
    if (cnt >= 0) {
#pragma unroll
      for (int e = 0; e < PF_E; e++) {
        if (e >= cnt) break;
        T f0, f1, w, w4;
        neighbour_q<T>(d, ring, dF, dWs, r.j[e], r.slot[e], q, f0, f1, w, w4);
        fwd_comp<T>(acc, r.co[0][e], r.co[1][e], r.co[2][e], f0, f1, w);
        if (q == 0 && sa_on) fwd_sa<T>(acc4, r.co[3][e], w4);
      }
    } else {
      const T* sc = (const T*)d.sc_f;
      const int nfs = d.nfs;
      for (int k = d.fs_ptr[p]; k < d.fs_ptr[p + 1]; k++) {
        T f0, f1, w, w4;
        neighbour_q<T>(d, ring, dF, dWs, d.fs_j[k], d.fs_slot[k], q, f0, f1, w, w4);
        fwd_comp<T>(acc, sc[k], sc[nfs + k], sc[2 * nfs + k], f0, f1, w);
        if (q == 0 && sa_on) fwd_sa<T>(acc4, sc[3 * nfs + k], w4);
      }
    }
  }
  const T dwq = inc_fwd<T>(acc, r.c[0]);
  const T dw4 = sa_on ? inc_fwd<T>(acc4, r.c[1]) : (T)0;
  T dw[4];
#pragma unroll
  for (int k = 0; k < 4; k++) dw[k] = shfl_q<T>(dwq, k);   // every lane of the warp takes part
  if (!live) return;
  T o[8];
  delta_flux<T>(r.w[0], r.w[1], r.w[2], r.c[2], r.c[3], r.c[4], dw[0], dw[1], dw[2], dw[3], o);
  const T o0 = q == 0 ? o[0] : (q == 1 ? o[2] : (q == 2 ? o[4] : o[6]));
  const T o1 = q == 0 ? o[1] : (q == 1 ? o[3] : (q == 2 ? o[5] : o[7]));
  const int slot = (p - pbase) % RING;
  ring[(2 * q) * RING + slot] = o0;
  ring[(2 * q + 1) * RING + slot] = o1;
  ring[(8 + q) * RING + slot] = dwq;
  const int i = r.i, pb = r.pb;
  T* recb = (T*)d.rec_b;
  dWs[q * n + i] = dwq;
  recb[(10 + q) * P + pb] = dwq;            // the backward sweep's copy of dW*
  dF[(2 * q) * n + i] = o0;
  dF[(2 * q + 1) * n + i] = o1;
  if (q == 0) {
    ring[12 * RING + slot] = dw4;
    dWs[4 * n + i] = dw4;
    recb[14 * P + pb] = dw4;
  }
}

// component q of one backward entry: an upper neighbour's increments, or a wall / symmetry
// ghost's (the ghost is formed whole, as with one thread per cell, and component q taken)
template <class T>
__device__ __forceinline__ void bwd_entry_q(const Dev& d, const T* ring, const T* dF, const T* dWo, int j, int slot,
                                            const T* ws, T sx, T sy, T sl, T sa, int q, bool sa_on, T& acc, T& acc4) {
  T f0, f1, w, w4;
  if (j >= 0) {
    neighbour_q<T>(d, ring, dF, dWo, j, slot, q, f0, f1, w, w4);
  } else {
    T f[8], wg[5];
    ghost_entry<T>(d, -1 - j, ws, f, wg);
    f0 = q == 0 ? f[0] : (q == 1 ? f[2] : (q == 2 ? f[4] : f[6]));
    f1 = q == 0 ? f[1] : (q == 1 ? f[3] : (q == 2 ? f[5] : f[7]));
    w = pick(wg, q);
    w4 = wg[4];
  }
  bwd_comp<T>(acc, sx, sy, sl, f0, f1, w);
  if (q == 0 && sa_on) bwd_sa<T>(acc4, sa, w4);
}

template <class T>
__device__ __forceinline__ void bwd_quad(const Dev& d, T* ring, int p, int pbase, const BwdRec<T>& r, int q,
                                         bool live, bool sa_on) {
  const int n = d.nc_pad;
  T* dWo = (T*)d.dW;
  T* dF = (T*)d.dF;
  T acc = (T)0, acc4 = (T)0;
  if (live) {
    const int cnt = r.cnt;
    if (cnt >= 0) {
#pragma unroll
      for (int e = 0; e < PF_E; e++) {
        if (e >= cnt) break;
        bwd_entry_q<T>(d, ring, dF, dWo, r.j[e], r.slot[e], r.ws, r.co[0][e], r.co[1][e], r.co[2][e], r.co[3][e],
                       q, sa_on, acc, acc4);
      }
    } else {
      const T* sc = (const T*)d.sc_b;
      const int nbs = d.nbs;
      for (int k = d.bs_ptr[p]; k < d.bs_ptr[p + 1]; k++)
        bwd_entry_q<T>(d, ring, dF, dWo, d.bs_j[k], d.bs_slot[k], r.ws, sc[k], sc[nbs + k], sc[2 * nbs + k],
                       sc[3 * nbs + k], q, sa_on, acc, acc4);
    }
  }
  const T wsq = pick(r.ws, q);
  const T dwq = inc_bwd<T>(wsq, acc, r.c[0]);
  const T dw4 = sa_on ? inc_bwd<T>(r.ws[4], acc4, r.c[1]) : (T)0;
  T dw[4];
#pragma unroll
  for (int k = 0; k < 4; k++) dw[k] = shfl_q<T>(dwq, k);
  if (!live) return;
  T o[8];
  delta_flux<T>(r.w[0], r.w[1], r.w[2], r.c[2], r.c[3], r.c[4], dw[0], dw[1], dw[2], dw[3], o);
  const T o0 = q == 0 ? o[0] : (q == 1 ? o[2] : (q == 2 ? o[4] : o[6]));
  const T o1 = q == 0 ? o[1] : (q == 1 ? o[3] : (q == 2 ? o[5] : o[7]));
  const int slot = (p - pbase) % RING;
  ring[(2 * q) * RING + slot] = o0;
  ring[(2 * q + 1) * RING + slot] = o1;
  ring[(8 + q) * RING + slot] = dwq;
  const int i = r.i;
  dWo[q * n + i] = dwq;
  dF[(2 * q) * n + i] = o0;
  dF[(2 * q + 1) * n + i] = o1;
  if (q == 0) {
    ring[12 * RING + slot] = dw4;
    dWo[4 * n + i] = dw4;
  }
}

template <class T>
__global__ void __launch_bounds__(QUAD_THREADS) k_sweep_fwd_quad(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  FwdRec<T>* stage = (FwdRec<T>*)(smem_raw + (size_t)13 * RING * sizeof(T));
  const int q = threadIdx.x % QUAD, cslot = threadIdx.x / QUAD, ncs = blockDim.x / QUAD;
  FwdRec<T>* st = stage + cslot;                     // the quad's staged record
  const int s = d.g_solve0 + blockIdx.x;
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  const bool sa_on = d.flow[s].sa_on;
  const int l0 = d.lvl_solve_ptr[s], l1 = d.lvl_solve_ptr[s + 1] - 1;
  const int pbase = d.fwd_lvl[l0];
  int b = d.fwd_lvl[l0], e = d.fwd_lvl[l0 + 1];
  int pm = b + cslot;
  if (l0 < l1 && pm < e) fwd_stage_q<T>(d, pm, st, q);
  for (int l = l0; l < l1; l++) {
    const int en = (l + 1 < l1) ? d.fwd_lvl[l + 2] : e;
    const bool mine = pm < e;
    FwdRec<T> cur;
    if (mine) cpa_wait_all();
    __syncwarp();                     // every lane's copies of the quad's record have landed
    if (mine) cur = *st;
    __syncwarp();                     // all lanes have read the stage before it is refilled
    const int pn = e + cslot;
    if (pn < en) fwd_stage_q<T>(d, pn, st, q);
    fwd_quad<T>(d, ring, pm, pbase, cur, q, mine, sa_on);
    // levels wider than the block's quads: further rounds, records read directly
    for (int base = b + ncs; base < e; base += ncs) {
      const int p = base + cslot;
      const bool live = p < e;
      FwdRec<T> xt;
      if (live) fwd_load_direct<T>(d, p, &xt);
      fwd_quad<T>(d, ring, p, pbase, xt, q, live, sa_on);
    }
    __syncthreads();
    b = e;
    e = en;
    pm = pn;
  }
}

template <class T>
__global__ void __launch_bounds__(QUAD_THREADS) k_sweep_bwd_quad(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  BwdRec<T>* stage = (BwdRec<T>*)(smem_raw + (size_t)13 * RING * sizeof(T));
  const int q = threadIdx.x % QUAD, cslot = threadIdx.x / QUAD, ncs = blockDim.x / QUAD;
  BwdRec<T>* st = stage + cslot;
  const int s = d.g_solve0 + blockIdx.x;
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  const bool sa_on = d.flow[s].sa_on;
  const int l0 = d.blvl_solve_ptr[s], l1 = d.blvl_solve_ptr[s + 1] - 1;
  const int pbase = d.bwd_lvl[l0];
  int b = d.bwd_lvl[l0], e = d.bwd_lvl[l0 + 1];
  int pm = b + cslot;
  if (l0 < l1 && pm < e) bwd_stage_q<T>(d, pm, st, q);
  for (int l = l0; l < l1; l++) {
    const int en = (l + 1 < l1) ? d.bwd_lvl[l + 2] : e;
    const bool mine = pm < e;
    BwdRec<T> cur;
    if (mine) cpa_wait_all();
    __syncwarp();
    if (mine) cur = *st;
    __syncwarp();
    const int pn = e + cslot;
    if (pn < en) bwd_stage_q<T>(d, pn, st, q);
    bwd_quad<T>(d, ring, pm, pbase, cur, q, mine, sa_on);
    for (int base = b + ncs; base < e; base += ncs) {
      const int p = base + cslot;
      const bool live = p < e;
      BwdRec<T> xt;
      if (live) bwd_load_direct<T>(d, p, &xt);
      bwd_quad<T>(d, ring, p, pbase, xt, q, live, sa_on);
    }
    __syncthreads();
    b = e;
    e = en;
    pm = pn;
  }
}

// ---- wide schedule: one launch per level, all solves ----
template <class T>
__global__ void k_sweep_fwd_level(Dev d, int b, int e) {
  const int k = b + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= e) return;
  const int i = d.wfwd_cells[k];
  const int s = d.cell_solve[i];
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  fwd_cell<T>(d, i, d.flow[s].sa_on);
}

template <class T>
__global__ void k_sweep_bwd_level(Dev d, int b, int e) {
  const int k = b + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= e) return;
  const int i = d.wbwd_cells[k];
  const int s = d.cell_solve[i];
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  bwd_cell<T>(d, i, d.flow[s].sa_on);
}

constexpr int WIDE_BLOCK = 128;

void launch_update(const Dev& d, int precision, cudaStream_t s) {
  if (precision == 1) k_update<float><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
  else if (precision == 2) k_update<df64><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
  else k_update<double><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
}

// dynamic shared memory of the narrow sweeps: the ring plus one staged record per thread
// (one staged record per thread)
template <class T>
static size_t fwd_smem() { return (size_t)13 * RING * sizeof(T) + (size_t)NARROW_THREADS * sizeof(FwdRec<T>); }
template <class T>
static size_t bwd_smem() { return (size_t)13 * RING * sizeof(T) + (size_t)NARROW_THREADS * sizeof(BwdRec<T>); }

template <class T, int C>
static void set_smem() {
  cudaFuncSetAttribute(k_sweep_fwd_narrow<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<T>());
  cudaFuncSetAttribute(k_sweep_bwd_narrow<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<T>());
}

template <class T>
static void set_smem_quad() {
  cudaFuncSetAttribute(k_sweep_fwd_quad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<T>());
  cudaFuncSetAttribute(k_sweep_bwd_quad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<T>());
}

void setup_sweeps() {
  set_smem<double, 1>(); set_smem<double, 2>(); set_smem<double, 4>(); set_smem<double, 8>();
  set_smem<float, 1>(); set_smem<float, 2>(); set_smem<float, 4>(); set_smem<float, 8>();
  set_smem<df64, 1>(); set_smem<df64, 2>(); set_smem<df64, 4>(); set_smem<df64, 8>();
  set_smem_quad<float>(); set_smem_quad<df64>();
}

// one block per solve (C = 1), or one cluster of C blocks per solve
template <class T, int C>
static void launch_narrow(bool fwd, const Dev& d, int threads, cudaStream_t s) {
  void (*k)(Dev) = fwd ? k_sweep_fwd_narrow<T, C> : k_sweep_bwd_narrow<T, C>;
  const size_t smem = fwd ? fwd_smem<T>() : bwd_smem<T>();
  if (C == 1) {
    k<<<d.g_nsolve, threads, smem, s>>>(d);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(d.g_nsolve * C));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, d);
}

template <class T>
static void launch_narrow_c(bool fwd, const Dev& d, int threads, cudaStream_t s) {
  if constexpr (!std::is_same<T, double>::value) {
    if (d.quad && d.sweep_cluster <= 1) {   // a quad of threads per cell
      void (*k)(Dev) = fwd ? k_sweep_fwd_quad<T> : k_sweep_bwd_quad<T>;
      k<<<d.g_nsolve, threads, fwd ? fwd_smem<T>() : bwd_smem<T>(), s>>>(d);
      return;
    }
  }
  switch (d.sweep_cluster) {
    case 2: launch_narrow<T, 2>(fwd, d, threads, s); break;
    case 4: launch_narrow<T, 4>(fwd, d, threads, s); break;
    case 8: launch_narrow<T, 8>(fwd, d, threads, s); break;
    default: launch_narrow<T, 1>(fwd, d, threads, s); break;
  }
}

void launch_sweep_prep(const Dev& d, int precision, cudaStream_t s) {
  if (precision == 1) k_sweep_prep<float><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
  else if (precision == 2) k_sweep_prep<df64><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
  else k_sweep_prep<double><<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
}

void launch_sweep_fwd(const Dev& d, int precision, int threads, cudaStream_t s) {
  if (d.wide) {
    for (int l = 0; l < d.n_wfwd; l++) {
      const int b = d.h_wfwd_ptr[l], e = d.h_wfwd_ptr[l + 1];
      const int g = (e - b + WIDE_BLOCK - 1) / WIDE_BLOCK;
      if (precision == 1) k_sweep_fwd_level<float><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
      else if (precision == 2) k_sweep_fwd_level<df64><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
      else k_sweep_fwd_level<double><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
    }
    return;
  }
  if (precision == 1) launch_narrow_c<float>(true, d, threads, s);
  else if (precision == 2) launch_narrow_c<df64>(true, d, threads, s);
  else launch_narrow_c<double>(true, d, threads, s);
}

void launch_sweep_bwd(const Dev& d, int precision, int threads, cudaStream_t s) {
  if (d.wide) {
    for (int l = 0; l < d.n_wbwd; l++) {
      const int b = d.h_wbwd_ptr[l], e = d.h_wbwd_ptr[l + 1];
      const int g = (e - b + WIDE_BLOCK - 1) / WIDE_BLOCK;
      if (precision == 1) k_sweep_bwd_level<float><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
      else if (precision == 2) k_sweep_bwd_level<df64><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
      else k_sweep_bwd_level<double><<<g, WIDE_BLOCK, 0, s>>>(d, b, e);
    }
    return;
  }
  if (precision == 1) launch_narrow_c<float>(false, d, threads, s);
  else if (precision == 2) launch_narrow_c<df64>(false, d, threads, s);
  else launch_narrow_c<double>(false, d, threads, s);
}

}  // namespace igks
