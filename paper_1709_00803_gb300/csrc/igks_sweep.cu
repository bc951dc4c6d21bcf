// igks_sweep.cu -- matrix-free LU-SGS forward and backward sweeps (Eq. 19-22 for the
// mean flow, Eq. 31-32 for the SA variable) with the FP64 state update, in FP64, FP32 or
// double-float.
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
//  - narrow: one block per solve (or a thread-block cluster) walks its levels with a
//    barrier between them (for orderings with hundreds of thin levels). The increments of
//    the last RING cells it produced stay in a shared-memory ring, so a cell usually reads
//    its neighbours' increments from shared memory; its record (stencil neighbours, ring
//    slots, coefficients and per-cell constants) is stored in sweep-position order, and a
//    level's records are brought into shared memory by bulk copies on an mbarrier, a few
//    levels ahead;
//  - wide: one launch per level covering that level's cells of every solve (for low-depth
//    orderings, e.g. multicolour, whose few levels hold thousands of cells each).
#include <cooperative_groups.h>
#include <float.h>

#include <cstddef>

#include <type_traits>

#include "igks_df64.cuh"
#include "igks_dev.h"
#include "igks_phys.cuh"

namespace cg = cooperative_groups;

namespace igks {

// The sweeps' arithmetic is written with explicitly rounded operations (fma_x, mul_x,
// add_x: __fma_rn / __dmul_rn / __dadd_rn in FP64, the __f*_rn intrinsics in FP32, the
// double-float operators): the compiler may not fuse or split them, so every schedule (one
// block or a cluster of blocks per solve, one launch per level) and every inlining
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

// the first BYTES bytes of src to dst (both 16-byte aligned) as 16-byte stores
template <size_t BYTES>
__device__ __forceinline__ void store_chunks(void* dst, const void* src) {
  static_assert(BYTES % 16 == 0, "whole chunks");
#pragma unroll
  for (int k = 0; k < (int)(BYTES / 16); k++)
    reinterpret_cast<uint4*>(dst)[k] = reinterpret_cast<const uint4*>(src)[k];
}

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
  // position-ordered records of the narrow schedule: the heads as whole 16-byte chunks
  // (the backward head's dW* slots are written by the forward sweep afterwards)
  const int pf = d.pos_f[i], pb = d.pos_b[i];
  FwdDyn<T>* rf = (FwdDyn<T>*)d.fdyn + pf;
  BwdDyn<T>* rb = (BwdDyn<T>*)d.bdyn + pb;
  const bool csr_f = d.fst[pf].cnt < 0, csr_b = d.bst[pb].cnt < 0;   // more entries than a record holds
  if (!wide) {
    FwdDyn<T> hf;
    BwdDyn<T> hb;
#pragma unroll
    for (int q = 0; q < 5; q++) hf.m[q] = (T)d.M[q * n + i];
    hf.w[0] = (T)r; hf.w[1] = (T)mx; hf.w[2] = (T)my;
#pragma unroll
    for (int q = 0; q < 5; q++) { hf.c[q] = cc[q]; hb.c[q] = cc[q]; hb.ws[q] = (T)0; }
#pragma unroll
    for (int q = 0; q < 5; q++) hb.w[q] = (T)d.W[q * n + i];
    for (int q = 0; q < (int)(sizeof(hf.pad0) / sizeof(T)); q++) hf.pad0[q] = (T)0;
    hb.pad0[0] = (T)0;
    store_chunks<offsetof(FwdDyn<T>, co)>(rf, &hf);
    store_chunks<offsetof(BwdDyn<T>, co)>(rb, &hb);
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
      const int xf = d.cf_to_ef[k], xb = d.cf_to_eb[k];   // record entry: position * PF_E + e
      alignas(16) const T ent[4] = {e0, e1, e2, e3};      // one entry: whole 16-byte chunks
      if (xf >= 0) store_chunks<sizeof(ent)>(((FwdDyn<T>*)d.fdyn)[xf / PF_E].co[xf % PF_E], ent);
      if (xb >= 0) store_chunks<sizeof(ent)>(((BwdDyn<T>*)d.bdyn)[xb / PF_E].co[xb % PF_E], ent);
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
  // a solve whose sweep wait ran out keeps its state (the increments are incomplete)
  const bool live = (i < d.nc_pad) && d.cell_solve[i] >= 0 && d.st[d.cell_solve[i]].state == 0 &&
                    !d.tmo[d.cell_solve[i]];
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
// Records. Each position has a static record (cell, neighbours, ring slots; 48 bytes) and
// a per-iteration record (FwdDyn / BwdDyn: 128 bytes in FP32, 240 / 256 in FP64 and
// double-float), both arrays of structures, so the records of one level are two contiguous
// ranges. With one block per solve the block brings a level's records into shared memory
// with two bulk copies (cp.async.bulk, the TMA engine's linear copy) completing on an
// mbarrier, NST levels ahead; the cells' threads only wait on the barrier and read. With a
// cluster of blocks per solve each thread stages its own record with 16-byte cp.async one
// level ahead.
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

// The increments of a record's PF_E entries. The ring reads of all entries are issued
// together, unconditionally (an unused entry or one whose neighbour left the ring reads a
// valid slot and its values are not used), so a cell waits for shared memory once rather
// than once per entry; the rare neighbours that left the ring are then read from global
// memory. Entries e >= cnt are not applied by the caller.
template <class T, int C = 1>
__device__ __forceinline__ void gather_entries(const Dev& d, const T* ring, const T* dF, const T* dWv, const int* j,
                                               const int* slot, int cnt, T (*f)[8], T (*w)[5]) {
#pragma unroll
  for (int e = 0; e < PF_E; e++) {
    const int sl = slot[e] >= 0 ? slot[e] : 0;
    const T* rb = ring_of<T, C>(ring, sl);
#pragma unroll
    for (int k = 0; k < 8; k++) f[e][k] = rb[k * RING + sl];
#pragma unroll
    for (int v = 0; v < 5; v++) w[e][v] = rb[(8 + v) * RING + sl];
  }
  const int n = d.nc_pad;
#pragma unroll
  for (int e = 0; e < PF_E; e++)
    if (e < cnt && slot[e] < 0 && j[e] >= 0) {
#pragma unroll
      for (int k = 0; k < 8; k++) f[e][k] = dF[k * n + j[e]];
#pragma unroll
      for (int v = 0; v < 5; v++) w[e][v] = dWv[v * n + j[e]];
    }
}

static_assert(sizeof(FwdDyn<df64>) == sizeof(FwdDyn<double>) && sizeof(BwdDyn<df64>) == sizeof(BwdDyn<double>),
              "double-float records");

// ---- asynchronous copies ----
// 16-byte cp.async (cluster schedule): global -> shared in the background, no registers held
__device__ __forceinline__ void cpa16(void* dst_smem, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// a record into registers with 16-byte loads (shared or global memory)
template <class R>
__device__ __forceinline__ R load_rec(const R* src) {
  R r;
#pragma unroll
  for (int k = 0; k < (int)(sizeof(R) / 16); k++) reinterpret_cast<uint4*>(&r)[k] = reinterpret_cast<const uint4*>(src)[k];
  return r;
}

template <class R>
__device__ __forceinline__ void cpa_record(R* dst, const R* src) {   // sizeof(R) is a multiple of 16
#pragma unroll
  for (int k = 0; k < (int)(sizeof(R) / 16); k++) cpa16((char*)dst + 16 * k, (const char*)src + 16 * k);
}

// mbarrier and bulk copy (one block per solve)
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {   // the producer's arrival
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for a phase of the barrier, at most limit tries; false when it ran out
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int limit) {
  for (int it = 0; it < limit; it++)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// ---- the work on one position (forward / backward), records in shared or global memory ----
template <class T, int C = 1>
__device__ __forceinline__ void fwd_process(const Dev& d, T* ring, int p, int pbase, const FwdStat& st,
                                            const FwdDyn<T>& dy, bool sa_on) {
  const int n = d.nc_pad;
  T* dWs = (T*)d.dWs;
  T* dF = (T*)d.dF;
  T acc[5];
#pragma unroll
  for (int v = 0; v < 5; v++) acc[v] = dy.m[v];
  const int cnt = st.cnt;
  if (cnt >= 0) {
    T f[PF_E][8], w[PF_E][5];
    gather_entries<T, C>(d, ring, dF, dWs, st.j, st.slot, cnt, f, w);
#pragma unroll
    for (int e = 0; e < PF_E; e++)
      if (e < cnt) fwd_acc<T>(acc, dy.co[e][0], dy.co[e][1], dy.co[e][2], dy.co[e][3], f[e], w[e], sa_on);
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
  for (int v = 0; v < 4; v++) dw[v] = inc_fwd<T>(acc[v], dy.c[0]);
  dw[4] = sa_on ? inc_fwd<T>(acc[4], dy.c[1]) : (T)0;
  T o[8];
  delta_flux<T>(dy.w[0], dy.w[1], dy.w[2], dy.c[2], dy.c[3], dy.c[4], dw[0], dw[1], dw[2], dw[3], o);
  const int slot = (p - pbase) % RING;
  ring_put<T>(ring, slot, o, dw);
  const int i = st.i;
  BwdDyn<T>* rb = (BwdDyn<T>*)d.bdyn + st.pb;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    dWs[v * n + i] = dw[v];
    rb->ws[v] = dw[v];                        // the backward sweep's copy of dW*
  }
#pragma unroll
  for (int k = 0; k < 8; k++) dF[k * n + i] = o[k];
}

template <class T>
__device__ __forceinline__ T mn_x(T a, T fx, T b, T fy) { return fma_x(a, fx, mul_x(b, fy)); }

// the increments of a wall / symmetry ghost (face fc) in the backward sweep: the boundary
// map of the cell's own forward increment ws, and the flux increment about the ghost state
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

// contribution of one backward entry: upper neighbour j (its increments from the ring or
// global memory), or a wall/symmetry ghost (j = -1 - face)
template <class T, int C>
__device__ __forceinline__ void bwd_entry(const Dev& d, const T* ring, const T* dF, const T* dWo, int j, int slot,
                                          const T* ws, T sx, T sy, T sl, T sa, bool sa_on, T* acc) {
  T f[8], w[5];
  if (j >= 0) neighbour<T, C>(d, ring, dF, dWo, j, slot, f, w);
  else ghost_entry<T>(d, -1 - j, ws, f, w);
  bwd_acc<T>(acc, sx, sy, sl, sa, f, w, sa_on);
}

template <class T, int C = 1>
__device__ __forceinline__ void bwd_process(const Dev& d, T* ring, int p, int pbase, const BwdStat& st,
                                            const BwdDyn<T>& dy, bool sa_on) {
  const int n = d.nc_pad;
  T* dWo = (T*)d.dW;
  T* dF = (T*)d.dF;
  T ws[5];
#pragma unroll
  for (int v = 0; v < 5; v++) ws[v] = dy.ws[v];
  T acc[5] = {0, 0, 0, 0, 0};
  const int cnt = st.cnt;
  if (cnt >= 0) {
    T f[PF_E][8], w[PF_E][5];
    gather_entries<T, C>(d, ring, dF, dWo, st.j, st.slot, cnt, f, w);
#pragma unroll
    for (int e = 0; e < PF_E; e++)
      if (e < cnt && st.j[e] < 0) ghost_entry<T>(d, -1 - st.j[e], ws, f[e], w[e]);   // wall / symmetry ghost
#pragma unroll
    for (int e = 0; e < PF_E; e++)
      if (e < cnt) bwd_acc<T>(acc, dy.co[e][0], dy.co[e][1], dy.co[e][2], dy.co[e][3], f[e], w[e], sa_on);
  } else {
    const T* sc = (const T*)d.sc_b;
    const int nbs = d.nbs;
    for (int k = d.bs_ptr[p]; k < d.bs_ptr[p + 1]; k++)
      bwd_entry<T, C>(d, ring, dF, dWo, d.bs_j[k], d.bs_slot[k], ws, sc[k], sc[nbs + k], sc[2 * nbs + k],
                      sc[3 * nbs + k], sa_on, acc);
  }
  T dw[5];
#pragma unroll
  for (int v = 0; v < 4; v++) dw[v] = inc_bwd<T>(ws[v], acc[v], dy.c[0]);
  dw[4] = sa_on ? inc_bwd<T>(ws[4], acc[4], dy.c[1]) : (T)0;
  T o[8];
  delta_flux<T>(dy.w[0], dy.w[1], dy.w[2], dy.c[2], dy.c[3], dy.c[4], dw[0], dw[1], dw[2], dw[3], o);
  ring_put<T>(ring, (p - pbase) % RING, o, dw);
  const int i = st.i;
#pragma unroll
  for (int v = 0; v < 5; v++) dWo[v * n + i] = dw[v];
#pragma unroll
  for (int k = 0; k < 8; k++) dF[k * n + i] = o[k];
}

// ---- one block per solve: levels staged by bulk copies NST levels ahead ----
constexpr int NST = 3;   // stage buffers (levels in flight)
template <class T>
__host__ __device__ constexpr int stage_max() { return sizeof(T) == 4 ? 256 : 128; }   // records per stage

template <class T, bool FWD>
struct Rec {
  using Stat = typename std::conditional<FWD, FwdStat, BwdStat>::type;
  using Dyn = typename std::conditional<FWD, FwdDyn<T>, BwdDyn<T>>::type;
};

// dynamic shared memory: ring | NST x stage_max static records | NST x stage_max dynamic
// records | NST mbarriers | abort flag
template <class T, bool FWD>
__host__ __device__ constexpr size_t stage_stat_off() { return (size_t)13 * RING * sizeof(T); }
template <class T, bool FWD>
__host__ __device__ constexpr size_t stage_dyn_off() {
  return stage_stat_off<T, FWD>() + (size_t)NST * stage_max<T>() * sizeof(typename Rec<T, FWD>::Stat);
}
template <class T, bool FWD>
__host__ __device__ constexpr size_t stage_bar_off() {
  return stage_dyn_off<T, FWD>() + (size_t)NST * stage_max<T>() * sizeof(typename Rec<T, FWD>::Dyn);
}
template <class T, bool FWD>
__host__ __device__ constexpr size_t bulk_smem() { return stage_bar_off<T, FWD>() + 8 * NST + 16; }

// issue the bulk copies of level [b, e) (its first stage_max records) into stage k
template <class T, bool FWD>
__device__ __forceinline__ void stage_level(const Dev& d, unsigned char* smem, int k, int b, int e) {
  using Stat = typename Rec<T, FWD>::Stat;
  using Dyn = typename Rec<T, FWD>::Dyn;
  const int nrec = min(e - b, stage_max<T>());
  const unsigned bar = (unsigned)__cvta_generic_to_shared(smem + stage_bar_off<T, FWD>() + 8 * k);
  const unsigned ss = (unsigned)__cvta_generic_to_shared(smem + stage_stat_off<T, FWD>()) +
                      (unsigned)(k * stage_max<T>() * sizeof(Stat));
  const unsigned sd = (unsigned)__cvta_generic_to_shared(smem + stage_dyn_off<T, FWD>()) +
                      (unsigned)(k * stage_max<T>() * sizeof(Dyn));
  const Stat* gs = (FWD ? (const Stat*)d.fst : (const Stat*)d.bst) + b;
  const Dyn* gd = (const Dyn*)(FWD ? d.fdyn : d.bdyn) + b;
  mbar_expect(bar, (unsigned)(nrec * (sizeof(Stat) + sizeof(Dyn))));
  bulk_g2s(ss, gs, (unsigned)(nrec * sizeof(Stat)), bar);
  bulk_g2s(sd, gd, (unsigned)(nrec * sizeof(Dyn)), bar);
}

// The sweep of one solve by one block. Level l (k = l - l0) sits in stage k % NST, phase
// (k / NST) & 1 of its barrier. Thread 0 issues the copies; every thread waits for its
// level's barrier (at most wait_limit tries: a wait that runs out marks the solve
// IGKS_TIMEOUT, the block stops after the level barrier, waits for its copies in flight,
// and the update leaves the solve's state untouched). Positions beyond stage_max of a wide
// level read their records from global memory.
template <class T, bool FWD>
__device__ __forceinline__ void sweep_bulk(const Dev& d) {
  using Stat = typename Rec<T, FWD>::Stat;
  using Dyn = typename Rec<T, FWD>::Dyn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  const Stat* sst = (const Stat*)(smem_raw + stage_stat_off<T, FWD>());
  const Dyn* sdy = (const Dyn*)(smem_raw + stage_dyn_off<T, FWD>());
  const unsigned bar0 = (unsigned)__cvta_generic_to_shared(smem_raw + stage_bar_off<T, FWD>());
  volatile int* abort_flag = (volatile int*)(smem_raw + stage_bar_off<T, FWD>() + 8 * NST);
  const int s = d.g_solve0 + blockIdx.x;
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;
  if (!FWD && d.tmo[s]) return;                       // the forward sweep of this solve gave up
  const bool sa_on = d.flow[s].sa_on;
  const int* lvl = FWD ? d.fwd_lvl : d.bwd_lvl;
  const int* lsp = FWD ? d.lvl_solve_ptr : d.blvl_solve_ptr;
  const int l0 = lsp[s], l1 = lsp[s + 1] - 1, nl = l1 - l0;
  if (nl <= 0) return;
  const Stat* gst = FWD ? (const Stat*)d.fst : (const Stat*)d.bst;
  const Dyn* gdy = (const Dyn*)(FWD ? d.fdyn : d.bdyn);
  const int limit = d.wait_limit;
  const int tid = threadIdx.x;
  int issued = 0;                                     // levels issued (thread 0)
  int nb = 0;                                         // offset of the next level to issue (thread 0)
  if (tid == 0) {
    for (int k = 0; k < NST; k++) mbar_init(bar0 + 8 * k, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    nb = lvl[l0];
    for (; issued < NST && issued < nl; issued++) {
      const int e = lvl[l0 + issued + 1];
      if (!(FWD && d.starve_test && issued == 1)) stage_level<T, FWD>(d, smem_raw, issued, nb, e);
      nb = e;
    }
  }
  __syncthreads();
  const int pbase = lvl[l0];
  int b = lvl[l0], e = lvl[l0 + 1];
  int k = 0;
  for (; k < nl; k++) {
    const int l = l0 + k;
    const int en = (k + 1 < nl) ? lvl[l + 2] : e;     // next level's end, loaded a level early
    const int st_k = k % NST;
    const int nnext = (tid == 0 && issued < nl) ? lvl[l0 + issued + 1] : 0;   // for the copy issued below
    const bool mine = b + tid < e;
    bool ok = true;
    if (mine) ok = mbar_wait(bar0 + 8 * st_k, (unsigned)((k / NST) & 1), limit);
    if (!ok) {
      d.tmo[s] = 1;
      *abort_flag = 1;
    } else {
      const int smax = stage_max<T>();
      for (int p = b + tid; p < e; p += blockDim.x) {
        const int q = p - b;
        Stat cs;
        Dyn cd;
        if (q < smax) {              // staged: shared-memory loads
          cs = load_rec(sst + st_k * smax + q);
          cd = load_rec(sdy + st_k * smax + q);
        } else {
          cs = load_rec(gst + p);
          cd = load_rec(gdy + p);
        }
        if constexpr (FWD) fwd_process<T>(d, ring, p, pbase, cs, cd, sa_on);
        else bwd_process<T>(d, ring, p, pbase, cs, cd, sa_on);
      }
    }
    __syncthreads();                                  // level done; stage st_k is free
    if (*abort_flag) break;
    if (tid == 0 && issued < nl) {
      // the stage was read by generic loads: order those before the async proxy's writes
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      stage_level<T, FWD>(d, smem_raw, issued % NST, nb, nnext);
      nb = nnext;
      issued++;
    }
    b = e;
    e = en;
  }
  // after a wait ran out: let the copies already issued land before the block exits
  if (tid == 0 && k < nl)
    for (int kk = k; kk < issued; kk++)
      if (!(FWD && d.starve_test && kk == 1)) mbar_wait(bar0 + 8 * (kk % NST), (unsigned)((kk / NST) & 1), limit);
}

template <class T>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_fwd_bulk(Dev d) { sweep_bulk<T, true>(d); }
template <class T>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_bwd_bulk(Dev d) { sweep_bulk<T, false>(d); }

// ---- a cluster of C blocks per solve: positions dealt round the blocks, records staged
// per thread with 16-byte cp.async one level ahead ----
// the first position at or after b that belongs to cluster block r (positions q = p - pbase
// are dealt round the C blocks: q % C == r)
template <int C>
__device__ __forceinline__ int first_own(int b, int pbase, int r) {
  return b + (((r - (b - pbase)) % C) + C) % C;
}

template <class T, bool FWD>
__host__ __device__ constexpr size_t cluster_smem() {
  return (size_t)13 * RING * sizeof(T) +
         (size_t)NARROW_THREADS * (sizeof(typename Rec<T, FWD>::Stat) + sizeof(typename Rec<T, FWD>::Dyn));
}

template <class T, bool FWD, int C>
__device__ __forceinline__ void sweep_cluster(const Dev& d) {
  using Stat = typename Rec<T, FWD>::Stat;
  using Dyn = typename Rec<T, FWD>::Dyn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = (T*)smem_raw;
  Stat* sst = (Stat*)(smem_raw + (size_t)13 * RING * sizeof(T)) + threadIdx.x;
  Dyn* sdy = (Dyn*)(smem_raw + (size_t)13 * RING * sizeof(T) + (size_t)NARROW_THREADS * sizeof(Stat)) + threadIdx.x;
  const int s = d.g_solve0 + blockIdx.x / C, r = blockIdx.x % C;   // one cluster of C blocks per solve
  if (d.st[s].state != 0 || d.flow[s].scheme == 1) return;         // uniform over the cluster
  cg::this_cluster().sync();                                       // every block runs before any remote read
  const bool sa_on = d.flow[s].sa_on;
  const int* lvl = FWD ? d.fwd_lvl : d.bwd_lvl;
  const int* lsp = FWD ? d.lvl_solve_ptr : d.blvl_solve_ptr;
  const int l0 = lsp[s], l1 = lsp[s + 1] - 1;
  const Stat* gst = FWD ? (const Stat*)d.fst : (const Stat*)d.bst;
  const Dyn* gdy = (const Dyn*)(FWD ? d.fdyn : d.bdyn);
  const int pbase = lvl[l0];
  const int step = C * (int)blockDim.x;
  int b = lvl[l0], e = lvl[l0 + 1];
  int pm = first_own<C>(b, pbase, r) + C * (int)threadIdx.x;   // this thread's position of the level
  if (l0 < l1 && pm < e) { cpa_record(sst, gst + pm); cpa_record(sdy, gdy + pm); cpa_commit(); }
  for (int l = l0; l < l1; l++) {
    const int en = (l + 1 < l1) ? lvl[l + 2] : e;
    const bool mine = pm < e;
    Stat cs;
    Dyn cd;
    if (mine) {
      cpa_wait_all();
      cs = load_rec(sst);        // this level's record into registers, freeing the stage
      cd = load_rec(sdy);
    }
    const int pn = first_own<C>(e, pbase, r) + C * (int)threadIdx.x;
    if (pn < en) { cpa_record(sst, gst + pn); cpa_record(sdy, gdy + pn); cpa_commit(); }
    if (mine) {
      if constexpr (FWD) fwd_process<T, C>(d, ring, pm, pbase, cs, cd, sa_on);
      else bwd_process<T, C>(d, ring, pm, pbase, cs, cd, sa_on);
    }
    for (int p = pm + step; p < e; p += step) {   // levels wider than the cluster's threads
      const Stat xs = load_rec(gst + p);
      const Dyn xd = load_rec(gdy + p);
      if constexpr (FWD) fwd_process<T, C>(d, ring, p, pbase, xs, xd, sa_on);
      else bwd_process<T, C>(d, ring, p, pbase, xs, xd, sa_on);
    }
    cg::this_cluster().sync();   // release/acquire over the cluster's shared and global writes
    b = e;
    e = en;
    pm = pn;
  }
}

template <class T, int C>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_fwd_cluster(Dev d) { sweep_cluster<T, true, C>(d); }
template <class T, int C>
__global__ void __launch_bounds__(NARROW_THREADS) k_sweep_bwd_cluster(Dev d) { sweep_cluster<T, false, C>(d); }

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

template <class T>
static void set_smem_t() {
  cudaFuncSetAttribute(k_sweep_fwd_bulk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bulk_smem<T, true>());
  cudaFuncSetAttribute(k_sweep_bwd_bulk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bulk_smem<T, false>());
  cudaFuncSetAttribute(k_sweep_fwd_cluster<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, true>());
  cudaFuncSetAttribute(k_sweep_bwd_cluster<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, false>());
  cudaFuncSetAttribute(k_sweep_fwd_cluster<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, true>());
  cudaFuncSetAttribute(k_sweep_bwd_cluster<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, false>());
  cudaFuncSetAttribute(k_sweep_fwd_cluster<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, true>());
  cudaFuncSetAttribute(k_sweep_bwd_cluster<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_smem<T, false>());
}

void setup_sweeps() {
  set_smem_t<double>();
  set_smem_t<float>();
  set_smem_t<df64>();
}

// one cluster of C blocks per solve
template <class T, int C>
static void launch_cluster(bool fwd, const Dev& d, int threads, cudaStream_t s) {
  void (*k)(Dev) = fwd ? k_sweep_fwd_cluster<T, C> : k_sweep_bwd_cluster<T, C>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(d.g_nsolve * C));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = fwd ? cluster_smem<T, true>() : cluster_smem<T, false>();
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
  switch (d.sweep_cluster) {
    case 2: launch_cluster<T, 2>(fwd, d, threads, s); break;
    case 4: launch_cluster<T, 4>(fwd, d, threads, s); break;
    case 8: launch_cluster<T, 8>(fwd, d, threads, s); break;
    default:   // one block per solve
      if (fwd) k_sweep_fwd_bulk<T><<<d.g_nsolve, threads, bulk_smem<T, true>(), s>>>(d);
      else k_sweep_bwd_bulk<T><<<d.g_nsolve, threads, bulk_smem<T, false>(), s>>>(d);
      break;
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
