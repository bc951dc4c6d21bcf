// igks_kernels.cu -- per-cell and per-solve kernels of the IGKS iteration on sm_103a:
// mesh geometry and wall distance (set-up), eddy viscosity, ghost cells (Section II.E),
// least-squares gradients with limiter and spectral radius (Eq. 6-10, 20-23), residual
// gather with the SA source (Eq. 16, 27-28a), residual norms and CFL adaptation (Eq. 25),
// and the end-of-iteration bookkeeping. The LU-SGS sweeps live in igks_sweep.cu.
//
// This translation unit is compiled without floating-point contraction (-fmad=false):
// its sums (polygon areas and centroids, least-squares normal equations, residual
// gathers) then round term by term in the order written, which keeps the gradients of
// highly stretched boundary-layer cells (normal matrices with condition numbers of
// 1e6-1e8) reproducible to the last bits.
//
// The work is HBM/latency bound (no dense contraction): loads are structure-of-arrays,
// per-cell reductions are done in registers, per-solve reductions in fixed order.
#include <float.h>

#include "igks_dev.h"
#include "igks_phys.cuh"

namespace igks {

// ===================================================================================
// set-up: geometry and wall distance
// ===================================================================================

__global__ void k_geometry_cells(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nc_pad || d.cell_solve[i] < 0) return;
  const double* X = d.xy;
  const double* Y = d.xy + d.nn;
  int b = d.cn_ptr[i], e = d.cn_ptr[i + 1];
  double a = 0.0, sx = 0.0, sy = 0.0;
  for (int k = b; k < e; k++) {
    int p = d.cn_node[k], q = d.cn_node[k + 1 < e ? k + 1 : b];
    double x0 = X[p], y0 = Y[p], x1 = X[q], y1 = Y[q];
    double c = x0 * y1 - x1 * y0;
    a += c;
    sx += (x0 + x1) * c;
    sy += (y0 + y1) * c;
  }
  a *= 0.5;
  d.area[i] = a;
  d.cx[i] = sx / (6.0 * a);
  d.cy[i] = sy / (6.0 * a);
  if (!(a > 0.0)) atomicOr(d.err + 0, 1);
}

__global__ void k_geometry_faces(Dev d) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nf) return;
  const double* X = d.xy;
  const double* Y = d.xy + d.nn;
  int a = d.fnode[f], b = d.fnode[d.nf + f];
  double dx = X[b] - X[a], dy = Y[b] - Y[a];
  double S = sqrt(dx * dx + dy * dy);
  double nx = dy / S, ny = -dx / S;
  double mx = 0.5 * (X[a] + X[b]), my = 0.5 * (Y[a] + Y[b]);
  int L = d.fL[f], R = d.fR[f];
  double cxl = d.cx[L], cyl = d.cy[L];
  double dL = (mx - cxl) * nx + (my - cyl) * ny;
  double cxr, cyr, dR;
  if (R >= 0) {
    cxr = d.cx[R]; cyr = d.cy[R];
    dR = -((mx - cxr) * nx + (my - cyr) * ny);
  } else {
    cxr = cxl + 2.0 * dL * nx;
    cyr = cyl + 2.0 * dL * ny;
    dR = dL;
  }
  d.fS[f] = S; d.fnx[f] = nx; d.fny[f] = ny; d.fmx[f] = mx; d.fmy[f] = my;
  d.fcx[f] = cxr; d.fcy[f] = cyr; d.fidL[f] = 1.0 / dL; d.fidR[f] = 1.0 / dR;
  d.fdn[f] = fabs((cxr - cxl) * nx + (cyr - cyl) * ny);
  if (!(dL > 0.0) || !(dR > 0.0) || !(S > 0.0)) atomicOr(d.err + 1, 1);
}

__global__ void k_wall_distance(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nc_pad) return;
  int s = d.cell_solve[i];
  if (s < 0) return;
  const double* X = d.xy;
  const double* Y = d.xy + d.nn;
  double px = d.cx[i], py = d.cy[i], dmin = 1e300;
  for (int k = d.wall_ptr[s]; k < d.wall_ptr[s + 1]; k++) {
    int f = d.wall_face[k];
    int a = d.fnode[f], b = d.fnode[d.nf + f];
    double ax = X[a], ay = Y[a], ex = X[b] - ax, ey = Y[b] - ay;
    double t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
    t = fmin(fmax(t, 0.0), 1.0);
    double qx = ax + t * ex - px, qy = ay + t * ey - py;
    dmin = fmin(dmin, sqrt(qx * qx + qy * qy));
  }
  d.wall_d[i] = dmin;
}

// The normal matrix of the least-squares gradient (Eq. 7) depends on the geometry only:
// accumulated here once, in the same order and roundings the gradient kernel used per
// iteration, with the correctly rounded reciprocal of its determinant.
__global__ void k_lsq_matrix(Dev d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nc_pad || d.cell_solve[i] < 0) return;
  const int n = d.nc_pad;
  const double xi = d.cx[i], yi = d.cy[i];
  double A00 = 0.0, A01 = 0.0, A11 = 0.0;
  for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
    const int f = d.cf_face[k];
    const int L = d.fL[f], R = d.fR[f];
    const int j = (L == i) ? R : L;
    double xk, yk;
    if (j >= 0) { xk = d.cx[j]; yk = d.cy[j]; } else { xk = d.fcx[f]; yk = d.fcy[f]; }
    const double dx = xk - xi, dy = yk - yi;
    A00 += dx * dx; A01 += dx * dy; A11 += dy * dy;
  }
  const double det = A00 * A11 - A01 * A01;
  d.lsq[i] = A00; d.lsq[n + i] = A01; d.lsq[2 * n + i] = A11; d.lsq[3 * n + i] = __drcp_rn(det);
}

void launch_geometry(const Dev& d, cudaStream_t s) {
  k_geometry_cells<<<(d.nc_pad + 255) / 256, 256, 0, s>>>(d);
  if (d.nf) k_geometry_faces<<<(d.nf + 255) / 256, 256, 0, s>>>(d);
  k_lsq_matrix<<<(d.nc_pad + 255) / 256, 256, 0, s>>>(d);
}

void launch_wall_distance(const Dev& d, cudaStream_t s) {
  k_wall_distance<<<(d.nc_pad + 255) / 256, 256, 0, s>>>(d);
}

// ===================================================================================
// iteration kernels
// ===================================================================================

__device__ __forceinline__ bool cell_live(const Dev& d, int i, int* solve) {
  if (i >= d.nc_pad) return false;
  int s = d.cell_solve[i];
  if (s < 0 || d.st[s].state != 0) return false;
  *solve = s;
  return true;
}

// velocity and sound speed of a state, in the order the face spectral radius uses them
__device__ __forceinline__ void speeds_of(const double* W, double* u, double* v, double* c) {
  const double p = pressure_of(W[0], W[1], W[2], W[3]);
  *u = W[1] / W[0];
  *v = W[2] / W[0];
  *c = sqrt(GAMMA * p / W[0]);
}

// laminar and eddy viscosity of every cell, and its velocity and sound speed (read by the
// face spectral radius of both cells of each face)
__global__ void __launch_bounds__(CELL_BLOCK) k_prep(Dev d) {
  int i = (d.g_blk0 + blockIdx.x) * CELL_BLOCK + threadIdx.x, s;
  if (!cell_live(d, i, &s)) return;
  const DevFlow& fl = d.flow[s];
  int n = d.nc_pad;
  double r = d.W[i], mx = d.W[n + i], my = d.W[2 * n + i], E = d.W[3 * n + i], nut = d.W[4 * n + i];
  // one reciprocal of the density serves the velocity, 1/(2 lambda) = p / rho and chi
  const double ir = __drcp_rn(r);
  const double u = mx * ir, v = my * ir;
  const double p = (GAMMA - 1.0) * (E - 0.5 * (mx * u + my * v));
  const double h = p * ir;
  const double mu = viscosity_h(fl, h);
  d.mu_l[i] = mu;
  double mt = 0.0;
  if (fl.sa_on && nut > 0.0) {   // mu_t = rho nu~ fv1 (Eq. 34)
    const double chi = nut * r * __drcp_rn(mu), c3 = chi * chi * chi;
    mt = r * nut * c3 * __drcp_rn(c3 + SA_CV1 * SA_CV1 * SA_CV1);
  }
  d.mu_t[i] = mt;
  d.pu[i] = u; d.pv[i] = v; d.pc[i] = sqrt(GAMMA * h);
}

// state of the cell across face f (ghost on a boundary)
__device__ __forceinline__ void across_W(const Dev& d, int f, int j, double* Wk) {
  if (j >= 0) {
    int n = d.nc_pad;
    for (int v = 0; v < 5; v++) Wk[v] = d.W[v * n + j];
  } else {
    for (int v = 0; v < 5; v++) Wk[v] = d.G[v * d.nf + f];
  }
}

// face spectral radius lambda_f = |Vbar.n| + cbar (+ viscous term) from the velocities and
// sound speeds of the two sides, always in the face's own left/right order so both cells
// get the same bits
__device__ __forceinline__ double face_lambda(const DevFlow& fl, double uL, double vL, double cL, double rL,
                                              double uR, double vR, double cR, double rR,
                                              double muL, double mtL, double muR, double mtR,
                                              double nx, double ny, double dn) {
  double ub = 0.5 * (uL + uR), vb = 0.5 * (vL + vR), cb = 0.5 * (cL + cR);
  double lam = fabs(ub * nx + vb * ny) + cb;
  if (fl.visc_sr) {
    double mub = 0.5 * (muL + muR), mtb = 0.5 * (mtL + mtR), rb = 0.5 * (rL + rR);
    lam += 2.0 * (mub + mtb) * GAMMA / (rb * fl.prandtl * dn);
  }
  return lam;
}

// per face: the ghost state of a boundary face (Section II.E) and the face spectral
// radius lambda_f of Eq. 21 (computed once per face, read by both cells' Lambda sums)
__global__ void k_ghost(Dev d) {
  int f = d.g_face0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.g_face0 + d.g_nface) return;
  int s = d.fsolve[f];
  if (d.st[s].state != 0) return;
  const DevFlow& fl = d.flow[s];
  const int L = d.fL[f], R = d.fR[f], n = d.nc_pad;
  double muR, mtR, uR, vR, cR, rR;
  if (R < 0) {
    double WL[5], WR[5];
    for (int v = 0; v < 5; v++) WL[v] = d.W[v * n + L];
    ghost_state(fl, d.fbc[f], d.fnx[f], d.fny[f], WL, WR);
    for (int v = 0; v < 5; v++) d.G[v * d.nf + f] = WR[v];
    muR = viscosity(fl, lambda_of(WR[0], WR[1], WR[2], WR[3]));
    mtR = eddy_viscosity(fl, WR[0], WR[4], muR);
    d.Gmu[f] = muR;
    d.Gmu[d.nf + f] = mtR;
    speeds_of(WR, &uR, &vR, &cR);
    rR = WR[0];
  } else {
    muR = d.mu_l[R];
    mtR = d.mu_t[R];
    uR = d.pu[R]; vR = d.pv[R]; cR = d.pc[R]; rR = d.W[R];
  }
  d.lam_f[f] = face_lambda(fl, d.pu[L], d.pv[L], d.pc[L], d.W[L], uR, vR, cR, rR, d.mu_l[L], d.mu_t[L], muR, mtR,
                           d.fnx[f], d.fny[f], d.fdn[f]);
}

void launch_prep(const Dev& d, cudaStream_t s) {
  k_prep<<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
}

void launch_ghost(const Dev& d, cudaStream_t s) {
  if (d.g_nface) k_ghost<<<(d.g_nface + 127) / 128, 128, 0, s>>>(d);
}

// Least-squares gradients (Eq. 7) of the conserved variables over the face neighbours
// (ghosts included), the limiter of Eq. 9-10, the vorticity for SA, Lambda_i from the face
// spectral radii and the per-solve minimum explicit time step (Eq. 23).
__global__ void __launch_bounds__(CELL_BLOCK) k_gradient(Dev d) {
  const int blk = d.g_blk0 + blockIdx.x;
  int i = blk * CELL_BLOCK + threadIdx.x, s = -1;
  bool live = cell_live(d, i, &s);
  double dtc = DBL_MAX;
  if (live) {
    const DevFlow& fl = d.flow[s];
    const int n = d.nc_pad;
    double Wi[5];
    for (int v = 0; v < 5; v++) Wi[v] = d.W[v * n + i];
    double xi = d.cx[i], yi = d.cy[i];
    double r0[4] = {0, 0, 0, 0}, r1[4] = {0, 0, 0, 0}, wmax[4], wmin[4];
    for (int v = 0; v < 4; v++) wmax[v] = wmin[v] = Wi[v];
    double Lam = 0.0;
    for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
      int f = d.cf_face[k];
      int L = d.fL[f], R = d.fR[f];
      int j = (L == i) ? R : L;
      double Wk[5], xk, yk;
      across_W(d, f, j, Wk);
      if (j >= 0) { xk = d.cx[j]; yk = d.cy[j]; } else { xk = d.fcx[f]; yk = d.fcy[f]; }
      double dx = xk - xi, dy = yk - yi;
#pragma unroll
      for (int v = 0; v < 4; v++) {
        double dw = Wk[v] - Wi[v];
        r0[v] += dx * dw;
        r1[v] += dy * dw;
        wmax[v] = fmax(wmax[v], Wk[v]);
        wmin[v] = fmin(wmin[v], Wk[v]);
      }
      Lam += 0.5 * d.lam_f[f] * d.fS[f];
    }
    // the geometry's normal matrix and 1/det (k_lsq_matrix)
    const double A00 = d.lsq[i], A01 = d.lsq[n + i], A11 = d.lsq[2 * n + i], idet = d.lsq[3 * n + i];
    double area = d.area[i];
    double b[8];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      b[2 * v] = (A11 * r0[v] - A01 * r1[v]) * idet;
      b[2 * v + 1] = (A00 * r1[v] - A01 * r0[v]) * idet;
      d.grad[(2 * v) * n + i] = b[2 * v];
      d.grad[(2 * v + 1) * n + i] = b[2 * v + 1];
    }
    double phi[4] = {1.0, 1.0, 1.0, 1.0};
    if (fl.limiter == 1) {
      // Barth-Jespersen: the smallest ratio over the vertices comes from the largest
      // excursion of each sign (correctly rounded division is monotone in the divisor),
      // so two divisions per variable give the same bits as one per vertex; and a
      // correctly rounded x / y with 0 < x < y stays below 1, so min(1, x / y) is 1
      // exactly when x >= y and the division is needed only where the limiter acts
      double up[4] = {0, 0, 0, 0}, dn[4] = {0, 0, 0, 0};
      for (int k = d.cn_ptr[i]; k < d.cn_ptr[i + 1]; k++) {
        int nd = d.cn_node[k];
        double ox = d.xy[nd] - xi, oy = d.xy[d.nn + nd] - yi;
#pragma unroll
        for (int v = 0; v < 4; v++) {
          double dv = b[2 * v] * ox + b[2 * v + 1] * oy;
          up[v] = fmax(up[v], dv);
          dn[v] = fmin(dn[v], dv);
        }
      }
#pragma unroll
      for (int v = 0; v < 4; v++) {
        const double hi = wmax[v] - Wi[v], lo = wmin[v] - Wi[v];
        if (up[v] > 0.0 && hi < up[v]) phi[v] = fmin(phi[v], hi / up[v]);
        if (dn[v] < 0.0 && lo > dn[v]) phi[v] = fmin(phi[v], lo / dn[v]);
      }
    } else if (fl.limiter == 2) {
      double h = sqrt(area);
      double eps2 = (fl.venkat_k * h) * (fl.venkat_k * h) * (fl.venkat_k * h);
      for (int k = d.cn_ptr[i]; k < d.cn_ptr[i + 1]; k++) {
        int nd = d.cn_node[k];
        double ox = d.xy[nd] - xi, oy = d.xy[d.nn + nd] - yi;
#pragma unroll
        for (int v = 0; v < 4; v++) {
          double dv = b[2 * v] * ox + b[2 * v + 1] * oy;
          double pv = 1.0;
          if (dv != 0.0) {
            double dp = dv > 0.0 ? wmax[v] - Wi[v] : wmin[v] - Wi[v];
            pv = ((dp * dp + eps2) * dv + 2.0 * dv * dv * dp) / (dv * (dp * dp + 2.0 * dv * dv + dv * dp + eps2));
          }
          phi[v] = fmin(phi[v], pv);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 4; v++) d.phi[v * n + i] = phi[v];
    const double ir = __drcp_rn(Wi[0]);
    double u = Wi[1] * ir, vv = Wi[2] * ir;
    double dudy = (b[3] - u * b[1]) * ir;
    double dvdx = (b[4] - vv * b[0]) * ir;
    d.omega[i] = fabs(dvdx - dudy);
    d.Lam[i] = Lam;
    dtc = fl.cfl_exp * area / Lam;
  }
  // block minimum -> one atomic per block; every block lies inside one solve
  __shared__ double red[CELL_BLOCK / 32];
  double m = dtc;
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < CELL_BLOCK / 32 ? red[threadIdx.x] : DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0 && m < DBL_MAX) {
      int bs = d.cell_solve[blk * CELL_BLOCK];
      // positive doubles order like their bit patterns
      if (bs >= 0) atomicMin(d.dt_bits + bs, (unsigned long long)__double_as_longlong(m));
    }
  }
}

void launch_gradient(const Dev& d, cudaStream_t s) {
  k_gradient<<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
}

// Residual M_i = -(1/dt) sum over the faces of cell i (ascending face order) of the signed
// face flux (Eq. 16), the SA right-hand side Omega Sr + R (Eq. 27-28a), the SA diagonal
// without its time term, and per-block partial norms of M_rho.
__global__ void __launch_bounds__(CELL_BLOCK) k_residual(Dev d) {
  const int blk = d.g_blk0 + blockIdx.x;
  int i = blk * CELL_BLOCK + threadIdx.x, s = -1;
  bool live = cell_live(d, i, &s);
  double rmax = 0.0, r2 = 0.0;
  if (live) {
    const DevFlow& fl = d.flow[s];
    const int n = d.nc_pad, nf = d.nf;
    double dt = __longlong_as_double((long long)d.dt_bits[s]);
    double acc[5] = {0, 0, 0, 0, 0}, sad = 0.0;
    for (int k = d.cf_ptr[i]; k < d.cf_ptr[i + 1]; k++) {
      int f = d.cf_face[k];
      if (d.fL[f] == i) {
#pragma unroll
        for (int v = 0; v < 4; v++) acc[v] += d.F[v * nf + f];
        acc[4] += d.F[4 * nf + f];
        sad += d.sa_a[2 * nf + f];
      } else {
#pragma unroll
        for (int v = 0; v < 4; v++) acc[v] -= d.F[v * nf + f];
        acc[4] += d.F[5 * nf + f];
        sad += d.sa_a[3 * nf + f];
      }
    }
    const double idt = __drcp_rn(dt);
#pragma unroll
    for (int v = 0; v < 4; v++) d.M[v * n + i] = -acc[v] * idt;
    double area = d.area[i];
    const double iarea = __drcp_rn(area);
    double m4 = 0.0, fw = 0.0, sdiag = 0.0;
    if (fl.sa_on) {
      // Eq. 28a with SA-noft2 and the 2012 clipping of S~; the wall distance enters through
      // 1/d, the viscosity ratio through chi = nu~ rho / mu, and x^(1/6) is cbrt(sqrt(x))
      const double ik2 = 1.0 / (SA_KAPPA * SA_KAPPA);
      double r = d.W[i], nut = d.W[4 * n + i];
      double chi = nut * r / d.mu_l[i], c3 = chi * chi * chi;
      double fv1 = c3 * __drcp_rn(c3 + SA_CV1 * SA_CV1 * SA_CV1);
      double fv2 = 1.0 - chi * __drcp_rn(1.0 + chi * fv1);
      double om = d.omega[i], idw = __drcp_rn(d.wall_d[i]);
      double nd2 = nut * idw * idw * ik2;              // nu~ / (kappa^2 d^2)
      double Sbar = fv2 * nd2;
      double St = (Sbar >= -SA_CV2 * om)
                      ? om + Sbar
                      : om + om * (SA_CV2 * SA_CV2 * om + SA_CV3 * Sbar) / ((SA_CV3 - 2.0 * SA_CV2) * om - Sbar);
      double rr = (nd2 < 10.0 * St) ? nd2 / St : 10.0;
      double r2_ = rr * rr, r6 = r2_ * r2_ * r2_;
      double g = rr + SA_CW2 * (r6 - rr);
      double g2 = g * g, g6 = g2 * g2 * g2;
      const double c6 = SA_CW3 * SA_CW3 * SA_CW3 * SA_CW3 * SA_CW3 * SA_CW3;
      fw = g * cbrt(sqrt((1.0 + c6) * __drcp_rn(g6 + c6)));
      double nd = nut * idw;
      double Sr = SA_CB1 * St * nut - SA_CW1 * fw * nd * nd;
      m4 = area * Sr + acc[4];
      sdiag = sad + area * 2.0 * SA_CW1 * fw * nut * idw * idw;
    }
    d.M[4 * n + i] = m4;
    d.fw[i] = fw;
    d.sa_diag[i] = sdiag;
    double mr = d.M[i];
    rmax = fabs(mr);
    double q = mr * iarea;
    r2 = q * q;
  }
  __shared__ double smax[CELL_BLOCK / 32], ssum[CELL_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) { smax[threadIdx.x >> 5] = rmax; ssum[threadIdx.x >> 5] = r2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < CELL_BLOCK / 32; w++) { a = fmax(a, smax[w]); b += ssum[w]; }
    d.part[blk] = a;
    d.part[d.n_cell_blocks + blk] = b;
  }
}

void launch_residual(const Dev& d, cudaStream_t s) {
  k_residual<<<d.g_nblk, CELL_BLOCK, 0, s>>>(d);
}

// per-solve norms in fixed block order, CFL adaptation (Eq. 25), stopping rule
__global__ void k_norms(Dev d) {
  int s = d.g_solve0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.g_solve0 + d.g_nsolve) return;
  SolveState& st = d.st[s];
  if (st.state != 0) return;
  const DevFlow& fl = d.flow[s];
  double rmax = 0.0, r2 = 0.0;
  for (int b = st.blk_begin; b < st.blk_end; b++) {
    rmax = fmax(rmax, d.part[b]);
    r2 += d.part[d.n_cell_blocks + b];
  }
  st.dt = __longlong_as_double((long long)d.dt_bits[s]);
  st.res_inf = rmax;
  st.res_l2 = sqrt(r2 / (double)(st.cell_end - st.cell_begin));
  double* h = d.hist + ((size_t)s * HIST + (size_t)(st.iter % HIST)) * 2;   // residual history
  h[0] = st.res_l2;
  h[1] = st.res_inf;
  if (st.iter == 0) {
    st.cfl = fl.cfl_init;
    st.res_l2_first = st.res_l2;
  } else {
    // Eq. 25; a residual that vanished exactly makes the ratio infinite (CFL to its cap),
    // two vanishing residuals in a row leave the CFL unchanged
    double c;
    if (st.res_inf > 0.0) c = st.cfl * st.res_inf_prev / st.res_inf;
    else c = (st.res_inf_prev > 0.0) ? fl.cfl_max : st.cfl;
    st.cfl = fmin(fmax(c, fl.cfl_min), fl.cfl_max);
  }
  st.res_inf_prev = st.res_inf;
  // converged at res_target times the first residual; an exactly zero residual (also at the
  // first iteration) has nothing left to fall
  st.pending = (st.res_l2 <= fl.res_target * st.res_l2_first) ? 1 : 0;
}

void launch_norms(const Dev& d, cudaStream_t s) {
  k_norms<<<(d.g_nsolve + 63) / 64, 64, 0, s>>>(d);
}

__global__ void k_end_iter(Dev d) {
  int s = d.g_solve0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.g_solve0 + d.g_nsolve) return;
  SolveState& st = d.st[s];
  if (st.state != 0) return;
  st.eq40 = __longlong_as_double((long long)d.eq40_bits[s]);
  const double e40 = d.flow[s].eq40_target;
  if (st.pending == 0 && e40 > 0.0 && st.eq40 <= e40) st.pending = 1;   // Eq. 40 criterion
  if (d.bad[s]) st.pending = -5;   // IGKS_DIVERGED
  if (d.tmo[s]) st.pending = -6;   // IGKS_TIMEOUT: a sweep wait ran out, the state was kept
  d.tmo[s] = 0;
  st.iter += 1;
  st.state = st.pending;
  d.dt_bits[s] = 0x7FF0000000000000ull;   // +inf: the next iteration's minimum starts here
  d.eq40_bits[s] = 0ull;
  d.bad[s] = 0;
}

void launch_end_iter(const Dev& d, cudaStream_t s) {
  k_end_iter<<<(d.g_nsolve + 63) / 64, 64, 0, s>>>(d);
}

// ===================================================================================
// whole-context state upload: a staged [5][nc_pad] state is checked per solve (density
// positive, energy finite) and committed only for the solves that pass
// ===================================================================================

__global__ void k_check_state(Dev d, const double* src, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nc_pad) return;
  const int s = d.cell_solve[i];
  if (s < 0) return;
  const int n = d.nc_pad;
  if (!(src[i] > 0.0) || !isfinite(src[3 * n + i])) atomicOr(bad + s, 1);
}

__global__ void k_commit_state(Dev d, const double* src, const int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nc_pad) return;
  const int s = d.cell_solve[i];
  if (s < 0 || bad[s]) return;
  const int n = d.nc_pad;
#pragma unroll
  for (int v = 0; v < 5; v++) d.W[v * n + i] = src[v * n + i];
}

void launch_set_state(const Dev& d, const double* staged, int* bad, cudaStream_t s) {
  const int g = (d.nc_pad + CELL_BLOCK - 1) / CELL_BLOCK;
  k_check_state<<<g, CELL_BLOCK, 0, s>>>(d, staged, bad);
  k_commit_state<<<g, CELL_BLOCK, 0, s>>>(d, staged, bad);
}

}  // namespace igks
