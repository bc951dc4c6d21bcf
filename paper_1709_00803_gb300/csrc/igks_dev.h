// igks_dev.h -- device data layout and launch entry points shared by the translation
// units of libigks (not part of the public ABI).
//
// Layout: every solve of a context is concatenated into one set of structure-of-arrays
// buffers in HBM. Cell ranges of consecutive solves start on multiples of CELL_ALIGN so
// that every block of the per-cell kernels belongs to exactly one solve (deterministic
// per-solve reductions without atomics on floating-point sums). Cells past a solve's end
// inside its aligned range are padding (cell_solve = -1) and are skipped everywhere.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace igks {

constexpr int KDOF = 3;                                  // internal degrees of freedom (Eq. 2)
constexpr double GAMMA = (KDOF + 4.0) / (KDOF + 2.0);    // 1.4
constexpr int CELL_ALIGN = 256;
constexpr int CELL_BLOCK = 256;                          // block of the per-cell kernels

// Spalart-Allmaras (SA-noft2 with the 2012 S-tilde clipping)
constexpr double SA_CB1 = 0.1355, SA_CB2 = 0.622, SA_SIGMA = 2.0 / 3.0, SA_KAPPA = 0.41;
constexpr double SA_CW1 = SA_CB1 / (SA_KAPPA * SA_KAPPA) + (1.0 + SA_CB2) / SA_SIGMA;
constexpr double SA_CW2 = 0.3, SA_CW3 = 2.0, SA_CV1 = 7.1, SA_CV2 = 0.7, SA_CV3 = 0.9;

struct DevFlow {
  double mach, re, prandtl, s_star, lam_inf, mu_inf, nut_inf, p_inf;
  double Winf[5];
  double cfl_exp, cfl_init, cfl_min, cfl_max, res_target, venkat_k, c_num;
  int sa_on, limiter, visc_sr, pad;
};

// per-solve iteration state, updated only on the device during iterations
struct SolveState {
  double dt, cfl, res_inf, res_l2, res_l2_first, res_inf_prev, eq40;
  int iter;
  int state;      // 0 running, 1 converged, <0 error; read by every kernel of an iteration
  int pending;    // state to take at the end of the current iteration
  int blk_begin, blk_end;      // per-cell-kernel blocks of this solve
  int cell_begin, cell_end;    // [begin, end) real cells
};

struct Dev {
  int n_solves;
  int nc_pad;               // total (padded) cells
  int nf;                   // total faces
  int nbf;                  // total boundary faces
  // nodes
  const double* xy;         // [2][nn]
  int nn;
  // cells
  const int* cell_solve;    // [nc_pad], -1 for padding
  const int* cf_ptr;        // [nc_pad+1] cell -> face CSR (ascending uploaded face order)
  const int* cf_face;
  const int* cn_ptr;        // [nc_pad+1] cell -> node CSR
  const int* cn_node;
  double* area; double* cx; double* cy; double* wall_d;
  double* W;                // [5][nc_pad]
  double* grad;             // [8][nc_pad] unlimited least-squares gradients, index 2v+{x,y}
  double* phi;              // [4][nc_pad]
  double* omega;            // [nc_pad] vorticity magnitude (SA)
  double* mu_l; double* mu_t;
  double* Lam;              // [nc_pad] sum over faces of (Lambda_c)_ij
  double* M;                // [5][nc_pad]
  double* fw;               // [nc_pad]
  double* sa_diag;          // [nc_pad] SA diagonal without the Omega/dt_imp term
  void* dWs;                // [5][nc_pad] of T (sweep type)
  void* dW;                 // [5][nc_pad] of T
  void* dF;                 // [8][nc_pad] of T: increments of the x and y Euler fluxes
  // faces
  const int* fL; const int* fR; const int* fbc; const int* fsolve;
  const int* fnode;         // [2][nf] face end nodes
  const int* bface;         // [nbf] boundary face ids
  double* fS; double* fnx; double* fny; double* fmx; double* fmy;
  double* fcx; double* fcy; // centre across the face (neighbour or ghost)
  double* fdL; double* fdR; double* fdn;   // normal distances centre->face, centre->centre
  double* lam_f;            // [nf]
  double* F;                // [6][nf]
  double* sa_a;             // [4][nf]: aLR, aRL, diag L, diag R
  double* G;                // [5][nf] ghost state (boundary faces)
  double* Gmu;              // [2][nf] ghost mu_l, mu_t
  // wall faces per solve (wall distance)
  const int* wall_face; const int* wall_ptr;   // wall_ptr[n_solves+1]
  // sweep schedule
  const int* fwd_order; const int* fwd_lvl;    // cell ids in level order; level offsets
  const int* bwd_order; const int* bwd_lvl;
  const int* lvl_solve_ptr;                     // [n_solves+1] into fwd_lvl (levels per solve)
  const int* blvl_solve_ptr;                    // [n_solves+1] into bwd_lvl
  // per solve
  const DevFlow* flow;
  SolveState* st;
  unsigned long long* dt_bits;   // [n_solves] atomic min of the explicit time step
  double* part;                  // [2][n_blocks] residual norm partials per cell block
  int n_cell_blocks;
  int* err;                      // [4] device error flags (mesh orientation, area)
};

// ---- launches (igks_kernels.cu / igks_flux.cu) ----
void launch_geometry(const Dev& d, cudaStream_t s);
void launch_wall_distance(const Dev& d, cudaStream_t s);
void launch_init_state(const Dev& d, int solve, cudaStream_t s);
void launch_prep(const Dev& d, cudaStream_t s);
void launch_ghost(const Dev& d, cudaStream_t s);
void launch_gradient(const Dev& d, cudaStream_t s);
void launch_flux(const Dev& d, cudaStream_t s);
void launch_residual(const Dev& d, cudaStream_t s);
void launch_norms(const Dev& d, cudaStream_t s);
void launch_sweep_fwd(const Dev& d, int precision, int threads, cudaStream_t s);
void launch_sweep_bwd(const Dev& d, int precision, int threads, cudaStream_t s);
void launch_end_iter(const Dev& d, cudaStream_t s);
constexpr int LAUNCHES_PER_ITER = 9;

}  // namespace igks
