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
  double cfl_exp, cfl_init, cfl_min, cfl_max, res_target, venkat_k, c_num, eq40_target;
  double pr_fix;   // 1/Pr - 1, the factor of the Prandtl-number fix
  int sa_on, limiter, visc_sr, scheme;
};

// per-solve iteration state, updated only on the device during iterations
constexpr int PF_E = 4;              // stencil entries held per sweep record

// static part of a narrow-sweep record: cell, entry count (-1: CSR stencil), the cell's
// backward position, and the entries' neighbours (j < 0: wall / symmetry ghost of face
// -1 - j) and shared-memory ring slots (-1: read from global memory)
struct alignas(16) FwdStat { int i, cnt, pb, pad; int j[PF_E], slot[PF_E]; };
struct alignas(16) BwdStat { int i, cnt, pad0, pad1; int j[PF_E], slot[PF_E]; };
// per-iteration part (T = double, float or double-float): forward: residual M[5], state
// (r, mx, my), 1/D, 1/a_ii, u, v, H and per entry (sx, sy, s lambda, SA coefficient);
// backward: state W[5], the same five constants, the forward increment dW*[5], entries.
// The head (up to the entries) and each entry's four coefficients are whole 16-byte
// chunks, so the pre-pass writes them with vector stores; every record is an odd number
// of chunks, so a warp reading its lanes' records from shared memory with 16-byte loads
// hits distinct banks.
template <class T>
struct alignas(16) FwdDyn {
  T m[5], w[3], c[5];
  T pad0[sizeof(T) == 4 ? 3 : 1];
  T co[PF_E][4];
  T pad1[4];
};
template <class T>
struct alignas(16) BwdDyn {
  T w[5], c[5], ws[5];
  T pad0[1];
  T co[PF_E][4];
  T pad1[sizeof(T) == 4 ? 4 : 2];
};
static_assert(sizeof(FwdStat) == 48 && sizeof(BwdStat) == 48, "static record size");
static_assert(sizeof(FwdDyn<float>) == 144 && sizeof(FwdDyn<double>) == 272, "forward record size");
static_assert(sizeof(BwdDyn<float>) == 144 && sizeof(BwdDyn<double>) == 272, "backward record size");

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
  double* pu; double* pv; double* pc;   // [nc_pad] velocity and sound speed of every cell (k_prep)
  double* lsq;              // [4][nc_pad] least-squares normal matrix A00, A01, A11 and 1/det (geometry)
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
  double* fidL; double* fidR; double* fdn; // reciprocal normal distances centre->face; centre->centre
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
  // sweep pre-pass results (type T of the sweep precision)
  void* sw_cell;                 // [5][nc_pad]: 1/D, 1/a_ii (SA), u, v, E + p
  void* sw_st;                   // [4][nnz]: signed hS nx, hS ny, hS lambda, SA coefficient
  int* sw_j;                     // [nnz] neighbour across each cell-face entry, -1 on a boundary
  int nnz;                       // entries of the cell -> face CSR
  // narrow schedule: stencils in sweep-position order (positions index fwd_order /
  // bwd_order). Forward entries are the lower neighbours, backward entries the upper
  // neighbours plus wall/symmetry ghosts (j = -1 - face). slot >= 0: the neighbour's
  // increments are still in the block's shared-memory ring at that slot.
  const int* fs_ptr; const int* fs_j; const int* fs_slot; const int* cf_to_fs;
  const int* bs_ptr; const int* bs_j; const int* bs_slot; const int* cf_to_bs;
  void* sc_f; void* sc_b;        // [4][entries] coefficients (T), written by the pre-pass
  int nfs, nbs;                  // entry counts
  // narrow schedule, per sweep position p (P = npos = all real cells): one record per
  // position and direction, array-of-structures so that a level's records are one
  // contiguous range (one bulk copy); the static part (cell, entry count, neighbours,
  // ring slots) is uploaded once, the per-iteration part written by the pre-pass. Up to
  // PF_E stencil entries per record (cnt < 0: more than that, use the CSR stencil above).
  int npos;
  const int* pos_f; const int* pos_b;            // [nc_pad] position of a cell (-1 padding)
  const FwdStat* fst; const BwdStat* bst;        // [P]
  void* fdyn; void* bdyn;                        // [P] FwdDyn<T> / BwdDyn<T>
  void* gprim;                                   // [6][nf] T: ghost r, mx, my, u, v, H of wall/symmetry faces
  const int* cf_to_ef; const int* cf_to_eb;      // [nnz] p * PF_E + e, or -1
  int wait_limit;                // spins of a device wait before it gives up (IGKS_TIMEOUT)
  int starve_test;               // test hook: the forward sweep never stages its second level
  int* tmo;                      // [n_solves] a sweep wait of the solve ran out this iteration
  // wide schedule: cells of each level of all solves
  int wide;                      // 1: one launch per level; 0: one block per solve
  int sweep_cluster;             // narrow schedule: blocks (a thread-block cluster) per solve
  const int* wfwd_cells; const int* wbwd_cells;
  const int* h_wfwd_ptr; const int* h_wbwd_ptr;   // HOST arrays of level offsets (launch sizes)
  int n_wfwd, n_wbwd;
  // per solve
  const DevFlow* flow;
  SolveState* st;
  unsigned long long* dt_bits;   // [n_solves] atomic min of the explicit time step
  unsigned long long* eq40_bits; // [n_solves] atomic max of the Eq. 40 ratio
  int* bad;                      // [n_solves] divergence flag of the current update
  double* part;                  // [2][n_blocks] residual norm partials per cell block
  double* hist;                  // [n_solves][HIST][2] residual norms of the last HIST iterations
  int n_cell_blocks;
  int flux_block;                // threads per block of the flux kernel (<= 128)
  int* err;                      // [4] device error flags (mesh orientation, area)
  // The range one launch of an iteration kernel covers: a group of consecutive solves
  // (the whole context unless the solves are split into groups that run on streams of
  // their own). Per-cell kernels take blocks [g_blk0, g_blk0 + g_nblk) of CELL_BLOCK
  // cells, per-face kernels faces [g_face0, g_face0 + g_nface), per-solve kernels and the
  // narrow sweeps solves [g_solve0, g_solve0 + g_nsolve).
  int g_blk0, g_nblk, g_face0, g_nface, g_solve0, g_nsolve;
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
void setup_sweeps();   // kernel attributes (shared-memory ring size), once per build
void launch_sweep_prep(const Dev& d, int precision, cudaStream_t s);
void launch_sweep_fwd(const Dev& d, int precision, int threads, cudaStream_t s);
void launch_sweep_bwd(const Dev& d, int precision, int threads, cudaStream_t s);
void launch_update(const Dev& d, int precision, cudaStream_t s);
void launch_end_iter(const Dev& d, cudaStream_t s);
// check a staged [5][nc_pad] state per solve (bad[s] = 1: non-physical) and copy the
// solves that pass into W
void launch_set_state(const Dev& d, const double* staged, int* bad, cudaStream_t s);
constexpr int N_KERNEL_KINDS = 11;   // kernels of one iteration (the wide sweeps launch per level)
constexpr int RING = 1024;           // shared-memory ring of the narrow sweeps (cells)
constexpr int NARROW_THREADS = 256;  // block of the narrow sweeps (one thread per cell of a level)
constexpr int DEFAULT_WAIT_LIMIT = 1 << 24;   // spins of a device wait (about a second)
constexpr int MAX_BATCH_GRAPH_ITERS = 64;     // iterations captured in one whole-batch graph at most
constexpr int WIDE_MAX_LEVELS = 64;  // automatic choice: wide schedule up to this many levels
constexpr int HIST = 1024;           // iterations of residual history kept per solve

}  // namespace igks
