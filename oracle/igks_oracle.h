/*
 * igks_oracle.h -- interface of the CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * The oracle is a plain, slow, single-threaded FP64 restatement of the implicit
 * gas-kinetic scheme of Pan, Zhong & Zhuo (arXiv:1709.00803). Only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. It shares no
 * code, header or table with the CUDA library: this header is the oracle's own.
 */
#ifndef IGKS_ORACLE_H
#define IGKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_flow {
  double mach, reynolds, aoa_deg, prandtl, t_ref, s_suth;
  int sa_on;
  int limiter;          /* 0 none, 1 Barth-Jespersen reading of Eq. 9, 2 Venkatakrishnan */
  double nut_ratio_inf, cfl_exp, cfl_init, cfl_min, cfl_max, res_target;
  double venkat_k, c_num;
  int visc_sr;
  int scheme;           /* 0: implicit, LU-SGS (Eq. 22); 1: explicit (Eq. 16) */
  double eq40_target;   /* if > 0: also converged when the Eq. 40 ratio is <= it */
} ora_flow;

typedef struct ora_solver ora_solver;

/* --- building blocks (pinned individually by the tests) --- */
void ora_moments_full(double U, double lam, double* m /*[10]*/);
void ora_moments_half(double U, double lam, int side /*+1: u>=0, -1: u<0*/, double* m /*[10]*/);
void ora_moments_xi(double lam, double* m /*[4]: <xi^0>,<xi^2>,<xi^4>,<xi^6>*/);
void ora_moment_matrix(double U, double V, double lam, double* M /*[16] row-major <psi_k psi_l>*/);
int  ora_moment_solve(double U, double V, double lam, const double* b /*[4]*/, double* a /*[4]*/);
void ora_time_weights(double dt, double tau, double* q /*[6]*/);
double ora_viscosity(const ora_flow* f, double lam);
int  ora_face_flux(const ora_flow* f, const double* WL, const double* WR,
                   const double* sLn, const double* sLt, const double* sRn, const double* sRt,
                   const double* WcL, const double* WcR, double dL, double dR,
                   double mut_face, double dt, double* F /*[4]*/, double* heat /*[1] or NULL*/);
void ora_euler_flux(const double* W, double nx, double ny, double* F /*[4]*/);
void ora_sa_source(double nut, double nu, double omega, double d,
                   double* out /*[6]: Sr, fw, S_tilde, r, fv1, fv2*/);

/* --- whole solver --- */
ora_solver* ora_create(int n_nodes, const double* xy, int n_cells, const int* cell_ptr,
                       const int* cell_nodes, int n_faces, const int* face_nodes,
                       const int* face_cells, const int* face_bc, const ora_flow* flow);
void ora_destroy(ora_solver* s);
void ora_init_freestream(ora_solver* s);
void ora_set_W(ora_solver* s, const double* W /*[5][N] SoA*/);
int  ora_iterate(ora_solver* s, int n_iter);   /* returns status: 0 ok, 1 converged, -5 diverged */
int  ora_get(const ora_solver* s, int which, double* out);
void ora_get_scalars(const ora_solver* s, double* out /*[ORA_NSCALARS]*/);
void ora_set_scalars(ora_solver* s, const double* in /*[ORA_NSCALARS]*/);

enum {
  ORA_W = 0,          /* [5][N]      conserved state + nu_tilde */
  ORA_GRAD = 1,       /* [4][2][N]   unlimited least-squares gradients (Eq. 7) */
  ORA_PHI = 2,        /* [4][N]      limiter factors (Eq. 9) */
  ORA_LAMBDA_F = 3,   /* [Nf]        face spectral radius */
  ORA_LAMBDA_C = 4,   /* [N]         sum of (Lambda_c)_ij over the faces of a cell */
  ORA_FLUX = 5,       /* [6][Nf]     time-integrated flux x S (4, global frame), SA face
                                     contribution to left cell, to right cell */
  ORA_RES = 6,        /* [5][N]      residual M (Eq. 16) and Omega Sr + R (Eq. 27) */
  ORA_DWSTAR = 7,     /* [5][N]      forward-sweep result */
  ORA_DW = 8,         /* [5][N]      backward-sweep result */
  ORA_GHOST = 9,      /* [5][Nf]     ghost states (zero on interior faces) */
  ORA_GEOM_CELL = 10, /* [4][N]      area, centroid x, centroid y, wall distance */
  ORA_GEOM_FACE = 11  /* [5][Nf]     length, nx, ny, midpoint x, midpoint y */
};

enum { ORA_S_DT = 0, ORA_S_CFL, ORA_S_RES_INF, ORA_S_RES_L2, ORA_S_RES_L2_FIRST,
       ORA_S_EQ40, ORA_S_ITER, ORA_S_STATUS, ORA_S_RES_INF_PREV, ORA_NSCALARS };

#ifdef __cplusplus
}
#endif
#endif
