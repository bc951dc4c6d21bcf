/*
 * igks_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of one steady iteration of the
 * implicit gas-kinetic scheme (IGKS) of Pan, Zhong & Zhuo, arXiv:1709.00803:
 *   Section II.A (Eq. 1-14)   BGK-NS gas-kinetic interface flux on an unstructured mesh,
 *   Section II.B (Eq. 15-25)  residual, matrix-free LU-SGS, time steps, CFL adaptation,
 *   Section II.C (Eq. 26-34)  Spalart-Allmaras source/fluxes and the turbulent tau,
 *   Section II.E              ghost-cell boundary conditions (values and increments).
 * Each step follows the paper's order and notation; where the paper is silent the
 * reading taken is stated at the step. There is no blocking, fusion or reordering: the
 * flux integrals are evaluated literally as moments of expanded polynomials in
 * (u, v, xi^2) against the Maxwellians of Eq. 2, and every linear system of Eq. 101,
 * 11 and 12 is solved by Gaussian elimination of its explicit 4x4 moment matrix, as the
 * paper states.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * this file. It shares no code with the CUDA library. Build with -ffp-contract=off.
 */
#include "igks_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KDOF 3                                  /* internal degrees of freedom (Eq. 2) */
#define GAMMA ((KDOF + 4.0) / (KDOF + 2.0))     /* 1.4 */
#define NMOM 10
#define PI_ 3.14159265358979323846

/* ===================================================================================
 * Maxwellian moments (Eq. 2).  <.> denotes (1/rho) * integral of (.) g dXi.
 * =================================================================================== */

/* <u^n> over the whole velocity space for a Maxwellian with mean U and lambda. */
void ora_moments_full(double U, double lam, double* m) {
  m[0] = 1.0;
  m[1] = U;
  for (int n = 0; n + 2 < NMOM; n++) m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

/* <u^n> over the half space u >= 0 (side = +1, H[u] = 1 incl. u = 0) or u < 0 (side = -1). */
void ora_moments_half(double U, double lam, int side, double* m) {
  double s = sqrt(lam);
  double e = exp(-lam * U * U) / sqrt(PI_ * lam);
  if (side > 0) {
    m[0] = 0.5 * erfc(-s * U);
    m[1] = U * m[0] + 0.5 * e;
  } else {
    m[0] = 0.5 * erfc(s * U);
    m[1] = U * m[0] - 0.5 * e;
  }
  for (int n = 0; n + 2 < NMOM; n++) m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

/* <xi^(2k)>, k = 0..3, for K internal components each of variance 1/(2 lambda). */
void ora_moments_xi(double lam, double* m) {
  double s2 = 1.0 / (2.0 * lam);
  m[0] = 1.0;
  m[1] = KDOF * s2;
  m[2] = KDOF * (KDOF + 2.0) * s2 * s2;
  m[3] = KDOF * (KDOF + 2.0) * (KDOF + 4.0) * s2 * s2 * s2;
}

/* ===================================================================================
 * Sparse polynomials in (u, v, xi^2): sum_k c_k u^pu v^pv (xi^2)^px.
 * =================================================================================== */
#define MAXT 512
typedef struct {
  int n;
  double c[MAXT];
  unsigned char pu[MAXT], pv[MAXT], px[MAXT];
} poly;

static void poly_zero(poly* p) { p->n = 0; }

static void poly_term(poly* p, double c, int pu, int pv, int px) {
  if (c == 0.0) return;
  if (p->n >= MAXT) abort();
  p->c[p->n] = c;
  p->pu[p->n] = (unsigned char)pu;
  p->pv[p->n] = (unsigned char)pv;
  p->px[p->n] = (unsigned char)px;
  p->n++;
}

/* psi_k of Eq. 101: (1, u, v, (u^2 + v^2 + xi^2)/2) */
static void poly_psi(poly* p, int k) {
  poly_zero(p);
  switch (k) {
    case 0: poly_term(p, 1.0, 0, 0, 0); break;
    case 1: poly_term(p, 1.0, 1, 0, 0); break;
    case 2: poly_term(p, 1.0, 0, 1, 0); break;
    default:
      poly_term(p, 0.5, 2, 0, 0);
      poly_term(p, 0.5, 0, 2, 0);
      poly_term(p, 0.5, 0, 0, 1);
  }
}

/* Taylor form of Eq. (100): a1 + a2 u + a3 v + a4 (u^2 + v^2 + xi^2)/2 */
static void poly_slope(poly* p, const double* a) {
  poly_zero(p);
  poly_term(p, a[0], 0, 0, 0);
  poly_term(p, a[1], 1, 0, 0);
  poly_term(p, a[2], 0, 1, 0);
  poly_term(p, 0.5 * a[3], 2, 0, 0);
  poly_term(p, 0.5 * a[3], 0, 2, 0);
  poly_term(p, 0.5 * a[3], 0, 0, 1);
}

static void poly_mul(poly* out, const poly* a, const poly* b) {
  poly r;
  poly_zero(&r);
  for (int i = 0; i < a->n; i++)
    for (int j = 0; j < b->n; j++)
      poly_term(&r, a->c[i] * b->c[j], a->pu[i] + b->pu[j], a->pv[i] + b->pv[j], a->px[i] + b->px[j]);
  *out = r;
}

static void poly_add(poly* y, double s, const poly* x) {
  for (int i = 0; i < x->n; i++) poly_term(y, s * x->c[i], x->pu[i], x->pv[i], x->px[i]);
}

/* multiply by u or v */
static void poly_shift(poly* out, const poly* a, int du, int dv) {
  poly r;
  poly_zero(&r);
  for (int i = 0; i < a->n; i++) poly_term(&r, a->c[i], a->pu[i] + du, a->pv[i] + dv, a->px[i]);
  *out = r;
}

/* moment of a polynomial: sum_k c_k <u^pu> <v^pv> <xi^(2 px)> */
static double poly_moment(const poly* p, const double* mu, const double* mv, const double* mx) {
  double s = 0.0;
  for (int i = 0; i < p->n; i++) {
    if (p->pu[i] >= NMOM || p->pv[i] >= NMOM || p->px[i] > 3) abort();
    s += p->c[i] * mu[p->pu[i]] * mv[p->pv[i]] * mx[p->px[i]];
  }
  return s;
}

/* A Maxwellian seen as a set of moment tables. */
typedef struct {
  double rho, U, V, lam;
  double mu[NMOM], mv[NMOM], mx[4];    /* full moments */
  double mup[NMOM], mun[NMOM];         /* half-space u moments, u >= 0 and u < 0 */
  double M[16];                        /* moment matrix <psi_k psi_l> of Eq. 101 */
} maxw;

void ora_moment_matrix(double U, double V, double lam, double* M);

static void maxw_set(maxw* g, double rho, double U, double V, double lam) {
  g->rho = rho; g->U = U; g->V = V; g->lam = lam;
  ora_moments_full(U, lam, g->mu);
  ora_moments_full(V, lam, g->mv);
  ora_moments_xi(lam, g->mx);
  ora_moments_half(U, lam, +1, g->mup);
  ora_moments_half(U, lam, -1, g->mun);
  ora_moment_matrix(U, V, lam, g->M);
}

/* <p> with half = 0 (full), +1 (u >= 0), -1 (u < 0) */
static double maxw_moment(const maxw* g, const poly* p, int half) {
  const double* mu = half > 0 ? g->mup : (half < 0 ? g->mun : g->mu);
  return poly_moment(p, mu, g->mv, g->mx);
}

/* ===================================================================================
 * Linear systems of Eq. 101 / 11 / 12: <a psi> = b, solved by Gaussian elimination of
 * the explicit moment matrix M_kl = <psi_k psi_l>.
 * =================================================================================== */
void ora_moment_matrix(double U, double V, double lam, double* M) {
  double mu[NMOM], mv[NMOM], mx[4];
  ora_moments_full(U, lam, mu);
  ora_moments_full(V, lam, mv);
  ora_moments_xi(lam, mx);
  for (int k = 0; k < 4; k++)
    for (int l = 0; l < 4; l++) {
      poly pk, pl, prod;
      poly_psi(&pk, k);
      poly_psi(&pl, l);
      poly_mul(&prod, &pk, &pl);
      M[4 * k + l] = poly_moment(&prod, mu, mv, mx);
    }
}

static int gauss_solve4(double* A, double* b, double* x) {
  int piv[4] = {0, 1, 2, 3};
  for (int c = 0; c < 4; c++) {
    int best = c;
    for (int r = c + 1; r < 4; r++)
      if (fabs(A[4 * piv[r] + c]) > fabs(A[4 * piv[best] + c])) best = r;
    int t = piv[c]; piv[c] = piv[best]; piv[best] = t;
    double d = A[4 * piv[c] + c];
    if (d == 0.0) return -1;
    for (int r = c + 1; r < 4; r++) {
      double f = A[4 * piv[r] + c] / d;
      for (int k = c; k < 4; k++) A[4 * piv[r] + k] -= f * A[4 * piv[c] + k];
      b[piv[r]] -= f * b[piv[c]];
    }
  }
  for (int c = 3; c >= 0; c--) {
    double s = b[piv[c]];
    for (int k = c + 1; k < 4; k++) s -= A[4 * piv[c] + k] * x[k];
    x[c] = s / A[4 * piv[c] + c];
  }
  return 0;
}

int ora_moment_solve(double U, double V, double lam, const double* b, double* a) {
  double M[16], rhs[4];
  ora_moment_matrix(U, V, lam, M);
  memcpy(rhs, b, sizeof rhs);
  return gauss_solve4(M, rhs, a);
}

/* ===================================================================================
 * Time integrals over [0, dt] of the six time weights of Eq. 13.
 *  q0 = int (1 - e^{-t/tau})            q1 = int (tau(-1 + e^{-t/tau}) + t e^{-t/tau})
 *  q2 = int tau(t/tau - 1 + e^{-t/tau}) q3 = int e^{-t/tau}
 *  q4 = int -(t + tau) e^{-t/tau}       q5 = int -tau e^{-t/tau}
 * =================================================================================== */
void ora_time_weights(double dt, double tau, double* q) {
  double x = dt / tau;
  double one_m_e = -expm1(-x);   /* 1 - e^{-dt/tau} */
  double e = exp(-x);
  q[0] = dt - tau * one_m_e;
  q[1] = 2.0 * tau * tau * one_m_e - tau * dt * (1.0 + e);
  q[2] = 0.5 * dt * dt - tau * dt + tau * tau * one_m_e;
  q[3] = tau * one_m_e;
  q[4] = -2.0 * tau * tau * one_m_e + tau * dt * e;
  q[5] = -tau * tau * one_m_e;
}

/* Sutherland's law relative to the free stream; T/T_inf = lambda_inf / lambda. */
double ora_viscosity(const ora_flow* f, double lam) {
  double lam_inf = GAMMA * f->mach * f->mach / 2.0;
  double tr = lam_inf / lam;
  double s = f->s_suth / f->t_ref;
  return (1.0 / f->reynolds) * tr * sqrt(tr) * (1.0 + s) / (tr + s);
}

/* primitive (rho, U, V, lambda) of a conserved state (rho, rho U, rho V, rho E) */
static void primitives(const double* W, double* rho, double* U, double* V, double* lam) {
  *rho = W[0];
  *U = W[1] / W[0];
  *V = W[2] / W[0];
  *lam = (KDOF + 2.0) * W[0] / (4.0 * (W[3] - 0.5 * W[0] * ((*U) * (*U) + (*V) * (*V))));
}

/* <a psi>_g = b by Gaussian elimination of g's moment matrix */
static int solve_about(const maxw* g, const double* b, double* a) {
  double M[16], rhs[4];
  memcpy(M, g->M, sizeof M);
  memcpy(rhs, b, sizeof rhs);
  return gauss_solve4(M, rhs, a);
}

/* Slope of Eq. 101 about Maxwellian g: solve <a psi>_g = dW / rho_g. */
static int slope_from(const maxw* g, const double* dW, double* a) {
  double b[4];
  for (int k = 0; k < 4; k++) b[k] = dW[k] / g->rho;
  return solve_about(g, b, a);
}

/* b_k = < P psi_k > over half-space `half` of g */
static void moments_psi(const maxw* g, const poly* P, int half, double* out) {
  for (int k = 0; k < 4; k++) {
    poly pk, prod;
    poly_psi(&pk, k);
    poly_mul(&prod, P, &pk);
    out[k] = maxw_moment(g, &prod, half);
  }
}

/* ===================================================================================
 * Interface flux, Eq. 4-14, in the face frame (x along the unit normal n from left to
 * right, y along t = (-n_y, n_x)). Inputs are conserved states with the momentum
 * rotated into that frame: face states W_L, W_R (Eq. 10), their limited normal and
 * tangential slopes, the centre states of the two cells (ghost on a boundary), their
 * normal distances to the face, the face eddy viscosity and the flux time step dt.
 * Output: F = int_0^dt int u psi f_cf (Eq. 14), with the Prandtl-number fix on F_E.
 * =================================================================================== */

typedef struct {
  maxw gl, gr, g0;
  double anl[4], atl[4], anr[4], atr[4], Al[4], Ar[4];   /* Eq. 4 slopes */
  double abl[4], abr[4], abt[4], Ab[4];                  /* Eq. 5 slopes */
  double q[6];
} face_state;

/* int_0^dt int w f_cf dXi dt for a weight polynomial w: the six lines of Eq. 13. */
static double fcf_integral(const face_state* s, const poly* w) {
  poly t, P, Q;
  double r = 0.0;
  /* line 1: (1 - e^{-t/tau}) g0 */
  r += s->q[0] * s->g0.rho * maxw_moment(&s->g0, w, 0);
  /* line 2: (abar_n^l H[u] + abar_n^r (1-H[u])) u + abar_t v, times g0 */
  poly_slope(&t, s->abl); poly_shift(&P, &t, 1, 0); poly_mul(&Q, w, &P);
  double l2 = maxw_moment(&s->g0, &Q, +1);
  poly_slope(&t, s->abr); poly_shift(&P, &t, 1, 0); poly_mul(&Q, w, &P);
  l2 += maxw_moment(&s->g0, &Q, -1);
  poly_slope(&t, s->abt); poly_shift(&P, &t, 0, 1); poly_mul(&Q, w, &P);
  l2 += maxw_moment(&s->g0, &Q, 0);
  r += s->q[1] * s->g0.rho * l2;
  /* line 3: Abar g0 */
  poly_slope(&t, s->Ab); poly_mul(&Q, w, &t);
  r += s->q[2] * s->g0.rho * maxw_moment(&s->g0, &Q, 0);
  /* lines 4-5: e^{-t/tau} (1 - (t + tau)(u a_n + v a_t)) H g^l, and the same for g^r */
  r += s->q[3] * (s->gl.rho * maxw_moment(&s->gl, w, +1) + s->gr.rho * maxw_moment(&s->gr, w, -1));
  {
    poly an, at, sum, Pn, Pt;
    poly_slope(&an, s->anl); poly_shift(&Pn, &an, 1, 0);
    poly_slope(&at, s->atl); poly_shift(&Pt, &at, 0, 1);
    poly_zero(&sum); poly_add(&sum, 1.0, &Pn); poly_add(&sum, 1.0, &Pt);
    poly_mul(&Q, w, &sum);
    double l4 = s->gl.rho * maxw_moment(&s->gl, &Q, +1);
    poly_slope(&an, s->anr); poly_shift(&Pn, &an, 1, 0);
    poly_slope(&at, s->atr); poly_shift(&Pt, &at, 0, 1);
    poly_zero(&sum); poly_add(&sum, 1.0, &Pn); poly_add(&sum, 1.0, &Pt);
    poly_mul(&Q, w, &sum);
    l4 += s->gr.rho * maxw_moment(&s->gr, &Q, -1);
    r += s->q[4] * l4;
  }
  /* line 6: e^{-t/tau} (-tau A^l H g^l - tau A^r (1-H) g^r) */
  poly_slope(&t, s->Al); poly_mul(&Q, w, &t);
  double l6 = s->gl.rho * maxw_moment(&s->gl, &Q, +1);
  poly_slope(&t, s->Ar); poly_mul(&Q, w, &t);
  l6 += s->gr.rho * maxw_moment(&s->gr, &Q, -1);
  r += s->q[5] * l6;
  return r;
}

/* time derivative A of Eq. 11: <(a_n u + a_t v + A) psi>_g = 0 */
static int time_slope(const maxw* g, const double* an, const double* at, double* A) {
  poly pa, pb, sum, Pn, Pt;
  double b[4], mom[4];
  poly_slope(&pa, an); poly_shift(&Pn, &pa, 1, 0);
  poly_slope(&pb, at); poly_shift(&Pt, &pb, 0, 1);
  poly_zero(&sum); poly_add(&sum, 1.0, &Pn); poly_add(&sum, 1.0, &Pt);
  moments_psi(g, &sum, 0, mom);
  for (int k = 0; k < 4; k++) b[k] = -mom[k];
  return solve_about(g, b, A);
}

int ora_face_flux(const ora_flow* f, const double* WL, const double* WR,
                  const double* sLn, const double* sLt, const double* sRn, const double* sRt,
                  const double* WcL, const double* WcR, double dL, double dR,
                  double mut_face, double dt, double* F, double* heat) {
  face_state s;
  double rho, U, V, lam;
  int err = 0;
  /* Maxwellians g^l, g^r of the reconstructed face states (Eq. 4) */
  primitives(WL, &rho, &U, &V, &lam);
  maxw_set(&s.gl, rho, U, V, lam);
  primitives(WR, &rho, &U, &V, &lam);
  maxw_set(&s.gr, rho, U, V, lam);
  if (!(s.gl.lam > 0 && s.gr.lam > 0 && s.gl.rho > 0 && s.gr.rho > 0)) return -1;
  /* non-equilibrium slopes a_n, a_t from Eq. 101, time slopes A from Eq. 11 */
  err |= slope_from(&s.gl, sLn, s.anl);
  err |= slope_from(&s.gl, sLt, s.atl);
  err |= slope_from(&s.gr, sRn, s.anr);
  err |= slope_from(&s.gr, sRt, s.atr);
  err |= time_slope(&s.gl, s.anl, s.atl, s.Al);
  err |= time_slope(&s.gr, s.anr, s.atr, s.Ar);
  /* equilibrium state at the interface: W0 = int psi (g^l H + g^r (1-H)) */
  double W0[4], ml[4], mr[4];
  {
    poly one;
    poly_zero(&one); poly_term(&one, 1.0, 0, 0, 0);
    moments_psi(&s.gl, &one, +1, ml);
    moments_psi(&s.gr, &one, -1, mr);
    for (int k = 0; k < 4; k++) W0[k] = s.gl.rho * ml[k] + s.gr.rho * mr[k];
  }
  primitives(W0, &rho, &U, &V, &lam);
  maxw_set(&s.g0, rho, U, V, lam);
  if (!(s.g0.lam > 0 && s.g0.rho > 0)) return -1;
  /* equilibrium slopes of Eq. 5: normal ones from the centre-to-interface differences on
   * each side, tangential one from the mean of the two limited tangential slopes */
  {
    double dl[4], dr[4], dt_[4];
    for (int k = 0; k < 4; k++) {
      dl[k] = (W0[k] - WcL[k]) / dL;
      dr[k] = (WcR[k] - W0[k]) / dR;
      dt_[k] = 0.5 * (sLt[k] + sRt[k]);
    }
    err |= slope_from(&s.g0, dl, s.abl);
    err |= slope_from(&s.g0, dr, s.abr);
    err |= slope_from(&s.g0, dt_, s.abt);
  }
  /* Abar from the compatibility condition (Eq. 12), in its standard reduced form:
   * <(abar_n^l u H + abar_n^r u (1-H) + abar_t v + Abar) psi>_{g0} = 0 */
  {
    double b[4], m1[4], m2[4], m3[4];
    poly t, P;
    poly_slope(&t, s.abl); poly_shift(&P, &t, 1, 0); moments_psi(&s.g0, &P, +1, m1);
    poly_slope(&t, s.abr); poly_shift(&P, &t, 1, 0); moments_psi(&s.g0, &P, -1, m2);
    poly_slope(&t, s.abt); poly_shift(&P, &t, 0, 1); moments_psi(&s.g0, &P, 0, m3);
    for (int k = 0; k < 4; k++) b[k] = -(m1[k] + m2[k] + m3[k]);
    err |= solve_about(&s.g0, b, s.Ab);
  }
  if (err) return -2;
  /* collision time: tau = (mu_l + mu_t)/p (Eq. 33-34) plus the pressure-jump term */
  double p0 = s.g0.rho / (2.0 * s.g0.lam);
  double pl = s.gl.rho / (2.0 * s.gl.lam), pr = s.gr.rho / (2.0 * s.gr.lam);
  double tau = (ora_viscosity(f, s.g0.lam) + mut_face) / p0 + f->c_num * fabs(pl - pr) / (pl + pr) * dt;
  ora_time_weights(dt, tau, s.q);
  /* Eq. 14: F_k = int int u psi_k f_cf */
  for (int k = 0; k < 4; k++) {
    poly pk, w;
    poly_psi(&pk, k);
    poly_shift(&w, &pk, 1, 0);
    F[k] = fcf_integral(&s, &w);
  }
  /* Prandtl fix: heat flux q = int int (u-U0)((u-U0)^2 + (v-V0)^2 + xi^2)/2 f_cf,
   * F_E += (1/Pr - 1) q */
  {
    double U0 = s.g0.U, V0 = s.g0.V;
    poly du, c2, w, tmp;
    poly_zero(&du); poly_term(&du, 1.0, 1, 0, 0); poly_term(&du, -U0, 0, 0, 0);
    poly_zero(&c2);
    poly_term(&c2, 1.0, 2, 0, 0); poly_term(&c2, -2.0 * U0, 1, 0, 0); poly_term(&c2, U0 * U0, 0, 0, 0);
    poly_term(&c2, 1.0, 0, 2, 0); poly_term(&c2, -2.0 * V0, 0, 1, 0); poly_term(&c2, V0 * V0, 0, 0, 0);
    poly_term(&c2, 1.0, 0, 0, 1);
    poly_mul(&tmp, &du, &c2);
    poly_zero(&w); poly_add(&w, 0.5, &tmp);
    double q = fcf_integral(&s, &w);
    if (heat) *heat = q;
    F[3] += (1.0 / f->prandtl - 1.0) * q;
  }
  return 0;
}

/* Inviscid flux F_E(W).n used by the matrix-free LU-SGS increments (Eq. 20). */
void ora_euler_flux(const double* W, double nx, double ny, double* F) {
  double rho = W[0], u = W[1] / rho, v = W[2] / rho;
  double p = (GAMMA - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
  double vn = u * nx + v * ny;
  F[0] = rho * vn;
  F[1] = W[1] * vn + p * nx;
  F[2] = W[2] * vn + p * ny;
  F[3] = (W[3] + p) * vn;
}

/* ===================================================================================
 * Solver.
 * =================================================================================== */

/* Spalart-Allmaras constants (SA-noft2 with the 2012 clipping of S-tilde); the paper
 * defers the model's constants to its reference. */
#define SA_CB1 0.1355
#define SA_CB2 0.622
#define SA_SIGMA (2.0 / 3.0)
#define SA_KAPPA 0.41
#define SA_CW1 (SA_CB1 / (SA_KAPPA * SA_KAPPA) + (1.0 + SA_CB2) / SA_SIGMA)
#define SA_CW2 0.3
#define SA_CW3 2.0
#define SA_CV1 7.1
#define SA_CV2 0.7
#define SA_CV3 0.9

struct ora_solver {
  ora_flow flow;
  int n_nodes, n_cells, n_faces;
  double* xy;
  int *cell_ptr, *cell_nodes;
  int *face_nodes, *face_cells, *face_bc;
  /* cell -> face lists in ascending face order */
  int *cf_ptr, *cf_face;
  /* geometry */
  double *area, *cx, *cy, *wall_d;
  double *fS, *fnx, *fny, *fmx, *fmy;
  double *gx, *gy;          /* centre of the cell across each face (ghost centre on a boundary) */
  /* state and work arrays, AoS per cell */
  double* W;                /* [N][5] */
  double* G;                /* [Nf][5] ghost state */
  double* grad;             /* [N][4][2] unlimited */
  double* phi;              /* [N][4] */
  double* lam_f;            /* [Nf] */
  double* Lam;              /* [N] */
  double* F;                /* [Nf][6] */
  double* M;                /* [N][5] */
  double* fw;               /* [N] */
  double* dWs;              /* [N][5] */
  double* dW;               /* [N][5] */
  double dt, cfl, res_inf, res_l2, res_l2_first, eq40, res_inf_prev;
  int iter, status;
};

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }
static int* ialloc(size_t n) { return (int*)calloc(n ? n : 1, sizeof(int)); }

static void freestream(const ora_flow* f, double* W) {
  double a = f->aoa_deg * PI_ / 180.0;
  double u = cos(a), v = sin(a), p = 1.0 / (GAMMA * f->mach * f->mach);
  W[0] = 1.0;
  W[1] = u;
  W[2] = v;
  W[3] = p / (GAMMA - 1.0) + 0.5 * (u * u + v * v);
  W[4] = f->sa_on ? f->nut_ratio_inf / f->reynolds : 0.0;
}

static double pressure(const double* W) {
  return (GAMMA - 1.0) * (W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0]);
}

/* lambda = rho / (2 p) */
static double lambda_of(const double* W) { return W[0] / (2.0 * pressure(W)); }

static double seg_dist(double px, double py, double ax, double ay, double bx, double by) {
  double dx = bx - ax, dy = by - ay;
  double t = ((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy);
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  double qx = ax + t * dx - px, qy = ay + t * dy - py;
  return sqrt(qx * qx + qy * qy);
}

ora_solver* ora_create(int n_nodes, const double* xy, int n_cells, const int* cell_ptr,
                       const int* cell_nodes, int n_faces, const int* face_nodes,
                       const int* face_cells, const int* face_bc, const ora_flow* flow) {
  ora_solver* s = (ora_solver*)calloc(1, sizeof(ora_solver));
  s->flow = *flow;
  s->n_nodes = n_nodes; s->n_cells = n_cells; s->n_faces = n_faces;
  s->xy = dalloc(2 * (size_t)n_nodes); memcpy(s->xy, xy, sizeof(double) * 2 * n_nodes);
  s->cell_ptr = ialloc(n_cells + 1); memcpy(s->cell_ptr, cell_ptr, sizeof(int) * (n_cells + 1));
  s->cell_nodes = ialloc(cell_ptr[n_cells]); memcpy(s->cell_nodes, cell_nodes, sizeof(int) * cell_ptr[n_cells]);
  s->face_nodes = ialloc(2 * n_faces); memcpy(s->face_nodes, face_nodes, sizeof(int) * 2 * n_faces);
  s->face_cells = ialloc(2 * n_faces); memcpy(s->face_cells, face_cells, sizeof(int) * 2 * n_faces);
  s->face_bc = ialloc(n_faces); memcpy(s->face_bc, face_bc, sizeof(int) * n_faces);
  /* cell -> faces, ascending face index */
  s->cf_ptr = ialloc(n_cells + 1);
  for (int f = 0; f < n_faces; f++) {
    s->cf_ptr[face_cells[2 * f] + 1]++;
    if (face_cells[2 * f + 1] >= 0) s->cf_ptr[face_cells[2 * f + 1] + 1]++;
  }
  for (int i = 0; i < n_cells; i++) s->cf_ptr[i + 1] += s->cf_ptr[i];
  s->cf_face = ialloc(s->cf_ptr[n_cells]);
  {
    int* fill = ialloc(n_cells);
    for (int f = 0; f < n_faces; f++) {
      int l = face_cells[2 * f], r = face_cells[2 * f + 1];
      s->cf_face[s->cf_ptr[l] + fill[l]++] = f;
      if (r >= 0) s->cf_face[s->cf_ptr[r] + fill[r]++] = f;
    }
    free(fill);
  }
  /* cell area and centroid of the polygon */
  s->area = dalloc(n_cells); s->cx = dalloc(n_cells); s->cy = dalloc(n_cells); s->wall_d = dalloc(n_cells);
  for (int i = 0; i < n_cells; i++) {
    double a = 0, sx = 0, sy = 0;
    int b = cell_ptr[i], e = cell_ptr[i + 1];
    for (int k = b; k < e; k++) {
      int p = cell_nodes[k], q = cell_nodes[k + 1 < e ? k + 1 : b];
      double x0 = xy[2 * p], y0 = xy[2 * p + 1], x1 = xy[2 * q], y1 = xy[2 * q + 1];
      double c = x0 * y1 - x1 * y0;
      a += c;
      sx += (x0 + x1) * c;
      sy += (y0 + y1) * c;
    }
    a *= 0.5;
    s->area[i] = a;
    s->cx[i] = sx / (6.0 * a);
    s->cy[i] = sy / (6.0 * a);
  }
  /* faces: length, unit normal (right-hand normal of a->b, out of the left cell), midpoint */
  s->fS = dalloc(n_faces); s->fnx = dalloc(n_faces); s->fny = dalloc(n_faces);
  s->fmx = dalloc(n_faces); s->fmy = dalloc(n_faces); s->gx = dalloc(n_faces); s->gy = dalloc(n_faces);
  for (int f = 0; f < n_faces; f++) {
    int a = face_nodes[2 * f], b = face_nodes[2 * f + 1];
    double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
    double S = sqrt(dx * dx + dy * dy);
    s->fS[f] = S;
    s->fnx[f] = dy / S;
    s->fny[f] = -dx / S;
    s->fmx[f] = 0.5 * (xy[2 * a] + xy[2 * b]);
    s->fmy[f] = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]);
    int l = face_cells[2 * f], r = face_cells[2 * f + 1];
    if (r >= 0) {
      s->gx[f] = s->cx[r];
      s->gy[f] = s->cy[r];
    } else {
      /* ghost centre: mirror image of the interior centre across the face line */
      double d = (s->fmx[f] - s->cx[l]) * s->fnx[f] + (s->fmy[f] - s->cy[l]) * s->fny[f];
      s->gx[f] = s->cx[l] + 2.0 * d * s->fnx[f];
      s->gy[f] = s->cy[l] + 2.0 * d * s->fny[f];
    }
  }
  /* wall distance for the SA model: brute force over the wall faces */
  for (int i = 0; i < n_cells; i++) {
    double dmin = 1e300;
    for (int f = 0; f < n_faces; f++) {
      if (face_bc[f] != 3 && face_bc[f] != 5) continue;
      int a = face_nodes[2 * f], b = face_nodes[2 * f + 1];
      double d = seg_dist(s->cx[i], s->cy[i], xy[2 * a], xy[2 * a + 1], xy[2 * b], xy[2 * b + 1]);
      if (d < dmin) dmin = d;
    }
    s->wall_d[i] = dmin;
  }
  s->W = dalloc(5 * (size_t)n_cells);
  s->G = dalloc(5 * (size_t)n_faces);
  s->grad = dalloc(8 * (size_t)n_cells);
  s->phi = dalloc(4 * (size_t)n_cells);
  s->lam_f = dalloc(n_faces);
  s->Lam = dalloc(n_cells);
  s->F = dalloc(6 * (size_t)n_faces);
  s->M = dalloc(5 * (size_t)n_cells);
  s->fw = dalloc(n_cells);
  s->dWs = dalloc(5 * (size_t)n_cells);
  s->dW = dalloc(5 * (size_t)n_cells);
  ora_init_freestream(s);
  return s;
}

void ora_destroy(ora_solver* s) {
  if (!s) return;
  void* ptrs[] = {s->xy, s->cell_ptr, s->cell_nodes, s->face_nodes, s->face_cells, s->face_bc,
                  s->cf_ptr, s->cf_face, s->area, s->cx, s->cy, s->wall_d, s->fS, s->fnx, s->fny,
                  s->fmx, s->fmy, s->gx, s->gy, s->W, s->G, s->grad, s->phi, s->lam_f, s->Lam,
                  s->F, s->M, s->fw, s->dWs, s->dW};
  for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; k++) free(ptrs[k]);
  free(s);
}

void ora_init_freestream(ora_solver* s) {
  double Wf[5];
  freestream(&s->flow, Wf);
  for (int i = 0; i < s->n_cells; i++) memcpy(s->W + 5 * i, Wf, sizeof Wf);
  s->iter = 0; s->status = 0; s->cfl = s->flow.cfl_init;
  s->res_inf_prev = 0; s->res_l2_first = 0;
}

void ora_set_W(ora_solver* s, const double* W) {
  for (int i = 0; i < s->n_cells; i++)
    for (int v = 0; v < 5; v++) s->W[5 * i + v] = W[(size_t)v * s->n_cells + i];
}

/* laminar kinematic viscosity and eddy viscosity mu_t = rho nu_tilde fv1 (Eq. 34) */
static double nu_lam(const ora_solver* s, const double* W) { return ora_viscosity(&s->flow, lambda_of(W)) / W[0]; }

static double mu_turb(const ora_solver* s, const double* W) {
  if (!s->flow.sa_on || W[4] <= 0.0) return 0.0;
  double chi = W[4] / nu_lam(s, W);
  double c3 = chi * chi * chi;
  return W[0] * W[4] * c3 / (c3 + SA_CV1 * SA_CV1 * SA_CV1);
}

/* ----- Section II.E: ghost state of a boundary face from the interior centre state ---- */
static void ghost_state(const ora_solver* s, int f, const double* Wi, double* Wg) {
  double nx = s->fnx[f], ny = s->fny[f];
  int bc = s->face_bc[f];
  if (bc == 3) {                /* non-slip wall: momentum and nu_tilde change sign */
    Wg[0] = Wi[0]; Wg[1] = -Wi[1]; Wg[2] = -Wi[2]; Wg[3] = Wi[3]; Wg[4] = -Wi[4];
  } else if (bc == 5) {         /* non-slip wall moving with the tangential part of the free-stream
                                   velocity: the ghost velocity mirrors the inside one about the
                                   wall velocity, same density and internal energy, nu_tilde sign */
    double Wf[5];
    freestream(&s->flow, Wf);
    double tx = -ny, ty = nx;
    double uw = (Wf[1] * tx + Wf[2] * ty) / Wf[0];
    double r = Wi[0], u = Wi[1] / r, v = Wi[2] / r;
    double ug = 2.0 * uw * tx - u, vg = 2.0 * uw * ty - v;
    Wg[0] = r; Wg[1] = r * ug; Wg[2] = r * vg;
    Wg[3] = Wi[3] - 0.5 * r * (u * u + v * v) + 0.5 * r * (ug * ug + vg * vg);
    Wg[4] = -Wi[4];
  } else if (bc == 2) {         /* symmetry: normal momentum changes sign */
    double mn = Wi[1] * nx + Wi[2] * ny;
    Wg[0] = Wi[0]; Wg[1] = Wi[1] - 2.0 * mn * nx; Wg[2] = Wi[2] - 2.0 * mn * ny; Wg[3] = Wi[3]; Wg[4] = Wi[4];
  } else if (bc == 4) {         /* outflow (Section II.E): the boundary-normal velocity is half the
                                   sum of the Riemann invariants R+ (inside) and R- (free stream);
                                   density, tangential velocity, temperature (lambda) and nu_tilde
                                   are the inside values */
    double Wf[5];
    freestream(&s->flow, Wf);
    double g = GAMMA;
    double ri = Wi[0], ui = Wi[1] / ri, vi = Wi[2] / ri, ci = sqrt(g * pressure(Wi) / ri);
    double co = sqrt(g * pressure(Wf) / Wf[0]);
    double uni = ui * nx + vi * ny, uno = (Wf[1] * nx + Wf[2] * ny) / Wf[0];
    double Rp = uni + 2.0 * ci / (g - 1.0);
    double Rm = uno - 2.0 * co / (g - 1.0);
    double ub = 0.5 * (Rp + Rm);
    double ut = ui - uni * nx, vt = vi - uni * ny;          /* tangential velocity, inside */
    double lam_i = (KDOF + 2.0) * ri / (4.0 * (Wi[3] - 0.5 * ri * (ui * ui + vi * vi)));
    double rb = ri;
    double bx = ub * nx + ut, by = ub * ny + vt;
    Wg[0] = rb; Wg[1] = rb * bx; Wg[2] = rb * by;
    Wg[3] = 0.5 * rb * (ub * ub + (ut * ut + vt * vt) + (KDOF + 2.0) / (2.0 * lam_i));
    Wg[4] = Wi[4];
  } else {                      /* free stream (Section II.E): the ghost holds the free stream */
    freestream(&s->flow, Wg);
  }
}

/* ghost increments used inside the sweeps: the boundary map applied to a cell increment */
static void ghost_increment(const ora_solver* s, int f, const double* dWi, double* dWg) {
  double nx = s->fnx[f], ny = s->fny[f];
  int bc = s->face_bc[f];
  if (bc == 3 || bc == 5) {   /* walls (a moving wall maps increments like a fixed one) */
    dWg[0] = dWi[0]; dWg[1] = -dWi[1]; dWg[2] = -dWi[2]; dWg[3] = dWi[3]; dWg[4] = -dWi[4];
  } else if (bc == 2) {
    double mn = dWi[1] * nx + dWi[2] * ny;
    dWg[0] = dWi[0]; dWg[1] = dWi[1] - 2.0 * mn * nx; dWg[2] = dWi[2] - 2.0 * mn * ny;
    dWg[3] = dWi[3]; dWg[4] = dWi[4];
  } else {
    for (int v = 0; v < 5; v++) dWg[v] = 0.0;
  }
}

/* state of the cell across face f as seen from cell i (ghost on a boundary) */
static const double* across(const ora_solver* s, int f, int i, int* j) {
  int l = s->face_cells[2 * f], r = s->face_cells[2 * f + 1];
  if (r < 0) { *j = -1; return s->G + 5 * f; }
  *j = (i == l) ? r : l;
  return s->W + 5 * (*j);
}

/* ---- step 1: ghost cells ---- */
static void step_ghosts(ora_solver* s) {
  for (int f = 0; f < s->n_faces; f++) {
    double* g = s->G + 5 * f;
    for (int v = 0; v < 5; v++) g[v] = 0.0;
    if (s->face_cells[2 * f + 1] < 0) ghost_state(s, f, s->W + 5 * s->face_cells[2 * f], g);
  }
}

/* ---- step 2: spectral radius (Eq. 20-21), explicit time step (Eq. 23) ---- */
static void step_spectral(ora_solver* s) {
  for (int f = 0; f < s->n_faces; f++) {
    int l = s->face_cells[2 * f], r = s->face_cells[2 * f + 1];
    const double* WL = s->W + 5 * l;
    const double* WR = r >= 0 ? s->W + 5 * r : s->G + 5 * f;
    double uL = WL[1] / WL[0], vL = WL[2] / WL[0], cL = sqrt(GAMMA * pressure(WL) / WL[0]);
    double uR = WR[1] / WR[0], vR = WR[2] / WR[0], cR = sqrt(GAMMA * pressure(WR) / WR[0]);
    double ub = 0.5 * (uL + uR), vb = 0.5 * (vL + vR), cb = 0.5 * (cL + cR);
    double lam = fabs(ub * s->fnx[f] + vb * s->fny[f]) + cb;
    if (s->flow.visc_sr) {
      double mub = 0.5 * (ora_viscosity(&s->flow, lambda_of(WL)) + ora_viscosity(&s->flow, lambda_of(WR)));
      double mtb = 0.5 * (mu_turb(s, WL) + mu_turb(s, WR));
      double rb = 0.5 * (WL[0] + WR[0]);
      double dn = fabs((s->gx[f] - s->cx[l]) * s->fnx[f] + (s->gy[f] - s->cy[l]) * s->fny[f]);
      lam += 2.0 * (mub + mtb) * GAMMA / (rb * s->flow.prandtl * dn);
    }
    s->lam_f[f] = lam;
  }
  double dt = DBL_MAX;
  for (int i = 0; i < s->n_cells; i++) {
    double L = 0.0;
    for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
      int f = s->cf_face[k];
      L += 0.5 * s->lam_f[f] * s->fS[f];
    }
    s->Lam[i] = L;
    double d = s->flow.cfl_exp * s->area[i] / L;
    if (d < dt) dt = d;
  }
  s->dt = dt;
}

/* ---- step 3: least-squares gradients (Eq. 6-7) and limiter (Eq. 9-10) ---- */
static void step_gradients(ora_solver* s) {
  for (int i = 0; i < s->n_cells; i++) {
    const double* Wi = s->W + 5 * i;
    double A00 = 0, A01 = 0, A11 = 0, r[4][2] = {{0}}, wmax[4], wmin[4];
    for (int v = 0; v < 4; v++) wmax[v] = wmin[v] = Wi[v];
    for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
      int f = s->cf_face[k], j;
      const double* Wk = across(s, f, i, &j);
      double xk = (j >= 0) ? s->cx[j] : s->gx[f];
      double yk = (j >= 0) ? s->cy[j] : s->gy[f];
      double dx = xk - s->cx[i], dy = yk - s->cy[i];
      A00 += dx * dx; A01 += dx * dy; A11 += dy * dy;
      for (int v = 0; v < 4; v++) {
        double dw = Wk[v] - Wi[v];
        r[v][0] += dx * dw;
        r[v][1] += dy * dw;
        if (Wk[v] > wmax[v]) wmax[v] = Wk[v];
        if (Wk[v] < wmin[v]) wmin[v] = Wk[v];
      }
    }
    double det = A00 * A11 - A01 * A01;
    for (int v = 0; v < 4; v++) {
      double bx = (A11 * r[v][0] - A01 * r[v][1]) / det;
      double by = (A00 * r[v][1] - A01 * r[v][0]) / det;
      s->grad[8 * i + 2 * v] = bx;
      s->grad[8 * i + 2 * v + 1] = by;
      double phi = 1.0;
      if (s->flow.limiter != 0) {
        double h = sqrt(s->area[i]);
        double eps2 = pow(s->flow.venkat_k * h, 3.0);
        for (int k = s->cell_ptr[i]; k < s->cell_ptr[i + 1]; k++) {
          int nd = s->cell_nodes[k];
          double d = bx * (s->xy[2 * nd] - s->cx[i]) + by * (s->xy[2 * nd + 1] - s->cy[i]);
          double pv = 1.0;
          if (s->flow.limiter == 1) {
            /* Eq. 9: ratio of the path extreme to the node-reconstructed extreme */
            if (d > 0.0) pv = fmin(1.0, (wmax[v] - Wi[v]) / d);
            else if (d < 0.0) pv = fmin(1.0, (wmin[v] - Wi[v]) / d);
          } else {
            double dp = d > 0.0 ? wmax[v] - Wi[v] : wmin[v] - Wi[v];
            if (d != 0.0)
              pv = ((dp * dp + eps2) * d + 2.0 * d * d * dp) / (d * (dp * dp + 2.0 * d * d + d * dp + eps2));
          }
          if (pv < phi) phi = pv;
        }
      }
      s->phi[4 * i + v] = phi;
    }
  }
}

/* rotate momentum of a conserved 4-vector into the face frame and back */
static void to_face(const double* W, double nx, double ny, double* R) {
  R[0] = W[0]; R[1] = W[1] * nx + W[2] * ny; R[2] = -W[1] * ny + W[2] * nx; R[3] = W[3];
}

/* boundary map in the face frame (wall: both momentum components, symmetry: normal) */
static void face_bc_map(int bc, const double* in, double* out) {
  out[0] = in[0]; out[3] = in[3];
  out[1] = -in[1];
  out[2] = (bc == 3) ? -in[2] : in[2];
}

/* ---- step 4: interface fluxes (Eq. 4-14, 33-34) and SA face fluxes (Eq. 28-30) ---- */
static int step_fluxes(ora_solver* s) {
  const ora_flow* fl = &s->flow;
  for (int f = 0; f < s->n_faces; f++) {
    int l = s->face_cells[2 * f], r = s->face_cells[2 * f + 1];
    int bc = s->face_bc[f];
    double nx = s->fnx[f], ny = s->fny[f], tx = -ny, ty = nx;
    const double* Wl = s->W + 5 * l;
    const double* Wr = r >= 0 ? s->W + 5 * r : s->G + 5 * f;
    /* reconstructed face states (Eq. 10) and limited slopes, global frame */
    double WLg[4], WRg[4], sLn[4], sLt[4], sRn[4], sRt[4];
    double dxl = s->fmx[f] - s->cx[l], dyl = s->fmy[f] - s->cy[l];
    for (int v = 0; v < 4; v++) {
      double gx = s->phi[4 * l + v] * s->grad[8 * l + 2 * v], gy = s->phi[4 * l + v] * s->grad[8 * l + 2 * v + 1];
      WLg[v] = Wl[v] + gx * dxl + gy * dyl;
      sLn[v] = gx * nx + gy * ny;
      sLt[v] = gx * tx + gy * ty;
    }
    double WL[4], WR[4], SLn[4], SLt[4], SRn[4], SRt[4], WcL[4], WcR[4];
    to_face(WLg, nx, ny, WL);
    to_face(sLn, nx, ny, SLn);
    to_face(sLt, nx, ny, SLt);
    to_face(Wl, nx, ny, WcL);
    to_face(Wr, nx, ny, WcR);
    double dL = dxl * nx + dyl * ny, dR;
    if (r >= 0) {
      double dxr = s->fmx[f] - s->cx[r], dyr = s->fmy[f] - s->cy[r];
      for (int v = 0; v < 4; v++) {
        double gx = s->phi[4 * r + v] * s->grad[8 * r + 2 * v], gy = s->phi[4 * r + v] * s->grad[8 * r + 2 * v + 1];
        WRg[v] = Wr[v] + gx * dxr + gy * dyr;
        sRn[v] = gx * nx + gy * ny;
        sRt[v] = gx * tx + gy * ty;
      }
      to_face(WRg, nx, ny, WR);
      to_face(sRn, nx, ny, SRn);
      to_face(sRt, nx, ny, SRt);
      dR = -(dxr * nx + dyr * ny);
    } else if (bc == 2 || bc == 3 || bc == 5) {
      /* mirror image of the left side: state mapped by the boundary condition, the
       * normal slope also reflected; a moving wall mirrors the tangential velocity about
       * the wall velocity (slopes map as at a fixed wall) */
      double tmp[4];
      int sb = bc == 5 ? 3 : bc;
      face_bc_map(sb, WL, WR);
      if (bc == 5) {
        double Wf[5];
        freestream(fl, Wf);
        double uw = (Wf[1] * tx + Wf[2] * ty) / Wf[0];
        double r = WL[0], ut = WL[2] / r, utg = 2.0 * uw - ut;
        WR[2] = r * utg;
        WR[3] = WL[3] - 0.5 * r * ut * ut + 0.5 * r * utg * utg;
      }
      face_bc_map(sb, SLn, tmp);
      for (int v = 0; v < 4; v++) SRn[v] = -tmp[v];
      face_bc_map(sb, SLt, SRt);
      dR = dL;
    } else {
      /* free stream and outflow: the ghost state, without slopes */
      for (int v = 0; v < 4; v++) { WR[v] = WcR[v]; SRn[v] = 0.0; SRt[v] = 0.0; }
      dR = dL;
    }
    double mut = 0.5 * (mu_turb(s, Wl) + mu_turb(s, Wr));
    double Fr[4];
    if (ora_face_flux(fl, WL, WR, SLn, SLt, SRn, SRt, WcL, WcR, dL, dR, mut, s->dt, Fr, NULL)) return -1;
    double S = s->fS[f];
    double* out = s->F + 6 * f;
    out[0] = Fr[0] * S;
    out[1] = (Fr[1] * nx - Fr[2] * ny) * S;
    out[2] = (Fr[1] * ny + Fr[2] * nx) * S;
    out[3] = Fr[3] * S;
    out[4] = out[5] = 0.0;
    if (fl->sa_on) {
      /* Eq. 29-30 with cell-centre velocities; conservative inviscid + viscous part,
       * anti-diffusion with the receiving cell's nu_tilde */
      double vni = (Wl[1] * nx + Wl[2] * ny) / Wl[0];
      double vnj = (Wr[1] * nx + Wr[2] * ny) / Wr[0];
      double up = 0.5 * (vni + fabs(vni)), um = 0.5 * (vnj - fabs(vnj));
      double dn = fabs((s->gx[f] - s->cx[l]) * nx + (s->gy[f] - s->cy[l]) * ny);
      double nui = nu_lam(s, Wl), nuj = nu_lam(s, Wr);
      double gradn = (Wr[4] - Wl[4]) / dn;
      double Finv = up * Wl[4] + um * Wr[4];
      double Fvis = 1.0 / (2.0 * SA_SIGMA) * ((nui + nuj) + (1.0 + SA_CB2) * (Wl[4] + Wr[4])) * gradn;
      double Fad_l = SA_CB2 / SA_SIGMA * Wl[4] * gradn;
      double Fad_r = SA_CB2 / SA_SIGMA * Wr[4] * (-gradn);
      out[4] = (-Finv + Fvis - Fad_l) * S;   /* R_l += */
      out[5] = (Finv - Fvis - Fad_r) * S;    /* R_r += */
    }
  }
  return 0;
}

/* Spalart-Allmaras source of Eq. 28a per unit volume, Sr = cb1 S~ nu~ - cw1 fw (nu~/d)^2
 * (SA-noft2; S~ with the 2012 clipping), for nu~ = nut, laminar kinematic viscosity nu,
 * vorticity magnitude omega and wall distance d. out: Sr, fw, S~, r, fv1, fv2. */
void ora_sa_source(double nut, double nu, double om, double d, double* out) {
  const double cv1 = SA_CV1, k2 = SA_KAPPA * SA_KAPPA;
  double chi = nut / nu, c3 = chi * chi * chi;
  double fv1 = c3 / (c3 + cv1 * cv1 * cv1);
  double fv2 = 1.0 - chi / (1.0 + chi * fv1);
  double Sbar = nut * fv2 / (k2 * d * d);
  double St;
  if (Sbar >= -SA_CV2 * om) St = om + Sbar;
  else St = om + om * (SA_CV2 * SA_CV2 * om + SA_CV3 * Sbar) / ((SA_CV3 - 2.0 * SA_CV2) * om - Sbar);
  double rr = (nut < 10.0 * St * k2 * d * d) ? nut / (St * k2 * d * d) : 10.0;
  double gg = rr + SA_CW2 * (pow(rr, 6.0) - rr);
  double c6 = pow(SA_CW3, 6.0);
  double fw = gg * pow((1.0 + c6) / (pow(gg, 6.0) + c6), 1.0 / 6.0);
  out[0] = SA_CB1 * St * nut - SA_CW1 * fw * (nut / d) * (nut / d);
  out[1] = fw;
  out[2] = St;
  out[3] = rr;
  out[4] = fv1;
  out[5] = fv2;
}

/* ---- step 5: residual M (Eq. 16) and the SA right-hand side (Eq. 27-28a) ---- */
static void step_residual(ora_solver* s) {
  for (int i = 0; i < s->n_cells; i++) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
      int f = s->cf_face[k];
      const double* Ff = s->F + 6 * f;
      if (s->face_cells[2 * f] == i) {
        for (int v = 0; v < 4; v++) acc[v] += Ff[v];
        acc[4] += Ff[4];
      } else {
        for (int v = 0; v < 4; v++) acc[v] -= Ff[v];
        acc[4] += Ff[5];
      }
    }
    double* Mi = s->M + 5 * i;
    for (int v = 0; v < 4; v++) Mi[v] = -acc[v] / s->dt;
    Mi[4] = 0.0;
    s->fw[i] = 0.0;
    if (s->flow.sa_on) {
      const double* Wi = s->W + 5 * i;
      double rho = Wi[0], u = Wi[1] / rho, v = Wi[2] / rho;
      const double* g = s->grad + 8 * i;
      double dudy = (g[3] - u * g[1]) / rho;
      double dvdx = (g[4] - v * g[0]) / rho;
      double om = fabs(dvdx - dudy);
      double src[6];
      ora_sa_source(Wi[4], nu_lam(s, Wi), om, s->wall_d[i], src);
      s->fw[i] = src[1];
      Mi[4] = s->area[i] * src[0] + acc[4];
    }
  }
}

/* ---- step 6: norms (Eq. 25) ---- */
static void step_norms(ora_solver* s) {
  double rinf = 0.0, r2 = 0.0;
  for (int i = 0; i < s->n_cells; i++) {
    double m = s->M[5 * i];
    if (fabs(m) > rinf) rinf = fabs(m);
    double q = m / s->area[i];
    r2 += q * q;
  }
  s->res_inf = rinf;
  s->res_l2 = sqrt(r2 / s->n_cells);
  if (s->iter == 0) {
    s->cfl = s->flow.cfl_init;
    s->res_l2_first = s->res_l2;
  } else {
    /* Eq. 25; a residual that vanished exactly makes the ratio infinite (CFL to its cap),
     * and two vanishing residuals in a row leave the CFL unchanged */
    double c;
    if (s->res_inf > 0.0) c = s->cfl * s->res_inf_prev / s->res_inf;
    else c = (s->res_inf_prev > 0.0) ? s->flow.cfl_max : s->cfl;
    if (c < s->flow.cfl_min) c = s->flow.cfl_min;
    if (c > s->flow.cfl_max) c = s->flow.cfl_max;
    s->cfl = c;
  }
  s->res_inf_prev = s->res_inf;
}

/* SA sweep coefficients of face f seen from cell i (reading of Eq. 31-32: frozen
 * viscous coefficient, upwind inviscid part). a_ij multiplies the neighbour increment,
 * diag is the face's contribution to a_ii. */
static void sa_coeffs(const ora_solver* s, int f, int i, const double* Wi, const double* Wj,
                      double nx, double ny, double* diag, double* aij) {
  int l = s->face_cells[2 * f];
  double dn = fabs((s->gx[f] - s->cx[l]) * s->fnx[f] + (s->gy[f] - s->cy[l]) * s->fny[f]);
  double vni = (Wi[1] * nx + Wi[2] * ny) / Wi[0];
  double vnj = (Wj[1] * nx + Wj[2] * ny) / Wj[0];
  double up = 0.5 * (vni + fabs(vni)), um = 0.5 * (vnj - fabs(vnj));
  double kap = 1.0 / (2.0 * SA_SIGMA) * ((nu_lam(s, Wi) + nu_lam(s, Wj)) + (1.0 + SA_CB2) * (Wi[4] + Wj[4]));
  double S = s->fS[f];
  *diag = S * (up + kap / dn);
  *aij = S * (um - kap / dn);
}

/* ---- steps 7-8: matrix-free LU-SGS sweeps (Eq. 19-22, 31-32) and update ---- */
static void step_sweeps(ora_solver* s) {
  int N = s->n_cells;
  const int sa = s->flow.sa_on;
  double* D = dalloc(N);
  double* Dsa = dalloc(N);
  for (int i = 0; i < N; i++) {
    /* D = Omega/dt_imp + sum (Lambda_c)_ij with dt_imp = CFL_imp Omega / Lambda (Eq. 20, 24) */
    double dtimp = s->cfl * s->area[i] / s->Lam[i];
    D[i] = s->area[i] / dtimp + s->Lam[i];
    if (sa) {
      const double* Wi = s->W + 5 * i;
      double a = s->area[i] / dtimp;
      for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
        int f = s->cf_face[k], j;
        const double* Wj = across(s, f, i, &j);
        double sg = (s->face_cells[2 * f] == i) ? 1.0 : -1.0;
        double dg, aij;
        sa_coeffs(s, f, i, Wi, Wj, sg * s->fnx[f], sg * s->fny[f], &dg, &aij);
        a += dg;
      }
      double d = s->wall_d[i];
      a += s->area[i] * 2.0 * SA_CW1 * s->fw[i] * Wi[4] / (d * d);
      Dsa[i] = a;
    }
  }
  /* forward sweep, i = 0 .. N-1, lower neighbours j < i */
  for (int i = 0; i < N; i++) {
    const double* Wi = s->W + 5 * i;
    double acc[5];
    for (int v = 0; v < 5; v++) acc[v] = s->M[5 * i + v];
    for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
      int f = s->cf_face[k], j;
      const double* Wj = across(s, f, i, &j);
      if (j < 0 || j >= i) continue;     /* boundary increments are zero in this sweep */
      double sg = (s->face_cells[2 * f] == i) ? 1.0 : -1.0;
      double nx = sg * s->fnx[f], ny = sg * s->fny[f], S = s->fS[f], lam = s->lam_f[f];
      const double* dWj = s->dWs + 5 * j;
      double Wp[4], F1[4], F0[4];
      for (int v = 0; v < 4; v++) Wp[v] = Wj[v] + dWj[v];
      ora_euler_flux(Wp, nx, ny, F1);
      ora_euler_flux(Wj, nx, ny, F0);
      for (int v = 0; v < 4; v++) acc[v] -= 0.5 * S * ((F1[v] - F0[v]) - lam * dWj[v]);
      if (sa) {
        double dg, aij;
        sa_coeffs(s, f, i, Wi, Wj, nx, ny, &dg, &aij);
        acc[4] -= aij * dWj[4];
      }
    }
    for (int v = 0; v < 4; v++) s->dWs[5 * i + v] = acc[v] / D[i];
    s->dWs[5 * i + 4] = sa ? acc[4] / Dsa[i] : 0.0;
  }
  /* backward sweep, i = N-1 .. 0, upper neighbours j > i; wall and symmetry ghosts take
   * the boundary map of the cell's own forward increment */
  for (int i = N - 1; i >= 0; i--) {
    const double* Wi = s->W + 5 * i;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = s->cf_ptr[i]; k < s->cf_ptr[i + 1]; k++) {
      int f = s->cf_face[k], j;
      const double* Wj = across(s, f, i, &j);
      double dWg[5];
      const double* dWj;
      if (j < 0) {
        if (s->face_bc[f] == 1 || s->face_bc[f] == 4) continue;   /* free-stream and outflow increments are zero */
        ghost_increment(s, f, s->dWs + 5 * i, dWg);
        dWj = dWg;
      } else {
        if (j <= i) continue;
        dWj = s->dW + 5 * j;
      }
      double sg = (s->face_cells[2 * f] == i) ? 1.0 : -1.0;
      double nx = sg * s->fnx[f], ny = sg * s->fny[f], S = s->fS[f], lam = s->lam_f[f];
      double Wp[4], F1[4], F0[4];
      for (int v = 0; v < 4; v++) Wp[v] = Wj[v] + dWj[v];
      ora_euler_flux(Wp, nx, ny, F1);
      ora_euler_flux(Wj, nx, ny, F0);
      for (int v = 0; v < 4; v++) acc[v] += 0.5 * S * ((F1[v] - F0[v]) - lam * dWj[v]);
      if (sa) {
        double dg, aij;
        sa_coeffs(s, f, i, Wi, Wj, nx, ny, &dg, &aij);
        acc[4] += aij * dWj[4];
      }
    }
    for (int v = 0; v < 4; v++) s->dW[5 * i + v] = s->dWs[5 * i + v] - acc[v] / D[i];
    s->dW[5 * i + 4] = sa ? s->dWs[5 * i + 4] - acc[4] / Dsa[i] : 0.0;
  }
  free(D);
  free(Dsa);
}

/* explicit scheme (Eq. 15, written as Eq. 16): W^{n+1} = W^n + dt M / Omega */
static void step_explicit(ora_solver* s) {
  for (int i = 0; i < s->n_cells; i++) {
    for (int v = 0; v < 4; v++) s->dW[5 * i + v] = s->dt * s->M[5 * i + v] / s->area[i];
    s->dW[5 * i + 4] = s->flow.sa_on ? s->dt * s->M[5 * i + 4] / s->area[i] : 0.0;
  }
}

static void step_update(ora_solver* s) {
  double eq40 = 0.0;
  int bad = 0;
  for (int i = 0; i < s->n_cells; i++) {
    double* Wi = s->W + 5 * i;
    const double* d = s->dW + 5 * i;
    double num = 0.0, den = 0.0;
    for (int v = 0; v < 4; v++) { num += d[v] * d[v]; den += Wi[v] * Wi[v]; }
    double r = sqrt(num) / sqrt(den);
    if (r > eq40) eq40 = r;
    for (int v = 0; v < 5; v++) Wi[v] += d[v];
    if (Wi[4] < 0.0) Wi[4] = 0.0;
    double p = pressure(Wi);
    if (!(Wi[0] > 0.0) || !(p > 0.0) || !isfinite(Wi[3]) || !isfinite(Wi[4])) bad = 1;
  }
  s->eq40 = eq40;
  if (bad) s->status = -5;
}

int ora_iterate(ora_solver* s, int n_iter) {
  for (int it = 0; it < n_iter; it++) {
    if (s->status < 0) return s->status;
    step_ghosts(s);
    step_spectral(s);
    step_gradients(s);
    if (step_fluxes(s)) { s->status = -5; return s->status; }
    step_residual(s);
    step_norms(s);
    if (s->flow.scheme == 1) step_explicit(s);
    else step_sweeps(s);
    step_update(s);
    s->iter++;
    if (s->status < 0) return s->status;
    /* converged when the density residual fell to res_target times its first value; a
     * residual that is exactly zero (also at the first iteration) has nothing left to fall */
    if ((s->res_l2 <= s->flow.res_target * s->res_l2_first) ||
        (s->flow.eq40_target > 0.0 && s->eq40 <= s->flow.eq40_target)) {
      s->status = 1;
      return 1;
    }
  }
  return s->status;
}

static void soa(const double* aos, int n, int w, double* out) {
  for (int i = 0; i < n; i++)
    for (int v = 0; v < w; v++) out[(size_t)v * n + i] = aos[(size_t)w * i + v];
}

int ora_get(const ora_solver* s, int which, double* out) {
  int N = s->n_cells, Nf = s->n_faces;
  switch (which) {
    case ORA_W: soa(s->W, N, 5, out); return 0;
    case ORA_GRAD: soa(s->grad, N, 8, out); return 0;
    case ORA_PHI: soa(s->phi, N, 4, out); return 0;
    case ORA_LAMBDA_F: memcpy(out, s->lam_f, sizeof(double) * Nf); return 0;
    case ORA_LAMBDA_C: memcpy(out, s->Lam, sizeof(double) * N); return 0;
    case ORA_FLUX: soa(s->F, Nf, 6, out); return 0;
    case ORA_RES: soa(s->M, N, 5, out); return 0;
    case ORA_DWSTAR: soa(s->dWs, N, 5, out); return 0;
    case ORA_DW: soa(s->dW, N, 5, out); return 0;
    case ORA_GHOST: soa(s->G, Nf, 5, out); return 0;
    case ORA_GEOM_CELL:
      memcpy(out, s->area, sizeof(double) * N);
      memcpy(out + N, s->cx, sizeof(double) * N);
      memcpy(out + 2 * N, s->cy, sizeof(double) * N);
      memcpy(out + 3 * N, s->wall_d, sizeof(double) * N);
      return 0;
    case ORA_GEOM_FACE:
      memcpy(out, s->fS, sizeof(double) * Nf);
      memcpy(out + Nf, s->fnx, sizeof(double) * Nf);
      memcpy(out + 2 * Nf, s->fny, sizeof(double) * Nf);
      memcpy(out + 3 * Nf, s->fmx, sizeof(double) * Nf);
      memcpy(out + 4 * Nf, s->fmy, sizeof(double) * Nf);
      return 0;
  }
  return -1;
}

void ora_get_scalars(const ora_solver* s, double* o) {
  o[ORA_S_DT] = s->dt; o[ORA_S_CFL] = s->cfl; o[ORA_S_RES_INF] = s->res_inf;
  o[ORA_S_RES_L2] = s->res_l2; o[ORA_S_RES_L2_FIRST] = s->res_l2_first; o[ORA_S_EQ40] = s->eq40;
  o[ORA_S_ITER] = s->iter; o[ORA_S_STATUS] = s->status; o[ORA_S_RES_INF_PREV] = s->res_inf_prev;
}

void ora_set_scalars(ora_solver* s, const double* in) {
  s->cfl = in[ORA_S_CFL]; s->res_l2_first = in[ORA_S_RES_L2_FIRST];
  s->iter = (int)in[ORA_S_ITER]; s->status = (int)in[ORA_S_STATUS];
  s->res_inf_prev = in[ORA_S_RES_INF_PREV];
}
