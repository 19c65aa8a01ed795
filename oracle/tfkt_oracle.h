/*
 * Oracle for the two-fluid kinetic scheme of Singh, Subramanian & Ansumali,
 * "Two-fluid kinetic theory for dilute polymer solutions" (arXiv 2201.10132).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 CPU restatement of the
 * discrete scheme of Sec. VI (D2Q9 solvent, D4Q25 polymer hyper-lattice,
 * trapezoidal time discretisation with the auxiliary population g) driven by
 * the Kolmogorov forcing of Sec. VII. Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may call it. It shares no code, header or
 * table with the CUDA library; the two are written independently from the
 * paper.
 *
 * Every function states the passage it follows. Readings of passages that are
 * silent, garbled or ambiguous are marked "reading:".
 */
#ifndef TFKT_ORACLE_H
#define TFKT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Physical inputs of a Kolmogorov run (Sec. VII: Re, Wi, beta; grid sizes). */
typedef struct {
  int32_t nx, ny;          /* r-grid, periodic */
  int32_t q_side;          /* S: S x S cell-centred Q-grid */
  double q_radius;         /* R: Q-nodes with |Q| <= R are kept (Q lattice units) */
  double re, wi, beta;     /* Re = U0 l / nu, Wi = U0 lambda_H / l, beta = eta_s/(eta_s+eta_p) */
  double u0;               /* laminar peak velocity, lattice units */
  int32_t k_periods;       /* forcing a0 sin(2 pi k_periods y / ny) */
  double tau2;             /* momentum relaxation time; <= 0 -> tau2 = tau1 */
  double ell;              /* Q-lattice spacing in r-lengths; <= 0 -> sqrt(2) */
  double fene_b;           /* FENE extensibility b in units of kT/H; 0 -> Hookean */
  int32_t qe_model;        /* 0: component momenta quasi-conserved (Sec. V, Eq. quasieq1);
                              1: component stresses quasi-conserved (Eq. quasieq2) */
} orc_phys;

/* Lattice-unit parameters used by the step. */
typedef struct {
  int32_t nx, ny, q_side;
  double q_radius;
  double tau1, tau2;       /* stress / momentum relaxation times */
  double H;                /* Hookean spring constant (r-length units) */
  double kappa;            /* 2 H tau2: Q-space drift rate (Q lattice units) */
  double ell;              /* Q-lattice spacing in r-lengths */
  double psi_tot;          /* sum_q psi of the initial state, per r-node */
  double sigma_q2;         /* variance of the initial Gaussian in Q (Q lattice units) */
  double a0;               /* forcing amplitude */
  double kf;               /* forcing wavenumber 2 pi k_periods / ny */
  double u0;               /* laminar amplitude (initial condition, mode 1) */
  double nu, nu_s, eta_p, lambda_h; /* reported, not used by the step */
  double fene_b;           /* FENE b (units of kT/H); 0 -> Hookean springs */
  int32_t qe_model;        /* 0: momentum quasi-equilibrium (tau1 = stress, tau2 = momentum
                              relaxation); 1: stress quasi-equilibrium (tau1 = momentum,
                              tau2 = stress relaxation) */
} orc_lattice;

typedef struct orc_state orc_state;

/* Fields of orc_fields, one plane of ny*nx doubles each. */
enum {
  ORC_F_RHO_S = 0, ORC_F_PSI_TOT, ORC_F_UX, ORC_F_UY,
  ORC_F_CXX, ORC_F_CXY, ORC_F_CYY, ORC_F_THXX, ORC_F_THXY, ORC_F_THYY,
  ORC_F_QRMS, ORC_F_VORT, ORC_NFIELDS
};
/* Diagnostics of orc_diagnostics. */
enum {
  ORC_D_MASS_S = 0, ORC_D_MASS_P, ORC_D_PX, ORC_D_PY, ORC_D_KE,
  ORC_D_ENSTROPHY, ORC_D_QRMS_MEAN, ORC_D_EY2, ORC_NDIAG
};

/* Physical -> lattice mapping; returns 0, or -1 on invalid input. */
int orc_map_params(const orc_phys* in, orc_lattice* out);

/* Velocity sets: writes 9 (D2Q9) or 25 (D4Q25) velocities, weights and the
   index of the opposite velocity. d2q9: c[9][2]; d4q25: c[25][4]. */
void orc_d2q9(int32_t* c, double* w, int32_t* opp);
void orc_d4q25(int32_t* c, double* w, int32_t* opp);

orc_state* orc_create(const orc_lattice* lat);
void orc_destroy(orc_state* st);
int32_t orc_nq(const orc_state* st);
/* Q-node coordinates (Q lattice units), nq each. */
void orc_q_nodes(const orc_state* st, double* qx, double* qy);
/* Initial psi(q) per r-node (the discretely normalised Gaussian). */
void orc_psi0(const orc_state* st, double* psi0);

/* Initial state: ic_mode 0 = rest, 1 = laminar U0 sin(kf y); plus the given
   perturbation velocity perturb[2][ny][nx] (may be NULL). */
void orc_init(orc_state* st, const double* perturb, int32_t ic_mode);

/* Direct access to the pre-collision populations g (after streaming):
   gs[ny][nx][9], gp[ny][nx][nq][25]. */
void orc_get_g(const orc_state* st, double* gs, double* gp);
void orc_set_g(orc_state* st, const double* gs, const double* gp);
/* Post-collision populations g' of the last orc_collide, same layout. */
void orc_get_gpost(const orc_state* st, double* gs, double* gp);
void orc_set_gpost(orc_state* st, const double* gs, const double* gp);

/* Replace the computed velocity gradient dU_b/dr_a by a fixed G[a][b]
   (homogeneous-flow test mode). enable = 0 restores the computed one. */
void orc_set_imposed_gradient(orc_state* st, const double* G, int32_t enable);

/* One collision (moments, U, gradients, equilibria, two-relaxation update). */
void orc_collide(orc_state* st);
/* Pull streaming of g' into g, periodic in r, bounce-back at the Q-disk edge. */
void orc_stream(orc_state* st);
/* n full steps: collide then stream. */
void orc_step(orc_state* st, int32_t n);

/* Macroscopic fields of the current g: out[ORC_NFIELDS][ny][nx];
   psi_out[ny][nx][nq] (may be NULL); E_out[2][ny][nx] elastic force (may be NULL). */
void orc_fields(orc_state* st, double* out, double* psi_out, double* e_out);
void orc_diagnostics(orc_state* st, double* out);

/* Set the number of OpenMP threads (<= 0: leave default); returns the count used. */
int32_t orc_set_threads(int32_t n);

#ifdef __cplusplus
}
#endif
#endif
