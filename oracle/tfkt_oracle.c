/*
 * Oracle for the two-fluid kinetic scheme (arXiv 2201.10132, Sec. VI-VII).
 * TEST INFRASTRUCTURE ONLY: plain FP64 CPU code, whole-array loops, no
 * blocking or fusion. Called only by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark. Shares nothing with the CUDA library.
 *
 * One time step n -> n+1 (orc_collide then orc_stream):
 *   A2  moments of g: rho_S, J_S(g); per (r,q): psi, J^r(g), J^Q(g)     (Sec. VI-A, VI-B)
 *   A3  per-q elastic drift D = F(Q) (Q . grad_r psi)/2, E = sum_q D     (Eq. poly_imposed_vel,
 *       first-order Taylor of psi(r - R_nu), as the paper does for I)   Sec. III, Eq. IDef)
 *   A4  mixture velocity rho U = J(g) + (E + rho a)/2                    (Sec. VI-C, moments of f)
 *   A5  grad U; J^r_eq = psi U + tau2 D; J^Q_eq = psi (Q . grad U - kappa Q)
 *   A6  g -> f momenta: J(f) = (2 tau2 J(g) + J_eq) / (2 tau2 + 1)
 *   A7  g' = (1-2b) g + 2b [(1 - tau1/tau2) f* + (tau1/tau2) f^eq] + (1-b) S,  b = 1/(2 tau1 + 1)
 *   A1  pull streaming, periodic in r, full bounce-back at the Q-disk edge
 *
 * Parity status: every function here is pinned by a CPU test (tables,
 * invariants, closed forms, limits); see the tests under tests/ named
 * test_oracle_*.
 */
#include "tfkt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct orc_state {
  orc_lattice L;
  int nx, ny, nq, S;
  int* qmap;              /* [S*S] grid cell -> q, or -1 outside the disk */
  int* qgi; int* qgj;     /* grid indices of node q */
  double* Qx; double* Qy; /* Q lattice coordinates of node q */
  double* psi0;           /* initial psi(q) */
  double* phi;            /* spring factor of Q-node q: 1 (Hookean) or 1/(1 - Q^2/Q0^2) (FENE) */
  int cs[9][2]; double ws[9]; int opps[9];
  int cp[25][4]; double wp[25]; int oppp[25];
  double* gs; double* gp;         /* pre-collision g (after streaming) */
  double* gs_post; double* gp_post; /* post-collision g' */
  /* work arrays, per r-node n = y*nx + x */
  double* rho_s; double* jsx; double* jsy;
  double* psi;                    /* [n][q] */
  double* jr; double* jq;         /* [n][q][2] */
  double* psitot; double* jpx; double* jpy;
  double* dq;                     /* [n][q][2] elastic drift D */
  double* ex; double* ey;
  double* ux; double* uy;
  double* gux; double* guy;       /* gradients: g?x[n][a] = d_a U_? */
  int imposed; double G[2][2];
};

/* ---------------------------------------------------------------- tables */

/* D2Q9 (Sec. VI-A). reading: the printed angle formula mixes axis and diagonal
   directions for i = 1..4; the standard set is used: i = 1..4 along the axes,
   i = 5..8 along the diagonals (length sqrt(2) c), weights 4/9, 1/9, 1/36. */
void orc_d2q9(int32_t* c, double* w, int32_t* opp) {
  static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int i = 0; i < 9; ++i) {
    c[2 * i] = cx[i];
    c[2 * i + 1] = cy[i];
    w[i] = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j)
      if (cx[j] == -cx[i] && cy[j] == -cy[i]) opp[i] = j;
}

/* D4Q25 on (r_x, r_y, Q_x, Q_y) (Sec. VI-B, Table dis_vel): the rest velocity
   and, for each of the 6 pairs of axes, the 4 sign combinations (+-c, +-c);
   weights w0 = 1/3, w1..24 = 1/36, c_sP^2 = 1/3 (c = 1). */
void orc_d4q25(int32_t* c, double* w, int32_t* opp) {
  int n = 0;
  for (int k = 0; k < 4; ++k) c[k] = 0;
  w[0] = 1.0 / 3.0;
  n = 1;
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b)
      for (int sa = 1; sa >= -1; sa -= 2)
        for (int sb = 1; sb >= -1; sb -= 2) {
          for (int k = 0; k < 4; ++k) c[4 * n + k] = 0;
          c[4 * n + a] = sa;
          c[4 * n + b] = sb;
          w[n] = 1.0 / 36.0;
          ++n;
        }
  for (int i = 0; i < 25; ++i)
    for (int j = 0; j < 25; ++j) {
      int same = 1;
      for (int k = 0; k < 4; ++k) same &= (c[4 * j + k] == -c[4 * i + k]);
      if (same) opp[i] = j;
    }
}

/* ------------------------------------------------------ parameter mapping */

/* Sec. VII defines Re = U l / nu, Wi = U tau_R / l, beta = eta_s/(eta_s+eta_p)
   and the forcing amplitude F = eta U / l^2. Lattice units dt = dr = 1,
   c_s^2 = 1/3, m_B = 1, rho_0 = 1.
   reading: nu_s = c_s^2 tau1 (the g-scheme has no -1/2 shift); the relaxation
   time of the Hookean dumbbell lambda_H = zeta/(4H) with zeta = m_B/tau2
   (Appendix A: tau = m_B/zeta), so H = 1/(4 lambda_H tau2) and the Q-drift
   rate 2H/zeta = 1/(2 lambda_H); the Q-space diffusivity 2 kT/zeta (Eq.
   Smoluchowski_new11) fixes the Q-lattice spacing ell = sqrt(2) r-lengths;
   the lattice psi counts beads (f_P sums f^II over both beads, Sec. VI-B), so
   the stress is Theta = (H ell^2 / 2) sum_q psi Q Q and psi_tot makes the
   polymer viscosity eta_p = (H ell^2 / 2) psi_tot sigma_Q^2 lambda_H (steady-shear
   stress of a Hookean dumbbell). */
int orc_map_params(const orc_phys* in, orc_lattice* out) {
  if (in->nx < 1 || in->ny < 1 || in->q_side < 1 || !(in->q_radius > 0)) return -1;
  if (!(in->re > 0) || !(in->beta > 0) || in->beta > 1 || !(in->u0 > 0)) return -1;
  if (in->k_periods < 1 || in->wi < 0 || in->fene_b < 0) return -1;
  if (in->qe_model != 0 && in->qe_model != 1) return -1;
  if (in->wi == 0 && in->beta < 1) return -1;
  memset(out, 0, sizeof *out);
  out->nx = in->nx;
  out->ny = in->ny;
  out->q_side = in->q_side;
  out->q_radius = in->q_radius;
  const double pi = 3.14159265358979323846;
  double kf = 2.0 * pi * in->k_periods / in->ny;
  double l = 1.0 / kf;
  double nu = in->u0 * l / in->re;
  double nu_s = in->beta * nu;
  /* reading: the viscosity comes from the stress relaxation time, nu_s = c_s^2 tau_s,
     and the drag / diffusion from the momentum relaxation time tau_m (the tau2
     input, default tau_s). Quasi-conserved momenta (Eq. quasieq1) need tau_s <=
     tau_m and relax the stress first (tau1 = tau_s, tau2 = tau_m); quasi-conserved
     stresses (Eq. quasieq2) need tau_m <= tau_s and swap the roles (Sec. V:
     viscosity from tau2, diffusion from tau1). */
  double tau_s = 3.0 * nu_s;
  double tau_m = in->tau2 > 0 ? in->tau2 : tau_s;
  double tau1, tau2;
  if (in->qe_model == 0) {
    if (tau_m < tau_s) return -1;
    tau1 = tau_s;
    tau2 = tau_m;
  } else {
    if (tau_m > tau_s) return -1;
    tau1 = tau_m;
    tau2 = tau_s;
  }
  double ell = in->ell > 0 ? in->ell : sqrt(2.0);
  double eta_p = (1.0 - in->beta) * nu;
  out->kf = kf;
  out->nu = nu;
  out->nu_s = nu_s;
  out->tau1 = tau1;
  out->tau2 = tau2;
  out->ell = ell;
  out->eta_p = eta_p;
  out->u0 = in->u0;
  out->a0 = nu * in->u0 * kf * kf;
  out->fene_b = in->fene_b;
  out->qe_model = in->qe_model;
  if (in->wi > 0) {
    double lam = in->wi * l / in->u0;
    out->lambda_h = lam;
    out->H = 1.0 / (4.0 * lam * tau_m);
    out->kappa = 2.0 * out->H * tau_m;
    out->sigma_q2 = tau_m / (3.0 * out->kappa);
    out->psi_tot = eta_p / (0.5 * out->H * ell * ell * out->sigma_q2 * lam);
  } else {
    out->lambda_h = 0;
    out->H = 0;
    out->kappa = 0;
    out->sigma_q2 = 1.0;
    out->psi_tot = 0;
  }
  /* FENE: every kept Q-node must lie strictly inside |Q| < Q0 = sqrt(b) sigma_Q */
  if (in->fene_b > 0 && in->q_radius * in->q_radius >= in->fene_b * out->sigma_q2) return -1;
  return 0;
}

/* ------------------------------------------------------------ life cycle */

static void* xcalloc(size_t n, size_t s) {
  void* p = calloc(n ? n : 1, s);
  if (!p) abort();
  return p;
}

orc_state* orc_create(const orc_lattice* lat) {
  orc_state* st = (orc_state*)xcalloc(1, sizeof(orc_state));
  st->L = *lat;
  st->nx = lat->nx;
  st->ny = lat->ny;
  st->S = lat->q_side;
  int S = st->S;
  st->qmap = (int*)xcalloc((size_t)S * S, sizeof(int));
  st->qgi = (int*)xcalloc((size_t)S * S, sizeof(int));
  st->qgj = (int*)xcalloc((size_t)S * S, sizeof(int));
  st->Qx = (double*)xcalloc((size_t)S * S, sizeof(double));
  st->Qy = (double*)xcalloc((size_t)S * S, sizeof(double));
  /* Cell-centred S x S grid, Q = (i - (S-1)/2, j - (S-1)/2), masked to the
     disk |Q| <= R (Sec. VI-D: the Q-domain is a circle); node order is
     row-major over (j, i). */
  int nq = 0;
  double R2 = lat->q_radius * lat->q_radius + 1e-9;
  for (int j = 0; j < S; ++j)
    for (int i = 0; i < S; ++i) {
      double qx = i - 0.5 * (S - 1), qy = j - 0.5 * (S - 1);
      if (qx * qx + qy * qy <= R2) {
        st->qmap[j * S + i] = nq;
        st->qgi[nq] = i;
        st->qgj[nq] = j;
        st->Qx[nq] = qx;
        st->Qy[nq] = qy;
        ++nq;
      } else {
        st->qmap[j * S + i] = -1;
      }
    }
  st->nq = nq;
  st->psi0 = (double*)xcalloc((size_t)nq, sizeof(double));
  st->phi = (double*)xcalloc((size_t)nq, sizeof(double));
  /* Spring law: Hookean F = H Q, or FENE F = H Q / (1 - |Q|^2 / Q0^2) with
     Q0^2 = b kT/H = b sigma_Q^2 in Q-lattice units (Sec. VI-D). The initial psi
     is the equilibrium of the spring: a Gaussian, or (1 - |Q|^2/Q0^2)^(b/2)
     (Eq. initail_condition), normalised on the masked grid. */
  double gsum = 0;
  for (int q = 0; q < nq; ++q) {
    double q2 = st->Qx[q] * st->Qx[q] + st->Qy[q] * st->Qy[q];
    double g;
    if (lat->fene_b > 0) {
      double s = 1.0 - q2 / (lat->fene_b * lat->sigma_q2);
      st->phi[q] = 1.0 / s;
      g = pow(s, 0.5 * lat->fene_b);
    } else {
      st->phi[q] = 1.0;
      g = exp(-q2 / (2.0 * lat->sigma_q2));
    }
    st->psi0[q] = g;
    gsum += g;
  }
  for (int q = 0; q < nq; ++q) st->psi0[q] = gsum > 0 ? lat->psi_tot * st->psi0[q] / gsum : 0.0;

  int32_t c9[18], opp9[9], c25[100], opp25[25];
  orc_d2q9(c9, st->ws, opp9);
  orc_d4q25(c25, st->wp, opp25);
  for (int i = 0; i < 9; ++i) {
    st->cs[i][0] = c9[2 * i];
    st->cs[i][1] = c9[2 * i + 1];
    st->opps[i] = opp9[i];
  }
  for (int i = 0; i < 25; ++i) {
    for (int k = 0; k < 4; ++k) st->cp[i][k] = c25[4 * i + k];
    st->oppp[i] = opp25[i];
  }

  size_t N = (size_t)st->nx * st->ny;
  st->gs = (double*)xcalloc(N * 9, sizeof(double));
  st->gs_post = (double*)xcalloc(N * 9, sizeof(double));
  st->gp = (double*)xcalloc(N * nq * 25, sizeof(double));
  st->gp_post = (double*)xcalloc(N * nq * 25, sizeof(double));
  st->rho_s = (double*)xcalloc(N, sizeof(double));
  st->jsx = (double*)xcalloc(N, sizeof(double));
  st->jsy = (double*)xcalloc(N, sizeof(double));
  st->psi = (double*)xcalloc(N * nq, sizeof(double));
  st->jr = (double*)xcalloc(N * nq * 2, sizeof(double));
  st->jq = (double*)xcalloc(N * nq * 2, sizeof(double));
  st->dq = (double*)xcalloc(N * nq * 2, sizeof(double));
  st->psitot = (double*)xcalloc(N, sizeof(double));
  st->jpx = (double*)xcalloc(N, sizeof(double));
  st->jpy = (double*)xcalloc(N, sizeof(double));
  st->ex = (double*)xcalloc(N, sizeof(double));
  st->ey = (double*)xcalloc(N, sizeof(double));
  st->ux = (double*)xcalloc(N, sizeof(double));
  st->uy = (double*)xcalloc(N, sizeof(double));
  st->gux = (double*)xcalloc(N * 2, sizeof(double));
  st->guy = (double*)xcalloc(N * 2, sizeof(double));
  return st;
}

void orc_destroy(orc_state* st) {
  if (!st) return;
  void* ptrs[] = {st->qmap, st->qgi, st->qgj, st->Qx, st->Qy, st->psi0, st->phi, st->gs, st->gp,
                  st->gs_post, st->gp_post, st->rho_s, st->jsx, st->jsy, st->psi, st->jr,
                  st->jq, st->dq, st->psitot, st->jpx, st->jpy, st->ex, st->ey, st->ux,
                  st->uy, st->gux, st->guy};
  for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; ++k) free(ptrs[k]);
  free(st);
}

int32_t orc_nq(const orc_state* st) { return st->nq; }

void orc_q_nodes(const orc_state* st, double* qx, double* qy) {
  for (int q = 0; q < st->nq; ++q) {
    qx[q] = st->Qx[q];
    qy[q] = st->Qy[q];
  }
}

void orc_psi0(const orc_state* st, double* psi0) { memcpy(psi0, st->psi0, sizeof(double) * st->nq); }

int32_t orc_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------ accessors */

void orc_get_g(const orc_state* st, double* gs, double* gp) {
  size_t N = (size_t)st->nx * st->ny;
  if (gs) memcpy(gs, st->gs, sizeof(double) * N * 9);
  if (gp) memcpy(gp, st->gp, sizeof(double) * N * st->nq * 25);
}
void orc_set_g(orc_state* st, const double* gs, const double* gp) {
  size_t N = (size_t)st->nx * st->ny;
  if (gs) memcpy(st->gs, gs, sizeof(double) * N * 9);
  if (gp) memcpy(st->gp, gp, sizeof(double) * N * st->nq * 25);
}
void orc_get_gpost(const orc_state* st, double* gs, double* gp) {
  size_t N = (size_t)st->nx * st->ny;
  if (gs) memcpy(gs, st->gs_post, sizeof(double) * N * 9);
  if (gp) memcpy(gp, st->gp_post, sizeof(double) * N * st->nq * 25);
}
void orc_set_gpost(orc_state* st, const double* gs, const double* gp) {
  size_t N = (size_t)st->nx * st->ny;
  if (gs) memcpy(st->gs_post, gs, sizeof(double) * N * 9);
  if (gp) memcpy(st->gp_post, gp, sizeof(double) * N * st->nq * 25);
}

void orc_set_imposed_gradient(orc_state* st, const double* G, int32_t enable) {
  st->imposed = enable ? 1 : 0;
  if (G)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) st->G[a][b] = G[2 * a + b];
}

/* -------------------------------------------------------------- helpers */

static inline int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Kolmogorov body force per unit mass, along x (Sec. VII, f = [F cos(y/l), 0]);
   reading: a(y) = a0 sin(kf y), the same profile shifted in phase. */
static inline double forcing(const orc_state* st, int y) { return st->L.a0 * sin(st->L.kf * y); }

/* Solvent equilibrium about velocity (ux, uy), Eq. dis_eq (c_sS^2 = 1/3). */
static inline double feq_solvent(double w, double rho, int cx, int cy, double ux, double uy) {
  double cu = cx * ux + cy * uy;
  return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
}

/* Linear polymer (quasi-)equilibrium, Eqs. feq_rq_space / fstar_rq_space (c_sP^2 = 1/3). */
static inline double feq_polymer(double w, double psi, const int* c, double jrx, double jry,
                                 double jqx, double jqy) {
  return w * (psi + 3.0 * (jrx * c[0] + jry * c[1] + jqx * c[2] + jqy * c[3]));
}

/* A2-A4: moments of the current g, the elastic drift D, E and U. */
static void macro(orc_state* st) {
  const int nx = st->nx, ny = st->ny, nq = st->nq;
  const double Hl2h = 0.5 * st->L.H * st->L.ell * st->L.ell;
  /* A2: moments */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      const double* g = st->gs + n * 9;
      double rho = 0, jx = 0, jy = 0;
      for (int i = 0; i < 9; ++i) {
        rho += g[i];
        jx += g[i] * st->cs[i][0];
        jy += g[i] * st->cs[i][1];
      }
      st->rho_s[n] = rho;
      st->jsx[n] = jx;
      st->jsy[n] = jy;
      double pt = 0, px = 0, py = 0;
      for (int q = 0; q < nq; ++q) {
        const double* f = st->gp + (n * nq + q) * 25;
        double p = 0, rx = 0, ry = 0, qx = 0, qy = 0;
        for (int i = 0; i < 25; ++i) {
          p += f[i];
          rx += f[i] * st->cp[i][0];
          ry += f[i] * st->cp[i][1];
          qx += f[i] * st->cp[i][2];
          qy += f[i] * st->cp[i][3];
        }
        st->psi[n * nq + q] = p;
        st->jr[(n * nq + q) * 2] = rx;
        st->jr[(n * nq + q) * 2 + 1] = ry;
        st->jq[(n * nq + q) * 2] = qx;
        st->jq[(n * nq + q) * 2 + 1] = qy;
        pt += p;
        px += rx;
        py += ry;
      }
      st->psitot[n] = pt;
      st->jpx[n] = px;
      st->jpy[n] = py;
    }
  /* A3: the bead-force term of Eq. poly_imposed_vel, sum_nu F_nu psi2(r - R_nu, Q),
     with psi2 the per-dumbbell pair density and R_nu = (-1)^nu Q/2, expanded to
     first order as the paper does for the impulse I (Sec. III, Eq. IDef):
     F(Q) [(Q . grad_r) psi2]. reading: the lattice psi counts beads, psi = 2 psi2
     to this order, so D(r,q) = (1/2) F(Q) [(Q . grad_r) psi]; this keeps the
     density equation of Appendix A (centre-of-mass diffusivity kT/(2 zeta)).
     F = H phi_q Q (phi_q = 1 Hookean, 1/(1 - Q^2/Q0^2) FENE), both in r-lengths:
     Q_phys = ell Q. Central differences
     (reading: stencil unspecified). */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      size_t nxp = (size_t)y * nx + wrap(x + 1, nx), nxm = (size_t)y * nx + wrap(x - 1, nx);
      size_t nyp = (size_t)wrap(y + 1, ny) * nx + x, nym = (size_t)wrap(y - 1, ny) * nx + x;
      double ex = 0, ey = 0;
      for (int q = 0; q < nq; ++q) {
        double dpx = 0.5 * (st->psi[nxp * nq + q] - st->psi[nxm * nq + q]);
        double dpy = 0.5 * (st->psi[nyp * nq + q] - st->psi[nym * nq + q]);
        double qgrad = st->Qx[q] * dpx + st->Qy[q] * dpy;
        double dx = Hl2h * st->phi[q] * st->Qx[q] * qgrad;
        double dy = Hl2h * st->phi[q] * st->Qy[q] * qgrad;
        st->dq[(n * nq + q) * 2] = dx;
        st->dq[(n * nq + q) * 2 + 1] = dy;
        ex += dx;
        ey += dy;
      }
      st->ex[n] = ex;
      st->ey[n] = ey;
    }
  /* A4: U of f. Summing the g -> f momentum relations over both species, with
     the body force applied by the same half-step rule:
     rho U = J_S(g) + J_P(g) + (E + rho a) / 2.
     reading: the printed U(f) = U(g) + (dt/2 tau) Theta/rho adds a tensor to a
     vector; Theta enters through its divergence E. */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double a = forcing(st, y);
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      double rho = st->rho_s[n] + st->psitot[n];
      st->ux[n] = (st->jsx[n] + st->jpx[n] + 0.5 * (st->ex[n] + rho * a)) / rho;
      st->uy[n] = (st->jsy[n] + st->jpy[n] + 0.5 * st->ey[n]) / rho;
    }
  }
  /* A5 (first half): grad U by central differences; gux[n][a] = d_a U_x. */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      size_t nxp = (size_t)y * nx + wrap(x + 1, nx), nxm = (size_t)y * nx + wrap(x - 1, nx);
      size_t nyp = (size_t)wrap(y + 1, ny) * nx + x, nym = (size_t)wrap(y - 1, ny) * nx + x;
      st->gux[n * 2] = 0.5 * (st->ux[nxp] - st->ux[nxm]);
      st->gux[n * 2 + 1] = 0.5 * (st->ux[nyp] - st->ux[nym]);
      st->guy[n * 2] = 0.5 * (st->uy[nxp] - st->uy[nxm]);
      st->guy[n * 2 + 1] = 0.5 * (st->uy[nyp] - st->uy[nym]);
    }
}

/* ------------------------------------------------------------- the step */

static void collide_stress_qe(orc_state* st);

void orc_collide(orc_state* st) {
  macro(st);
  if (st->L.qe_model == 1) {
    collide_stress_qe(st);
    return;
  }
  const int nx = st->nx, ny = st->ny, nq = st->nq;
  const double tau1 = st->L.tau1, tau2 = st->L.tau2, kappa = st->L.kappa;
  const double b = 1.0 / (2.0 * tau1 + 1.0); /* beta = dt / (2 tau1 + dt) */
  const double r = tau1 / tau2;
  const double c2 = 2.0 * tau2;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double a = forcing(st, y);
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      double Ux = st->ux[n], Uy = st->uy[n];
      double rho_s = st->rho_s[n];
      double rho = rho_s + st->psitot[n];
      /* velocity gradient G[a][b] = d_a U_b */
      double G00, G01, G10, G11;
      if (st->imposed) {
        G00 = st->G[0][0]; G01 = st->G[0][1]; G10 = st->G[1][0]; G11 = st->G[1][1];
      } else {
        G00 = st->gux[n * 2];     /* d_x U_x */
        G01 = st->guy[n * 2];     /* d_x U_y */
        G10 = st->gux[n * 2 + 1]; /* d_y U_x */
        G11 = st->guy[n * 2 + 1]; /* d_y U_y */
      }
      /* A6, solvent: J_S(f) = (2 tau2 J_S(g) + rho_S U + tau2 rho a) / (2 tau2 + 1);
         the force density rho a acts on the solvent (reading: forcing scheme unstated). */
      double jfx = (c2 * st->jsx[n] + rho_s * Ux + tau2 * rho * a) / (c2 + 1.0);
      double jfy = (c2 * st->jsy[n] + rho_s * Uy) / (c2 + 1.0);
      double usx = jfx / rho_s, usy = jfy / rho_s;
      /* A7, solvent: two-relaxation update with the Guo source of force rho a. */
      const double* g = st->gs + n * 9;
      double* gpost = st->gs_post + n * 9;
      for (int i = 0; i < 9; ++i) {
        int cx = st->cs[i][0], cy = st->cs[i][1];
        double fstar = feq_solvent(st->ws[i], rho_s, cx, cy, usx, usy);
        double feq = feq_solvent(st->ws[i], rho_s, cx, cy, Ux, Uy);
        /* Guo source w_i [3 (c - U) + 9 (c . U) c] . F with F = (rho a, 0). */
        double cu = cx * Ux + cy * Uy;
        double src = st->ws[i] * (3.0 * (cx - Ux) + 9.0 * cu * cx) * rho * a;
        gpost[i] = (1.0 - 2.0 * b) * g[i] + 2.0 * b * ((1.0 - r) * fstar + r * feq) + (1.0 - b) * src;
      }
      /* A5-A7, polymer, per Q-node. */
      for (int q = 0; q < nq; ++q) {
        size_t nqq = n * nq + q;
        double psi = st->psi[nqq];
        double Qx = st->Qx[q], Qy = st->Qy[q];
        /* Eq. poly_imposed_vel: J^r_eq = psi U + D / zeta, 1/zeta = tau2 (m_B = 1) */
        double jrex = psi * Ux + tau2 * st->dq[nqq * 2];
        double jrey = psi * Uy + tau2 * st->dq[nqq * 2 + 1];
        /* J^Q_eq = psi (Q . grad U) - psi 2F/zeta; in Q lattice units the
           spacing ell cancels and 2F/zeta = kappa Q with kappa = 2 H tau2. */
        double jqex = psi * (Qx * G00 + Qy * G10 - kappa * st->phi[q] * Qx);
        double jqey = psi * (Qx * G01 + Qy * G11 - kappa * st->phi[q] * Qy);
        double jrfx = (c2 * st->jr[nqq * 2] + jrex) / (c2 + 1.0);
        double jrfy = (c2 * st->jr[nqq * 2 + 1] + jrey) / (c2 + 1.0);
        double jqfx = (c2 * st->jq[nqq * 2] + jqex) / (c2 + 1.0);
        double jqfy = (c2 * st->jq[nqq * 2 + 1] + jqey) / (c2 + 1.0);
        const double* f = st->gp + nqq * 25;
        double* fpost = st->gp_post + nqq * 25;
        for (int i = 0; i < 25; ++i) {
          double fstar = feq_polymer(st->wp[i], psi, st->cp[i], jrfx, jrfy, jqfx, jqfy);
          double feq = feq_polymer(st->wp[i], psi, st->cp[i], jrex, jrey, jqex, jqey);
          fpost[i] = (1.0 - 2.0 * b) * f[i] + 2.0 * b * ((1.0 - r) * fstar + r * feq);
        }
      }
    }
  }
}

/* Collision with the component stresses quasi-conserved (Sec. V, Eq. quasieq2;
   Sec. VI: f*_S with P_S, f**_P with P^r, P^rQ, P^Q). The targets carry the
   equilibrium momenta (rho_S U for the solvent, J^r_eq and J^Q_eq for the
   polymer, as in the momentum model but with the momentum relaxation time
   tau1 = tau_m) and the current stresses of f; the trapezoidal g-scheme then
   reads g' = (1 - 2 beta) g + 2 beta [(1 - tau1/tau2) f** + (tau1/tau2) f^eq] with
   beta = 1/(2 tau1 + 1). The stresses of f follow from those of g as the
   momenta do in the other model, g = f - (Omega + S)/2 with Omega moving the
   stress at the rate 1/tau2 only and the Guo source S (force F = (rho a, 0) on
   the solvent) adding F U + U F: P_S(f) = (2 tau2 P_S(g) + P_eq + tau2 (F U + U F))
   / (2 tau2 + 1); the polymer carries no source, so P(f) = (2 tau2 P(g) + P_eq) /
   (2 tau2 + 1) for its three blocks.
   reading: the printed quasi-equilibria lack the Hermite normalisations; they
   are the ones that give <f**, vv> = P (1/(2 c_s^4) = 9/2 for the diagonal
   blocks, 1/c_s^4 = 9 for the r-Q block), as the text requires of f**.
   reading: the forcing enters as in the momentum model (Guo source on the
   solvent, half-force shift of U). */
static void collide_stress_qe(orc_state* st) {
  const int nx = st->nx, ny = st->ny, nq = st->nq;
  const double tau1 = st->L.tau1, tau2 = st->L.tau2, kappa = st->L.kappa;
  const double b = 1.0 / (2.0 * tau1 + 1.0);
  const double r = tau1 / tau2;
  const double c2 = 2.0 * tau2;
  const double cs2 = 1.0 / 3.0;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double a = forcing(st, y);
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      double Ux = st->ux[n], Uy = st->uy[n];
      double rho_s = st->rho_s[n];
      double rho = rho_s + st->psitot[n];
      double G00, G01, G10, G11;
      if (st->imposed) {
        G00 = st->G[0][0]; G01 = st->G[0][1]; G10 = st->G[1][0]; G11 = st->G[1][1];
      } else {
        G00 = st->gux[n * 2]; G01 = st->guy[n * 2]; G10 = st->gux[n * 2 + 1]; G11 = st->guy[n * 2 + 1];
      }
      /* solvent: P_S(g), P_eq = rho_S (c_s^2 I + U U), P_S(f) */
      const double* g = st->gs + n * 9;
      double* gpost = st->gs_post + n * 9;
      double pxx = 0, pxy = 0, pyy = 0;
      for (int i = 0; i < 9; ++i) {
        int cx = st->cs[i][0], cy = st->cs[i][1];
        pxx += g[i] * cx * cx;
        pxy += g[i] * cx * cy;
        pyy += g[i] * cy * cy;
      }
      double exx = rho_s * (cs2 + Ux * Ux), exy = rho_s * Ux * Uy, eyy = rho_s * (cs2 + Uy * Uy);
      double Fx = rho * a; /* F = (rho a, 0): F U + U F = (2 Fx Ux, Fx Uy; Fx Uy, 0) */
      double fxx = (c2 * pxx + exx + tau2 * 2.0 * Fx * Ux) / (c2 + 1.0);
      double fxy = (c2 * pxy + exy + tau2 * Fx * Uy) / (c2 + 1.0);
      double fyy = (c2 * pyy + eyy) / (c2 + 1.0);
      for (int i = 0; i < 9; ++i) {
        int cx = st->cs[i][0], cy = st->cs[i][1];
        /* f*_S = w [rho_S + rho_S c.U / c_s^2 + (P_S - rho_S c_s^2 I):(cc - c_s^2 I) / (2 c_s^4)] */
        double hxx = cx * cx - cs2, hxy = (double)(cx * cy), hyy = cy * cy - cs2;
        double pneq = (fxx - rho_s * cs2) * hxx + 2.0 * fxy * hxy + (fyy - rho_s * cs2) * hyy;
        double fss = st->ws[i] * (rho_s + 3.0 * rho_s * (cx * Ux + cy * Uy) + 4.5 * pneq);
        double feq = feq_solvent(st->ws[i], rho_s, cx, cy, Ux, Uy);
        double cu = cx * Ux + cy * Uy;
        double src = st->ws[i] * (3.0 * (cx - Ux) + 9.0 * cu * cx) * rho * a;
        gpost[i] = (1.0 - 2.0 * b) * g[i] + 2.0 * b * ((1.0 - r) * fss + r * feq) + (1.0 - b) * src;
      }
      /* polymer, per Q-node */
      for (int q = 0; q < nq; ++q) {
        size_t nqq = n * nq + q;
        double psi = st->psi[nqq];
        double Qx = st->Qx[q], Qy = st->Qy[q];
        double jrex = psi * Ux + tau1 * st->dq[nqq * 2];
        double jrey = psi * Uy + tau1 * st->dq[nqq * 2 + 1];
        double jqex = psi * (Qx * G00 + Qy * G10 - kappa * st->phi[q] * Qx);
        double jqey = psi * (Qx * G01 + Qy * G11 - kappa * st->phi[q] * Qy);
        const double* f = st->gp + nqq * 25;
        double* fpost = st->gp_post + nqq * 25;
        /* second moments of g: P^r (vv), P^rQ (v Qdot), P^Q (Qdot Qdot); c = (vx, vy, Qx', Qy') */
        double P[4][4];
        for (int u = 0; u < 4; ++u)
          for (int v = 0; v < 4; ++v) P[u][v] = 0.0;
        for (int i = 0; i < 25; ++i)
          for (int u = 0; u < 4; ++u)
            for (int v = 0; v < 4; ++v) P[u][v] += f[i] * st->cp[i][u] * st->cp[i][v];
        /* P(f) = (2 tau2 P(g) + P_eq) / (2 tau2 + 1), P_eq = psi c_s^2 I (linear equilibrium) */
        for (int u = 0; u < 4; ++u)
          for (int v = 0; v < 4; ++v) P[u][v] = (c2 * P[u][v] + (u == v ? psi * cs2 : 0.0)) / (c2 + 1.0);
        for (int i = 0; i < 25; ++i) {
          const int* c = st->cp[i];
          /* (P^r - psi c_s^2 I):(vv - c_s^2 I) / (2 c_s^4) + (P^Q - psi c_s^2 I):(QQ - c_s^2 I) / (2 c_s^4)
             + P^rQ : (v Qdot) / c_s^4 */
          double sdiag = 0.0, scross = 0.0;
          for (int blk = 0; blk < 2; ++blk)
            for (int u = 2 * blk; u < 2 * blk + 2; ++u)
              for (int v = 2 * blk; v < 2 * blk + 2; ++v)
                sdiag += (P[u][v] - (u == v ? psi * cs2 : 0.0)) * (c[u] * c[v] - (u == v ? cs2 : 0.0));
          for (int u = 0; u < 2; ++u)
            for (int v = 2; v < 4; ++v) scross += P[u][v] * c[u] * c[v];
          double fss = feq_polymer(st->wp[i], psi, c, jrex, jrey, jqex, jqey) +
                       st->wp[i] * (4.5 * sdiag + 9.0 * scross);
          double feq = feq_polymer(st->wp[i], psi, c, jrex, jrey, jqex, jqey);
          fpost[i] = (1.0 - 2.0 * b) * f[i] + 2.0 * b * ((1.0 - r) * fss + r * feq);
        }
      }
    }
  }
}

/* A1: pull streaming. Solvent: g_i(r) = g'_i(r - c_i), periodic (Sec. VII).
   Polymer: g_i(r, Q) = g'_i(r - v_i, Q - Qdot_i) if Q - Qdot_i lies in the disk,
   else g'_{-i}(r, Q). reading: full (halfway) bounce-back reverses all four
   components, so the population returns to its own (r, Q) node. */
void orc_stream(orc_state* st) {
  const int nx = st->nx, ny = st->ny, nq = st->nq, S = st->S;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      for (int i = 0; i < 9; ++i) {
        size_t src = (size_t)wrap(y - st->cs[i][1], ny) * nx + wrap(x - st->cs[i][0], nx);
        st->gs[n * 9 + i] = st->gs_post[src * 9 + i];
      }
      for (int q = 0; q < nq; ++q)
        for (int i = 0; i < 25; ++i) {
          int si = st->qgi[q] - st->cp[i][2], sj = st->qgj[q] - st->cp[i][3];
          int sq = (si >= 0 && si < S && sj >= 0 && sj < S) ? st->qmap[sj * S + si] : -1;
          double v;
          if (sq >= 0) {
            size_t src = (size_t)wrap(y - st->cp[i][1], ny) * nx + wrap(x - st->cp[i][0], nx);
            v = st->gp_post[(src * nq + sq) * 25 + i];
          } else {
            v = st->gp_post[(n * nq + q) * 25 + st->oppp[i]];
          }
          st->gp[(n * nq + q) * 25 + i] = v;
        }
    }
}

void orc_step(orc_state* st, int32_t n) {
  for (int32_t k = 0; k < n; ++k) {
    orc_collide(st);
    orc_stream(st);
  }
}

/* ------------------------------------------------------ initial condition */

/* Initial state (Sec. VI-D, VII). reading: Hookean dumbbells in place of FENE,
   so psi(r, Q, 0) is the Gaussian exp(-|Q|^2 / (2 sigma_Q^2)) normalised on the
   masked grid to sum psi_tot; the flow starts from rest (ic_mode 0) or from the
   laminar profile (ic_mode 1), plus the supplied perturbation; g = f^eq of
   these fields with J^r_eq = psi U and J^Q_eq = psi (Q . grad U - kappa Q)
   (grad_r psi = 0 initially), grad U by central differences. */
void orc_init(orc_state* st, const double* perturb, int32_t ic_mode) {
  const int nx = st->nx, ny = st->ny, nq = st->nq;
  size_t N = (size_t)nx * ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      double ux = ic_mode == 1 ? st->L.u0 * sin(st->L.kf * y) : 0.0;
      double uy = 0.0;
      if (perturb) {
        ux += perturb[n];
        uy += perturb[N + n];
      }
      st->ux[n] = ux;
      st->uy[n] = uy;
    }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t n = (size_t)y * nx + x;
      size_t nxp = (size_t)y * nx + wrap(x + 1, nx), nxm = (size_t)y * nx + wrap(x - 1, nx);
      size_t nyp = (size_t)wrap(y + 1, ny) * nx + x, nym = (size_t)wrap(y - 1, ny) * nx + x;
      double G00 = 0.5 * (st->ux[nxp] - st->ux[nxm]);
      double G10 = 0.5 * (st->ux[nyp] - st->ux[nym]);
      double G01 = 0.5 * (st->uy[nxp] - st->uy[nxm]);
      double G11 = 0.5 * (st->uy[nyp] - st->uy[nym]);
      double Ux = st->ux[n], Uy = st->uy[n];
      for (int i = 0; i < 9; ++i)
        st->gs[n * 9 + i] = feq_solvent(st->ws[i], 1.0, st->cs[i][0], st->cs[i][1], Ux, Uy);
      for (int q = 0; q < nq; ++q) {
        double psi = st->psi0[q];
        double Qx = st->Qx[q], Qy = st->Qy[q];
        double jrx = psi * Ux, jry = psi * Uy;
        double jqx = psi * (Qx * G00 + Qy * G10 - st->L.kappa * st->phi[q] * Qx);
        double jqy = psi * (Qx * G01 + Qy * G11 - st->L.kappa * st->phi[q] * Qy);
        for (int i = 0; i < 25; ++i)
          st->gp[(n * nq + q) * 25 + i] = feq_polymer(st->wp[i], psi, st->cp[i], jrx, jry, jqx, jqy);
      }
    }
}

/* ------------------------------------------------------------ observables */

/* Fields of the current g (Sec. VII diagnostics): rho_S, psi_tot, U; the
   conformation C = ell^2 sum_q psi Q Q / psi_tot (r-lengths); the elastic
   stress Theta = (ell^2 / 2) sum_q psi Q F(Q) (Sec. III, Eq. IDef; (H ell^2 / 2)
   sum_q phi_q psi Q Q with the spring factor phi_q, psi counting beads); Q_rms = sqrt(<psi Q^2> / <psi>); vorticity d_x U_y - d_y U_x. */
void orc_fields(orc_state* st, double* out, double* psi_out, double* e_out) {
  macro(st);
  const int nx = st->nx, ny = st->ny, nq = st->nq;
  size_t N = (size_t)nx * ny;
  const double l2 = st->L.ell * st->L.ell, H = st->L.H;
  for (size_t n = 0; n < N; ++n) {
    double sxx = 0, sxy = 0, syy = 0, fxx = 0, fxy = 0, fyy = 0;
    for (int q = 0; q < nq; ++q) {
      double p = st->psi[n * nq + q];
      sxx += p * st->Qx[q] * st->Qx[q];
      sxy += p * st->Qx[q] * st->Qy[q];
      syy += p * st->Qy[q] * st->Qy[q];
      fxx += st->phi[q] * p * st->Qx[q] * st->Qx[q];
      fxy += st->phi[q] * p * st->Qx[q] * st->Qy[q];
      fyy += st->phi[q] * p * st->Qy[q] * st->Qy[q];
    }
    double pt = st->psitot[n];
    out[ORC_F_RHO_S * N + n] = st->rho_s[n];
    out[ORC_F_PSI_TOT * N + n] = pt;
    out[ORC_F_UX * N + n] = st->ux[n];
    out[ORC_F_UY * N + n] = st->uy[n];
    double cxx = pt != 0 ? l2 * sxx / pt : 0, cxy = pt != 0 ? l2 * sxy / pt : 0,
           cyy = pt != 0 ? l2 * syy / pt : 0;
    out[ORC_F_CXX * N + n] = cxx;
    out[ORC_F_CXY * N + n] = cxy;
    out[ORC_F_CYY * N + n] = cyy;
    out[ORC_F_THXX * N + n] = 0.5 * H * l2 * fxx;
    out[ORC_F_THXY * N + n] = 0.5 * H * l2 * fxy;
    out[ORC_F_THYY * N + n] = 0.5 * H * l2 * fyy;
    out[ORC_F_QRMS * N + n] = sqrt(cxx + cyy);
    /* d_x U_y - d_y U_x */
    out[ORC_F_VORT * N + n] = st->guy[n * 2] - st->gux[n * 2 + 1];
    if (e_out) {
      e_out[n] = st->ex[n];
      e_out[N + n] = st->ey[n];
    }
  }
  if (psi_out) memcpy(psi_out, st->psi, sizeof(double) * N * nq);
}

/* Global diagnostics (Sec. VII): masses, momentum sum rho U, kinetic energy,
   enstrophy (1/2) sum omega^2, mean Q_rms, and sum U_y^2 (growth indicator). */
void orc_diagnostics(orc_state* st, double* out) {
  const int nx = st->nx, ny = st->ny;
  size_t N = (size_t)nx * ny;
  double* f = (double*)xcalloc(N * ORC_NFIELDS, sizeof(double));
  orc_fields(st, f, NULL, NULL);
  double d[ORC_NDIAG] = {0};
  for (size_t n = 0; n < N; ++n) {
    double rho = f[ORC_F_RHO_S * N + n] + f[ORC_F_PSI_TOT * N + n];
    double ux = f[ORC_F_UX * N + n], uy = f[ORC_F_UY * N + n];
    double w = f[ORC_F_VORT * N + n];
    d[ORC_D_MASS_S] += f[ORC_F_RHO_S * N + n];
    d[ORC_D_MASS_P] += f[ORC_F_PSI_TOT * N + n];
    d[ORC_D_PX] += rho * ux;
    d[ORC_D_PY] += rho * uy;
    d[ORC_D_KE] += 0.5 * rho * (ux * ux + uy * uy);
    d[ORC_D_ENSTROPHY] += 0.5 * w * w;
    d[ORC_D_QRMS_MEAN] += f[ORC_F_QRMS * N + n];
    d[ORC_D_EY2] += uy * uy;
  }
  d[ORC_D_QRMS_MEAN] /= (double)N;
  memcpy(out, d, sizeof d);
  free(f);
}
