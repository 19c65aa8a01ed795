// Host side of libtfkt: parameter mapping, lattice tables, workspace layout
// and the extern "C" entry points declared in include/tfkt.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"

namespace tfkt {

thread_local std::string g_last_error;

tfkt_status fail(tfkt_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

tfkt_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  if (c) c->poisoned = true;
  return fail(TFKT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TFKT_CUDA(ctx, ...)                                             \
  do {                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                     \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #__VA_ARGS__);   \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Physical -> lattice parameters (Sec. VII definitions Re = U0 l / nu,
// Wi = U0 lambda_H / l, beta = eta_s / (eta_s + eta_p), F = eta U0 / l^2):
// nu_s = c_s^2 tau1 (trapezoidal scheme), lambda_H = zeta / (4 H) with
// zeta = m_B / tau2 (Appendix A), Q-drift 2 H / zeta = kappa, Q spacing
// ell = sqrt(2) from the Q-diffusivity 2 kT / zeta of Eq. Smoluchowski_new11,
// and psi_tot from eta_p = (H ell^2 / 2) psi_tot sigma_Q^2 lambda_H
// (psi counts beads). FENE springs keep this mapping (H, lambda_H and the
// stress scale n kT lambda_H of the Hookean dumbbell of the same H) and add
// Q0^2 = b kT/H = b sigma_Q^2, inside which every Q-node must lie.
tfkt_status map_params(const tfkt_params* p, Lattice* L) {
  if (!p) return fail(TFKT_EINVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1) return fail(TFKT_EINVAL, "nx and ny must be >= 1");
  if (p->q_side < 1 || p->q_side > 64) return fail(TFKT_EINVAL, "q_side must be in [1, 64]");
  if (!(p->q_radius > 0)) return fail(TFKT_EINVAL, "q_radius must be > 0");
  if (!(p->re > 0)) return fail(TFKT_EINVAL, "re must be > 0");
  if (!(p->beta > 0) || p->beta > 1) return fail(TFKT_EINVAL, "beta must be in (0, 1]");
  if (!(p->u0 > 0) || p->u0 > 0.2) return fail(TFKT_EINVAL, "u0 must be in (0, 0.2]");
  if (p->k_periods < 1) return fail(TFKT_EINVAL, "k_periods must be >= 1");
  if (!(p->wi >= 0)) return fail(TFKT_EINVAL, "wi must be >= 0");
  if (p->wi == 0 && p->beta < 1) return fail(TFKT_EINVAL, "wi = 0 needs beta = 1 (no polymer)");
  if (p->precision != TFKT_FP64 && p->precision != TFKT_FP32 && p->precision != TFKT_FP16)
    return fail(TFKT_EINVAL, "unknown precision");
  if (p->ic_mode != 0 && p->ic_mode != 1) return fail(TFKT_EINVAL, "ic_mode must be 0 or 1");
  if (!(p->fene_b >= 0)) return fail(TFKT_EINVAL, "fene_b must be >= 0 (0: Hookean)");
  if (p->qe_model != TFKT_QE_MOMENTUM && p->qe_model != TFKT_QE_STRESS)
    return fail(TFKT_EINVAL, "unknown qe_model");
  Lattice l;
  l.nx = p->nx;
  l.ny = p->ny;
  l.S = p->q_side;
  l.q_radius = p->q_radius;
  l.ic_mode = p->ic_mode;
  l.precision = p->precision;
  l.fene_b = p->fene_b;
  l.qe_model = p->qe_model;
  const double kf = 2.0 * M_PI * p->k_periods / p->ny;
  const double len = 1.0 / kf;
  l.kf = kf;
  l.u0 = p->u0;
  l.nu = p->u0 * len / p->re;
  l.nu_s = p->beta * l.nu;
  // the viscosity comes from the stress relaxation time tau_s = 3 nu_s, the drag and
  // diffusion from the momentum relaxation time tau_m (tau2 input, default tau_s);
  // the momentum model relaxes the stress first (tau1 = tau_s <= tau2 = tau_m), the
  // stress model the momenta (tau1 = tau_m <= tau2 = tau_s), Sec. V
  const double tau_s = 3.0 * l.nu_s;
  l.tau_m = p->tau2 > 0 ? p->tau2 : tau_s;
  if (l.qe_model == TFKT_QE_MOMENTUM) {
    if (l.tau_m < tau_s) return fail(TFKT_EINVAL, "momentum model: tau2 must be >= 3 beta nu");
    l.tau1 = tau_s;
    l.tau2 = l.tau_m;
  } else {
    if (l.tau_m > tau_s) return fail(TFKT_EINVAL, "stress model: tau2 must be <= 3 beta nu");
    l.tau1 = l.tau_m;
    l.tau2 = tau_s;
  }
  l.ell = p->ell > 0 ? p->ell : std::sqrt(2.0);
  l.eta_p = (1.0 - p->beta) * l.nu;
  l.a0 = l.nu * p->u0 * kf * kf;
  if (p->wi > 0) {
    l.lambda_h = p->wi * len / p->u0;
    l.H = 1.0 / (4.0 * l.lambda_h * l.tau_m);
    l.kappa = 2.0 * l.H * l.tau_m;
    l.sigma_q2 = l.tau_m / (3.0 * l.kappa);
    l.psi_tot = l.eta_p / (0.5 * l.H * l.ell * l.ell * l.sigma_q2 * l.lambda_h);
  } else {
    l.lambda_h = 0;
    l.H = 0;
    l.kappa = 0;
    l.sigma_q2 = 1.0;
    l.psi_tot = 0;
  }
  // Q-disk nodes
  int nq = 0;
  const double R2 = p->q_radius * p->q_radius + 1e-9;
  for (int j = 0; j < l.S; ++j)
    for (int i = 0; i < l.S; ++i) {
      const double qx = i - 0.5 * (l.S - 1), qy = j - 0.5 * (l.S - 1);
      if (qx * qx + qy * qy <= R2) ++nq;
    }
  if (nq < 1) return fail(TFKT_EINVAL, "the Q-disk holds no node");
  if (l.fene_b > 0 && p->q_radius * p->q_radius >= l.fene_b * l.sigma_q2)
    return fail(TFKT_EINVAL, "FENE: q_radius must be < Q0 = sqrt(fene_b sigma_q2)");
  l.nq = nq;
  l.pitch = align_up((size_t)l.nx, 32);
  l.plane = (size_t)l.ny * l.pitch;
  l.npl = 9 + 25 * nq;
  l.nm = nq + M_NSCALAR;
  *L = l;
  return TFKT_OK;
}

size_t real_size(const Lattice& L) { return L.precision == TFKT_FP64 ? 8 : 4; }
double polymer_scale(const Lattice& L) {
  if (L.precision != TFKT_FP16 || !(L.psi_tot > 0)) return 1.0;
  // typical stored value w_i psi0(q) ~ psi_tot / (36 nq): scale it to about one
  const double target = 36.0 * L.nq / L.psi_tot;
  return std::ldexp(1.0, (int)std::lround(std::log2(target)));
}

size_t store_size(const Lattice& L) {
  return L.precision == TFKT_FP64 ? 8 : (L.precision == TFKT_FP16 ? 2 : 4);
}

// 9 + 25 nq plane slots of the storage type, and under FP16 storage the nine
// FP32 solvent planes after them (the layout of solvent_planes).
size_t population_bytes(const Lattice& L) {
  const size_t slots = (size_t)L.npl * L.plane * store_size(L);
  return L.precision == TFKT_FP16 ? slots + 9 * L.plane * sizeof(float) : slots;
}

// Blocks of the diagnostics reduction: one or more rows each, at most 8 per SM.
int diag_blocks_for(const Lattice& L) { return L.ny < 8 * 152 ? L.ny : 8 * 152; }

// Workspace layout; returns the total size.
size_t layout(const Lattice& L, Workspace* w) {
  const size_t sz = real_size(L), A = 256;
  size_t o = 0;
  // a population buffer also stages field output (doubles) and the initial perturbation
  const size_t N = (size_t)L.nx * L.ny;
  size_t pop = population_bytes(L);
  if (pop < (size_t)TFKT_NFIELDS * N * sizeof(double)) pop = (size_t)TFKT_NFIELDS * N * sizeof(double);
  w->off_pop[0] = o;
  o = align_up(o + pop, A);
  w->off_pop[1] = o;
  o = align_up(o + pop, A);
  w->off_M = o;
  o = align_up(o + (size_t)L.nm * L.plane * sz, A);
  w->off_U = o;
  o = align_up(o + 2 * L.plane * sz, A);
  w->off_tab = o;
  const size_t tab = (5 * (size_t)L.nq + 25 * (size_t)L.nq + 2 * (size_t)L.ny) * sz +
                     25 * (size_t)L.nq * sizeof(int) + 10 * A;
  o = align_up(o + tab, A);
  w->off_part = o;
  o = align_up(o + (size_t)diag_blocks_for(L) * TFKT_NDIAG * sizeof(double), A);
  w->off_diag = o;
  o = align_up(o + TFKT_NDIAG * sizeof(double), A);
  if (fused_path(L)) {
    w->off_M2 = o;
    o = align_up(o + (size_t)L.nm * L.plane * sz, A);
    w->off_exp = o;
    o = align_up(o + fused_export_capacity(L.nx, L.ny, L.nq) * sz, A);
    w->off_ftab = o;
    o = align_up(o + (size_t)L.nq * (9 * sizeof(int) + sz + 25 * sizeof(long long)) + 2 * A, A);
  }
  return o;
}

int opposite25(int i) {
  const V4 c = c25(i);
  for (int j = 0; j < 25; ++j) {
    const V4 d = c25(j);
    if (d.rx == -c.rx && d.ry == -c.ry && d.qx == -c.qx && d.qy == -c.qy) return j;
  }
  return -1;
}

// Q-nodes (cell-centred S x S grid inside the disk |Q| <= R, Sec. VI-D),
// the spring force per unit H, phi_q Q, the initial psi0(q) (the spring's
// equilibrium: Gaussian, or (1 - Q^2/Q0^2)^(b/2) for FENE, normalised on the
// masked grid to psi_tot), the pull table with bounce-back at the disk edge,
// the forcing a(y) = a0 sin(kf y) (Sec. VII) and the initial base flow.
HostTables build_tables(const Lattice& L) {
  HostTables t;
  std::vector<int> qmap((size_t)L.S * L.S, -1), gi, gj;
  const double R2 = L.q_radius * L.q_radius + 1e-9;
  for (int j = 0; j < L.S; ++j)
    for (int i = 0; i < L.S; ++i) {
      const double qx = i - 0.5 * (L.S - 1), qy = j - 0.5 * (L.S - 1);
      if (qx * qx + qy * qy <= R2) {
        qmap[(size_t)j * L.S + i] = (int)t.qx.size();
        t.qx.push_back(qx);
        t.qy.push_back(qy);
        gi.push_back(i);
        gj.push_back(j);
      }
    }
  double gsum = 0;
  for (int q = 0; q < L.nq; ++q) {
    const double q2 = t.qx[q] * t.qx[q] + t.qy[q] * t.qy[q];
    double g, phi;
    if (L.fene_b > 0) {
      const double u = 1.0 - q2 / (L.fene_b * L.sigma_q2);
      phi = 1.0 / u;
      g = std::pow(u, 0.5 * L.fene_b);
    } else {
      phi = 1.0;
      g = std::exp(-q2 / (2.0 * L.sigma_q2));
    }
    t.fx.push_back(L.fene_b > 0 ? phi * t.qx[q] : t.qx[q]);
    t.fy.push_back(L.fene_b > 0 ? phi * t.qy[q] : t.qy[q]);
    t.psi0.push_back(g);
    gsum += g;
  }
  for (double& v : t.psi0) v = gsum > 0 ? L.psi_tot * v / gsum : 0.0;
  t.pull.resize((size_t)L.nq * 25);
  t.delta.resize((size_t)L.nq * 25);
  for (int q = 0; q < L.nq; ++q)
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const int si = gi[q] - c.qx, sj = gj[q] - c.qy;
      const int sq = (si >= 0 && si < L.S && sj >= 0 && sj < L.S) ? qmap[(size_t)sj * L.S + si] : -1;
      if (sq >= 0) {
        t.pull[(size_t)q * 25 + i] = 9 + 25 * sq + i;
        t.delta[(size_t)q * 25 + i] = w25(i) * (t.psi0[sq] - t.psi0[q]);
      } else {
        t.pull[(size_t)q * 25 + i] = ~(9 + 25 * q + opposite25(i));
        t.delta[(size_t)q * 25 + i] = 0.0;
      }
    }
  // forcing and laminar profile of each row, at its global row (a slab's rows are
  // rows of a larger run)
  const int nyg = L.ny_global > 0 ? L.ny_global : L.ny;
  for (int y = 0; y < L.ny; ++y) {
    const int yg = ((L.y_origin + y) % nyg + nyg) % nyg;
    t.arow.push_back(L.a0 * std::sin(L.kf * yg));
    t.urow.push_back(L.ic_mode == 1 ? L.u0 * std::sin(L.kf * yg) : 0.0);
  }
  return t;
}

namespace {

template <typename real>
KernelArgs<real> make_args(const Ctx* c, const HostTables* ht = nullptr) {
  const Lattice& L = c->L;
  char* base = (char*)c->ws.base;
  KernelArgs<real> a{};
  a.src = base + c->ws.off_pop[c->cur];
  a.dst = base + c->ws.off_pop[c->cur ^ 1];
  a.M = (real*)(base + (c->mcur ? c->ws.off_M2 : c->ws.off_M));
  a.U = (real*)(base + c->ws.off_U);
  a.perturb = nullptr;
  a.nx = L.nx;
  a.ny = L.ny;
  a.nq = L.nq;
  a.pitch = L.pitch;
  a.plane = L.plane;
  const double b = 1.0 / (2.0 * L.tau1 + 1.0);
  a.tau2 = (real)L.tau2;
  a.c2 = (real)(2.0 * L.tau2);
  a.inv_c2p1 = (real)(1.0 / (2.0 * L.tau2 + 1.0));
  a.om2b = (real)(1.0 - 2.0 * b);
  a.tb = (real)(2.0 * b);
  a.omb = (real)(1.0 - b);
  a.r = (real)(L.tau1 / L.tau2);
  a.omr = (real)(1.0 - L.tau1 / L.tau2);
  a.kappa = (real)L.kappa;
  a.hl2h = (real)(0.5 * L.H * L.ell * L.ell);
  a.tau_m = (real)L.tau_m;
  a.qe = L.qe_model;
  a.rho0 = (real)(1.0 + L.psi_tot);
  a.psi_tot0 = (real)L.psi_tot;
  a.l2 = (real)(L.ell * L.ell);
  a.H = (real)L.H;
  a.pscale = (real)polymer_scale(L);
  a.pinv = (real)(1.0 / polymer_scale(L));
  // tables
  char* tb = base + c->ws.off_tab;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = tb + o;
    o = align_up(o + bytes, 256);
    return p;
  };
  const size_t nq = L.nq;
  a.tab.qx = (const real*)take(nq * sizeof(real));
  a.tab.qy = (const real*)take(nq * sizeof(real));
  a.tab.fx = (const real*)take(nq * sizeof(real));
  a.tab.fy = (const real*)take(nq * sizeof(real));
  a.tab.psi0 = (const real*)take(nq * sizeof(real));
  a.tab.pull = (const int*)take(nq * 25 * sizeof(int));
  a.tab.delta = (const real*)take(nq * 25 * sizeof(real));
  a.tab.arow = (const real*)take((size_t)L.ny * sizeof(real));
  a.tab.urow = (const real*)take((size_t)L.ny * sizeof(real));
  (void)ht;
  return a;
}

template <typename real>
FusedArgs<real> make_fused(const Ctx* c) {
  const Lattice& L = c->L;
  char* base = (char*)c->ws.base;
  FusedArgs<real> f{};
  f.Min = (const real*)(base + (c->mcur ? c->ws.off_M2 : c->ws.off_M));
  f.Mout = (real*)(base + (c->mcur ? c->ws.off_M : c->ws.off_M2));
  f.exports = (real*)(base + c->ws.off_exp);
  f.tgt = (const int*)(base + c->ws.off_ftab);
  f.dpsi = (const real*)(base + c->ws.off_ftab + align_up((size_t)L.nq * 9 * sizeof(int), 256));
  f.poff = (const long long*)((const char*)f.dpsi + align_up((size_t)L.nq * sizeof(real), 256));
  f.dvx = (real)c->dvx;
  f.dvy = (real)c->dvy;
  return f;
}

template <typename real>
tfkt_status upload_fused_tables(Ctx* c, const HostTables& t) {
  std::vector<int> tgt;
  std::vector<double> dpsi;
  std::vector<long long> poff;
  fused_tables(c->L, t, tgt, dpsi, c->dvx, c->dvy, poff);
  FusedArgs<real> f = make_fused<real>(c);
  std::vector<real> d(dpsi.begin(), dpsi.end());
  TFKT_CUDA(c, cudaMemcpy((void*)f.poff, poff.data(), poff.size() * sizeof(long long),
                          cudaMemcpyHostToDevice));
  TFKT_CUDA(c, cudaMemcpy((void*)f.tgt, tgt.data(), tgt.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  TFKT_CUDA(c, cudaMemcpy((void*)f.dpsi, d.data(), d.size() * sizeof(real),
                          cudaMemcpyHostToDevice));
  return TFKT_OK;
}

template <typename real>
tfkt_status upload_tables(Ctx* c, const HostTables& t) {
  KernelArgs<real> a = make_args<real>(c);
  auto put = [&](const void* dptr, const std::vector<double>& v) -> cudaError_t {
    std::vector<real> h(v.begin(), v.end());
    return cudaMemcpy((void*)dptr, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice);
  };
  TFKT_CUDA(c, put(a.tab.qx, t.qx));
  TFKT_CUDA(c, put(a.tab.qy, t.qy));
  TFKT_CUDA(c, put(a.tab.fx, t.fx));
  TFKT_CUDA(c, put(a.tab.fy, t.fy));
  TFKT_CUDA(c, put(a.tab.psi0, t.psi0));
  TFKT_CUDA(c, cudaMemcpy((void*)a.tab.pull, t.pull.data(), t.pull.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  TFKT_CUDA(c, put(a.tab.delta, t.delta));
  TFKT_CUDA(c, put(a.tab.arow, t.arow));
  TFKT_CUDA(c, put(a.tab.urow, t.urow));
  if (c->fused) return upload_fused_tables<real>(c, t);
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status init_state(Ctx* c, const double* perturb) {
  const Lattice& L = c->L;
  KernelArgs<real> a = make_args<real>(c);
  // The buffer that the first step writes is free now: stage the perturbation there.
  double* dpert = nullptr;
  if (perturb) {
    dpert = (double*)((char*)c->ws.base + c->ws.off_pop[1]);
    TFKT_CUDA(c, cudaMemcpyAsync(dpert, perturb, sizeof(double) * 2 * (size_t)L.nx * L.ny,
                                 cudaMemcpyHostToDevice, c->stream));
  }
  a.perturb = dpert;
  a.dst = (char*)c->ws.base + c->ws.off_pop[0];
  TFKT_CUDA(c, launch_init<real, S>(a, c->stream));   // populations and their moments
  c->cur = 0;
  c->m_valid = true;
  TFKT_CUDA(c, cudaStreamSynchronize(c->stream));
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status ensure_moments(Ctx* c) {
  if (c->m_valid) return TFKT_OK;
  KernelArgs<real> a = make_args<real>(c);
  TFKT_CUDA(c, launch_moments<real, S>(a, c->stream));
  c->m_valid = true;
  return TFKT_OK;
}

// One step. Fused path: the step kernel also produces the next state's
// moment planes (completed at tile borders by the fix-up kernel), so the
// moments stay valid. Two-pass path: moments kernel, then the step kernel.
template <typename real, typename S>
tfkt_status do_step(Ctx* c, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    tfkt_status s = ensure_moments<real, S>(c);
    if (s != TFKT_OK) return s;
    KernelArgs<real> a = make_args<real>(c);
    if (c->fused) {
      FusedArgs<real> f = make_fused<real>(c);
      if (c->lpm_pending) f.rshp = (const real*)c->lpm_rshp;
      TFKT_CUDA(c, launch_step_fused<real, S>(a, f, c->stream));
      TFKT_CUDA(c, launch_fixup<real>(a, f, c->stream));
      c->lpm_pending = false;
      c->mcur ^= 1;
    } else {
      TFKT_CUDA(c, launch_step<real, S>(a, c->stream));
      c->m_valid = false;
    }
    c->cur ^= 1;
    ++c->step;
  }
  return TFKT_OK;
}

// tfkt_step with an event pair around each launch (profiling only).
template <typename real, typename S>
tfkt_status do_step_profiled(Ctx* c, int64_t n, double* ms, int64_t* launches) {
  // An event pair around every launch, recorded without waiting, so that the
  // launches stay queued back to back as in tfkt_step; the times are read once
  // per CHUNK launches (and at the end), which is when the host waits.
  constexpr int CHUNK = 64;
  cudaEvent_t ev[2 * CHUNK];
  int created = 0;
  struct Guard {
    cudaEvent_t* e;
    int* n;
    ~Guard() {
      for (int k = 0; k < *n; ++k) cudaEventDestroy(e[k]);
    }
  } guard{ev, &created};
  for (; created < 2 * CHUNK; ++created) TFKT_CUDA(c, cudaEventCreate(&ev[created]));
  double acc[TFKT_NKERNELS] = {};
  int64_t cnt[TFKT_NKERNELS] = {};
  int kinds[CHUNK];
  int pending = 0;
  auto drain = [&]() -> tfkt_status {
    if (pending == 0) return TFKT_OK;
    TFKT_CUDA(c, cudaEventSynchronize(ev[2 * pending - 1]));
    for (int k = 0; k < pending; ++k) {
      float t = 0;
      TFKT_CUDA(c, cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]));
      acc[kinds[k]] += t;
      ++cnt[kinds[k]];
    }
    pending = 0;
    return TFKT_OK;
  };
  auto timed = [&](int kind, auto&& launch) -> tfkt_status {
    if (pending == CHUNK) {
      tfkt_status s = drain();
      if (s != TFKT_OK) return s;
    }
    TFKT_CUDA(c, cudaEventRecord(ev[2 * pending], c->stream));
    TFKT_CUDA(c, launch());
    TFKT_CUDA(c, cudaEventRecord(ev[2 * pending + 1], c->stream));
    kinds[pending++] = kind;
    return TFKT_OK;
  };
  for (int64_t k = 0; k < n; ++k) {
    if (!c->m_valid) {
      KernelArgs<real> a = make_args<real>(c);
      tfkt_status s = timed(TFKT_K_MOMENTS, [&] { return launch_moments<real, S>(a, c->stream); });
      if (s != TFKT_OK) return s;
      c->m_valid = true;
    }
    KernelArgs<real> a = make_args<real>(c);
    if (c->fused) {
      FusedArgs<real> f = make_fused<real>(c);
      if (c->lpm_pending) f.rshp = (const real*)c->lpm_rshp;
      tfkt_status s =
          timed(TFKT_K_FUSED, [&] { return launch_step_fused<real, S>(a, f, c->stream); });
      if (s != TFKT_OK) return s;
      c->lpm_pending = false;
      s = timed(TFKT_K_FIXUP, [&] { return launch_fixup<real>(a, f, c->stream); });
      if (s != TFKT_OK) return s;
      c->mcur ^= 1;
    } else {
      tfkt_status s = timed(TFKT_K_STEP, [&] { return launch_step<real, S>(a, c->stream); });
      if (s != TFKT_OK) return s;
      c->m_valid = false;
    }
    c->cur ^= 1;
    ++c->step;
  }
  tfkt_status s = drain();
  if (s != TFKT_OK) return s;
  for (int j = 0; j < TFKT_NKERNELS; ++j) {
    ms[j] += acc[j];
    if (launches) launches[j] += cnt[j];
  }
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status do_fields(Ctx* c, uint32_t mask, double* dst, int dst_is_device) {
  const Lattice& L = c->L;
  tfkt_status s = ensure_moments<real, S>(c);
  if (s != TFKT_OK) return s;
  KernelArgs<real> a = make_args<real>(c);
  TFKT_CUDA(c, launch_velocity<real>(a, c->stream));
  const size_t nf = (size_t)__builtin_popcount(mask);
  const size_t bytes = nf * (size_t)L.nx * L.ny * sizeof(double);
  // Host destination: stage in the population buffer that the next step overwrites.
  double* out = dst_is_device ? dst : (double*)a.dst;
  TFKT_CUDA(c, launch_fields<real>(a, mask, out, c->stream));
  if (!dst_is_device) {
    TFKT_CUDA(c, cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream));
    TFKT_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status do_psi(Ctx* c, double* dst, int dst_is_device) {
  const Lattice& L = c->L;
  tfkt_status s = ensure_moments<real, S>(c);
  if (s != TFKT_OK) return s;
  KernelArgs<real> a = make_args<real>(c);
  const size_t bytes = (size_t)L.nq * L.nx * L.ny * sizeof(double);
  double* out = dst_is_device ? dst : (double*)a.dst;
  TFKT_CUDA(c, launch_psi<real>(a, out, c->stream));
  if (!dst_is_device) {
    TFKT_CUDA(c, cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream));
    TFKT_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status do_populations(Ctx* c, double* host) {
  const Lattice& L = c->L;
  if (c->lpm_pending) {
    tfkt_status s = ctx_lpm_flush(c);
    if (s != TFKT_OK) return s;
  }
  KernelArgs<real> a = make_args<real>(c);
  const size_t N = (size_t)L.nx * L.ny;
  double* tmp = nullptr;
  TFKT_CUDA(c, cudaMallocAsync((void**)&tmp, (size_t)L.npl * N * sizeof(double), c->stream));
  cudaError_t e = launch_populations<real, S>(a, tmp, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, tmp, (size_t)L.npl * N * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
  cudaError_t f = cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "populations");
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status do_diag(Ctx* c, double* out) {
  tfkt_status s = ensure_moments<real, S>(c);
  if (s != TFKT_OK) return s;
  KernelArgs<real> a = make_args<real>(c);
  TFKT_CUDA(c, launch_velocity<real>(a, c->stream));
  double* part = (double*)((char*)c->ws.base + c->ws.off_part);
  double* dout = (double*)((char*)c->ws.base + c->ws.off_diag);
  TFKT_CUDA(c, launch_diag<real>(a, part, c->diag_blocks, dout, c->stream));
  TFKT_CUDA(c, cudaMemcpyAsync(out, dout, TFKT_NDIAG * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  TFKT_CUDA(c, cudaStreamSynchronize(c->stream));
  static const char* const names[TFKT_NDIAG] = {"mass_s", "mass_p", "px", "py", "ke",
                                                "enstrophy", "qrms_mean", "ey2", "umax",
                                                "qrms_max"};
  for (int j = 0; j < TFKT_NDIAG; ++j)
    if (!std::isfinite(out[j]))
      return fail(TFKT_ENAN, std::string("non-finite diagnostic ") + names[j] + " at step " +
                                 std::to_string(c->step));
  return TFKT_OK;
}

// Compute and storage types of a context: FP64 (double, double), FP32
// (float, float), FP16 storage computed in FP32 (float, __half).
#define DISPATCH(c, fn, ...)                                       \
  ((c)->L.precision == TFKT_FP64   ? fn<double, double>(__VA_ARGS__) \
   : (c)->L.precision == TFKT_FP32 ? fn<float, float>(__VA_ARGS__)   \
                                   : fn<float, __half>(__VA_ARGS__))

tfkt_status check_ctx(const Ctx* c) {
  if (!c) return fail(TFKT_EINVAL, "context is NULL");
  if (c->poisoned) return fail(TFKT_ESTATE, "context poisoned by an earlier CUDA error");
  return TFKT_OK;
}

}  // namespace
}  // namespace tfkt

using namespace tfkt;

struct tfkt_ctx : public Ctx {};

namespace tfkt {
Ctx* ctx_of(tfkt_ctx* c) { return c; }
size_t ctx_layout(const Lattice& L) {
  Workspace w;
  return layout(L, &w);
}
template <typename real>
KernelArgs<real> ctx_args(const Ctx* c) {
  return make_args<real>(c);
}
template <typename real>
FusedArgs<real> ctx_fused(const Ctx* c) {
  return make_fused<real>(c);
}
template KernelArgs<float> ctx_args<float>(const Ctx*);
template FusedArgs<float> ctx_fused<float>(const Ctx*);
tfkt_status ctx_reinit(Ctx* c, const double* perturb) {
  c->cur = 0;
  c->mcur = 0;
  c->step = 0;
  c->lpm_pending = false;
  c->lpm_step = -1;
  return DISPATCH(c, init_state, c, perturb);
}
tfkt_status ctx_ensure_moments_f32(Ctx* c) {
  if (c->L.precision != TFKT_FP32) return fail(TFKT_EINVAL, "FP32 context expected");
  return ensure_moments<float, float>(c);
}
tfkt_status ctx_ensure_moments(Ctx* c) { return DISPATCH(c, ensure_moments, c); }
}  // namespace tfkt

extern "C" {

tfkt_status tfkt_required_bytes(const tfkt_params* p, size_t* bytes) {
  if (!bytes) return fail(TFKT_EINVAL, "bytes is NULL");
  Lattice L;
  tfkt_status s = map_params(p, &L);
  if (s != TFKT_OK) return s;
  Workspace w;
  *bytes = layout(L, &w);
  return TFKT_OK;
}

tfkt_status tfkt_create(const tfkt_params* p, const double* perturb, void* dev_workspace,
                        size_t workspace_bytes, void* stream, tfkt_ctx** out) {
  NvtxRange nvtx_range("tfkt_create");
  if (!out) return fail(TFKT_EINVAL, "out is NULL");
  *out = nullptr;
  Lattice L;
  tfkt_status s = map_params(p, &L);
  if (s != TFKT_OK) return s;
  return ctx_create(L, perturb, dev_workspace, workspace_bytes, stream, out);
}

}  // extern "C"

namespace tfkt {
tfkt_status ctx_create(const Lattice& L, const double* perturb, void* dev_workspace,
                       size_t workspace_bytes, void* stream, tfkt_ctx** out) {
  tfkt_status s = TFKT_OK;
  tfkt_ctx* c = new (std::nothrow) tfkt_ctx();
  if (!c) return fail(TFKT_ENOMEM, "host allocation failed");
  c->L = L;
  c->stream = (cudaStream_t)stream;
  c->fused = fused_path(L);
  const size_t need = layout(L, &c->ws);
  c->diag_blocks = diag_blocks_for(L);
  if (dev_workspace) {
    if (workspace_bytes < need) {
      delete c;
      return fail(TFKT_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
    }
    if (((uintptr_t)dev_workspace) % 256 != 0) {
      delete c;
      return fail(TFKT_EINVAL, "workspace must be 256-byte aligned");
    }
    c->ws.base = dev_workspace;
    c->ws.owned = false;
  } else {
    cudaError_t e = cudaMalloc(&c->ws.base, need);
    if (e != cudaSuccess) {
      delete c;
      cudaGetLastError();
      return fail(TFKT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->ws.owned = true;
  }
  c->ws.bytes = need;
  HostTables t = build_tables(L);
  s = L.precision == TFKT_FP64 ? upload_tables<double>(c, t) : upload_tables<float>(c, t);
  if (s == TFKT_OK) s = DISPATCH(c, init_state, c, perturb);
  if (s != TFKT_OK) {
    if (c->ws.owned) cudaFree(c->ws.base);
    delete c;
    return s;
  }
  *out = c;
  return TFKT_OK;
}
}  // namespace tfkt

extern "C" {

tfkt_status tfkt_step(tfkt_ctx* c, int64_t n) {
  NvtxRange nvtx_range("tfkt_step");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (n < 0) return fail(TFKT_EINVAL, "n must be >= 0");
  return DISPATCH(c, do_step, c, n);
}

tfkt_status tfkt_step_profiled(tfkt_ctx* c, int64_t n, double* kernel_ms, int64_t* launches) {
  NvtxRange nvtx_range("tfkt_step_profiled");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (n < 0 || !kernel_ms) return fail(TFKT_EINVAL, "n must be >= 0 and kernel_ms non-NULL");
  return DISPATCH(c, do_step_profiled, c, n, kernel_ms, launches);
}

tfkt_status tfkt_moments(tfkt_ctx* c, uint32_t mask, double* dst, size_t bytes, int dst_is_device) {
  NvtxRange nvtx_range("tfkt_moments");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (!dst) return fail(TFKT_EINVAL, "dst is NULL");
  if (mask == 0 || (mask >> TFKT_NFIELDS) != 0) return fail(TFKT_EINVAL, "bad field mask");
  const size_t need = (size_t)__builtin_popcount(mask) * c->L.nx * c->L.ny * sizeof(double);
  if (bytes < need) return fail(TFKT_EINVAL, "dst too small");
  return DISPATCH(c, do_fields, c, mask, dst, dst_is_device);
}

tfkt_status tfkt_psi(tfkt_ctx* c, double* dst, size_t bytes, int dst_is_device) {
  NvtxRange nvtx_range("tfkt_psi");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (!dst) return fail(TFKT_EINVAL, "dst is NULL");
  if (bytes < (size_t)c->L.nq * c->L.nx * c->L.ny * sizeof(double))
    return fail(TFKT_EINVAL, "dst too small");
  return DISPATCH(c, do_psi, c, dst, dst_is_device);
}

tfkt_status tfkt_diagnostics(tfkt_ctx* c, double* out) {
  NvtxRange nvtx_range("tfkt_diagnostics");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (!out) return fail(TFKT_EINVAL, "out is NULL");
  return DISPATCH(c, do_diag, c, out);
}

tfkt_status tfkt_populations(tfkt_ctx* c, double* host_dst, size_t bytes) {
  NvtxRange nvtx_range("tfkt_populations");
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  if (!host_dst) return fail(TFKT_EINVAL, "dst is NULL");
  if (bytes < (size_t)c->L.npl * c->L.nx * c->L.ny * sizeof(double))
    return fail(TFKT_EINVAL, "dst too small");
  return DISPATCH(c, do_populations, c, host_dst);
}

tfkt_status tfkt_get_info(const tfkt_ctx* c, tfkt_info* info) {
  if (!c || !info) return fail(TFKT_EINVAL, "NULL argument");
  const Lattice& L = c->L;
  tfkt_info i{};
  i.nx = L.nx;
  i.ny = L.ny;
  i.nq = L.nq;
  i.precision = L.precision;
  i.tau1 = L.tau1;
  i.tau2 = L.tau2;
  i.H = L.H;
  i.kappa = L.kappa;
  i.ell = L.ell;
  i.psi_tot = L.psi_tot;
  i.sigma_q2 = L.sigma_q2;
  i.a0 = L.a0;
  i.kf = L.kf;
  i.nu = L.nu;
  i.nu_s = L.nu_s;
  i.eta_p = L.eta_p;
  i.lambda_h = L.lambda_h;
  i.fene_b = L.fene_b;
  i.qe_model = L.qe_model;
  i.step = c->step;
  i.workspace_bytes = c->ws.bytes;
  i.pitch = L.pitch;
  // each population read once and written once, each moment plane read and written once
  i.bytes_per_node_step = 2 * population_bytes(L) / L.plane + (size_t)L.nm * 2 * real_size(L);
  *info = i;
  return TFKT_OK;
}

tfkt_status tfkt_lattice(int32_t* c9, int32_t* c25v) {
  if (c9)
    for (int i = 0; i < 9; ++i) {
      c9[2 * i] = c9x(i);
      c9[2 * i + 1] = c9y(i);
    }
  if (c25v)
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      c25v[4 * i] = c.rx;
      c25v[4 * i + 1] = c.ry;
      c25v[4 * i + 2] = c.qx;
      c25v[4 * i + 3] = c.qy;
    }
  return TFKT_OK;
}

tfkt_status tfkt_sync(tfkt_ctx* c) {
  tfkt_status s = check_ctx(c);
  if (s != TFKT_OK) return s;
  TFKT_CUDA(c, cudaStreamSynchronize(c->stream));
  return TFKT_OK;
}

tfkt_status tfkt_destroy(tfkt_ctx* c) {
  if (!c) return TFKT_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (c->ws.owned && c->ws.base) {
    cudaError_t f = cudaFree(c->ws.base);
    if (e == cudaSuccess) e = f;
  }
  if (c->lpm) {
    cudaError_t f = cudaFree(c->lpm);
    if (e == cudaSuccess) e = f;
  }
  delete c;
  if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("destroy: ") + cudaGetErrorString(e));
  return TFKT_OK;
}

const char* tfkt_status_string(tfkt_status s) {
  switch (s) {
    case TFKT_OK: return "ok";
    case TFKT_EINVAL: return "invalid argument";
    case TFKT_ENOMEM: return "out of device memory";
    case TFKT_ECUDA: return "CUDA error";
    case TFKT_ENAN: return "non-finite value";
    case TFKT_ESTATE: return "context poisoned";
    case TFKT_EIO: return "checkpoint file error";
    case TFKT_ETIMEOUT: return "bounded wait ran out";
  }
  return "unknown status";
}

const char* tfkt_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
