// Device kernels of the two-fluid kinetic step (arXiv 2201.10132, Sec. VI-VII).
//
// Storage: structure-of-arrays planes of ny rows x pitch elements, x fastest.
// Population planes 0..8 hold the solvent (D2Q9), plane 9 + 25 q + i the
// polymer velocity i at Q-node q (D4Q25). A buffer holds post-collision g'
// values that have not been streamed yet, stored as deviations from rest:
// g' - w_i (solvent, rho_0 = 1) and g' - w_i psi0(q) (polymer). The pull at
// node r reads g'_i(r - c_r, q - Qdot_i), or g'_{-i}(r, q) when q - Qdot_i
// leaves the Q-disk (bounce-back), and adds the shift difference delta(q, i).
//
// Moment planes M: delta psi(q) (q < nq), then delta rho (total), J_x, J_y
// (total momentum of g), and delta Theta_xx, xy, yy = (H ell^2 / 2) sum_q
// delta psi phi_q Q Q, all of the pulled (pre-collision) state.
#include "tfkt_internal.cuh"

namespace tfkt {

namespace {

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// The nine pull offsets of node (x, y): source displaced by (sx, sy).
struct Offsets {
  size_t o[9];
};

__device__ __forceinline__ Offsets node_offsets(int x, int y, int nx, int ny, size_t pitch) {
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t rm = (size_t)ym * pitch, r0 = (size_t)y * pitch, rp = (size_t)yp * pitch;
  Offsets f;
  f.o[0] = rm + xm; f.o[1] = rm + x; f.o[2] = rm + xp;
  f.o[3] = r0 + xm; f.o[4] = r0 + x; f.o[5] = r0 + xp;
  f.o[6] = rp + xm; f.o[7] = rp + x; f.o[8] = rp + xp;
  return f;
}

// Mixture velocity U of f at node n (Sec. VI-C, moments of f): summing the
// g -> f momentum relations over both species with the body force applied
// by the same half-step rule gives rho U = J(g) + (E + rho a) / 2, where the
// elastic force E = div Theta (Sec. III, Eq. IDef) by central differences.
template <typename real>
__device__ __forceinline__ void mixture_velocity(const KernelArgs<real>& a, int x, int y,
                                                 real& ux, real& uy, real& rho) {
  const int nq = a.nq;
  const size_t P = a.plane;
  const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
  const size_t n = (size_t)y * a.pitch + x;
  const size_t nxm = (size_t)y * a.pitch + xm, nxp = (size_t)y * a.pitch + xp;
  const size_t nym = (size_t)ym * a.pitch + x, nyp = (size_t)yp * a.pitch + x;
  const real* M = a.M;
  const real* Txx = M + (size_t)(nq + M_THXX) * P;
  const real* Txy = M + (size_t)(nq + M_THXY) * P;
  const real* Tyy = M + (size_t)(nq + M_THYY) * P;
  rho = a.rho0 + M[(size_t)(nq + M_DRHO) * P + n];
  const real jx = M[(size_t)(nq + M_JX) * P + n];
  const real jy = M[(size_t)(nq + M_JY) * P + n];
  const real ex = real(0.5) * (Txx[nxp] - Txx[nxm]) + real(0.5) * (Txy[nyp] - Txy[nym]);
  const real ey = real(0.5) * (Txy[nxp] - Txy[nxm]) + real(0.5) * (Tyy[nyp] - Tyy[nym]);
  const real f = a.tab.arow[y];
  ux = (jx + real(0.5) * (ex + rho * f)) / rho;
  uy = (jy + real(0.5) * ey) / rho;
}

// ------------------------------------------------------------------ init
// g = f^eq of the initial fields (Sec. VI-D): rho_S = 1, psi = psi0(q),
// U = base flow + perturbation, J^r_eq = psi U, J^Q_eq = psi (Q . grad U -
// kappa Q) (grad_r psi = 0). Each value is written to the slot that the
// first pull reads for it, so the first step starts from exactly this state.
// For the same reason the pulled populations of a node are its own stored
// values: the kernel also writes the state's moment planes M, rebuilding each
// value from its stored form and summing exactly as moments_kernel does, so
// the moments need no second pass over the populations.
template <typename real, typename S>
__global__ void __launch_bounds__(256) init_kernel(KernelArgs<real> a) {
  using SS = SolventT<S>;
  SS* __restrict__ sdst = solvent_planes<S>(a.dst, a.plane, a.nq);
  S* __restrict__ dst = (S*)a.dst;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const int nx = a.nx, ny = a.ny;
  auto U0 = [&](int xx, int yy, real& ux, real& uy) {
    const size_t k = (size_t)yy * nx + xx;
    ux = a.tab.urow[yy] + (a.perturb ? real(a.perturb[k]) : real(0));
    uy = a.perturb ? real(a.perturb[(size_t)nx * ny + k]) : real(0);
  };
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  real ux, uy, uxa, uya, uxb, uyb;
  U0(x, y, ux, uy);
  U0(xp, y, uxa, uya);
  U0(xm, y, uxb, uyb);
  const real G00 = real(0.5) * (uxa - uxb), G01 = real(0.5) * (uya - uyb);
  U0(x, yp, uxa, uya);
  U0(x, ym, uxb, uyb);
  const real G10 = real(0.5) * (uxa - uxb), G11 = real(0.5) * (uya - uyb);
  const Offsets off = node_offsets(x, y, nx, ny, a.pitch);
  const size_t P = a.plane;
  const real usq = ux * ux + uy * uy;
  real drho = 0, jx = 0, jy = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const real cu = real(c9x(i)) * ux + real(c9y(i)) * uy;
    const real h = real(w9(i)) * (real(3) * cu + real(4.5) * cu * cu - real(1.5) * usq);
    const SS st = to_store<SS>(h);
    sdst[(size_t)i * P + off.o[shift_index(-c9x(i), -c9y(i))]] = st;
    const real v = from_store<real>(st);
    drho += v;
    jx += real(c9x(i)) * v;
    jy += real(c9y(i)) * v;
  }
  real txx = 0, txy = 0, tyy = 0;
  for (int q = 0; q < a.nq; ++q) {
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q], psi = a.tab.psi0[q];
    const real Fx = a.tab.fx[q], Fy = a.tab.fy[q];
    const real jrx = psi * ux, jry = psi * uy;
    const real jqx = psi * (Qx * G00 + Qy * G10 - a.kappa * Fx);
    const real jqy = psi * (Qx * G01 + Qy * G11 - a.kappa * Fy);
    real dpsi = 0, rx = 0, ry = 0;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const real h = real(w25(i)) * real(3) *
                     (jrx * real(c.rx) + jry * real(c.ry) + jqx * real(c.qx) + jqy * real(c.qy));
      const int e = a.tab.pull[q * 25 + i];
      const size_t o = e >= 0 ? off.o[shift_index(-c.rx, -c.ry)] : off.o[4];
      const int p = e >= 0 ? e : ~e;
      const S st = to_store<S>((h - a.tab.delta[q * 25 + i]) * a.pscale);
      dst[(size_t)p * P + o] = st;
      const real v = from_store<real>(st) * a.pinv + a.tab.delta[q * 25 + i];
      dpsi += v;
      rx += real(c.rx) * v;
      ry += real(c.ry) * v;
    }
    a.M[(size_t)q * P + off.o[4]] = dpsi;
    drho += dpsi;
    jx += rx;
    jy += ry;
    txx += dpsi * Fx * Qx;
    txy += dpsi * Fx * Qy;
    tyy += dpsi * Fy * Qy;
  }
  const size_t n = off.o[4];
  const int nq = a.nq;
  a.M[(size_t)(nq + M_DRHO) * P + n] = drho;
  a.M[(size_t)(nq + M_JX) * P + n] = jx;
  a.M[(size_t)(nq + M_JY) * P + n] = jy;
  a.M[(size_t)(nq + M_THXX) * P + n] = a.hl2h * txx;
  a.M[(size_t)(nq + M_THXY) * P + n] = a.hl2h * txy;
  a.M[(size_t)(nq + M_THYY) * P + n] = a.hl2h * tyy;
}

// --------------------------------------------------------------- moments
// Pull-read every population of node (x, y) and write its moments to M
// (Sec. VI-A / VI-B moment definitions; Theta of Sec. III, Eq. IDef, with the
// spring force H phi_q Q).
template <typename real, typename S>
__global__ void __launch_bounds__(256) moments_kernel(KernelArgs<real> a) {
  // The pull tables go to shared memory, and the populations of Q-node q + 1
  // are loaded into each register as soon as Q-node q has used it, so the
  // loads of one Q-node are in flight while the previous one is summed.
  extern __shared__ __align__(16) unsigned char mom_smem[];
  const int nq = a.nq;
  real* s_delta = reinterpret_cast<real*>(mom_smem);
  int* s_pull = reinterpret_cast<int*>(mom_smem + sizeof(real) * (size_t)nq * 25);
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int k = tid; k < nq * 25; k += TX * TY) {
    s_delta[k] = a.tab.delta[k];
    s_pull[k] = a.tab.pull[k];
  }
  __syncthreads();
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const Offsets off = node_offsets(x, y, a.nx, a.ny, a.pitch);
  const size_t P = a.plane;
  const size_t n = off.o[4];
  const S* __restrict__ src = (const S*)a.src;
  const SolventT<S>* __restrict__ ssrc = solvent_planes<S>(a.src, P, a.nq);
  auto pull = [&](int q, int i) {
    const V4 c = c25(i);
    const int e = s_pull[q * 25 + i];
    const size_t o = e >= 0 ? off.o[shift_index(-c.rx, -c.ry)] : off.o[4];
    return src[(size_t)(e >= 0 ? e : ~e) * P + o];
  };
  S h[25];
  if (nq > 0) {
#pragma unroll
    for (int i = 0; i < 25; ++i) h[i] = pull(0, i);
  }
  real drho = 0, jx = 0, jy = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const real v = from_store<real>(ssrc[(size_t)i * P + off.o[shift_index(-c9x(i), -c9y(i))]]);
    drho += v;
    jx += real(c9x(i)) * v;
    jy += real(c9y(i)) * v;
  }
  real txx = 0, txy = 0, tyy = 0;
  for (int q = 0; q < nq; ++q) {
    const bool more = q + 1 < nq;
    real dpsi = 0, rx = 0, ry = 0;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const real v = from_store<real>(h[i]) * a.pinv + s_delta[q * 25 + i];
      if (more) h[i] = pull(q + 1, i);
      dpsi += v;
      rx += real(c.rx) * v;
      ry += real(c.ry) * v;
    }
    a.M[(size_t)q * P + n] = dpsi;
    drho += dpsi;
    jx += rx;
    jy += ry;
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q], Fx = a.tab.fx[q], Fy = a.tab.fy[q];
    txx += dpsi * Fx * Qx;
    txy += dpsi * Fx * Qy;
    tyy += dpsi * Fy * Qy;
  }
  a.M[(size_t)(nq + M_DRHO) * P + n] = drho;
  a.M[(size_t)(nq + M_JX) * P + n] = jx;
  a.M[(size_t)(nq + M_JY) * P + n] = jy;
  a.M[(size_t)(nq + M_THXX) * P + n] = a.hl2h * txx;
  a.M[(size_t)(nq + M_THXY) * P + n] = a.hl2h * txy;
  a.M[(size_t)(nq + M_THYY) * P + n] = a.hl2h * tyy;
}

// ------------------------------------------------------------------ step
// One collision of the pulled state, written unstreamed to dst:
//   U from M (tile + 1-node halo in shared memory), grad U by central
//   differences; solvent J_S(f) = (2 tau2 J_S(g) + rho_S U + tau2 rho a) /
//   (2 tau2 + 1), u_S = J_S(f) / rho_S; polymer J^r_eq = psi U + tau2 D,
//   D = (H ell^2 / 2) phi_q Q (Q . grad_r psi), J^Q_eq = psi (Q . grad U - kappa phi_q Q)
//   (phi_q Q = spring force / H: phi_q = 1 Hookean, 1 / (1 - Q^2/Q0^2) FENE),
//   J(f) = (2 tau2 J(g) + J_eq) / (2 tau2 + 1);
//   g' = (1 - 2 beta) g + 2 beta [(1 - tau1/tau2) f* + (tau1/tau2) f^eq]
//        + (1 - beta) S_i,   beta = 1 / (2 tau1 + 1)
// with the quadratic solvent equilibria (Eq. dis_eq), the linear polymer
// equilibria (Eqs. feq_rq_space, fstar_rq_space) and the Guo source S_i of the
// force density rho a (solvent only).
template <typename real, typename S>
__global__ void __launch_bounds__(256) step_kernel(KernelArgs<real> a) {
  __shared__ real sUx[TY + 2][TX + 2];
  __shared__ real sUy[TY + 2][TX + 2];
  // pull tables in shared memory (dynamic: nq * 25 shift differences, then plane entries)
  extern __shared__ __align__(16) unsigned char step_smem[];
  real* s_delta = reinterpret_cast<real*>(step_smem);
  int* s_pull = reinterpret_cast<int*>(step_smem + sizeof(real) * (size_t)a.nq * 25);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int k = tid; k < a.nq * 25; k += TX * TY) {
    s_delta[k] = a.tab.delta[k];
    s_pull[k] = a.tab.pull[k];
  }
  for (int k = tid; k < (TX + 2) * (TY + 2); k += TX * TY) {
    const int hx = k % (TX + 2), hy = k / (TX + 2);
    const int gx = wrapi(x0 - 1 + hx, a.nx), gy = wrapi(y0 - 1 + hy, a.ny);
    real ux, uy, rho;
    mixture_velocity(a, gx, gy, ux, uy, rho);
    sUx[hy][hx] = ux;
    sUy[hy][hx] = uy;
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  if (x >= a.nx || y >= a.ny) return;
  const real Ux = sUx[ty + 1][tx + 1], Uy = sUy[ty + 1][tx + 1];
  const real G00 = real(0.5) * (sUx[ty + 1][tx + 2] - sUx[ty + 1][tx]);  // d_x U_x
  const real G01 = real(0.5) * (sUy[ty + 1][tx + 2] - sUy[ty + 1][tx]);  // d_x U_y
  const real G10 = real(0.5) * (sUx[ty + 2][tx + 1] - sUx[ty][tx + 1]);  // d_y U_x
  const real G11 = real(0.5) * (sUy[ty + 2][tx + 1] - sUy[ty][tx + 1]);  // d_y U_y

  const Offsets off = node_offsets(x, y, a.nx, a.ny, a.pitch);
  const size_t P = a.plane;
  const size_t n = off.o[4];
  const int nq = a.nq;
  const real rho = a.rho0 + a.M[(size_t)(nq + M_DRHO) * P + n];
  const real force = rho * a.tab.arow[y];
  using SS = SolventT<S>;
  const S* __restrict__ src = (const S*)a.src;
  S* __restrict__ dst = (S*)a.dst;
  const SS* __restrict__ ssrc = solvent_planes<S>(a.src, P, a.nq);
  SS* __restrict__ sdst = solvent_planes<S>(a.dst, P, a.nq);

  // ---- solvent
  {
    real h[9];
    real drs = 0, jsx = 0, jsy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      h[i] = from_store<real>(ssrc[(size_t)i * P + off.o[shift_index(-c9x(i), -c9y(i))]]);
      drs += h[i];
      jsx += real(c9x(i)) * h[i];
      jsy += real(c9y(i)) * h[i];
    }
    const real rs = real(1) + drs;
    const real jfx = (a.c2 * jsx + rs * Ux + a.tau2 * force) * a.inv_c2p1;
    const real jfy = (a.c2 * jsy + rs * Uy) * a.inv_c2p1;
    const real usx = jfx / rs, usy = jfy / rs;
    const real vx = a.omr * usx + a.r * Ux, vy = a.omr * usy + a.r * Uy;
    const real sq = a.omr * (usx * usx + usy * usy) + a.r * (Ux * Ux + Uy * Uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const real cx = real(c9x(i)), cy = real(c9y(i));
      const real cus = cx * usx + cy * usy, cu = cx * Ux + cy * Uy;
      const real feq_dev =
          real(w9(i)) * (drs + rs * (real(3) * (cx * vx + cy * vy) +
                                     real(4.5) * (a.omr * cus * cus + a.r * cu * cu) -
                                     real(1.5) * sq));
      const real srcterm = real(w9(i)) * (real(3) * (cx - Ux) + real(9) * cu * cx) * force;
      sdst[(size_t)i * P + n] = to_store<SS>(a.om2b * h[i] + a.tb * feq_dev + a.omb * srcterm);
    }
  }

  // ---- polymer, one Q-node at a time; the populations (and psi neighbours) of
  // Q-node q + 1 are loaded while Q-node q is collided
  const size_t nxm = off.o[3], nxp = off.o[5], nym = off.o[1], nyp = off.o[7];
  auto pull = [&](int q, int i) {
    const V4 c = c25(i);
    const int e = s_pull[q * 25 + i];
    const size_t o = e >= 0 ? off.o[shift_index(-c.rx, -c.ry)] : off.o[4];
    return from_store<real>(src[(size_t)(e >= 0 ? e : ~e) * P + o]);
  };
  real h[25], mn[4];
  if (nq > 0) {
#pragma unroll
    for (int i = 0; i < 25; ++i) h[i] = pull(0, i);
    mn[0] = a.M[nxp];
    mn[1] = a.M[nxm];
    mn[2] = a.M[nyp];
    mn[3] = a.M[nym];
  }
  for (int q = 0; q < nq; ++q) {
    const bool more = q + 1 < nq;
    const real dpx = real(0.5) * (mn[0] - mn[1]);
    const real dpy = real(0.5) * (mn[2] - mn[3]);
    if (more) {
      const real* Mq = a.M + (size_t)(q + 1) * P;
      mn[0] = Mq[nxp];
      mn[1] = Mq[nxm];
      mn[2] = Mq[nyp];
      mn[3] = Mq[nym];
    }
    real dpsi = 0, rx = 0, ry = 0, qx = 0, qy = 0;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      h[i] = h[i] * a.pinv + s_delta[q * 25 + i];
      dpsi += h[i];
      rx += real(c.rx) * h[i];
      ry += real(c.ry) * h[i];
      qx += real(c.qx) * h[i];
      qy += real(c.qy) * h[i];
    }
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q], Fx = a.tab.fx[q], Fy = a.tab.fy[q];
    const real psi = a.tab.psi0[q] + dpsi;
    const real qg = Qx * dpx + Qy * dpy;
    const real jrex = psi * Ux + a.tau2 * a.hl2h * Fx * qg;
    const real jrey = psi * Uy + a.tau2 * a.hl2h * Fy * qg;
    const real jqex = psi * (Qx * G00 + Qy * G10 - a.kappa * Fx);
    const real jqey = psi * (Qx * G01 + Qy * G11 - a.kappa * Fy);
    // mixture (1 - r) J(f) + r J_eq of the two equilibria's momenta
    const real mrx = a.omr * (a.c2 * rx + jrex) * a.inv_c2p1 + a.r * jrex;
    const real mry = a.omr * (a.c2 * ry + jrey) * a.inv_c2p1 + a.r * jrey;
    const real mqx = a.omr * (a.c2 * qx + jqex) * a.inv_c2p1 + a.r * jqex;
    const real mqy = a.omr * (a.c2 * qy + jqey) * a.inv_c2p1 + a.r * jqey;
    S* dq = dst + (size_t)(9 + 25 * q) * P + n;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const real fdev = real(w25(i)) * (dpsi + real(3) * (mrx * real(c.rx) + mry * real(c.ry) +
                                                           mqx * real(c.qx) + mqy * real(c.qy)));
      dq[(size_t)i * P] = to_store<S>((a.om2b * h[i] + a.tb * fdev) * a.pscale);
      if (more) h[i] = pull(q + 1, i);
    }
  }
}

// The same step with the component stresses quasi-conserved (Sec. V, Eq.
// quasieq2; f*_S and f**_P of Sec. VI): the targets carry the equilibrium
// momenta (rho_S U; J^r_eq = psi U + tau1 D, J^Q_eq) and the current stresses
// of f, P(f) = (2 tau2 P(g) + P_eq [+ tau2 (F U + U F) for the solvent]) /
// (2 tau2 + 1), entered through the second-order Hermite terms normalised so
// that <f**, vv> = P; momenta relax at tau1, stresses at tau2.
template <typename real, typename S>
__global__ void __launch_bounds__(256) step_stress_kernel(KernelArgs<real> a) {
  __shared__ real sUx[TY + 2][TX + 2];
  __shared__ real sUy[TY + 2][TX + 2];
  // pull tables in shared memory (dynamic: nq * 25 shift differences, then plane entries)
  extern __shared__ __align__(16) unsigned char stress_smem[];
  real* s_delta = reinterpret_cast<real*>(stress_smem);
  int* s_pull = reinterpret_cast<int*>(stress_smem + sizeof(real) * (size_t)a.nq * 25);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int k = tid; k < a.nq * 25; k += TX * TY) {
    s_delta[k] = a.tab.delta[k];
    s_pull[k] = a.tab.pull[k];
  }
  for (int k = tid; k < (TX + 2) * (TY + 2); k += TX * TY) {
    const int hx = k % (TX + 2), hy = k / (TX + 2);
    const int gx = wrapi(x0 - 1 + hx, a.nx), gy = wrapi(y0 - 1 + hy, a.ny);
    real ux, uy, rho;
    mixture_velocity(a, gx, gy, ux, uy, rho);
    sUx[hy][hx] = ux;
    sUy[hy][hx] = uy;
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  if (x >= a.nx || y >= a.ny) return;
  const real Ux = sUx[ty + 1][tx + 1], Uy = sUy[ty + 1][tx + 1];
  const real G00 = real(0.5) * (sUx[ty + 1][tx + 2] - sUx[ty + 1][tx]);
  const real G01 = real(0.5) * (sUy[ty + 1][tx + 2] - sUy[ty + 1][tx]);
  const real G10 = real(0.5) * (sUx[ty + 2][tx + 1] - sUx[ty][tx + 1]);
  const real G11 = real(0.5) * (sUy[ty + 2][tx + 1] - sUy[ty][tx + 1]);
  const Offsets off = node_offsets(x, y, a.nx, a.ny, a.pitch);
  const size_t P = a.plane;
  const size_t n = off.o[4];
  const int nq = a.nq;
  const real rho = a.rho0 + a.M[(size_t)(nq + M_DRHO) * P + n];
  const real force = rho * a.tab.arow[y];
  using SS = SolventT<S>;
  const S* __restrict__ src = (const S*)a.src;
  S* __restrict__ dst = (S*)a.dst;
  const SS* __restrict__ ssrc = solvent_planes<S>(a.src, P, a.nq);
  SS* __restrict__ sdst = solvent_planes<S>(a.dst, P, a.nq);
  const real cs2 = real(1) / real(3);
  const real rmix = a.r, omr = a.omr;

  // ---- solvent
  {
    real h[9];
    real drs = 0, pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      h[i] = from_store<real>(ssrc[(size_t)i * P + off.o[shift_index(-c9x(i), -c9y(i))]]);
      drs += h[i];
      pxx += real(c9x(i) * c9x(i)) * h[i];
      pxy += real(c9x(i) * c9y(i)) * h[i];
      pyy += real(c9y(i) * c9y(i)) * h[i];
    }
    const real rs = real(1) + drs;
    // P(g) - P_eq from the deviations (P(g) = c_s^2 I + sum h c c, P_eq = rho_S (c_s^2 I + U U)),
    // then P(f) - rho_S c_s^2 I = [2 tau2 (P(g) - P_eq) + tau2 (F U + U F)] / (2 tau2 + 1) + rho_S U U
    const real dxx = pxx - drs * cs2 - rs * Ux * Ux, dxy = pxy - rs * Ux * Uy;
    const real dyy = pyy - drs * cs2 - rs * Uy * Uy;
    const real fxx = (a.c2 * dxx + a.tau2 * real(2) * force * Ux) * a.inv_c2p1 + rs * Ux * Ux;
    const real fxy = (a.c2 * dxy + a.tau2 * force * Uy) * a.inv_c2p1 + rs * Ux * Uy;
    const real fyy = a.c2 * dyy * a.inv_c2p1 + rs * Uy * Uy;
    const real usq = Ux * Ux + Uy * Uy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const real cx = real(c9x(i)), cy = real(c9y(i));
      const real cu = cx * Ux + cy * Uy;
      const real pneq = fxx * (cx * cx - cs2) + real(2) * fxy * cx * cy + fyy * (cy * cy - cs2);
      const real fss_dev = real(w9(i)) * (drs + real(3) * rs * cu + real(4.5) * pneq);
      const real feq_dev = real(w9(i)) * (drs + rs * (real(3) * cu + real(4.5) * cu * cu - real(1.5) * usq));
      const real srcterm = real(w9(i)) * (real(3) * (cx - Ux) + real(9) * cu * cx) * force;
      sdst[(size_t)i * P + n] =
          to_store<SS>(a.om2b * h[i] + a.tb * (omr * fss_dev + rmix * feq_dev) + a.omb * srcterm);
    }
  }

  // ---- polymer, one Q-node at a time; the populations (and psi neighbours) of
  // Q-node q + 1 are loaded while Q-node q is collided
  const size_t nxm = off.o[3], nxp = off.o[5], nym = off.o[1], nyp = off.o[7];
  auto pull = [&](int q, int i) {
    const V4 c = c25(i);
    const int e = s_pull[q * 25 + i];
    const size_t o = e >= 0 ? off.o[shift_index(-c.rx, -c.ry)] : off.o[4];
    return from_store<real>(src[(size_t)(e >= 0 ? e : ~e) * P + o]);
  };
  real h[25], mn[4];
  if (nq > 0) {
#pragma unroll
    for (int i = 0; i < 25; ++i) h[i] = pull(0, i);
    mn[0] = a.M[nxp];
    mn[1] = a.M[nxm];
    mn[2] = a.M[nyp];
    mn[3] = a.M[nym];
  }
  for (int q = 0; q < nq; ++q) {
    const bool more = q + 1 < nq;
    const real dpx = real(0.5) * (mn[0] - mn[1]);
    const real dpy = real(0.5) * (mn[2] - mn[3]);
    if (more) {
      const real* Mq = a.M + (size_t)(q + 1) * P;
      mn[0] = Mq[nxp];
      mn[1] = Mq[nxm];
      mn[2] = Mq[nyp];
      mn[3] = Mq[nym];
    }
    real dpsi = 0;
    // second moments of the deviations: vv (3), v Qdot (4), Qdot Qdot (3)
    real rxx = 0, rxy = 0, ryy = 0, cxx = 0, cxy = 0, cyx = 0, cyy = 0, qxx = 0, qxy = 0, qyy = 0;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      h[i] = h[i] * a.pinv + s_delta[q * 25 + i];
      dpsi += h[i];
      rxx += real(c.rx * c.rx) * h[i];
      rxy += real(c.rx * c.ry) * h[i];
      ryy += real(c.ry * c.ry) * h[i];
      cxx += real(c.rx * c.qx) * h[i];
      cxy += real(c.rx * c.qy) * h[i];
      cyx += real(c.ry * c.qx) * h[i];
      cyy += real(c.ry * c.qy) * h[i];
      qxx += real(c.qx * c.qx) * h[i];
      qxy += real(c.qx * c.qy) * h[i];
      qyy += real(c.qy * c.qy) * h[i];
    }
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q], Fx = a.tab.fx[q], Fy = a.tab.fy[q];
    const real psi = a.tab.psi0[q] + dpsi;
    const real qg = Qx * dpx + Qy * dpy;
    const real jrex = psi * Ux + a.tau_m * a.hl2h * Fx * qg;
    const real jrey = psi * Uy + a.tau_m * a.hl2h * Fy * qg;
    const real jqex = psi * (Qx * G00 + Qy * G10 - a.kappa * Fx);
    const real jqey = psi * (Qx * G01 + Qy * G11 - a.kappa * Fy);
    // P(g) - P_eq = (the deviations' moments) - dpsi c_s^2 I on the diagonal blocks (P_eq =
    // psi c_s^2 I), so P(f) - P_eq = 2 tau2 (P(g) - P_eq) / (2 tau2 + 1)
    auto dg = [&](real m) { return a.c2 * (m - dpsi * cs2) * a.inv_c2p1; };
    auto od = [&](real m) { return a.c2 * m * a.inv_c2p1; };
    const real Rxx = dg(rxx), Rxy = od(rxy), Ryy = dg(ryy);
    const real Qxx = dg(qxx), Qxy = od(qxy), Qyy = dg(qyy);
    const real Cxx = od(cxx), Cxy = od(cxy), Cyx = od(cyx), Cyy = od(cyy);
    S* dq = dst + (size_t)(9 + 25 * q) * P + n;
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const real vx = real(c.rx), vy = real(c.ry), wx = real(c.qx), wy = real(c.qy);
      const real lin = dpsi + real(3) * (jrex * vx + jrey * vy + jqex * wx + jqey * wy);
      const real sdiag = Rxx * (vx * vx - cs2) + real(2) * Rxy * vx * vy + Ryy * (vy * vy - cs2) +
                         Qxx * (wx * wx - cs2) + real(2) * Qxy * wx * wy + Qyy * (wy * wy - cs2);
      const real scross = Cxx * vx * wx + Cxy * vx * wy + Cyx * vy * wx + Cyy * vy * wy;
      const real fss_dev = real(w25(i)) * (lin + real(4.5) * sdiag + real(9) * scross);
      const real feq_dev = real(w25(i)) * lin;
      dq[(size_t)i * P] = to_store<S>((a.om2b * h[i] + a.tb * (omr * fss_dev + rmix * feq_dev)) * a.pscale);
      if (more) h[i] = pull(q + 1, i);
    }
  }
}

// ------------------------------------------------------------- observers
template <typename real>
__global__ void __launch_bounds__(256) velocity_kernel(KernelArgs<real> a) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  real ux, uy, rho;
  mixture_velocity(a, x, y, ux, uy, rho);
  const size_t n = (size_t)y * a.pitch + x;
  a.U[n] = ux;
  a.U[a.plane + n] = uy;
}

// Per-node observables (Sec. VII): rho_S, psi_tot, U, C, Theta, Q_rms, vorticity,
// the ones in `mask` (others are left unset). The sums over the Q-nodes run in
// FP64 (the second moments behind C_xy and Theta_xy cancel between Q-nodes of
// opposite sign, which FP32 sums would resolve only to ~1e-7 of the diagonal
// ones) and only as far as the requested fields need them.
constexpr uint32_t FIELDS_PSUM = (1u << TFKT_F_RHO_S) | (1u << TFKT_F_PSI_TOT) | (1u << TFKT_F_CXX) |
                                 (1u << TFKT_F_CXY) | (1u << TFKT_F_CYY) | (1u << TFKT_F_QRMS);
constexpr uint32_t FIELDS_CONF = (1u << TFKT_F_CXX) | (1u << TFKT_F_CXY) | (1u << TFKT_F_CYY) |
                                 (1u << TFKT_F_QRMS);
constexpr uint32_t FIELDS_STRESS = (1u << TFKT_F_THXX) | (1u << TFKT_F_THXY) | (1u << TFKT_F_THYY);

template <typename real>
__device__ void node_fields(const KernelArgs<real>& a, int x, int y, uint32_t mask,
                            double f[TFKT_NFIELDS]) {
  const size_t P = a.plane;
  const size_t n = (size_t)y * a.pitch + x;
  const int nq = a.nq;
  double pt = 0, sxx = 0, sxy = 0, syy = 0, fxx = 0, fxy = 0, fyy = 0;
  if (mask & (FIELDS_PSUM | FIELDS_STRESS)) {
    const bool conf = mask & FIELDS_CONF, stress = mask & FIELDS_STRESS;
    for (int q = 0; q < nq; ++q) {
      const double p = double(a.tab.psi0[q]) + double(a.M[(size_t)q * P + n]);
      const double Qx = a.tab.qx[q], Qy = a.tab.qy[q];
      pt += p;
      if (conf) {
        sxx += p * Qx * Qx;
        sxy += p * Qx * Qy;
        syy += p * Qy * Qy;
      }
      if (stress) {
        const double Fx = a.tab.fx[q], Fy = a.tab.fy[q];
        fxx += p * Fx * Qx;
        fxy += p * Fx * Qy;
        fyy += p * Fy * Qy;
      }
    }
  }
  const double ptd = pt;
  const double rho = double(a.rho0) + double(a.M[(size_t)(nq + M_DRHO) * P + n]);
  const double l2 = a.l2, hh = 0.5 * double(a.H) * l2;
  f[TFKT_F_RHO_S] = rho - ptd;
  f[TFKT_F_PSI_TOT] = ptd;
  f[TFKT_F_UX] = a.U[n];
  f[TFKT_F_UY] = a.U[P + n];
  const double cxx = ptd != 0 ? l2 * double(sxx) / ptd : 0, cxy = ptd != 0 ? l2 * double(sxy) / ptd : 0,
               cyy = ptd != 0 ? l2 * double(syy) / ptd : 0;
  f[TFKT_F_CXX] = cxx;
  f[TFKT_F_CXY] = cxy;
  f[TFKT_F_CYY] = cyy;
  f[TFKT_F_THXX] = hh * double(fxx);
  f[TFKT_F_THXY] = hh * double(fxy);
  f[TFKT_F_THYY] = hh * double(fyy);
  f[TFKT_F_QRMS] = sqrt(cxx + cyy);
  if (mask & (1u << TFKT_F_VORT)) {
    const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
    const double duy_dx = 0.5 * (double(a.U[P + (size_t)y * a.pitch + xp]) -
                                 double(a.U[P + (size_t)y * a.pitch + xm]));
    const double dux_dy =
        0.5 * (double(a.U[(size_t)yp * a.pitch + x]) - double(a.U[(size_t)ym * a.pitch + x]));
    f[TFKT_F_VORT] = duy_dx - dux_dy;
  }
}

template <typename real>
__global__ void __launch_bounds__(256) fields_kernel(KernelArgs<real> a, uint32_t mask,
                                                     double* out) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  double f[TFKT_NFIELDS];
  node_fields(a, x, y, mask, f);
  const size_t N = (size_t)a.nx * a.ny, k = (size_t)y * a.nx + x;
  int slot = 0;
  for (int j = 0; j < TFKT_NFIELDS; ++j)
    if (mask & (1u << j)) out[(size_t)(slot++) * N + k] = f[j];
}

template <typename real>
__global__ void __launch_bounds__(256) psi_kernel(KernelArgs<real> a, double* out) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t n = (size_t)y * a.pitch + x, k = (size_t)y * a.nx + x;
  for (int q = 0; q < a.nq; ++q)
    out[k * a.nq + q] = double(a.tab.psi0[q]) + double(a.M[(size_t)q * a.plane + n]);
}

// Stored populations with the storage shift added back, as doubles.
template <typename real, typename S>
__global__ void __launch_bounds__(256) populations_kernel(KernelArgs<real> a, double* out) {
  const S* src = (const S*)a.src;
  const SolventT<S>* ssrc = solvent_planes<S>(a.src, a.plane, a.nq);
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t n = (size_t)y * a.pitch + x, k = (size_t)y * a.nx + x,
               N = (size_t)a.nx * a.ny;
  for (int i = 0; i < 9; ++i)
    out[(size_t)i * N + k] = w9(i) + from_store<double>(ssrc[(size_t)i * a.plane + n]);
  for (int q = 0; q < a.nq; ++q)
    for (int i = 0; i < 25; ++i) {
      const int p = 9 + 25 * q + i;
      out[(size_t)p * N + k] = w25(i) * double(a.tab.psi0[q]) +
                               from_store<double>(src[(size_t)p * a.plane + n]) * double(a.pinv);
    }
}

// Global diagnostics: per-block FP64 partial sums over a fixed node
// partition (grid-stride, fixed order), then one block sums the partials in
// block order: the result does not depend on scheduling.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
  return v;
}

// Maximum of non-negative values (|u|^2, Q_rms) that keeps a NaN once it has
// met one (fmax would drop it), so that a non-finite node shows in the maximum
// diagnostics too. For IEEE values with the sign bit clear the order of the
// bit patterns read as unsigned integers is the numeric order, and every NaN
// (of either sign) lies above +inf: one integer maximum.
__device__ __forceinline__ float nan_max(float m, float v) {
  return __uint_as_float(max(__float_as_uint(m), __float_as_uint(v)));
}
__device__ __forceinline__ double nan_max(double m, double v) {
  return __longlong_as_double((long long)max((unsigned long long)__double_as_longlong(m),
                                             (unsigned long long)__double_as_longlong(v)));
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v = nan_max(v, __shfl_down_sync(0xffffffffu, v, s));
  return v;
}
// Diagnostics reduced by maximum rather than by sum.
__host__ __device__ constexpr bool diag_is_max(int j) {
  return j == TFKT_D_U2_MAX || j == TFKT_D_QRMS_MAX;
}

// Block partials of the global diagnostics (Sec. VII follows the enstrophy
// and Q_rms): sums, and the maxima of |u|^2 (a Mach-number guard, since the
// lattice scheme holds only for |u| well below c_s) and of Q_rms. A block takes whole rows, a thread every DIAG_THREADS-th
// node of a row. Per node only what the sums need is formed, in the context's
// precision and as deviations from the rest state (sum_q delta psi, and
// sum_q delta psi Q^2 for Q_rms); the rest-state constants are added once.
// Values are summed in that precision along a row segment of one thread and
// in FP64 across segments, blocks and the final reduction: FP64 arithmetic,
// slow on this GPU, stays out of the per-node work of FP32 contexts, while
// FP64 contexts keep FP64 throughout.
// |Q|^2 of every Q-node is staged in shared memory; a node's moment planes
// are loaded eight at a time so that several loads are in flight per thread
// (the sums still run in Q-node order).
template <typename real>
__global__ void __launch_bounds__(DIAG_THREADS) diag_partial_kernel(KernelArgs<real> a,
                                                                    double* partials) {
  extern __shared__ unsigned char diag_smem[];
  real* q2 = reinterpret_cast<real*>(diag_smem);
  const int nq = a.nq;
  const size_t P = a.plane;
  for (int q = threadIdx.x; q < nq; q += DIAG_THREADS) {
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q];
    q2[q] = Qx * Qx + Qy * Qy;
  }
  __syncthreads();
  real s0 = 0;   // sum_q psi0(q) |Q|^2 of the rest state
  for (int q = 0; q < nq; ++q) s0 += a.tab.psi0[q] * q2[q];
  double acc[TFKT_NDIAG] = {};
  for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
    const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
    real r[TFKT_NDIAG] = {};
    for (int x = threadIdx.x; x < a.nx; x += DIAG_THREADS) {
      const size_t n = (size_t)y * a.pitch + x;
      real dpt = 0, sq = 0;
      const real* mp = a.M + n;
      int q = 0;
      for (; q + 8 <= nq; q += 8) {
        real m[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) m[k] = mp[(size_t)(q + k) * P];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          dpt += m[k];
          sq += m[k] * q2[q + k];
        }
      }
      for (; q < nq; ++q) {
        const real m = mp[(size_t)q * P];
        dpt += m;
        sq += m * q2[q];
      }
      const real drho = a.M[(size_t)(nq + M_DRHO) * P + n];
      const real pt = a.psi_tot0 + dpt, rho = a.rho0 + drho;
      const real ux = a.U[n], uy = a.U[P + n];
      const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
      const real w = real(0.5) * (a.U[P + (size_t)y * a.pitch + xp] - a.U[P + (size_t)y * a.pitch + xm]) -
                     real(0.5) * (a.U[(size_t)yp * a.pitch + x] - a.U[(size_t)ym * a.pitch + x]);
      r[TFKT_D_MASS_S] += drho - dpt;   // rho_s minus its rest value rho0 - psi_tot0
      r[TFKT_D_MASS_P] += dpt;          // psi_tot minus psi_tot0
      r[TFKT_D_PX] += rho * ux;
      r[TFKT_D_PY] += rho * uy;
      r[TFKT_D_KE] += real(0.5) * rho * (ux * ux + uy * uy);
      r[TFKT_D_ENSTROPHY] += real(0.5) * w * w;
      const real qrms = pt != real(0) ? sqrt(a.l2 * (s0 + sq) / pt) : real(0);
      r[TFKT_D_QRMS_MEAN] += qrms;
      r[TFKT_D_EY2] += uy * uy;
      r[TFKT_D_U2_MAX] = nan_max(r[TFKT_D_U2_MAX], ux * ux + uy * uy);
      r[TFKT_D_QRMS_MAX] = nan_max(r[TFKT_D_QRMS_MAX], qrms);
    }
#pragma unroll
    for (int j = 0; j < TFKT_NDIAG; ++j)
      acc[j] = diag_is_max(j) ? nan_max(acc[j], double(r[j])) : acc[j] + double(r[j]);
  }
  __shared__ double red[DIAG_THREADS / 32][TFKT_NDIAG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < TFKT_NDIAG; ++j) {
    const double v = diag_is_max(j) ? warp_max(acc[j]) : warp_sum(acc[j]);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < TFKT_NDIAG) {
    const int j = threadIdx.x;
    double s = 0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w)
      s = diag_is_max(j) ? nan_max(s, red[w][j]) : s + red[w][j];
    partials[(size_t)blockIdx.x * TFKT_NDIAG + j] = s;
  }
}

// base_s, base_p: the masses of the rest state, N (rho0 - psi_tot0) and N psi_tot0.
// One warp per diagnostic: lanes stride over the block partials, then a fixed
// shuffle tree (the order does not depend on scheduling).
__global__ void diag_final_kernel(const double* partials, int nblocks, double inv_n, double base_s,
                                  double base_p, double* out) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j >= TFKT_NDIAG) return;
  const bool mx = diag_is_max(j);
  double s = 0;
  for (int b = lane; b < nblocks; b += 32) {
    const double v = partials[(size_t)b * TFKT_NDIAG + j];
    s = mx ? nan_max(s, v) : s + v;
  }
  s = mx ? warp_max(s) : warp_sum(s);
  if (lane == 0) {
    if (j == TFKT_D_MASS_S) s += base_s;
    if (j == TFKT_D_MASS_P) s += base_p;
    if (j == TFKT_D_QRMS_MEAN) s *= inv_n;
    if (j == TFKT_D_U2_MAX) s = sqrt(s);   // reported as max |u|
    out[j] = s;
  }
}

inline dim3 node_grid(int nx, int ny) { return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY); }

}  // namespace

template <typename real, typename S>
cudaError_t launch_init(const KernelArgs<real>& a, cudaStream_t s) {
  init_kernel<real, S><<<node_grid(a.nx, a.ny), dim3(TX, TY), 0, s>>>(a);
  return cudaGetLastError();
}
template <typename real, typename S>
cudaError_t launch_moments(const KernelArgs<real>& a, cudaStream_t s) {
  const size_t smem = (sizeof(real) + sizeof(int)) * (size_t)a.nq * 25;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(moments_kernel<real, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  moments_kernel<real, S><<<node_grid(a.nx, a.ny), dim3(TX, TY), smem, s>>>(a);
  return cudaGetLastError();
}
template <typename real, typename S>
cudaError_t launch_step(const KernelArgs<real>& a, cudaStream_t s) {
  const size_t smem = (sizeof(real) + sizeof(int)) * (size_t)a.nq * 25;   // pull tables
  if (a.qe == TFKT_QE_STRESS) {
    if (smem > 40 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(step_stress_kernel<real, S>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    step_stress_kernel<real, S><<<node_grid(a.nx, a.ny), dim3(TX, TY), smem, s>>>(a);
  } else {
    if (smem > 40 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(step_kernel<real, S>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    step_kernel<real, S><<<node_grid(a.nx, a.ny), dim3(TX, TY), smem, s>>>(a);
  }
  return cudaGetLastError();
}
template <typename real>
cudaError_t launch_velocity(const KernelArgs<real>& a, cudaStream_t s) {
  velocity_kernel<real><<<node_grid(a.nx, a.ny), dim3(TX, TY), 0, s>>>(a);
  return cudaGetLastError();
}
template <typename real>
cudaError_t launch_fields(const KernelArgs<real>& a, uint32_t mask, double* out, cudaStream_t s) {
  fields_kernel<real><<<node_grid(a.nx, a.ny), dim3(TX, TY), 0, s>>>(a, mask, out);
  return cudaGetLastError();
}
template <typename real>
cudaError_t launch_psi(const KernelArgs<real>& a, double* out, cudaStream_t s) {
  psi_kernel<real><<<node_grid(a.nx, a.ny), dim3(TX, TY), 0, s>>>(a, out);
  return cudaGetLastError();
}
template <typename real, typename S>
cudaError_t launch_populations(const KernelArgs<real>& a, double* out, cudaStream_t s) {
  populations_kernel<real, S><<<node_grid(a.nx, a.ny), dim3(TX, TY), 0, s>>>(a, out);
  return cudaGetLastError();
}
template <typename real>
cudaError_t launch_diag(const KernelArgs<real>& a, double* partials, int nblocks, double* out,
                        cudaStream_t s) {
  diag_partial_kernel<real><<<nblocks, DIAG_THREADS, (size_t)a.nq * sizeof(real), s>>>(a, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double N = (double)a.nx * a.ny;
  diag_final_kernel<<<1, 32 * TFKT_NDIAG, 0, s>>>(partials, nblocks, 1.0 / N,
                                     N * ((double)a.rho0 - (double)a.psi_tot0), N * (double)a.psi_tot0,
                                     out);
  return cudaGetLastError();
}

#define TFKT_INSTANTIATE_POP(real, S)                                                          \
  template cudaError_t launch_init<real, S>(const KernelArgs<real>&, cudaStream_t);           \
  template cudaError_t launch_moments<real, S>(const KernelArgs<real>&, cudaStream_t);        \
  template cudaError_t launch_step<real, S>(const KernelArgs<real>&, cudaStream_t);           \
  template cudaError_t launch_populations<real, S>(const KernelArgs<real>&, double*,          \
                                                   cudaStream_t);
#define TFKT_INSTANTIATE(real)                                                                 \
  template cudaError_t launch_velocity<real>(const KernelArgs<real>&, cudaStream_t);          \
  template cudaError_t launch_fields<real>(const KernelArgs<real>&, uint32_t, double*,        \
                                           cudaStream_t);                                     \
  template cudaError_t launch_psi<real>(const KernelArgs<real>&, double*, cudaStream_t);      \
  template cudaError_t launch_diag<real>(const KernelArgs<real>&, double*, int, double*,      \
                                         cudaStream_t);
TFKT_INSTANTIATE(float)
TFKT_INSTANTIATE(double)
TFKT_INSTANTIATE_POP(double, double)
TFKT_INSTANTIATE_POP(float, float)
TFKT_INSTANTIATE_POP(float, __half)

}  // namespace tfkt
