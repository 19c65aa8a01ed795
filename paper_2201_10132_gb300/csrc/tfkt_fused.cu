// Fused single-pass step: pull-stream, moments, collision and write-back of
// every population of a 32 x 8 tile, plus the moment planes of the NEXT step,
// in one read and one write of the populations (Sec. VI-C update; moments of
// Sec. VI-A / VI-B; elastic stress of Sec. III).
//
// The next step's moments of node y are sums of post-collision populations
// arriving at y: g'_i(y - c_r, q) lands on (y, q + Qdot_i), or bounces back to
// (y, q) as the opposite velocity when q + Qdot_i leaves the Q-disk. A tile
// writes its post-collision values into shared memory and every thread sums,
// in a fixed order, the arrivals at its own node from sources inside the tile;
// 84 threads do the same for the ring of nodes around the tile. Arrivals from
// neighbouring tiles reach a border node through those tiles' ring exports,
// which the fix-up kernel adds in a fixed order. No atomics: results do not
// depend on scheduling.
//
// M planes written for step n+1: interior nodes get final values (delta psi,
// delta rho, J, delta Theta); border nodes get the tile's raw partial sums in
// the delta psi, delta rho and J planes, completed by the fix-up kernel.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "tfkt_fused.cuh"

namespace tfkt {
namespace {
// Exchange buffer: per velocity a plane of (H + 2) rows of HX = TX + 2 cells,
// the tile plus a one-node zero halo, and two zero rows before the first and
// after the last plane. A ring node's pull of a velocity that cannot reach it
// from the tile falls up to two nodes out; in this layout such a read wraps
// into a halo cell of the same or the neighbouring plane (or the end rows),
// which all stay zero, so the ring sums need neither masks nor a wider halo.
// Shared memory is kept small: what two blocks leave of the SM's 256 KB is the
// L1 through which the pulls' global loads return, and the loads in flight
// need it.
template <typename real>
struct Smem {
  real* hb;          // [20][H+2][HX] collided values of the r-moving velocities, zero halo
  real* A;           // [nq][NT] own-node arrival sums per Q-node
  real* Ar;          // [nq][RING] ring-node arrival sums per Q-node
  real* Ux;          // [H+2][TX+2] velocity on the tile and its ring; shares the
  real* Uy;          // space of A, which is cleared only after its last use
  long long* ptab;   // [nq][PQ] per pull: its source plane in the current source buffer, as
                     // a pointer, or (lean variant) as an element offset
  real* delta;       // [nq][DG] pull shift difference of each Q-displacement group that
                     // moves in Q (the same for the group's members; zero where the pull bounces)
  int* aoff;         // [nq][AQ] per Q-displacement group: byte offset in A of its target
                     // Q-node's row; a displacement that leaves the disk targets q itself
  uint32_t* bmask;   // [nq] bit g set when displacement group g leaves the disk
};

constexpr int PQ = 26;   // per-Q-node stride of the pull table (entry pairs 16-byte aligned)
constexpr int AQ = 12;   // per-Q-node stride of the target table (three 16-byte loads)

template <typename real, int H>
__host__ __device__ constexpr size_t smem_layout(int nq, size_t* o_A, size_t* o_Ar, size_t* o_poff,
                                                 size_t* o_delta, size_t* o_aoff, size_t* o_bm) {
  size_t o = sizeof(real) * (20 * Geo<H>::HSZ + 2 * HPAD);
  o = (o + 15) & ~(size_t)15;
  *o_A = o;
  const size_t a_elems = (size_t)nq * Geo<H>::NT, u_elems = 2 * (H + 2) * (TX + 2);
  o += sizeof(real) * (a_elems > u_elems ? a_elems : u_elems);
  *o_Ar = o;
  o += sizeof(real) * (size_t)nq * Geo<H>::RING;
  o = (o + 15) & ~(size_t)15;
  *o_poff = o;
  o += sizeof(long long) * (size_t)nq * PQ;
  *o_delta = o;
  o += sizeof(real) * (size_t)nq * DG;
  o = (o + 15) & ~(size_t)15;
  *o_aoff = o;
  o += sizeof(int) * (size_t)nq * AQ;
  *o_bm = o;
  o += sizeof(uint32_t) * (size_t)nq;
  return o;
}

template <typename real, int H>
__device__ __forceinline__ Smem<real> carve(unsigned char* base, int nq) {
  size_t oA, oAr, op, od, oa, ob;
  smem_layout<real, H>(nq, &oA, &oAr, &op, &od, &oa, &ob);
  Smem<real> s;
  s.hb = (real*)base + HPAD;
  s.A = (real*)(base + oA);
  s.Ar = (real*)(base + oAr);
  s.Ux = s.A;
  s.Uy = s.Ux + (H + 2) * (TX + 2);
  s.ptab = (long long*)(base + op);
  s.delta = (real*)(base + od);
  s.aoff = (int*)(base + oa);
  s.bmask = (uint32_t*)(base + ob);
  return s;
}

// The four Q-displacement groups of the velocities that move on one Q-axis
// (1: -Q_y, 3: -Q_x, 5: +Q_x, 7: +Q_y) and the k-th of their four members,
// all of which also move in r. The r-diagonals with Q at rest (1..4) are
// group 4 and the Q-diagonals with r at rest (21..24) the corner groups.
__host__ __device__ constexpr int axis_group(int k) { return 2 * k + 1; }
// A velocity of Q-displacement group g (g != 4).
__host__ __device__ constexpr int group_member(int g) {
  for (int i = 1; i < 25; ++i)
    if (qgroup(c25(i)) == g) return i;
  return 0;
}
__host__ __device__ constexpr int axis_vel(int g, int k) {
  int seen = 0;
  for (int i = 5; i <= 20; ++i)
    if (qgroup(c25(i)) == g) {
      if (seen == k) return i;
      ++seen;
    }
  return -1;
}

// One tile (btx, bty) of an ntx x nty tile grid; shared by the single-run and
// the batched kernels. LEAN (the batched kernel, whose arguments sit in shared
// memory and which already runs at its register limit) addresses the pulls by
// offsets and sums the moments velocity by velocity; the single-run kernel
// uses a table of source-plane pointers and pairwise moment sums, which cost
// registers but fewer instructions (measured: each is faster in one kernel and
// slower in the other). STRESS: the collision with the component stresses
// quasi-conserved (Sec. V, Eq. quasieq2; f*_S and f**_P of Sec. VI), whose
// targets carry the equilibrium momenta and the current stresses of f; it needs
// the second moments of every Q-node's populations (single-run kernel only).
template <typename real, typename S, bool RESHAPE, int H, bool LEAN, bool STRESS = false>
__device__ __forceinline__ void fused_body(const KernelArgs<real>& a, const FusedArgs<real>& fa,
                                           int btx, int bty, int ntx, int nty,
                                           unsigned char* smem_raw) {
  constexpr int NT = Geo<H>::NT, RING = Geo<H>::RING, HSZ = Geo<H>::HSZ;
  constexpr int TY = H;     // tile height within this body
  constexpr uint32_t AROW = NT * sizeof(real);   // bytes of one Q-node row of A (a power of two)
  const int nq = a.nq;
  Smem<real> sm = carve<real, H>(smem_raw, nq);
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TX + lx;
  const int x0 = btx * TX, y0 = bty * TY;
  const int x = x0 + lx, y = y0 + ly;
  const size_t P = a.plane;
  const real* __restrict__ Min = fa.Min;
  real* __restrict__ Mout = fa.Mout;
  using SS = SolventT<S>;
  const S* __restrict__ src = (const S*)a.src;
  S* __restrict__ dst = (S*)a.dst;
  const SS* __restrict__ ssrc = solvent_planes<S>(a.src, P, a.nq);
  SS* __restrict__ sdst = solvent_planes<S>(a.dst, P, a.nq);

  // pull offsets within a plane (32-bit: a plane holds < 2^31 elements)
  const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
  const int pitch = (int)a.pitch;
  uint32_t off[9];
  off[0] = ym * pitch + xm; off[1] = ym * pitch + x; off[2] = ym * pitch + xp;
  off[3] = y * pitch + xm;  off[4] = y * pitch + x;  off[5] = y * pitch + xp;
  off[6] = yp * pitch + xm; off[7] = yp * pitch + x; off[8] = yp * pitch + xp;
  const uint32_t n = off[4];

  // ---- stage: tables, zeroed accumulators and exchange halo, U on the tile and its ring
  for (int k = tid; k < nq; k += NT) {
    uint32_t m = 0;
    for (int g = 0; g < 9; ++g)
      if (fa.tgt[k * 9 + g] < 0) m |= 1u << g;
    sm.bmask[k] = m;
  }
  for (int k = tid; k < nq * AQ; k += NT) {
    const int q = k / AQ, g = k % AQ;
    const int t = g < 9 ? fa.tgt[q * 9 + g] : -1;
    sm.aoff[k] = (t >= 0 ? t : q) * (int)AROW;
  }
  for (int k = tid; k < nq * PQ; k += NT) {
    const int q = k / PQ, i = k % PQ;
    const long long e = i < 25 ? fa.poff[q * 25 + i] : 0;
    if constexpr (LEAN) sm.ptab[k] = e;
    else sm.ptab[k] = reinterpret_cast<long long>(src + e);
  }
  for (int k = tid; k < nq * DG; k += NT) {
    const int q = k / DG, s = k % DG;
    sm.delta[k] = a.tab.delta[q * 25 + group_member(s < 4 ? s : s + 1)];
  }
  for (int k = tid; k < 20 * HSZ + 2 * HPAD; k += NT) sm.hb[k - HPAD] = real(0);
  for (int k = tid; k < nq * RING; k += NT) sm.Ar[k] = real(0);
  for (int k = tid; k < (TX + 2) * (TY + 2); k += NT) {
    const int hx = k % (TX + 2), hy = k / (TX + 2);
    int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
    gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
    gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
    real ux, uy;
    velocity_at(a, Min, gx, gy, ux, uy);
    sm.Ux[k] = ux;
    sm.Uy[k] = uy;
  }
  __syncthreads();

  const int c = (ly + 1) * (TX + 2) + (lx + 1);
  const real Ux = sm.Ux[c], Uy = sm.Uy[c];
  const real G00 = real(0.5) * (sm.Ux[c + 1] - sm.Ux[c - 1]);                    // d_x U_x
  const real G01 = real(0.5) * (sm.Uy[c + 1] - sm.Uy[c - 1]);                    // d_x U_y
  const real G10 = real(0.5) * (sm.Ux[c + TX + 2] - sm.Ux[c - TX - 2]);          // d_y U_x
  const real G11 = real(0.5) * (sm.Uy[c + TX + 2] - sm.Uy[c - TX - 2]);          // d_y U_y

  // exchange-buffer cells: own node, and (threads < RING) one ring node; a
  // source outside the tile falls on the zero halo, so the sums need no masks
  const int hcell = (ly + 1) * HX + (lx + 1);
  const bool ring_thread = tid < RING;
  int rex = 0, rey = 0;
  if (ring_thread) ring_coords<H>(tid, rex, rey);
  const int rcell = (rey + 1) * HX + (rex + 1);

  const real rho = a.rho0 + Min[(size_t)(nq + M_DRHO) * P + n];
  const real force = rho * a.tab.arow[y];
  real jx_arr = 0, jy_arr = 0, ms_arr = 0;    // own-node arrivals (momentum, solvent mass)
  real jx_r = 0, jy_r = 0, ms_r = 0;          // ring-node arrivals

  // The pull table's entries of Q-node q for velocities i and i + 1 (i even).
  auto entry_pair = [&](int q, int i) {
    return *reinterpret_cast<const longlong2*>(sm.ptab + q * PQ + i);
  };
  // Source address of the pull of velocity i at a Q-node whose table entry is e
  // and whose bounce mask is bm. The pull bounces when q - Qdot_i leaves the disk
  // (the opposite group 8 - g): the entry then names the opposite velocity's
  // plane, and the source is the node itself. The r-diagonals never bounce.
  auto pull_addr = [&](auto I, long long e, uint32_t bm) -> const S* {
    constexpr int i = decltype(I)::value;
    constexpr V4 cv = c25(i);
    uint32_t o = off[shift_index(-cv.rx, -cv.ry)];
    if constexpr (moves_r(i) && qgroup(cv) != 4) {
      if ((bm >> (8 - qgroup(cv))) & 1u) o = off[4];
    }
    if constexpr (LEAN) return src + (e + o);
    else return reinterpret_cast<const S*>(e) + o;
  };
  // The populations of a Q-node are loaded one Q-node ahead: register h[i] is
  // refilled for Q-node q + 1 as soon as the collision of Q-node q has used it,
  // so the loads are in flight during the exchange and the barriers. A
  // converted storage type (FP16) is refilled into hr[i] in its stored form and
  // converted where the next Q-node starts, so that no conversion waits for a
  // load before the barriers (h[i] and hr[i] are never live at once).
  constexpr bool RAW = std::is_same<S, real>::value;
  S hr[25];
  real h[25], mn[4];
  long long e_odd = 0;   // the second entry of the last pair read from the pull table
  if (nq > 0) {
    const uint32_t bm0 = sm.bmask[0];
    static_for<0, 25>([&](auto I) {
      constexpr int i = decltype(I)::value;
      long long e;
      if constexpr (i % 2 == 0) {
        const longlong2 pr = entry_pair(0, i);
        e = pr.x;
        e_odd = pr.y;
      } else {
        e = e_odd;
      }
      if constexpr (RAW) h[i] = *pull_addr(I, e, bm0);
      else hr[i] = *pull_addr(I, e, bm0);
    });
    mn[0] = Min[off[5]];
    mn[1] = Min[off[3]];
    mn[2] = Min[off[7]];
    mn[3] = Min[off[1]];
  }

  // ---- solvent
  if constexpr (STRESS) {
    // stress quasi-equilibrium: f*_S carries rho_S U and the stress of f,
    // P(f) - rho_S c_s^2 I = [2 tau2 (P(g) - P_eq) + tau2 (F U + U F)] / (2 tau2 + 1) + rho_S U U
    real hs[9];
    real drs = 0, pxx = 0, pxy = 0, pyy = 0;
    static_for<0, 9>([&](auto I) {
      constexpr int i = I;
      hs[i] = from_store<real>(ssrc[(size_t)i * P + off[shift_index(-c9x(i), -c9y(i))]]);
      drs += hs[i];
      acc<c9x(i) * c9x(i)>(pxx, hs[i]);
      acc<c9x(i) * c9y(i)>(pxy, hs[i]);
      acc<c9y(i) * c9y(i)>(pyy, hs[i]);
    });
    const real cs2 = real(1) / real(3);
    const real rs = real(1) + drs;
    const real dxx = pxx - drs * cs2 - rs * Ux * Ux, dxy = pxy - rs * Ux * Uy;
    const real dyy = pyy - drs * cs2 - rs * Uy * Uy;
    const real fxx = (a.c2 * dxx + a.tau2 * real(2) * force * Ux) * a.inv_c2p1 + rs * Ux * Ux;
    const real fxy = (a.c2 * dxy + a.tau2 * force * Uy) * a.inv_c2p1 + rs * Ux * Uy;
    const real fyy = a.c2 * dyy * a.inv_c2p1 + rs * Uy * Uy;
    const real usq = Ux * Ux + Uy * Uy;
    static_for<0, 9>([&](auto I) {
      constexpr int i = I;
      constexpr real cx = real(c9x(i)), cy = real(c9y(i));
      const real cu = cx * Ux + cy * Uy;
      const real pneq = fxx * (cx * cx - cs2) + real(2) * fxy * cx * cy + fyy * (cy * cy - cs2);
      const real fss_dev = real(w9(i)) * (drs + real(3) * rs * cu + real(4.5) * pneq);
      const real feq_dev = real(w9(i)) * (drs + rs * (real(3) * cu + real(4.5) * cu * cu - real(1.5) * usq));
      const real srcterm = real(w9(i)) * (real(3) * (cx - Ux) + real(9) * cu * cx) * force;
      const real hp = a.om2b * hs[i] + a.tb * (a.omr * fss_dev + a.r * feq_dev) + a.omb * srcterm;
      sdst[(size_t)i * P + n] = to_store<SS>(hp);
      if constexpr (i == 0) ms_arr += hp;
      else sm.hb[(i - 1) * HSZ + hcell] = hp;
    });
  } else
  {
    real hs[9];
    real drs = 0, jsx = 0, jsy = 0;
    static_for<0, 9>([&](auto I) {
      constexpr int i = I;
      hs[i] = from_store<real>(ssrc[(size_t)i * P + off[shift_index(-c9x(i), -c9y(i))]]);
      drs += hs[i];
      acc<c9x(i)>(jsx, hs[i]);
      acc<c9y(i)>(jsy, hs[i]);
    });
    const real rs = real(1) + drs;
    const real jfx = (a.c2 * jsx + rs * Ux + a.tau2 * force) * a.inv_c2p1;
    const real jfy = (a.c2 * jsy + rs * Uy) * a.inv_c2p1;
    const real usx = jfx / rs, usy = jfy / rs;
    const real vx = a.omr * usx + a.r * Ux, vy = a.omr * usy + a.r * Uy;
    const real sq = a.omr * (usx * usx + usy * usy) + a.r * (Ux * Ux + Uy * Uy);
    static_for<0, 9>([&](auto I) {
      constexpr int i = I;
      real cus = 0, cu = 0, cv = 0;
      acc<c9x(i)>(cus, usx); acc<c9y(i)>(cus, usy);
      acc<c9x(i)>(cu, Ux);   acc<c9y(i)>(cu, Uy);
      acc<c9x(i)>(cv, vx);   acc<c9y(i)>(cv, vy);
      // Guo source (3 (c - U) + 9 (c . U) c) . (force, 0)
      real gx = -real(3) * Ux;
      acc<c9x(i)>(gx, real(3) + real(9) * cu);
      const real feq_dev = real(w9(i)) * (drs + rs * (real(3) * cv +
                                                      real(4.5) * (a.omr * cus * cus + a.r * cu * cu) -
                                                      real(1.5) * sq));
      const real hp = a.om2b * hs[i] + a.tb * feq_dev + a.omb * real(w9(i)) * gx * force;
      sdst[(size_t)i * P + n] = to_store<SS>(hp);
      if constexpr (i == 0) ms_arr += hp;
      else sm.hb[(i - 1) * HSZ + hcell] = hp;
    });
  }
  __syncthreads();
  static_for<1, 8>([&](auto I) {
    constexpr int i = I;
    const real v = sm.hb[(i - 1) * HSZ + hcell - (c9y(i) * HX + c9x(i))];
    ms_arr += v;
    acc<c9x(i)>(jx_arr, v);
    acc<c9y(i)>(jy_arr, v);
  });
  if (ring_thread) {
    static_for<1, 8>([&](auto I) {
      constexpr int i = I;
      const real v = sm.hb[(i - 1) * HSZ + rcell - (c9y(i) * HX + c9x(i))];
      ms_r += v;
      acc<c9x(i)>(jx_r, v);
      acc<c9y(i)>(jy_r, v);
    });
  }
  __syncthreads();
  // every thread has read the staged velocity (it shares A's space): clear
  // this thread's column of the arrival sums
  for (int p = 0; p < nq; ++p) sm.A[p * NT + tid] = real(0);

  // a learned block's pending increment: dpsi(q) = p0(q) (B0 Qx^2 + B1 Qx Qy + B2 Qy^2 + B3)
  real B0 = 0, B1 = 0, B2 = 0, B3 = 0, rpt0 = 0;
  if constexpr (RESHAPE) {
    B0 = fa.rshp[n];
    B1 = fa.rshp[P + n];
    B2 = fa.rshp[2 * P + n];
    B3 = fa.rshp[3 * P + n];
    rpt0 = real(1) / a.psi_tot0;
  }
  char* const Acol = reinterpret_cast<char*>(sm.A) + tid * sizeof(real);

  // ---- polymer, one Q-node at a time
  for (int q = 0; q < nq; ++q) {
    const uint32_t bm = sm.bmask[q];
    {
      real dl[DG];
      load_vec<DG>(dl, sm.delta + q * DG);
      static_for<0, 25>([&](auto I) {   // unscale (FP16 storage), shift to this Q-node
        constexpr int i = I, g = qgroup(c25(i));
        if constexpr (g == 4) {
          if constexpr (!RAW) h[i] = from_store<real>(hr[i]) * a.pinv;
        } else {
          constexpr int sl = g < 4 ? g : g - 1;
          if constexpr (RAW) h[i] += dl[sl];
          else h[i] = from_store<real>(hr[i]) * a.pinv + dl[sl];
        }
      });
    }
    if constexpr (RESHAPE) {
      // added as the linear quasi-equilibrium w_i [dpsi + 3 (v_i . dpsi U + Qdot_i . dpsi
      // (Q . grad U - kappa Q))] with this step's U and grad U (Hookean springs)
      const real Qx = a.tab.qx[q], Qy = a.tab.qy[q];
      const real dps = a.tab.psi0[q] * rpt0 * (B0 * Qx * Qx + B1 * Qx * Qy + B2 * Qy * Qy + B3);
      const real t1 = real(3) * dps * Ux, t2 = real(3) * dps * Uy;
      const real t3 = real(3) * dps * (Qx * G00 + Qy * G10 - a.kappa * Qx);
      const real t4 = real(3) * dps * (Qx * G01 + Qy * G11 - a.kappa * Qy);
      static_for<0, 25>([&](auto I) {
        constexpr int i = I;
        real v = dps;
        acc<c25(i).rx>(v, t1);
        acc<c25(i).ry>(v, t2);
        acc<c25(i).qx>(v, t3);
        acc<c25(i).qy>(v, t4);
        h[i] += real(w25(i)) * v;
      });
    }
    const real dpx = real(0.5) * (mn[0] - mn[1]);
    const real dpy = real(0.5) * (mn[2] - mn[3]);
    const bool more = q + 1 < nq;
    const uint32_t bmn = more ? sm.bmask[q + 1] : 0u;
    if (more) {
      const real* Mq = Min + (size_t)(q + 1) * P;
      mn[0] = Mq[off[5]];
      mn[1] = Mq[off[3]];
      mn[2] = Mq[off[7]];
      mn[3] = Mq[off[1]];
    }
    real dpsi = 0, rx = 0, ry = 0, qx = 0, qy = 0;
    // STRESS: second moments of the deviations on the four axes (rx, ry, qx, qy):
    // diagonal t[k] and the six off-diagonal pairs t2[pr], in the pair order below
    real t[4] = {0, 0, 0, 0}, t2[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (LEAN) {
      static_for<0, 25>([&](auto I) {
        constexpr int i = I;
        dpsi += h[i];
        acc<c25(i).rx>(rx, h[i]);
        acc<c25(i).ry>(ry, h[i]);
        acc<c25(i).qx>(qx, h[i]);
        acc<c25(i).qy>(qy, h[i]);
      });
    } else {
      // the four velocities (+-1, +-1) on a component pair (a, b) give their
      // sum and the a- and b-momenta from two differences
      dpsi = h[0];
      static_for<0, 6>([&](auto PR) {
        constexpr int pr = PR;   // pairs (rx,ry) (rx,qx) (rx,qy) (ry,qx) (ry,qy) (qx,qy)
        constexpr int ca = pr < 3 ? 0 : (pr < 5 ? 1 : 2);
        constexpr int cb = pr == 0 ? 1 : (pr == 1 ? 2 : (pr == 2 ? 3 : (pr == 3 ? 2 : 3)));
        constexpr int ipp = pair_vel(ca, cb, 1, 1), ipm = pair_vel(ca, cb, 1, -1);
        constexpr int imp = pair_vel(ca, cb, -1, 1), imm = pair_vel(ca, cb, -1, -1);
        static_assert(ipp > 0 && ipm > 0 && imp > 0 && imm > 0, "D4Q25 pair velocities");
        const real d1 = h[ipp] - h[imm], d2 = h[ipm] - h[imp];
        const real s1 = h[ipp] + h[imm], s2 = h[ipm] + h[imp];
        dpsi += s1 + s2;
        if constexpr (STRESS) {
          // the four velocities have c_a^2 = c_b^2 = 1 and c_a c_b = +1 (pp, mm) or -1 (pm, mp)
          const real sg = s1 + s2;
          t[ca] += sg;
          t[cb] += sg;
          t2[pr] += s1 - s2;
        }
        const real ma = d1 + d2, mb = d1 - d2;
        auto addc = [&](auto K, real v) {
          constexpr int k = decltype(K)::value;
          if constexpr (k == 0) rx += v;
          else if constexpr (k == 1) ry += v;
          else if constexpr (k == 2) qx += v;
          else qy += v;
        };
        addc(std::integral_constant<int, ca>(), ma);
        addc(std::integral_constant<int, cb>(), mb);
      });
    }
    const real Qx = a.tab.qx[q], Qy = a.tab.qy[q], Fx = a.tab.fx[q], Fy = a.tab.fy[q];
    const real psi = a.tab.psi0[q] + dpsi;
    const real qg = Qx * dpx + Qy * dpy;
    const real jrex = psi * Ux + a.tau_m * a.hl2h * Fx * qg;
    const real jrey = psi * Uy + a.tau_m * a.hl2h * Fy * qg;
    const real jqex = psi * (Qx * G00 + Qy * G10 - a.kappa * Fx);
    const real jqey = psi * (Qx * G01 + Qy * G11 - a.kappa * Fy);
    // 3 x the momenta of the mixed equilibrium (1 - r) f* + r f^eq, times the
    // relaxation weight 2 beta w_i of the moving velocities (w_i = 1/36): a
    // moving population then takes an add per nonzero component and one FMA
    const real tw = a.tb * real(1.0 / 36.0), tw3 = real(3) * tw;
    real mrx, mry, mqx, mqy;
    // STRESS: the second-order Hermite terms of f**, times the relaxation weight
    // and (1 - r): per axis sk[k] = 4.5 (P(f) - P_eq)_kk, s0 = -1.5 tr, and per
    // pair sp[pr] = 9 (P(f) - P_eq)_ab, with P(f) - P_eq = 2 tau2 (P(g) - P_eq) / (2 tau2 + 1)
    // and P_eq = psi c_s^2 I on the diagonal blocks; a moving velocity on the pair
    // (a, b) adds sk[a] + sk[b] + s0 + c_a c_b sp[pr], the rest velocity s0
    real sk[4], sp[6], s0 = 0;
    if constexpr (STRESS) {
      // both targets carry the equilibrium momenta
      mrx = tw3 * jrex;
      mry = tw3 * jrey;
      mqx = tw3 * jqex;
      mqy = tw3 * jqey;
      const real cs2 = real(1) / real(3);
      const real kf = tw * a.omr * a.c2 * a.inv_c2p1;
      real tr = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const real dk = t[k] - dpsi * cs2;
        tr += dk;
        sk[k] = real(4.5) * kf * dk;
      }
      s0 = real(-1.5) * kf * tr;
#pragma unroll
      for (int k = 0; k < 6; ++k) sp[k] = real(9) * kf * t2[k];
    } else {
      mrx = tw3 * (a.omr * (a.c2 * rx + jrex) * a.inv_c2p1 + a.r * jrex);
      mry = tw3 * (a.omr * (a.c2 * ry + jrey) * a.inv_c2p1 + a.r * jrey);
      mqx = tw3 * (a.omr * (a.c2 * qx + jqex) * a.inv_c2p1 + a.r * jqex);
      mqy = tw3 * (a.omr * (a.c2 * qy + jqey) * a.inv_c2p1 + a.r * jqey);
    }
    const real wdpsi = tw * dpsi;
    S* dq = dst + (size_t)(9 + 25 * q) * P + n;
    // post-collision values that stay on this r-node, per Q-displacement group
    // (rest velocity and Q-diagonals; a group that leaves the disk targets q)
    real grp[9];
#pragma unroll
    for (int g = 0; g < 9; ++g) grp[g] = real(0);
    static_for<0, 25>([&](auto I) {
      constexpr int i = I;
      static_assert(i == 0 || w25(i) == 1.0 / 36.0, "moving weights");
      real d = i == 0 ? a.tb * real(w25(0)) * dpsi : wdpsi;
      acc<c25(i).rx>(d, mrx);
      acc<c25(i).ry>(d, mry);
      acc<c25(i).qx>(d, mqx);
      acc<c25(i).qy>(d, mqy);
      if constexpr (STRESS) {
        if constexpr (i == 0) {
          d += real(12) * s0;                       // w0 / w = 12
        } else {
          constexpr V4 cv = c25(i);
          constexpr int ka = cv.rx != 0 ? 0 : (cv.ry != 0 ? 1 : 2);
          constexpr int kb = cv.qy != 0 ? 3 : (cv.qx != 0 ? 2 : 1);
          constexpr int pr = ka == 0 ? kb - 1 : (ka == 1 ? kb + 1 : 5);
          constexpr int sab = comp_of(cv, ka) * comp_of(cv, kb);
          d += sk[ka] + sk[kb] + s0;
          acc<sab>(d, sp[pr]);
        }
      }
      const real hp = a.om2b * h[i] + d;
      if constexpr (std::is_same<S, real>::value) dq[(size_t)i * P] = hp;
      else dq[(size_t)i * P] = to_store<S>(hp * a.pscale);
      // an r-moving value goes through the exchange buffer (whether it bounces is
      // settled where the arrivals are summed); the others stay on this r-node
      if constexpr (moves_r(i)) sm.hb[(i - 1) * HSZ + hcell] = hp;
      else grp[qgroup(c25(i))] += hp;
      if (more) {
        long long e;
        if constexpr (i % 2 == 0) {
          const longlong2 pr = entry_pair(q + 1, i);
          e = pr.x;
          e_odd = pr.y;
        } else {
          e = e_odd;
        }
        if constexpr (RAW) h[i] = *pull_addr(I, e, bmn);
        else hr[i] = *pull_addr(I, e, bmn);
      }
    });
    __syncthreads();
    // arrivals from the other r-nodes of the tile. A Q-axis group whose
    // displacement leaves the disk bounces back: its values stay on their own
    // r-node (and Q-node) with the r-velocity reversed, so the node takes its own
    // values of that group, with negated momentum, and no neighbour's.
    static_for<1, 4>([&](auto I) {   // r-diagonals, Q at rest (group 4): never bounce
      constexpr int i = I;
      constexpr V4 cv = c25(i);
      const real v = sm.hb[(i - 1) * HSZ + hcell - (cv.ry * HX + cv.rx)];
      grp[4] += v;
      acc<cv.rx>(jx_arr, v);
      acc<cv.ry>(jy_arr, v);
    });
    static_for<0, 4>([&](auto GI) {
      constexpr int g = axis_group(GI);
      if ((bm >> g) & 1u) {
        static_for<0, 4>([&](auto K) {
          constexpr int i = axis_vel(g, K);
          constexpr V4 cv = c25(i);
          const real v = sm.hb[(i - 1) * HSZ + hcell];
          grp[g] += v;
          acc<-cv.rx>(jx_arr, v);
          acc<-cv.ry>(jy_arr, v);
        });
      } else {
        static_for<0, 4>([&](auto K) {
          constexpr int i = axis_vel(g, K);
          constexpr V4 cv = c25(i);
          const real v = sm.hb[(i - 1) * HSZ + hcell - (cv.ry * HX + cv.rx)];
          grp[g] += v;
          acc<cv.rx>(jx_arr, v);
          acc<cv.ry>(jy_arr, v);
        });
      }
    });
    int to[AQ];
    load_vec<AQ>(to, sm.aoff + q * AQ);
#pragma unroll
    for (int g = 0; g < 9; ++g) *reinterpret_cast<real*>(Acol + to[g]) += grp[g];
    if (ring_thread) {
      // a ring node takes the tile's values of the groups that do not bounce
      real g4 = 0;
      static_for<1, 4>([&](auto I) {
        constexpr int i = I;
        constexpr V4 cv = c25(i);
        const real v = sm.hb[(i - 1) * HSZ + rcell - (cv.ry * HX + cv.rx)];
        g4 += v;
        acc<cv.rx>(jx_r, v);
        acc<cv.ry>(jy_r, v);
      });
      sm.Ar[q * RING + tid] += g4;
      static_for<0, 4>([&](auto GI) {
        constexpr int g = axis_group(GI);
        if (!((bm >> g) & 1u)) {
          real s = 0;
          static_for<0, 4>([&](auto K) {
            constexpr int i = axis_vel(g, K);
            constexpr V4 cv = c25(i);
            const real v = sm.hb[(i - 1) * HSZ + rcell - (cv.ry * HX + cv.rx)];
            s += v;
            acc<cv.rx>(jx_r, v);
            acc<cv.ry>(jy_r, v);
          });
          sm.Ar[((uint32_t)to[g] / AROW) * RING + tid] += s;
        }
      });
    }
    __syncthreads();
  }

  // ---- flush the next step's moments
  const bool border = lx == 0 || lx == TX - 1 || ly == 0 || ly == TY - 1;
  if (!border) {
    real drho = ms_arr, txx = 0, txy = 0, tyy = 0;
    for (int p = 0; p < nq; ++p) {
      const real d = sm.A[p * NT + tid] + fa.dpsi[p];
      Mout[(size_t)p * P + n] = d;
      drho += d;
      const real Qx = a.tab.qx[p], Qy = a.tab.qy[p], Fx = a.tab.fx[p], Fy = a.tab.fy[p];
      txx += d * Fx * Qx;
      txy += d * Fx * Qy;
      tyy += d * Fy * Qy;
    }
    Mout[(size_t)(nq + M_DRHO) * P + n] = drho;
    Mout[(size_t)(nq + M_JX) * P + n] = jx_arr + fa.dvx;
    Mout[(size_t)(nq + M_JY) * P + n] = jy_arr + fa.dvy;
    Mout[(size_t)(nq + M_THXX) * P + n] = a.hl2h * txx;
    Mout[(size_t)(nq + M_THXY) * P + n] = a.hl2h * txy;
    Mout[(size_t)(nq + M_THYY) * P + n] = a.hl2h * tyy;
  } else {
    for (int p = 0; p < nq; ++p) Mout[(size_t)p * P + n] = sm.A[p * NT + tid];
    Mout[(size_t)(nq + M_DRHO) * P + n] = ms_arr;
    Mout[(size_t)(nq + M_JX) * P + n] = jx_arr;
    Mout[(size_t)(nq + M_JY) * P + n] = jy_arr;
  }
  if (ring_thread) {
    const size_t ntiles = (size_t)ntx * nty;
    const size_t tile = (size_t)bty * ntx + btx;
    real* ex = fa.exports;
    for (int p = 0; p < nq; ++p) ex[((size_t)p * ntiles + tile) * RING + tid] = sm.Ar[p * RING + tid];
    ex[((size_t)(nq + 0) * ntiles + tile) * RING + tid] = ms_r;
    ex[((size_t)(nq + 1) * ntiles + tile) * RING + tid] = jx_r;
    ex[((size_t)(nq + 2) * ntiles + tile) * RING + tid] = jy_r;
  }
}

template <typename real, typename S, bool RESHAPE, bool STRESS = false>
__global__ void __launch_bounds__(Geo<TY>::NT, 2)
step_fused_kernel(KernelArgs<real> a, FusedArgs<real> fa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fused_body<real, S, RESHAPE, TY, false, STRESS>(a, fa, blockIdx.x, blockIdx.y, gridDim.x,
                                                  gridDim.y, smem_raw);
}


// Completes the border nodes of every tile: own partial sums plus the ring
// exports of the neighbouring tiles (left, right, down, up, then the four
// diagonal neighbours at corners), plus the constant shift terms; then
// delta rho and delta Theta. One block per tile. Pass A takes one (plane,
// border node) item per thread at a time, FIX_BATCH items with all their loads
// issued first, so that many loads are in flight; it writes the final delta
// psi planes and J and keeps delta psi and the raw delta rho in shared memory.
// Pass B sums delta rho and Theta over the Q-nodes of each border node in the
// same order as the tile body.
constexpr int FIX_T = 256;       // threads of a fix-up block
constexpr int FIX_BATCH = 4;     // items per thread whose loads are issued together

template <int H>
constexpr int fix_nodes() { return 2 * TX + 2 * (H - 2); }

template <typename real, int H>
size_t fix_smem_bytes(int nq) { return (size_t)(nq + 1) * fix_nodes<H>() * sizeof(real); }

template <typename real, int H>
__device__ __forceinline__ void fixup_body(const KernelArgs<real>& a, const FusedArgs<real>& fa,
                                           int tx, int ty, int ntx, int nty, real* s_d) {
  constexpr int TY = H, RING = Geo<H>::RING;
  constexpr int NB = fix_nodes<H>();
  __shared__ uint32_t s_n[NB];        // node offset within a plane
  __shared__ uint32_t s_nc[NB];       // contributing neighbour tiles (1 to 3)
  __shared__ size_t s_e[3][NB];       // their export positions (tile * RING + ring position)
  const int tid = threadIdx.x;
  const size_t ntiles = (size_t)ntx * nty;
  const int nq = a.nq;
  const size_t P = a.plane;
  if (tid < NB) {
    const int k = tid;
    int lx, ly;
    if (k < TX) { lx = k; ly = 0; }
    else if (k < 2 * TX) { lx = k - TX; ly = TY - 1; }
    else if (k < 2 * TX + TY - 2) { lx = 0; ly = 1 + (k - 2 * TX); }
    else { lx = TX - 1; ly = 1 + (k - 2 * TX - (TY - 2)); }
    s_n[k] = (uint32_t)((size_t)(ty * TY + ly) * a.pitch + (tx * TX + lx));
    int ctile[3] = {0, 0, 0}, cpos[3] = {0, 0, 0}, nc = 0;
    auto tile_of = [&](int dx, int dy) {
      const int ax = (tx + dx + ntx) % ntx, ay = (ty + dy + nty) % nty;
      return ay * ntx + ax;
    };
    if (lx == 0) { ctile[nc] = tile_of(-1, 0); cpos[nc++] = ring_pos<H>(TX, ly); }
    if (lx == TX - 1) { ctile[nc] = tile_of(1, 0); cpos[nc++] = ring_pos<H>(-1, ly); }
    if (ly == 0) { ctile[nc] = tile_of(0, -1); cpos[nc++] = ring_pos<H>(lx, TY); }
    if (ly == TY - 1) { ctile[nc] = tile_of(0, 1); cpos[nc++] = ring_pos<H>(lx, -1); }
    if (lx == 0 && ly == 0) { ctile[nc] = tile_of(-1, -1); cpos[nc++] = ring_pos<H>(TX, TY); }
    if (lx == TX - 1 && ly == 0) { ctile[nc] = tile_of(1, -1); cpos[nc++] = ring_pos<H>(-1, TY); }
    if (lx == 0 && ly == TY - 1) { ctile[nc] = tile_of(-1, 1); cpos[nc++] = ring_pos<H>(TX, -1); }
    if (lx == TX - 1 && ly == TY - 1) { ctile[nc] = tile_of(1, 1); cpos[nc++] = ring_pos<H>(-1, -1); }
    s_nc[k] = nc;
#pragma unroll
    for (int c = 0; c < 3; ++c) s_e[c][k] = (size_t)ctile[c] * RING + cpos[c];
  }
  __syncthreads();
  real* M = fa.Mout;
  const real* ex = fa.exports;
  const size_t estride = ntiles * RING;
  // planes j < nq: delta psi(q = j); j = nq, nq + 1, nq + 2: delta rho, J_x, J_y
  // (the moment planes and the export planes use the same index)
  const int nitems = (nq + 3) * NB;
  for (int b0 = 0; b0 < nitems; b0 += FIX_T * FIX_BATCH) {
    real v[FIX_BATCH];
#pragma unroll
    for (int u = 0; u < FIX_BATCH; ++u) {
      const int it = b0 + u * FIX_T + tid;
      if (it < nitems) {
        const int j = it / NB, k = it - j * NB;
        real w = M[(size_t)j * P + s_n[k]];
        const uint32_t nc = s_nc[k];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c < (int)nc) w += ex[(size_t)j * estride + s_e[c][k]];
        v[u] = w;
      }
    }
#pragma unroll
    for (int u = 0; u < FIX_BATCH; ++u) {
      const int it = b0 + u * FIX_T + tid;
      if (it < nitems) {
        const int j = it / NB, k = it - j * NB;
        if (j < nq) {
          const real d = v[u] + fa.dpsi[j];
          M[(size_t)j * P + s_n[k]] = d;
          s_d[j * NB + k] = d;
        } else if (j == nq) {
          s_d[nq * NB + k] = v[u];
        } else {
          M[(size_t)j * P + s_n[k]] = v[u] + (j == nq + 1 ? fa.dvx : fa.dvy);
        }
      }
    }
  }
  __syncthreads();
  if (tid < NB) {
    const size_t n = s_n[tid];
    real drho = s_d[nq * NB + tid], txx = 0, txy = 0, tyy = 0;
    for (int p = 0; p < nq; ++p) {
      const real d = s_d[p * NB + tid];
      drho += d;
      const real Qx = a.tab.qx[p], Qy = a.tab.qy[p], Fx = a.tab.fx[p], Fy = a.tab.fy[p];
      txx += d * Fx * Qx;
      txy += d * Fx * Qy;
      tyy += d * Fy * Qy;
    }
    M[(size_t)(nq + M_DRHO) * P + n] = drho;
    M[(size_t)(nq + M_THXX) * P + n] = a.hl2h * txx;
    M[(size_t)(nq + M_THXY) * P + n] = a.hl2h * txy;
    M[(size_t)(nq + M_THYY) * P + n] = a.hl2h * tyy;
  }
}

template <typename real>
__global__ void __launch_bounds__(FIX_T) fixup_kernel(KernelArgs<real> a, FusedArgs<real> fa) {
  extern __shared__ __align__(16) unsigned char fix_raw[];
  fixup_body<real, TY>(a, fa, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, (real*)fix_raw);
}

// ---------------------------------------------------------------- batches
// Many independent runs in one launch: block b is tile b of the concatenated
// tile lists; it finds its run, copies that run's arguments (for the current
// buffer parity) into shared memory and advances the tile like the
// single-run kernel.
__device__ __forceinline__ int find_run(const int* tile_start, int nruns, int t) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ void copy_words(T* dst, const T* src, int tid, int nthreads) {
  static_assert(sizeof(T) % 4 == 0, "");
  const int* s = (const int*)src;
  int* d = (int*)dst;
  for (int k = tid; k < (int)(sizeof(T) / 4); k += nthreads) d[k] = s[k];
}

template <typename real, typename S, int H>
__global__ void __launch_bounds__(Geo<H>::NT, Geo<H>::MINB)
step_fused_batch_kernel(const BatchRun<real>* runs, const int* tile_start, int nruns, int parity) {
  constexpr int NT = Geo<H>::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ KernelArgs<real> sa;
  __shared__ FusedArgs<real> sf;
  __shared__ int s_run;
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (tid == 0) s_run = find_run(tile_start, nruns, blockIdx.x);
  __syncthreads();
  const BatchRun<real>& br = runs[s_run];
  copy_words(&sa, &br.a[parity], tid, NT);
  copy_words(&sf, &br.f[parity], tid, NT);
  __syncthreads();
  const int local = blockIdx.x - tile_start[s_run];
  fused_body<real, S, false, H, true>(sa, sf, local % br.ntx, local / br.ntx, br.ntx, br.nty,
                                       smem_raw);
}

template <typename real, int H>
__global__ void __launch_bounds__(FIX_T) fixup_batch_kernel(const BatchRun<real>* runs,
                                                          const int* tile_start, int nruns,
                                                          int parity) {
  __shared__ KernelArgs<real> sa;
  __shared__ FusedArgs<real> sf;
  __shared__ int s_run;
  if (threadIdx.x == 0) s_run = find_run(tile_start, nruns, blockIdx.x);
  __syncthreads();
  const BatchRun<real>& br = runs[s_run];
  copy_words(&sa, &br.a[parity], threadIdx.x, blockDim.x);
  copy_words(&sf, &br.f[parity], threadIdx.x, blockDim.x);
  __syncthreads();
  const int local = blockIdx.x - tile_start[s_run];
  extern __shared__ __align__(16) unsigned char fix_raw[];
  fixup_body<real, H>(sa, sf, local % br.ntx, local / br.ntx, br.ntx, br.nty, (real*)fix_raw);
}

}  // namespace

template <int H>
size_t smem_bytes_h(int nq, size_t real_bytes) {
  size_t a, b, c, d, e, f;
  return real_bytes == 8 ? smem_layout<double, H>(nq, &a, &b, &c, &d, &e, &f)
                         : smem_layout<float, H>(nq, &a, &b, &c, &d, &e, &f);
}

size_t fused_smem_bytes(int nq, size_t real_bytes, int ty) {
  switch (ty) {
    case 4: return smem_bytes_h<4>(nq, real_bytes);
    case 8: return smem_bytes_h<8>(nq, real_bytes);
    case 16: return smem_bytes_h<16>(nq, real_bytes);
    default: return ~(size_t)0;
  }
}

size_t fused_export_elems(int nx, int ny, int nq, int ty) {
  const size_t ring = 2 * (TX + 2) + 2 * (size_t)ty;
  return (size_t)(nx / TX) * (ny / ty) * ring * (size_t)(nq + 3);
}

size_t fused_export_capacity(int nx, int ny, int nq) {
  size_t m = 0;
  for (int ty : {4, 8, 16})
    if (ny % ty == 0) m = std::max(m, fused_export_elems(nx, ny, nq, ty));
  return m;
}

bool fused_supported(int nx, int ny, int nq, size_t real_bytes, int ty) {
  return nx % TX == 0 && ny % ty == 0 &&
         fused_smem_bytes(nq, real_bytes, ty) <= 227 * 1024;
}

bool fused_path(const Lattice& L) {
  return fused_supported(L.nx, L.ny, L.nq, L.precision == TFKT_FP64 ? 8 : 4);
}

template <typename real, typename S>
cudaError_t launch_step_fused(const KernelArgs<real>& a, const FusedArgs<real>& f, cudaStream_t s) {
  const size_t smem = fused_smem_bytes(a.nq, sizeof(real), TY);
  const dim3 grid(a.nx / TX, a.ny / TY), block(TX, TY);
  if (f.rshp) {
    // a learned block's increment rides on this step's pull (FP32 storage only)
    if constexpr (std::is_same<real, float>::value && std::is_same<S, float>::value) {
      cudaError_t e = cudaFuncSetAttribute(step_fused_kernel<real, S, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      step_fused_kernel<real, S, true><<<grid, block, smem, s>>>(a, f);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (a.qe == TFKT_QE_STRESS) {
    cudaError_t e = cudaFuncSetAttribute(step_fused_kernel<real, S, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    step_fused_kernel<real, S, false, true><<<grid, block, smem, s>>>(a, f);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(step_fused_kernel<real, S, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  step_fused_kernel<real, S, false><<<grid, block, smem, s>>>(a, f);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fixup(const KernelArgs<real>& a, const FusedArgs<real>& f, cudaStream_t s) {
  const size_t smem = fix_smem_bytes<real, TY>(a.nq);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fixup_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  fixup_kernel<real><<<dim3(a.nx / TX, a.ny / TY), FIX_T, smem, s>>>(a, f);
  return cudaGetLastError();
}

// Batches that launch each run's own single-run kernels (graph branches): the
// attribute is set once here, so the launches below make no other API call.
cudaError_t prepare_single_fp32(int max_nq) {
  const size_t smem = fused_smem_bytes(max_nq, sizeof(float), TY);
  cudaError_t e = cudaFuncSetAttribute(step_fused_kernel<float, float, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const size_t fsmem = fix_smem_bytes<float, TY>(max_nq);
  if (e == cudaSuccess && fsmem > 48 * 1024)
    e = cudaFuncSetAttribute(fixup_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fsmem);
  return e;
}

cudaError_t launch_single_fp32(const KernelArgs<float>& a, const FusedArgs<float>& f,
                               cudaStream_t s) {
  const dim3 grid(a.nx / TX, a.ny / TY), block(TX, TY);
  step_fused_kernel<float, float, false><<<grid, block, fused_smem_bytes(a.nq, sizeof(float), TY), s>>>(
      a, f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  fixup_kernel<float><<<grid, FIX_T, fix_smem_bytes<float, TY>(a.nq), s>>>(a, f);
  return cudaGetLastError();
}

template <int H>
cudaError_t prepare_batch_h(int max_nq) {
  const size_t smem = fused_smem_bytes(max_nq, sizeof(float), H);
  return cudaFuncSetAttribute(step_fused_batch_kernel<float, float, H>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_batch(int max_nq, int ty) {
  switch (ty) {
    case 4: return prepare_batch_h<4>(max_nq);
    case 8: return prepare_batch_h<8>(max_nq);
    case 16: return prepare_batch_h<16>(max_nq);
    default: return cudaErrorInvalidValue;
  }
}

template <int H>
cudaError_t launch_batch_step_h(const BatchRun<float>* runs, const int* tile_start, int nruns,
                                int total_tiles, int max_nq, int parity, cudaStream_t s) {
  const size_t smem = fused_smem_bytes(max_nq, sizeof(float), H);
  step_fused_batch_kernel<float, float, H><<<total_tiles, dim3(TX, H), smem, s>>>(
      runs, tile_start, nruns, parity);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t fsmem = fix_smem_bytes<float, H>(max_nq);
  if (fsmem > 48 * 1024) {
    e = cudaFuncSetAttribute(fixup_batch_kernel<float, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fsmem);
    if (e != cudaSuccess) return e;
  }
  fixup_batch_kernel<float, H><<<total_tiles, FIX_T, fsmem, s>>>(runs, tile_start, nruns, parity);
  return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchRun<float>* runs, const int* tile_start, int nruns,
                              int total_tiles, int max_nq, int parity, cudaStream_t s, int ty) {
  switch (ty) {
    case 4: return launch_batch_step_h<4>(runs, tile_start, nruns, total_tiles, max_nq, parity, s);
    case 8: return launch_batch_step_h<8>(runs, tile_start, nruns, total_tiles, max_nq, parity, s);
    case 16:
      return launch_batch_step_h<16>(runs, tile_start, nruns, total_tiles, max_nq, parity, s);
    default: return cudaErrorInvalidValue;
  }
}

// Host-side tables of the fused kernel: target Q-node of every
// (Q-node, Q-displacement group), -1 where the displacement leaves the disk;
// the per-Q-node sum of the pull shift differences; their r-momentum sum.
void fused_tables(const Lattice& L, const HostTables& t, std::vector<int>& tgt,
                  std::vector<double>& dpsi, double& dvx, double& dvy,
                  std::vector<long long>& poff) {
  poff.resize((size_t)L.nq * 25);
  for (size_t k = 0; k < poff.size(); ++k) {
    const int e = t.pull[k];
    poff[k] = (long long)(e >= 0 ? e : ~e) * (long long)L.plane;
  }
  tgt.assign((size_t)L.nq * 9, -1);
  std::vector<int> qmap((size_t)L.S * L.S, -1);
  std::vector<int> gi(L.nq), gj(L.nq);
  for (int q = 0; q < L.nq; ++q) {
    gi[q] = (int)lround(t.qx[q] + 0.5 * (L.S - 1));
    gj[q] = (int)lround(t.qy[q] + 0.5 * (L.S - 1));
    qmap[(size_t)gj[q] * L.S + gi[q]] = q;
  }
  for (int q = 0; q < L.nq; ++q)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = gi[q] + dx, j = gj[q] + dy;
        const int tq = (i >= 0 && i < L.S && j >= 0 && j < L.S) ? qmap[(size_t)j * L.S + i] : -1;
        tgt[(size_t)q * 9 + qgroup9(dx, dy)] = tq;
      }
  dpsi.assign(L.nq, 0.0);
  dvx = dvy = 0;
  for (int q = 0; q < L.nq; ++q)
    for (int i = 0; i < 25; ++i) {
      const double d = t.delta[(size_t)q * 25 + i];
      dpsi[q] += d;
      dvx += c25(i).rx * d;
      dvy += c25(i).ry * d;
    }
}

template cudaError_t launch_step_fused<double, double>(const KernelArgs<double>&,
                                                        const FusedArgs<double>&, cudaStream_t);
template cudaError_t launch_step_fused<float, float>(const KernelArgs<float>&,
                                                      const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_step_fused<float, __half>(const KernelArgs<float>&,
                                                       const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_fixup<double>(const KernelArgs<double>&, const FusedArgs<double>&,
                                          cudaStream_t);
template cudaError_t launch_fixup<float>(const KernelArgs<float>&, const FusedArgs<float>&,
                                         cudaStream_t);

}  // namespace tfkt
