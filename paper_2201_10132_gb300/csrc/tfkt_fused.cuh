// Helpers of the fused single-pass step kernels (tfkt_fused.cu): compile-time
// loops, the tile geometry and its ring of border nodes, D4Q25 velocity
// properties, and the mixture velocity of a node from the moment planes.
#pragma once

#include <type_traits>
#include <utility>

#include "tfkt_internal.cuh"

namespace tfkt {
namespace {

// Calls f(std::integral_constant<int, B + k>) for k = 0 .. N-1: a loop whose
// index is a compile-time constant in the body.
template <int B, typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, B + Is>{}), ...);
}
template <int B, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl<B>(f, std::make_integer_sequence<int, N>{});
}

// Tile geometry for a tile height H (the width is one warp, TX): threads /
// nodes per tile, ring nodes around it, the exchange buffer's rows and plane.
// The single-run path uses H = TY; batches pick H by timing (tfkt_batch.cu).
template <int H>
struct Geo {
  static constexpr int NT = TX * H;
  static constexpr int RING = 2 * (TX + 2) + 2 * H;
  static constexpr int HY = H + 4;
  static constexpr int HSZ = (TX + 2) * (H + 2);
  static constexpr int MINB = NT >= 512 ? 1 : 512 / NT;   // blocks per SM at 128 registers
};

// Ring position of frame coordinates (ex, ey) in [-1, TX] x [-1, H] \ tile.
template <int H>
__host__ __device__ constexpr int ring_pos(int ex, int ey) {
  return ey == -1 ? ex + 1
       : ey == H ? TX + 3 + ex
       : ex == -1 ? 2 * TX + 4 + ey
                  : 2 * TX + 4 + H + ey;
}
template <int H>
__device__ __forceinline__ void ring_coords(int k, int& ex, int& ey) {
  if (k < TX + 2) { ex = k - 1; ey = -1; }
  else if (k < 2 * TX + 4) { ex = k - (TX + 3); ey = H; }
  else if (k < 2 * TX + 4 + H) { ex = -1; ey = k - (2 * TX + 4); }
  else { ex = TX; ey = k - (2 * TX + 4 + H); }
}

// Q-displacement group of a velocity: (qy + 1) * 3 + (qx + 1); 4 = no Q motion.
__host__ __device__ constexpr int qgroup(const V4 c) { return (c.qy + 1) * 3 + (c.qx + 1); }
__host__ __device__ constexpr int qgroup9(int cx, int cy) { return (cy + 1) * 3 + (cx + 1); }


template <typename T>
__device__ __forceinline__ T __int_as_T(int v) {
  if constexpr (std::is_same<T, float>::value) return __int_as_float(v);
  else return (T)v;
}

// Adds s * v for a compile-time s in {-1, 0, 1} (no multiply by a zero
// coefficient, which IEEE arithmetic would not let the compiler drop).
template <int S, typename real>
__device__ __forceinline__ void acc(real& sum, real v) {
  if constexpr (S == 1) sum += v;
  else if constexpr (S == -1) sum -= v;
}

// Component k (0..3 = rx, ry, qx, qy) of a velocity, and the index of the
// D4Q25 velocity with components ca = sa, cb = sb and zero elsewhere (every
// moving velocity is +-1 on exactly one pair of components).
__host__ __device__ constexpr int comp_of(const V4 c, int k) {
  return k == 0 ? c.rx : (k == 1 ? c.ry : (k == 2 ? c.qx : c.qy));
}
__host__ __device__ constexpr int pair_vel(int ca, int cb, int sa, int sb) {
  for (int i = 1; i < 25; ++i) {
    bool ok = true;
    for (int k = 0; k < 4; ++k) {
      const int want = k == ca ? sa : (k == cb ? sb : 0);
      ok = ok && comp_of(c25(i), k) == want;
    }
    if (ok) return i;
  }
  return -1;
}

// Velocities 1..20 move in r (they reach other r-nodes); 0 and 21..24 do not.
__host__ __device__ constexpr bool moves_r(int i) { return i >= 1 && i <= 20; }

// Loads N values (N a multiple of the vector width) from 16-byte aligned shared memory.
template <int N, typename T>
__device__ __forceinline__ void load_vec(T* out, const T* src) {
  if constexpr (sizeof(T) == 4) {
    static_assert(N % 4 == 0, "");
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const int4 v = reinterpret_cast<const int4*>(src)[k];
      out[4 * k] = __int_as_T<T>(v.x);
      out[4 * k + 1] = __int_as_T<T>(v.y);
      out[4 * k + 2] = __int_as_T<T>(v.z);
      out[4 * k + 3] = __int_as_T<T>(v.w);
    }
  } else {
    static_assert(N % 2 == 0, "");
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 v = reinterpret_cast<const double2*>(src)[k];
      out[2 * k] = v.x;
      out[2 * k + 1] = v.y;
    }
  }
}

// Exchange buffer constants of the fused kernel (its layout is described where
// the buffer is carved) and the size of the per-Q-node shift table.
constexpr int HX = TX + 2;
constexpr int HPAD = 2 * HX;     // zero cells before the first and after the last plane
constexpr int DG = 8;            // per-Q-node entries of the shift table: the groups that move in Q

template <typename real>
__device__ __forceinline__ void velocity_at(const KernelArgs<real>& a, const real* M, int x, int y,
                                            real& ux, real& uy) {
  const int nq = a.nq;
  const size_t P = a.plane;
  const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
  const size_t n = (size_t)y * a.pitch + x;
  const size_t nxm = (size_t)y * a.pitch + xm, nxp = (size_t)y * a.pitch + xp;
  const size_t nym = (size_t)ym * a.pitch + x, nyp = (size_t)yp * a.pitch + x;
  const real* Txx = M + (size_t)(nq + M_THXX) * P;
  const real* Txy = M + (size_t)(nq + M_THXY) * P;
  const real* Tyy = M + (size_t)(nq + M_THYY) * P;
  const real rho = a.rho0 + M[(size_t)(nq + M_DRHO) * P + n];
  const real jx = M[(size_t)(nq + M_JX) * P + n];
  const real jy = M[(size_t)(nq + M_JY) * P + n];
  const real ex = real(0.5) * (Txx[nxp] - Txx[nxm]) + real(0.5) * (Txy[nyp] - Txy[nym]);
  const real ey = real(0.5) * (Txy[nxp] - Txy[nxm]) + real(0.5) * (Tyy[nyp] - Tyy[nym]);
  const real f = a.tab.arow[y];
  ux = (jx + real(0.5) * (ex + rho * f)) / rho;
  uy = (jy + real(0.5) * ey) / rho;
}

}  // namespace
}  // namespace tfkt
