// Learned polymer macro-step (the paper has no learned component; the block
// is built on the scheme of Sec. VI): one plain step, the network's
// conformation K steps ahead checked tile by tile against the plain step's
// rate, K solvent-only sub-steps under the interpolated polymer stress, and
// an equilibrium-shaped increment that moves the polymer populations to the
// predicted conformation. FP32, Hookean springs, fused-path contexts.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"
#include "tfkt_mlp.cuh"
#include "tfkt_umma.cuh"

namespace tfkt {

const MlpDev& mlp_dev(const tfkt_mlp* net);

namespace {

// Scratch planes of the learned block (ny * pitch floats each).
enum { L_PSI = 0, L_C1 = 1, L_DP = 4, L_JP = 6, L_CNEW = 8, L_CPREV = 11, L_B = 14, L_NPLANES = 18 };

struct LpmArgs {
  float* p;                 // scratch planes, plane k at p + k * plane
  int* counter;             // tiles that fell back; counter[1]: a tensor-core wait timed out
  float S0[3];              // sum_q psi0 Q_a Q_b (xx, xy, yy), Q lattice units
  float m0[3];              // second moments of the normalised equilibrium p0 = psi0 / psi_tot0
  float M0inv[9];           // inverse of M0[a][b] = sum_q p0 qq_a w_b (qq_b - m0_b), w = 1, 2, 1
  float rpt0;               // 1 / psi_tot0
  float ce;                 // lattice equilibrium C_xx (r-lengths^2)
  float l2, hl2h, H, tau2, kappa, inv_lambda;
  int K, tile, mode;
  float threshold;
  int inject_wait_timeout;  // fault injection: no tensor-core work, waits bounded to a few polls
};

__device__ __forceinline__ int wrap_i(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

struct Nbr {
  size_t o[9];              // node offsets of the 3 x 3 neighbourhood (dy major)
};
__device__ __forceinline__ Nbr nbr(int x, int y, int nx, int ny, size_t pitch) {
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const size_t rm = (size_t)ym * pitch, r0 = (size_t)y * pitch, rp = (size_t)yp * pitch;
  Nbr f;
  f.o[0] = rm + xm; f.o[1] = rm + x; f.o[2] = rm + xp;
  f.o[3] = r0 + xm; f.o[4] = r0 + x; f.o[5] = r0 + xp;
  f.o[6] = rp + xm; f.o[7] = rp + x; f.o[8] = rp + xp;
  return f;
}

// psi_tot and C = ell^2 sum_q psi Q Q / psi_tot of node n from the moment planes.
__device__ __forceinline__ void node_conformation(const KernelArgs<float>& a, const LpmArgs& l,
                                                  size_t n, float& pt, float C[3]) {
  const size_t P = a.plane;
  float s = 0.f;
  for (int q = 0; q < a.nq; ++q) s += a.M[(size_t)q * P + n];
  pt = a.psi_tot0 + s;
  const float r = l.l2 / pt;
  C[0] = r * (l.S0[0] + a.M[(size_t)(a.nq + M_THXX) * P + n] / l.hl2h);
  C[1] = r * (l.S0[1] + a.M[(size_t)(a.nq + M_THXY) * P + n] / l.hl2h);
  C[2] = r * (l.S0[2] + a.M[(size_t)(a.nq + M_THYY) * P + n] / l.hl2h);
}

// Pulled solvent moments (deviation of rho_S from 1, J_S) of node (x, y).
__device__ __forceinline__ void solvent_pull_moments(const float* src, size_t P, const Nbr& nb,
                                                     float& drs, float& jx, float& jy) {
  drs = jx = jy = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float h = src[(size_t)i * P + nb.o[shift_index(-c9x(i), -c9y(i))]];
    drs += h;
    jx += float(c9x(i)) * h;
    jy += float(c9y(i)) * h;
  }
}

__global__ void __launch_bounds__(256) conf_kernel(KernelArgs<float> a, LpmArgs l, int out_plane) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t n = (size_t)y * a.pitch + x, P = a.plane;
  float pt, C[3];
  node_conformation(a, l, n, pt, C);
  for (int c = 0; c < 3; ++c) l.p[(size_t)(out_plane + c) * P + n] = C[c];
}

// After the plain step: psi_tot, C(t + 1), the polymer momentum J_P = J - J_S and
// its offset dP = J_P - psi_tot U - tau2 E from the slaved value.
__global__ void __launch_bounds__(256) prepare_kernel(KernelArgs<float> a, LpmArgs l) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t P = a.plane;
  const Nbr nb = nbr(x, y, a.nx, a.ny, a.pitch);
  const size_t n = nb.o[4];
  float pt, C[3];
  node_conformation(a, l, n, pt, C);
  float drs, jsx, jsy;
  solvent_pull_moments((const float*)a.src, P, nb, drs, jsx, jsy);
  const float* Txx = a.M + (size_t)(a.nq + M_THXX) * P;
  const float* Txy = a.M + (size_t)(a.nq + M_THXY) * P;
  const float* Tyy = a.M + (size_t)(a.nq + M_THYY) * P;
  const float ex = 0.5f * (Txx[nb.o[5]] - Txx[nb.o[3]]) + 0.5f * (Txy[nb.o[7]] - Txy[nb.o[1]]);
  const float ey = 0.5f * (Txy[nb.o[5]] - Txy[nb.o[3]]) + 0.5f * (Tyy[nb.o[7]] - Tyy[nb.o[1]]);
  const float jpx = a.M[(size_t)(a.nq + M_JX) * P + n] - jsx;
  const float jpy = a.M[(size_t)(a.nq + M_JY) * P + n] - jsy;
  const float ux = a.U[n], uy = a.U[P + n];
  float* p = l.p;
  p[(size_t)L_PSI * P + n] = pt;
  for (int c = 0; c < 3; ++c) p[(size_t)(L_C1 + c) * P + n] = C[c];
  p[(size_t)L_JP * P + n] = jpx;
  p[(size_t)(L_JP + 1) * P + n] = jpy;
  p[(size_t)L_DP * P + n] = jpx - pt * ux - l.tau2 * ex;
  p[(size_t)(L_DP + 1) * P + n] = jpy - pt * uy - l.tau2 * ey;
}

// Features of node (x, y) from U (a.U) and C(t + 1) (plane L_C1); C_dep returned too.
__device__ __forceinline__ void node_features(const KernelArgs<float>& a, const LpmArgs& l, int x,
                                              int y, float f[NIN], float cdep[3]) {
  const size_t P = a.plane;
  const float* Ux = a.U;
  const float* Uy = a.U + P;
  auto at = [&](int xx, int yy) { return (size_t)wrap_i(yy, a.ny) * a.pitch + wrap_i(xx, a.nx); };
  const float K = (float)l.K;
  // departure point of the parcel arriving at (x, y): bilinear interpolation of C
  const size_t n = (size_t)y * a.pitch + x;
  const float px = (float)x - K * Ux[n], py = (float)y - K * Uy[n];
  const float fx0 = floorf(px), fy0 = floorf(py);
  const float fx = px - fx0, fy = py - fy0;
  int x0 = (int)fx0 % a.nx, y0 = (int)fy0 % a.ny;
  if (x0 < 0) x0 += a.nx;
  if (y0 < 0) y0 += a.ny;
  const int x1 = x0 + 1 == a.nx ? 0 : x0 + 1, y1 = y0 + 1 == a.ny ? 0 : y0 + 1;
  const size_t n00 = (size_t)y0 * a.pitch + x0, n01 = (size_t)y0 * a.pitch + x1;
  const size_t n10 = (size_t)y1 * a.pitch + x0, n11 = (size_t)y1 * a.pitch + x1;
  for (int c = 0; c < 3; ++c) {
    const float* C = l.p + (size_t)(L_C1 + c) * P;
    cdep[c] = (1.f - fy) * ((1.f - fx) * C[n00] + fx * C[n01]) + fy * ((1.f - fx) * C[n10] + fx * C[n11]);
  }
  const float rce = 1.f / l.ce;
  f[0] = (cdep[0] - l.ce) * rce;
  f[1] = cdep[1] * rce;
  f[2] = (cdep[2] - l.ce) * rce;
  int k = 3;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int xx = x + dx, yy = y + dy;
      const float g00 = 0.5f * (Ux[at(xx + 1, yy)] - Ux[at(xx - 1, yy)]);   // dU_x/dx
      const float g01 = 0.5f * (Uy[at(xx + 1, yy)] - Uy[at(xx - 1, yy)]);   // dU_y/dx
      const float g10 = 0.5f * (Ux[at(xx, yy + 1)] - Ux[at(xx, yy - 1)]);   // dU_x/dy
      const float g11 = 0.5f * (Uy[at(xx, yy + 1)] - Uy[at(xx, yy - 1)]);   // dU_y/dy
      f[k++] = K * g00;
      f[k++] = K * g01;
      f[k++] = K * g10;
      f[k++] = K * g11;
    }
  f[39] = K * l.inv_lambda;
}

// One block per check tile: the network's C_new for every node, the tile's
// largest disagreement with the plain rate, and the fallback.
//
// The network runs on the fifth-generation tensor cores (tcgen05): the block is
// two groups of 128 threads, and each group takes 128 nodes at a time, one node
// per thread and per TMEM lane. Every thread forms its node's 40 standardised
// features, splits them into a bfloat16 high part and remainder, and writes them
// as its row of the K-major operands in shared memory; one thread issues the
// layer's MMAs (bf16 operands, FP32 accumulators in 64 TMEM columns) for the
// high part and the remainder against the bfloat16 weights, and commits them to
// the group's mbarrier. Each thread then loads its row of accumulators from TMEM,
// adds the bias, applies GELU and writes the next layer's operand row. The
// 64 -> 3 output layer (too narrow for the tensor cores) runs on the CUDA cores
// in FP32. A wait that does not complete within its bound sets counter[1],
// skips the TMEM reads (the tile falls back) and still frees the TMEM.
constexpr int NET_GROUPS = 2;
constexpr int NET_THREADS = 128 * NET_GROUPS;
constexpr int NET_K1 = 48;                       // layer-1 inner size: NIN padded to 3 steps of 16
constexpr uint32_t NET_SBO1 = NET_K1 / 8 * 128;  // operand bytes per 8 rows, K = 48
constexpr uint32_t NET_SBO2 = NH / 8 * 128;      // K = 64
constexpr uint32_t NET_IDESC = umma::idesc_bf16_f32(128, NH);
constexpr uint32_t NET_MAX_POLLS = 1u << 22;
static_assert(NIN <= NET_K1 && NH == 64 && NOUT == 3, "tensor-core tiling of the network");

struct NetSmem {
  __nv_bfloat16 w1[NH * NET_K1];                 // K-major operand layout, in >= NIN zero
  __nv_bfloat16 w2[NH * NH];
  __nv_bfloat16 act[NET_GROUPS][2][128 * NH];    // per group: high part and remainder rows
  float w3[NOUT][NH];
  float b1[NH], b2[NH], b3[NOUT];
  float mx[NIN], rsx[NIN], mt[NOUT], st[NOUT];
  uint64_t mbar[NET_GROUPS];
  uint32_t tmem;
};
constexpr size_t net_smem_bytes() { return sizeof(NetSmem) + 128; }

// Byte offset of element (r, k) in a K-major operand with sbo bytes per 8 rows.
__host__ __device__ constexpr uint32_t op_offset(int r, int k, uint32_t sbo) {
  return (uint32_t)(r / 8) * sbo + (uint32_t)(k / 8) * 128u + (uint32_t)(r % 8) * 16u +
         (uint32_t)(k % 8) * 2u;
}

// Writes 8 values v[8 c .. 8 c + 7] of row r, split into high part and remainder,
// as one 16-byte chunk of each operand.
__device__ __forceinline__ void write_row(__nv_bfloat16* hi, __nv_bfloat16* lo, int r, const float* v,
                                          int nchunks, uint32_t sbo) {
  for (int c = 0; c < nchunks; ++c) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tc_split(v[8 * c + 2 * j], v[8 * c + 2 * j + 1], h[j], l[j]);
    const uint32_t off = op_offset(r, 8 * c, sbo);
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(hi) + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(lo) + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(NET_THREADS) net_kernel(KernelArgs<float> a, LpmArgs l, MlpDev net) {
  extern __shared__ __align__(16) unsigned char net_smem[];
  __shared__ float red[NET_THREADS];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid >> 7, r = tid & 127;         // group, row (node) within the group
  const size_t P = a.plane;
  const int T = l.tile;
  const int tx0 = blockIdx.x * T, ty0 = blockIdx.y * T;
  const float* C1 = l.p + (size_t)L_C1 * P;
  const float* Cp = l.p + (size_t)L_CPREV * P;
  float* Cn = l.p + (size_t)L_CNEW * P;
  const float Kf = (float)l.K;
  if (l.mode == TFKT_LPM_FROZEN) {
    for (int k = tid; k < T * T; k += blockDim.x) {
      const int x = tx0 + k % T, y = ty0 + k / T;
      if (x >= a.nx || y >= a.ny) continue;
      const size_t n = (size_t)y * a.pitch + x;
      for (int c = 0; c < 3; ++c) Cn[(size_t)c * P + n] = C1[(size_t)c * P + n];
    }
    return;
  }
  // 128-byte aligned view of the dynamic shared memory
  NetSmem& s = *reinterpret_cast<NetSmem*>(
      (unsigned char*)(((uintptr_t)net_smem + 127) & ~(uintptr_t)127));
  // weights into the operand layout, the rest as FP32
  for (int e = tid; e < NH * NET_K1; e += blockDim.x) {
    const int o = e / NET_K1, i = e % NET_K1;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(s.w1) + op_offset(o, i, NET_SBO1)) =
        i < NIN ? net.wmat[o * NIN + i] : __float2bfloat16(0.0f);
  }
  for (int e = tid; e < NH * NH; e += blockDim.x) {
    const int o = e / NH, i = e % NH;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(s.w2) + op_offset(o, i, NET_SBO2)) =
        net.wmat[NH * NIN + o * NH + i];
  }
  for (int e = tid; e < NOUT * NH; e += blockDim.x)
    s.w3[e / NH][e % NH] = __bfloat162float(net.wmat[NH * NIN + NH * NH + e]);
  for (int k = tid; k < NH; k += blockDim.x) {
    s.b1[k] = net.master[OB1 + k];
    s.b2[k] = net.master[OB2 + k];
  }
  for (int k = tid; k < NIN; k += blockDim.x) {
    s.mx[k] = net.master[OMX + k];
    s.rsx[k] = 1.0f / net.master[OSX + k];
  }
  for (int k = tid; k < NOUT; k += blockDim.x) {
    s.b3[k] = net.master[OB3 + k];
    s.mt[k] = net.master[OMT + k];
    s.st[k] = net.master[OST + k];
  }
  if (tid == 0)
    for (int q = 0; q < NET_GROUPS; ++q) umma::mbar_init(&s.mbar[q], 1);
  if (warp == 0) umma::tmem_alloc(&s.tmem, 64 * NET_GROUPS);
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = s.tmem + 64u * g;                          // the group's 64 columns
  const uint32_t tmem_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's lanes
  __nv_bfloat16* ahi = s.act[g][0];
  __nv_bfloat16* alo = s.act[g][1];
  const uint32_t ahi_a = umma::smem_addr(ahi), alo_a = umma::smem_addr(alo);
  const uint32_t w1_a = umma::smem_addr(s.w1), w2_a = umma::smem_addr(s.w2);
  // fault injection (tests): no MMA is issued, so no wait can complete
  const bool issue = !l.inject_wait_timeout;
  const uint32_t polls = issue ? NET_MAX_POLLS : 64u;
  uint32_t phase = 0;
  bool failed = false;
  float worst = 0.f;
  const int npass = (T * T + NET_THREADS - 1) / NET_THREADS;      // same count in both groups
  for (int pass = 0; pass < npass; ++pass) {
    const int k = pass * NET_THREADS + g * 128 + r;
    const int x = tx0 + k % T, y = ty0 + k / T;
    const bool ok = k < T * T && x < a.nx && y < a.ny;
    float f[NET_K1], cdep[3] = {0.f, 0.f, 0.f};
    if (ok) {
      node_features(a, l, x, y, f, cdep);
#pragma unroll
      for (int i = 0; i < NIN; ++i) f[i] = (f[i] - s.mx[i]) * s.rsx[i];
    } else {
#pragma unroll
      for (int i = 0; i < NIN; ++i) f[i] = 0.f;
    }
#pragma unroll
    for (int i = NIN; i < NET_K1; ++i) f[i] = 0.f;
    // layer 1: [128 x 48] x [48 x 64]
    write_row(ahi, alo, r, f, NET_K1 / 8, NET_SBO1);
    umma::fence_proxy_async();
    umma::fence_before_sync();
    umma::bar_sync(1 + g, 128);
    if (r == 0 && issue) {
      umma::fence_after_sync();
      for (int ks = 0; ks < NET_K1 / 16; ++ks) {
        const uint64_t bd = umma::desc_kmajor(w1_a + 256u * ks, 128u, NET_SBO1);
        umma::mma_bf16(tmem, umma::desc_kmajor(ahi_a + 256u * ks, 128u, NET_SBO1), bd, NET_IDESC,
                       ks > 0);
        umma::mma_bf16(tmem, umma::desc_kmajor(alo_a + 256u * ks, 128u, NET_SBO1), bd, NET_IDESC,
                       true);
      }
      umma::commit(&s.mbar[g]);
    }
    const bool done1 = umma::mbar_wait(&s.mbar[g], phase, polls);
    phase ^= 1u;
    umma::fence_after_sync();
    float h[NH];
    if (done1) {
      float v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        umma::ld_x32(tmem_row + 32u * half, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) h[32 * half + j] = gelu(v[j] + s.b1[32 * half + j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NH; ++j) h[j] = 0.f;
    }
    // layer 2: [128 x 64] x [64 x 64] (the layer-1 operands are consumed: reuse them)
    write_row(ahi, alo, r, h, NH / 8, NET_SBO2);
    umma::fence_proxy_async();
    umma::fence_before_sync();
    umma::bar_sync(1 + g, 128);
    if (r == 0 && issue) {
      umma::fence_after_sync();
      for (int ks = 0; ks < NH / 16; ++ks) {
        const uint64_t bd = umma::desc_kmajor(w2_a + 256u * ks, 128u, NET_SBO2);
        umma::mma_bf16(tmem, umma::desc_kmajor(ahi_a + 256u * ks, 128u, NET_SBO2), bd, NET_IDESC,
                       ks > 0);
        umma::mma_bf16(tmem, umma::desc_kmajor(alo_a + 256u * ks, 128u, NET_SBO2), bd, NET_IDESC,
                       true);
      }
      umma::commit(&s.mbar[g]);
    }
    const bool done2 = umma::mbar_wait(&s.mbar[g], phase, polls);
    phase ^= 1u;
    umma::fence_after_sync();
    float o[NOUT] = {s.b3[0], s.b3[1], s.b3[2]};
    if (done2) {
      float v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        umma::ld_x32(tmem_row + 32u * half, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float hj = gelu(v[j] + s.b2[32 * half + j]);
#pragma unroll
          for (int c = 0; c < NOUT; ++c) o[c] = fmaf(s.w3[c][32 * half + j], hj, o[c]);
        }
      }
    }
    // the next pass's layer-1 MMAs overwrite these TMEM columns and operands only
    // after every thread of the group has passed its next barrier
    umma::fence_before_sync();
    if (!(done1 && done2)) {
      failed = true;
      if (r == 0) atomicExch(l.counter + 1, 1);
    }
    if (ok) {
      const size_t n = (size_t)y * a.pitch + x;
      for (int c = 0; c < 3; ++c) {
        const float cn = cdep[c] + l.ce * (o[c] * s.st[c] + s.mt[c]);
        Cn[(size_t)c * P + n] = cn;
        const float c1 = C1[(size_t)c * P + n];
        const float plain = c1 + Kf * (c1 - Cp[(size_t)c * P + n]);
        worst = fmaxf(worst, fabsf(cn - plain) / l.ce);
      }
    }
  }
  if (failed) {
    // the tile falls back; before the TMEM is freed, wait (again bounded) for the
    // group's last MMAs to complete
    worst = __int_as_float(0x7f800000);
    if (r == 0) umma::mbar_wait(&s.mbar[g], phase ^ 1u, polls);
  }
  red[tid] = worst;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = fmaxf(red[tid], red[tid + w]);
    __syncthreads();
  }
  if (!(red[0] <= l.threshold)) {      // NaN falls back too
    if (tid == 0) atomicAdd(l.counter, 1);
    for (int k = tid; k < T * T; k += blockDim.x) {
      const int x = tx0 + k % T, y = ty0 + k / T;
      if (x >= a.nx || y >= a.ny) continue;
      const size_t n = (size_t)y * a.pitch + x;
      for (int c = 0; c < 3; ++c) Cn[(size_t)c * P + n] = C1[(size_t)c * P + n];
    }
  }
  // every TMEM load has completed (the reduction's barriers follow them)
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(s.tmem, 64 * NET_GROUPS);
}

// Training features of every node (node order y-major, nx per row).
__global__ void __launch_bounds__(256) features_kernel(KernelArgs<float> a, LpmArgs l, float* X,
                                                       float* Cdep) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  float f[NIN], cdep[3];
  node_features(a, l, x, y, f, cdep);
  const size_t k = (size_t)y * a.nx + x;
  for (int i = 0; i < NIN; ++i) X[k * NIN + i] = f[i];
  for (int c = 0; c < 3; ++c) Cdep[k * 3 + c] = cdep[c];
}

__global__ void __launch_bounds__(256) targets_kernel(KernelArgs<float> a, LpmArgs l,
                                                      const float* Cdep, float* T) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  float pt, C[3];
  node_conformation(a, l, (size_t)y * a.pitch + x, pt, C);
  const size_t k = (size_t)y * a.nx + x;
  for (int c = 0; c < 3; ++c) T[k * 3 + c] = (C[c] - Cdep[k * 3 + c]) / l.ce;
}

// One solvent sub-step: pull, U under the interpolated polymer stress with the
// polymer momentum slaved (rho_S U = J_S + (tau2 + 1/2) E + rho a / 2 + dP), and
// the plain step's solvent collision.
__global__ void __launch_bounds__(256) solvent_kernel(KernelArgs<float> a, LpmArgs l,
                                                     const float* __restrict__ src,
                                                     float* __restrict__ dst, float frac) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t P = a.plane;
  const Nbr nb = nbr(x, y, a.nx, a.ny, a.pitch);
  const size_t n = nb.o[4];
  float h[9], drs = 0.f, jsx = 0.f, jsy = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    h[i] = src[(size_t)i * P + nb.o[shift_index(-c9x(i), -c9y(i))]];
    drs += h[i];
    jsx += float(c9x(i)) * h[i];
    jsy += float(c9y(i)) * h[i];
  }
  const float* psi = l.p + (size_t)L_PSI * P;
  auto theta = [&](int c, size_t m) {
    const float c1 = l.p[(size_t)(L_C1 + c) * P + m];
    const float cn = l.p[(size_t)(L_CNEW + c) * P + m];
    return 0.5f * l.H * psi[m] * (c1 + frac * (cn - c1));
  };
  const float ex = 0.5f * (theta(0, nb.o[5]) - theta(0, nb.o[3])) + 0.5f * (theta(1, nb.o[7]) - theta(1, nb.o[1]));
  const float ey = 0.5f * (theta(1, nb.o[5]) - theta(1, nb.o[3])) + 0.5f * (theta(2, nb.o[7]) - theta(2, nb.o[1]));
  const float rs = 1.f + drs;
  const float rho = rs + psi[n];
  const float force = rho * a.tab.arow[y];
  const float t = l.tau2 + 0.5f;
  const float Ux = (jsx + t * ex + 0.5f * force + l.p[(size_t)L_DP * P + n]) / rs;
  const float Uy = (jsy + t * ey + l.p[(size_t)(L_DP + 1) * P + n]) / rs;
  const float jfx = (a.c2 * jsx + rs * Ux + a.tau2 * force) * a.inv_c2p1;
  const float jfy = (a.c2 * jsy + rs * Uy) * a.inv_c2p1;
  const float usx = jfx / rs, usy = jfy / rs;
  const float vx = a.omr * usx + a.r * Ux, vy = a.omr * usy + a.r * Uy;
  const float sq = a.omr * (usx * usx + usy * usy) + a.r * (Ux * Ux + Uy * Uy);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float cx = float(c9x(i)), cy = float(c9y(i));
    const float cus = cx * usx + cy * usy, cu = cx * Ux + cy * Uy;
    const float feq_dev = float(w9(i)) * (drs + rs * (3.f * (cx * vx + cy * vy) +
                                                      4.5f * (a.omr * cus * cus + a.r * cu * cu) -
                                                      1.5f * sq));
    const float srcterm = float(w9(i)) * (3.f * (cx - Ux) + 9.f * cu * cx) * force;
    dst[(size_t)i * P + n] = a.om2b * h[i] + a.tb * feq_dev + a.omb * srcterm;
  }
}

// Move the polymer's Q-distribution of every node to C_new at unchanged psi_tot:
// dpsi(q) = psi_tot p0(q) sum_ab w_ab beta_ab (Q_a Q_b - m0_ab), beta = M0^-1 (C_new - C)/ell^2
// (equilibrium-weighted, so the 3 x 3 system is a constant, well-conditioned one).
// Rewrite the moment planes of the state (polymer part with dpsi, solvent part
// from the last sub-step) and keep psi_tot times the coefficients of the
// quadratic form for apply_kernel: dpsi(q) = p0(q) (B0 Qx^2 + B1 Qx Qy + B2 Qy^2 + B3).
__global__ void __launch_bounds__(256) reshape_kernel(KernelArgs<float> a, LpmArgs l) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t P = a.plane;
  const Nbr nb = nbr(x, y, a.nx, a.ny, a.pitch);
  const size_t n = nb.o[4];
  const int nq = a.nq;
  float pt, C[3];
  node_conformation(a, l, n, pt, C);
  float d[3];
  for (int c = 0; c < 3; ++c) d[c] = (l.p[(size_t)(L_CNEW + c) * P + n] - C[c]) / l.l2;
  float beta[3];
  for (int r = 0; r < 3; ++r)
    beta[r] = l.M0inv[3 * r] * d[0] + l.M0inv[3 * r + 1] * d[1] + l.M0inv[3 * r + 2] * d[2];
  const float B0 = pt * beta[0], B1 = pt * 2.f * beta[1], B2 = pt * beta[2];
  const float B3 = -pt * (beta[0] * l.m0[0] + 2.f * beta[1] * l.m0[1] + beta[2] * l.m0[2]);
  float* p = l.p;
  p[(size_t)L_B * P + n] = B0;
  p[(size_t)(L_B + 1) * P + n] = B1;
  p[(size_t)(L_B + 2) * P + n] = B2;
  p[(size_t)(L_B + 3) * P + n] = B3;
  float sum = 0.f, txx = 0.f, txy = 0.f, tyy = 0.f;
  for (int q = 0; q < nq; ++q) {
    const float qx = a.tab.qx[q], qy = a.tab.qy[q];
    const float dpsi = a.tab.psi0[q] * l.rpt0 * (B0 * qx * qx + B1 * qx * qy + B2 * qy * qy + B3);
    const float dv = a.M[(size_t)q * P + n] + dpsi;
    a.M[(size_t)q * P + n] = dv;
    sum += dv;
    txx += dpsi * qx * qx;
    txy += dpsi * qx * qy;
    tyy += dpsi * qy * qy;
  }
  float drs, jsx, jsy;
  solvent_pull_moments((const float*)a.src, P, nb, drs, jsx, jsy);
  a.M[(size_t)(nq + M_DRHO) * P + n] = drs + sum;
  a.M[(size_t)(nq + M_JX) * P + n] = jsx + p[(size_t)L_JP * P + n];
  a.M[(size_t)(nq + M_JY) * P + n] = jsy + p[(size_t)(L_JP + 1) * P + n];
  a.M[(size_t)(nq + M_THXX) * P + n] += l.hl2h * txx;
  a.M[(size_t)(nq + M_THXY) * P + n] += l.hl2h * txy;
  a.M[(size_t)(nq + M_THYY) * P + n] += l.hl2h * tyy;
  for (int c = 0; c < 3; ++c) p[(size_t)(L_CPREV + c) * P + n] = p[(size_t)(L_CNEW + c) * P + n];
}

// Add to every stored polymer population the increment that its pull delivers
// to (x, q, i): dg_i = w_i [dpsi + 3 (v_i . dpsi U + Qdot_i . dpsi (Q . grad U - kappa Q))],
// dpsi from reshape_kernel's coefficients, U and grad U those of the reshaped
// state (a.U). The pull is a permutation of the stored slots, so every slot is
// written by one thread. (The block itself leaves the increment to the next
// step's pull, which adds the same values; this kernel serves readers of the
// stored populations in between.)
__global__ void __launch_bounds__(256) apply_kernel(KernelArgs<float> a, LpmArgs l) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const size_t P = a.plane;
  const Nbr nb = nbr(x, y, a.nx, a.ny, a.pitch);
  const size_t n = nb.o[4];
  const float* Ux = a.U;
  const float* Uy = a.U + P;
  const float ux = Ux[n], uy = Uy[n];
  const float G00 = 0.5f * (Ux[nb.o[5]] - Ux[nb.o[3]]), G01 = 0.5f * (Uy[nb.o[5]] - Uy[nb.o[3]]);
  const float G10 = 0.5f * (Ux[nb.o[7]] - Ux[nb.o[1]]), G11 = 0.5f * (Uy[nb.o[7]] - Uy[nb.o[1]]);
  const float b0 = l.p[(size_t)L_B * P + n], b1 = l.p[(size_t)(L_B + 1) * P + n];
  const float b2 = l.p[(size_t)(L_B + 2) * P + n], b3 = l.p[(size_t)(L_B + 3) * P + n];
  float* pop = (float*)a.src;
  for (int q = 0; q < a.nq; ++q) {
    const float qx = a.tab.qx[q], qy = a.tab.qy[q];
    const float dpsi = a.tab.psi0[q] * l.rpt0 * (b0 * qx * qx + b1 * qx * qy + b2 * qy * qy + b3);
    const float jrx = dpsi * ux, jry = dpsi * uy;
    const float jqx = dpsi * (qx * G00 + qy * G10 - l.kappa * qx);
    const float jqy = dpsi * (qx * G01 + qy * G11 - l.kappa * qy);
    size_t slot[25];
    float v[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) {     // every load of the Q-node before any store
      const V4 c = c25(i);
      const int e = a.tab.pull[q * 25 + i];
      slot[i] = (size_t)(e >= 0 ? e : ~e) * P + (e >= 0 ? nb.o[shift_index(-c.rx, -c.ry)] : nb.o[4]);
      v[i] = pop[slot[i]];
    }
#pragma unroll
    for (int i = 0; i < 25; ++i) {
      const V4 c = c25(i);
      const float dg = float(w25(i)) *
                       (dpsi + 3.f * (float(c.rx) * jrx + float(c.ry) * jry + float(c.qx) * jqx + float(c.qy) * jqy));
      pop[slot[i]] = v[i] + dg * a.pscale;
    }
  }
}

dim3 node_grid2(int nx, int ny) { return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY); }

tfkt_status lpm_err(cudaError_t e, const char* what) {
  return fail(TFKT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LPM_CUDA(...)                                         \
  do {                                                        \
    cudaError_t e_ = (__VA_ARGS__);                           \
    if (e_ != cudaSuccess) return lpm_err(e_, #__VA_ARGS__);  \
  } while (0)

tfkt_status check(Ctx* c, int K) {
  const Lattice& L = c->L;
  if (L.precision != TFKT_FP32) return fail(TFKT_EINVAL, "the learned block needs an FP32 context");
  if (!c->fused) return fail(TFKT_EINVAL, "the learned block needs nx % 32 == 0 and ny % 8 == 0");
  if (!(L.psi_tot > 0)) return fail(TFKT_EINVAL, "the learned block needs a polymer (beta < 1)");
  if (L.fene_b != 0) return fail(TFKT_EINVAL, "the learned block is for Hookean springs");
  if (L.qe_model != TFKT_QE_MOMENTUM)
    return fail(TFKT_EINVAL, "the learned block uses the momentum quasi-equilibrium");
  if (L.nq < 4) return fail(TFKT_EINVAL, "the learned block needs at least 4 Q-nodes");
  if (K < 2 || K > 64 || (K & 1)) return fail(TFKT_EINVAL, "K must be even, 2 <= K <= 64");
  // a block reaches further than the ghost rows of a slab refreshed once per step
  if (c->slab_ny != 0) return fail(TFKT_EINVAL, "the learned block does not run on a slab context");
  if (c->poisoned) return fail(TFKT_ESTATE, "context is poisoned by an earlier CUDA error");
  return TFKT_OK;
}

tfkt_status setup(Ctx* c, int K, LpmArgs* l) {
  const Lattice& L = c->L;
  if (!c->lpm) {
    const size_t bytes = (size_t)L_NPLANES * L.plane * sizeof(float) + 256;
    LPM_CUDA(cudaMalloc(&c->lpm, bytes));
    c->lpm_step = -1;
  }
  const HostTables t = build_tables(L);
  double S0[3] = {0, 0, 0}, sxx = 0, ps = 0;
  for (int q = 0; q < L.nq; ++q) {
    S0[0] += t.psi0[q] * t.qx[q] * t.qx[q];
    S0[1] += t.psi0[q] * t.qx[q] * t.qy[q];
    S0[2] += t.psi0[q] * t.qy[q] * t.qy[q];
    ps += t.psi0[q];
  }
  sxx = S0[0];
  // equilibrium-weighted reshape: m0 and the inverse of M0 (3 x 3, in double)
  double m0[3] = {S0[0] / ps, S0[1] / ps, S0[2] / ps}, M0[3][3] = {};
  const double wgt[3] = {1.0, 2.0, 1.0};
  for (int q = 0; q < L.nq; ++q) {
    const double p0 = t.psi0[q] / ps;
    const double qq[3] = {t.qx[q] * t.qx[q], t.qx[q] * t.qy[q], t.qy[q] * t.qy[q]};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M0[r][c] += p0 * qq[r] * wgt[c] * (qq[c] - m0[c]);
  }
  const double det = M0[0][0] * (M0[1][1] * M0[2][2] - M0[1][2] * M0[2][1]) -
                     M0[0][1] * (M0[1][0] * M0[2][2] - M0[1][2] * M0[2][0]) +
                     M0[0][2] * (M0[1][0] * M0[2][1] - M0[1][1] * M0[2][0]);
  if (!(std::fabs(det) > 0)) return fail(TFKT_EINVAL, "the Q-disk's second moments are degenerate");
  double inv[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
      inv[r][c] = (M0[r1][c1] * M0[r2][c2] - M0[r1][c2] * M0[r2][c1]) / det;
    }
  LpmArgs a{};
  for (int k = 0; k < 3; ++k) a.m0[k] = (float)m0[k];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) a.M0inv[3 * r + c] = (float)inv[r][c];
  a.rpt0 = (float)(1.0 / L.psi_tot);
  a.p = (float*)c->lpm;
  a.counter = (int*)((char*)c->lpm + (size_t)L_NPLANES * L.plane * sizeof(float));
  for (int k = 0; k < 3; ++k) a.S0[k] = (float)S0[k];
  const double l2 = L.ell * L.ell;
  a.ce = (float)(l2 * sxx / ps);
  a.l2 = (float)l2;
  a.hl2h = (float)(0.5 * L.H * l2);
  a.H = (float)L.H;
  a.tau2 = (float)L.tau2;
  a.kappa = (float)L.kappa;
  a.inv_lambda = (float)(1.0 / L.lambda_h);
  a.K = K;
  *l = a;
  return TFKT_OK;
}

}  // namespace

// Add the pending increment to the stored populations now (for readers of the
// populations): U and grad U of the reshaped state, then the slot updates.
tfkt_status ctx_lpm_flush(Ctx* c) {
  if (!c->lpm_pending) return TFKT_OK;
  LpmArgs l;
  tfkt_status s = setup(c, 2, &l);
  if (s != TFKT_OK) return s;
  const Lattice& L = c->L;
  KernelArgs<float> a = ctx_args<float>(c);
  LPM_CUDA(launch_velocity<float>(a, c->stream));
  apply_kernel<<<node_grid2(L.nx, L.ny), dim3(TX, TY), 0, c->stream>>>(a, l);
  LPM_CUDA(cudaGetLastError());
  c->lpm_pending = false;
  return TFKT_OK;
}

}  // namespace tfkt

using namespace tfkt;

extern "C" tfkt_status tfkt_lpm_run(tfkt_ctx* cc, const tfkt_mlp* net, const tfkt_lpm_opts* o,
                                    int64_t nblocks, int64_t* flagged) {
  NvtxRange nvtx_range("tfkt_lpm_run");
  if (!cc || !o) return fail(TFKT_EINVAL, "NULL argument");
  Ctx* c = ctx_of(cc);
  tfkt_status s = check(c, o->K);
  if (s != TFKT_OK) return s;
  if (o->tile < 1 || o->tile > 64) return fail(TFKT_EINVAL, "tile must be in [1, 64]");
  if (o->mode != TFKT_LPM_NET && o->mode != TFKT_LPM_FROZEN) return fail(TFKT_EINVAL, "unknown mode");
  if (o->mode == TFKT_LPM_NET && !net) return fail(TFKT_EINVAL, "the network is NULL");
  if (!(o->threshold >= 0)) return fail(TFKT_EINVAL, "threshold must be >= 0");
  if (nblocks < 0) return fail(TFKT_EINVAL, "nblocks must be >= 0");
  LpmArgs l;
  if ((s = setup(c, o->K, &l)) != TFKT_OK) return s;
  l.tile = o->tile;
  l.mode = o->mode;
  l.threshold = o->threshold;
  l.inject_wait_timeout = o->inject_wait_timeout != 0;
  if ((s = ctx_ensure_moments_f32(c)) != TFKT_OK) return s;
  const Lattice& L = c->L;
  cudaStream_t st = c->stream;
  const dim3 grid = node_grid2(L.nx, L.ny), blk(TX, TY);
  const dim3 tiles((L.nx + o->tile - 1) / o->tile, (L.ny + o->tile - 1) / o->tile);
  MlpDev nd{};
  if (net) nd = mlp_dev(net);
  LPM_CUDA(cudaMemsetAsync(l.counter, 0, 2 * sizeof(int), st));
  for (int64_t b = 0; b < nblocks; ++b) {
    if (c->lpm_step != c->step) {
      conf_kernel<<<grid, blk, 0, st>>>(ctx_args<float>(c), l, L_CPREV);
      LPM_CUDA(cudaGetLastError());
    }
    if ((s = tfkt_step(cc, 1)) != TFKT_OK) return s;
    KernelArgs<float> a = ctx_args<float>(c);
    LPM_CUDA(launch_velocity<float>(a, st));
    prepare_kernel<<<grid, blk, 0, st>>>(a, l);
    LPM_CUDA(cudaGetLastError());
    const size_t nsm = net_smem_bytes();
    LPM_CUDA(cudaFuncSetAttribute(net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm));
    net_kernel<<<tiles, NET_THREADS, nsm, st>>>(a, l, nd);
    LPM_CUDA(cudaGetLastError());
    for (int j = 0; j < o->K; ++j) {
      KernelArgs<float> aj = ctx_args<float>(c);
      solvent_kernel<<<grid, blk, 0, st>>>(aj, l, (const float*)aj.src, (float*)aj.dst,
                                           (float)j / (float)o->K);
      LPM_CUDA(cudaGetLastError());
      c->cur ^= 1;
    }
    a = ctx_args<float>(c);
    reshape_kernel<<<grid, blk, 0, st>>>(a, l);
    LPM_CUDA(cudaGetLastError());
    // the increment rides on the next step's pull (tfkt_step, or the next block)
    c->lpm_pending = true;
    c->lpm_rshp = l.p + (size_t)L_B * L.plane;
    c->step += o->K;
    c->lpm_step = c->step;
  }
  int h[2] = {0, 0};
  LPM_CUDA(cudaMemcpyAsync(h, l.counter, sizeof(h), cudaMemcpyDeviceToHost, st));
  LPM_CUDA(cudaStreamSynchronize(st));
  if (flagged) *flagged = h[0];
  if (h[1])
    return fail(TFKT_ETIMEOUT, "a tensor-core wait of the network kernel ran out "
                               "(the affected tiles fell back to the plain step)");
  return TFKT_OK;
}

extern "C" tfkt_status tfkt_lpm_features(tfkt_ctx* cc, int32_t K, float* X, float* Cdep) {
  NvtxRange nvtx_range("tfkt_lpm_features");
  if (!cc || !X || !Cdep) return fail(TFKT_EINVAL, "NULL argument");
  Ctx* c = ctx_of(cc);
  tfkt_status s = check(c, K);
  if (s != TFKT_OK) return s;
  LpmArgs l;
  if ((s = setup(c, K, &l)) != TFKT_OK) return s;
  if ((s = ctx_ensure_moments_f32(c)) != TFKT_OK) return s;
  const Lattice& L = c->L;
  const dim3 grid = node_grid2(L.nx, L.ny), blk(TX, TY);
  KernelArgs<float> a = ctx_args<float>(c);
  LPM_CUDA(launch_velocity<float>(a, c->stream));
  conf_kernel<<<grid, blk, 0, c->stream>>>(a, l, L_C1);
  LPM_CUDA(cudaGetLastError());
  features_kernel<<<grid, blk, 0, c->stream>>>(a, l, X, Cdep);
  LPM_CUDA(cudaGetLastError());
  return TFKT_OK;
}

extern "C" tfkt_status tfkt_lpm_targets(tfkt_ctx* cc, const float* Cdep, float* T) {
  NvtxRange nvtx_range("tfkt_lpm_targets");
  if (!cc || !Cdep || !T) return fail(TFKT_EINVAL, "NULL argument");
  Ctx* c = ctx_of(cc);
  tfkt_status s = check(c, 2);
  if (s != TFKT_OK) return s;
  LpmArgs l;
  if ((s = setup(c, 2, &l)) != TFKT_OK) return s;
  if ((s = ctx_ensure_moments_f32(c)) != TFKT_OK) return s;
  const Lattice& L = c->L;
  targets_kernel<<<node_grid2(L.nx, L.ny), dim3(TX, TY), 0, c->stream>>>(ctx_args<float>(c), l, Cdep, T);
  LPM_CUDA(cudaGetLastError());
  return TFKT_OK;
}
