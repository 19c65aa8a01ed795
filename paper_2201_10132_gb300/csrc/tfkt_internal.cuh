// Internal declarations of libtfkt: lattice tables, context layout, kernel
// arguments and launchers. Not part of the C-ABI (include/tfkt.h is).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "tfkt.h"

namespace tfkt {

// Scoped NVTX range naming one call of the C interface (create, step,
// diagnostics, ...) on a profiler timeline. NVTX v3 is header-only; with no
// tool attached a push or pop is a call into an empty function.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- lattices
// D2Q9 (Sec. VI-A): rest, the four axis velocities, the four diagonals.
// The paper's printed angle formula mixes axes and diagonals for i = 1..4;
// the standard set is used.
__host__ __device__ constexpr int c9x(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int c9y(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr double w9(int i) {
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// D4Q25 on (r_x, r_y, Q_x, Q_y) (Sec. VI-B, Table dis_vel), grouped by the
// r-displacement so that a block of velocities shares one pull offset:
//   0        rest
//   1..4     (+-1, +-1, 0, 0)   r-diagonals, Q at rest
//   5..8     (+-1, 0, +-1, 0)   9..12  (+-1, 0, 0, +-1)
//   13..16   (0, +-1, +-1, 0)   17..20 (0, +-1, 0, +-1)
//   21..24   (0, 0, +-1, +-1)   Q-diagonals, r at rest
// Weights 1/3 (rest) and 1/36, c_sP^2 = 1/3.
struct V4 {
  int rx, ry, qx, qy;
};
__host__ __device__ constexpr V4 c25(int i) {
  // sign pattern of the four members of each group: (+,+), (+,-), (-,+), (-,-)
  // for the mixed groups; the two diagonal groups follow the D2Q9 diagonal order.
  return i == 0 ? V4{0, 0, 0, 0}
       : i <= 4 ? V4{c9x(i + 4), c9y(i + 4), 0, 0}
       : i <= 8 ? V4{(i - 5) < 2 ? 1 : -1, 0, ((i - 5) & 1) ? -1 : 1, 0}
       : i <= 12 ? V4{(i - 9) < 2 ? 1 : -1, 0, 0, ((i - 9) & 1) ? -1 : 1}
       : i <= 16 ? V4{0, (i - 13) < 2 ? 1 : -1, ((i - 13) & 1) ? -1 : 1, 0}
       : i <= 20 ? V4{0, (i - 17) < 2 ? 1 : -1, 0, ((i - 17) & 1) ? -1 : 1}
                 : V4{0, 0, c9x(i - 16), c9y(i - 16)};
}
__host__ __device__ constexpr double w25(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 36.0; }

// Index of the pull offset for a source displaced by (sx, sy) in {-1,0,1}^2.
__host__ __device__ constexpr int shift_index(int sx, int sy) { return (sy + 1) * 3 + (sx + 1); }

constexpr int TX = 32;   // tile width (one warp along x)
constexpr int TY = 8;    // tile height of the single-run path (batches choose 4, 8 or 16)

// --------------------------------------------------------------- contexts
// Derived lattice parameters (lattice units).
struct Lattice {
  int nx = 0, ny = 0, S = 0, nq = 0;
  double q_radius = 0;
  double tau1 = 0, tau2 = 0, H = 0, kappa = 0, ell = 0, psi_tot = 0, sigma_q2 = 0;
  double a0 = 0, kf = 0, u0 = 0, nu = 0, nu_s = 0, eta_p = 0, lambda_h = 0;
  int ic_mode = 0, precision = 0;
  double fene_b = 0;  // 0: Hookean springs; > 0: FENE extensibility b
  int qe_model = 0;   // tfkt_qe_model
  double tau_m = 0;   // momentum relaxation time (drag, Q-drift, bead diffusion)
  size_t pitch = 0;   // elements per stored row
  size_t plane = 0;   // elements per plane (ny * pitch)
  int npl = 0;        // population planes: 9 + 25 nq
  int nm = 0;         // moment planes: nq + 6
  // Rows of a slab of a larger run (tfkt_slab_*): local row y holds global row
  // (y_origin + y) mod ny_global; the forcing and the laminar profile follow the
  // global row. ny_global = 0: the context is the whole run.
  int y_origin = 0;
  int ny_global = 0;
};

// Moment field planes (M): delta psi(q) for q < nq, then these.
enum { M_DRHO = 0, M_JX, M_JY, M_THXX, M_THXY, M_THYY, M_NSCALAR };

// Device tables of a context (one copy per precision in use).
template <typename real>
struct Tables {
  const real* qx;        // [nq] Q_x (Q lattice units)
  const real* qy;        // [nq]
  const real* fx;        // [nq] phi_q Q_x: spring force / H (phi_q = 1 Hookean,
  const real* fy;        //      1 / (1 - Q^2/Q0^2) FENE); equal to Q bit for bit when Hookean
  const real* psi0;      // [nq] storage shift of the polymer: w_i psi0(q)
  const int* pull;       // [nq*25]: >= 0 source plane (shifted by -c_r); < 0: ~plane, bounce-back
  const real* delta;     // [nq*25]: w_i (psi0(q - Qdot_i) - psi0(q)), 0 for bounce-back
  const real* arow;      // [ny] forcing a(y)
  const real* urow;      // [ny] initial base flow U_x(y)
};

// Conversions between the storage type S of the populations and the compute
// type real (FP16 storage is computed in FP32; round to nearest on store).
template <typename real, typename S>
__host__ __device__ __forceinline__ real from_store(S v) { return (real)v; }
template <>
__host__ __device__ __forceinline__ float from_store<float, __half>(__half v) { return __half2float(v); }
template <>
__host__ __device__ __forceinline__ double from_store<double, __half>(__half v) {
  return (double)__half2float(v);
}
template <typename S, typename real>
__host__ __device__ __forceinline__ S to_store(real v) { return (S)v; }
template <>
__host__ __device__ __forceinline__ __half to_store<__half, float>(float v) { return __float2half_rn(v); }

// Storage type of the nine solvent planes. FP16 storage keeps them in FP32:
// the solvent carries nearly all of the mixture momentum, and its stored
// deviations w_i (3 c_i.u + ...) ~ 1e-2 round in FP16 to ~1e-5, the size of a
// small velocity perturbation's share of them; they are 9 of 9 + 25 nq planes,
// so FP32 costs ~1% of the bytes. FP64 and FP32 store them like the polymer.
template <typename S> struct SolventStore { using type = S; };
template <> struct SolventStore<__half> { using type = float; };
template <typename S> using SolventT = typename SolventStore<S>::type;

// A population buffer of storage S holds 9 + 25 nq plane slots of S, `plane`
// elements each: polymer plane k (k >= 9) in slot k. Solvent planes of the
// storage type itself fill slots 0..8; FP32 solvent planes under FP16 storage
// follow the last slot instead (slots 0..8 stay unused), so that the polymer
// planes keep the addresses they have when every plane is FP16.
template <typename S>
__host__ __device__ __forceinline__ const SolventT<S>* solvent_planes(const void* buf, size_t plane,
                                                                       int nq) {
  if (sizeof(SolventT<S>) == sizeof(S)) return (const SolventT<S>*)buf;
  return (const SolventT<S>*)((const S*)buf + (size_t)(9 + 25 * nq) * plane);
}
template <typename S>
__host__ __device__ __forceinline__ SolventT<S>* solvent_planes(void* buf, size_t plane, int nq) {
  return const_cast<SolventT<S>*>(solvent_planes<S>((const void*)buf, plane, nq));
}

template <typename real>
struct KernelArgs {
  const void* src;               // populations read (pull): plane slots, see solvent_planes
  void* dst;                     // populations written
  real* M;                       // moment planes
  real* U;                       // scratch: 2 planes (U_x, U_y)
  const double* perturb;         // [2][ny][nx] (init only)
  int nx, ny, nq;
  size_t pitch, plane;
  real tau2, c2, inv_c2p1;       // tau2, 2 tau2, 1 / (2 tau2 + 1)
  real om2b, tb, omb;            // 1 - 2 beta, 2 beta, 1 - beta
  real r, omr;                   // tau1 / tau2, 1 - tau1 / tau2
  real kappa, hl2h;              // kappa, H ell^2 / 2
  real tau_m;                    // momentum relaxation time (tau2, or tau1 in the stress model)
  int qe;                        // tfkt_qe_model
  real rho0;                     // 1 + psi_tot: total density of the rest state
  real psi_tot0;
  real l2, H;
  real pscale, pinv;             // polymer storage scale (a power of two) and its inverse
  Tables<real> tab;
};

// Extra arguments of the fused step and its border fix-up.
template <typename real>
struct FusedArgs {
  const real* Min;      // complete moment planes of the state being stepped
  real* Mout;           // moment planes of the next state (written)
  real* exports;        // [nq + 3][tiles][ring] arrivals at ring nodes from each tile
  const int* tgt;       // [nq][9] target Q-node per Q-displacement group, -1: bounce-back
  const real* dpsi;     // [nq] sum over i of the pull shift differences of Q-node q
  const long long* poff;  // [nq*25] element offset of each pull's source plane
  real dvx, dvy;        // r-momentum of all pull shift differences
  // Pending increment of a learned block (or null): per node the coefficients
  // B0..B3 (4 planes) of dpsi(q) = p0(q) (B0 Qx^2 + B1 Qx Qy + B2 Qy^2 + B3), added to
  // the pulled polymer populations as a linear quasi-equilibrium (FP32 only).
  const real* rshp;
};

// One run of a batch: its kernel arguments for both buffer parities.
template <typename real>
struct BatchRun {
  KernelArgs<real> a[2];
  FusedArgs<real> f[2];
  int ntx, nty;
  int pad[2];
};

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  bool owned = false;
  size_t off_pop[2] = {0, 0};
  size_t off_M = 0, off_U = 0, off_tab = 0, off_part = 0, off_diag = 0;
  size_t off_M2 = 0, off_exp = 0, off_ftab = 0;  // fused path: second M, ring exports, tables
};

struct Ctx {
  Lattice L;
  Workspace ws;
  cudaStream_t stream = nullptr;
  int cur = 0;            // population buffer holding the state
  bool m_valid = false;   // M holds the moments of the current state
  bool poisoned = false;
  int64_t step = 0;
  int diag_blocks = 0;
  bool fused = false;     // grid fits the fused single-pass kernel
  int mcur = 0;           // moment buffer (0: off_M, 1: off_M2) of the current state
  double dvx = 0, dvy = 0;  // r-momentum of all pull shift differences (fused path)
  void* lpm = nullptr;    // scratch of the learned block (allocated on first use)
  int64_t lpm_step = -1;  // step whose conformation the learned block's scratch holds
  bool lpm_pending = false;        // an increment waits to be added at the next pull
  const float* lpm_rshp = nullptr; // its coefficient planes
  bool in_batch = false;  // a run of a tfkt_batch (its buffer parity belongs to the batch)
  int slab_y0 = 0;        // a slab context (tfkt_slab_create): first owned global row,
  int slab_ny = 0;        // owned rows (0: not a slab); the ghost rows are around them
};

// Host helpers (tfkt_api.cu).
tfkt_status fail(tfkt_status s, const std::string& msg);
size_t align_up(size_t v, size_t a);
tfkt_status map_params(const tfkt_params* p, Lattice* L);
size_t real_size(const Lattice& L);   // bytes of the compute type (moment planes, tables)
size_t store_size(const Lattice& L);  // bytes of the population storage type
size_t population_bytes(const Lattice& L);  // one population buffer: solvent + polymer planes
// Polymer populations are stored as (deviation x scale): a power of two that
// brings them to order one in FP16 storage (exact, so FP16 keeps its full 11
// bits instead of falling into the subnormal range); 1 for FP32 and FP64.
double polymer_scale(const Lattice& L);
struct HostTables {
  std::vector<double> qx, qy, fx, fy, psi0, delta, arow, urow;
  std::vector<int> pull;
};
HostTables build_tables(const Lattice& L);

// Launchers (tfkt_kernels.cu). Each returns the launch status.
template <typename real, typename S>
cudaError_t launch_init(const KernelArgs<real>& a, cudaStream_t s);
template <typename real, typename S>
cudaError_t launch_moments(const KernelArgs<real>& a, cudaStream_t s);
template <typename real, typename S>
cudaError_t launch_step(const KernelArgs<real>& a, cudaStream_t s);
template <typename real>
cudaError_t launch_velocity(const KernelArgs<real>& a, cudaStream_t s);
template <typename real>
cudaError_t launch_fields(const KernelArgs<real>& a, uint32_t mask, double* out, cudaStream_t s);
template <typename real>
cudaError_t launch_psi(const KernelArgs<real>& a, double* out, cudaStream_t s);
template <typename real, typename S>
cudaError_t launch_populations(const KernelArgs<real>& a, double* out, cudaStream_t s);
template <typename real>
cudaError_t launch_diag(const KernelArgs<real>& a, double* partials, int nblocks, double* out,
                        cudaStream_t s);

// Fused single-pass step (tfkt_fused.cu).
size_t fused_smem_bytes(int nq, size_t real_bytes, int ty = TY);
size_t fused_export_elems(int nx, int ny, int nq, int ty = TY);
// ring-export elements enough for every tile height the grid allows (4, 8, 16)
size_t fused_export_capacity(int nx, int ny, int nq);
bool fused_supported(int nx, int ny, int nq, size_t real_bytes, int ty = TY);
void fused_tables(const Lattice& L, const HostTables& t, std::vector<int>& tgt,
                  std::vector<double>& dpsi, double& dvx, double& dvy,
                  std::vector<long long>& poff);
template <typename real, typename S>
cudaError_t launch_step_fused(const KernelArgs<real>& a, const FusedArgs<real>& f, cudaStream_t s);
template <typename real>
cudaError_t launch_fixup(const KernelArgs<real>& a, const FusedArgs<real>& f, cudaStream_t s);
// Whether a context of this lattice takes the fused path (tile multiples and the
// kernel's shared memory; either quasi-equilibrium).
bool fused_path(const Lattice& L);

// Each run's single-run FP32 kernels (fused step + fix-up) without API calls
// besides the launches, after prepare_single_fp32 for the largest nq.
cudaError_t prepare_single_fp32(int max_nq);
cudaError_t launch_single_fp32(const KernelArgs<float>& a, const FusedArgs<float>& f,
                               cudaStream_t s);
// Batched fused step (FP32): all tiles of all runs in one launch of each kernel.
cudaError_t prepare_batch(int max_nq, int ty);
cudaError_t launch_batch_step(const BatchRun<float>* runs, const int* tile_start, int nruns,
                              int total_tiles, int max_nq, int parity, cudaStream_t s, int ty);
// Access to a context's internals and argument builders (tfkt_api.cu).
Ctx* ctx_of(tfkt_ctx* c);
// A context of an already mapped lattice: workspace, tables, initial state
// (tfkt_create does the mapping first; tfkt_slab_create adjusts the rows).
tfkt_status ctx_create(const Lattice& L, const double* perturb, void* dev_workspace,
                       size_t workspace_bytes, void* stream, tfkt_ctx** out);
size_t ctx_layout(const Lattice& L);
template <typename real>
KernelArgs<real> ctx_args(const Ctx* c);
template <typename real>
FusedArgs<real> ctx_fused(const Ctx* c);
// Make the moment planes of an FP32 context (of any context) current (tfkt_api.cu).
tfkt_status ctx_ensure_moments_f32(Ctx* c);
tfkt_status ctx_ensure_moments(Ctx* c);
// Write the initial state (Sec. VI-D) again, from this perturbation (tfkt_api.cu).
tfkt_status ctx_reinit(Ctx* c, const double* perturb);
// Add a pending learned-block increment to the stored populations (tfkt_lpm.cu).
tfkt_status ctx_lpm_flush(Ctx* c);

constexpr int DIAG_THREADS = 256;

}  // namespace tfkt
