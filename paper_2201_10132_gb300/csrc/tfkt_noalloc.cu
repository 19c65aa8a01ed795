// tfkt_moments_noalloc: the macroscopic-field path (moments -> velocity ->
// fields kernels) for callers that must not allocate device memory, e.g. code
// running inside a memory-capped arena or a host framework whose allocator
// may not be entered at that point. Its scratch (moment planes, velocity
// planes, lattice tables) lives in one file-scope device array instead of an
// allocation; the caller passes the populations and the output buffer.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "tfkt_internal.cuh"

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TFKT_NOALLOC_SCRATCH_BYTES];

namespace tfkt {
namespace {

// Device address of g_noalloc_scratch, looked up once per device. In host
// code the symbol's name only stands for it; only this address may be given
// to a kernel.
constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
// Parameters whose lattice tables the array of each device holds (valid once
// an upload has completed); a call with the same parameters reuses them.
tfkt_params g_tables_of[kMaxDevices];
bool g_tables_valid[kMaxDevices] = {};

bool same_params(const tfkt_params& a, const tfkt_params& b) {
  return a.nx == b.nx && a.ny == b.ny && a.q_side == b.q_side && a.q_radius == b.q_radius &&
         a.re == b.re && a.wi == b.wi && a.beta == b.beta && a.u0 == b.u0 &&
         a.k_periods == b.k_periods && a.tau2 == b.tau2 && a.ell == b.ell &&
         a.ic_mode == b.ic_mode && a.precision == b.precision && a.fene_b == b.fene_b &&
         a.qe_model == b.qe_model;
}

tfkt_status scratch_address(void** out, int* device) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(TFKT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(TFKT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  *device = dev;
  return TFKT_OK;
}

template <typename real, typename S>
tfkt_status moments_noalloc(const tfkt_params& p, const Lattice& L, const void* pops,
                            uint32_t mask, double* dst, cudaStream_t stream) {
  // scratch layout: M planes, U planes, then the tables
  const size_t sz = sizeof(real), A = 256, nq = L.nq;
  size_t o = 0;
  const size_t off_M = o;
  o = align_up(o + (size_t)L.nm * L.plane * sz, A);
  const size_t off_U = o;
  o = align_up(o + 2 * L.plane * sz, A);
  constexpr int NT = 9, KPULL = 5;
  size_t off_t[NT];
  const size_t tsz[NT] = {nq * sz, nq * sz, nq * sz, nq * sz, nq * sz, nq * 25 * sizeof(int),
                          nq * 25 * sz, (size_t)L.ny * sz, (size_t)L.ny * sz};
  for (int k = 0; k < NT; ++k) {
    off_t[k] = o;
    o = align_up(o + tsz[k], A);
  }
  if (o > (size_t)TFKT_NOALLOC_SCRATCH_BYTES)
    return fail(TFKT_EINVAL, "grid too large for tfkt_moments_noalloc: needs " + std::to_string(o) +
                                 " bytes of scratch, the static scratch holds " +
                                 std::to_string((size_t)TFKT_NOALLOC_SCRATCH_BYTES));
  void* base = nullptr;
  int dev = 0;
  tfkt_status s = scratch_address(&base, &dev);
  if (s != TFKT_OK) return s;
  char* b = (char*)base;

  // Lattice tables: uploaded when the array does not hold those of these
  // parameters yet (the first call on the device, or other parameters than the
  // last upload). The host copies are pageable, so the stream is synchronised
  // before they go out of scope; a call that finds its tables in place only
  // queues the kernels.
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_tables_valid[dev] || !same_params(g_tables_of[dev], p)) {
      g_tables_valid[dev] = false;
      const HostTables t = build_tables(L);
      const std::vector<double>* src[NT] = {&t.qx,    &t.qy,    &t.fx,   &t.fy,  &t.psi0,
                                            nullptr, &t.delta, &t.arow, &t.urow};
      std::vector<real> conv[NT];
      for (int k = 0; k < NT; ++k) {
        if (k == KPULL) {
          e = cudaMemcpyAsync(b + off_t[k], t.pull.data(), tsz[k], cudaMemcpyHostToDevice, stream);
        } else {
          conv[k].assign(src[k]->begin(), src[k]->end());
          e = cudaMemcpyAsync(b + off_t[k], conv[k].data(), tsz[k], cudaMemcpyHostToDevice, stream);
        }
        if (e != cudaSuccess)
          return fail(TFKT_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
      }
      e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
      g_tables_of[dev] = p;
      g_tables_valid[dev] = true;
    }
  }

  KernelArgs<real> a{};
  a.src = pops;
  a.dst = nullptr;
  a.M = (real*)(b + off_M);
  a.U = (real*)(b + off_U);
  a.nx = L.nx;
  a.ny = L.ny;
  a.nq = L.nq;
  a.pitch = L.pitch;
  a.plane = L.plane;
  a.tau2 = (real)L.tau2;
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
  a.tab.qx = (const real*)(b + off_t[0]);
  a.tab.qy = (const real*)(b + off_t[1]);
  a.tab.fx = (const real*)(b + off_t[2]);
  a.tab.fy = (const real*)(b + off_t[3]);
  a.tab.psi0 = (const real*)(b + off_t[4]);
  a.tab.pull = (const int*)(b + off_t[5]);
  a.tab.delta = (const real*)(b + off_t[6]);
  a.tab.arow = (const real*)(b + off_t[7]);
  a.tab.urow = (const real*)(b + off_t[8]);
  // every plane read below is written first by these kernels: the moments
  // kernel writes all M planes of every node, the velocity kernel both U
  // planes of every node, so nothing needs clearing between calls (the tables
  // are those of these parameters, checked above)
  if ((e = launch_moments<real, S>(a, stream)) != cudaSuccess ||
      (e = launch_velocity<real>(a, stream)) != cudaSuccess ||
      (e = launch_fields<real>(a, mask, dst, stream)) != cudaSuccess)
    return fail(TFKT_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return TFKT_OK;
}

}  // namespace
}  // namespace tfkt

extern "C" tfkt_status tfkt_moments_noalloc(const tfkt_params* p, const void* pops,
                                            uint32_t field_mask, double* dst, size_t bytes,
                                            void* stream) {
  using namespace tfkt;
  Lattice L;
  tfkt_status s = map_params(p, &L);
  if (s != TFKT_OK) return s;
  if (!pops || !dst) return fail(TFKT_EINVAL, "pops and dst must be device pointers");
  if (field_mask == 0 || (field_mask >> TFKT_NFIELDS) != 0) return fail(TFKT_EINVAL, "bad field mask");
  const size_t need = (size_t)__builtin_popcount(field_mask) * L.nx * L.ny * sizeof(double);
  if (bytes < need) return fail(TFKT_EINVAL, "dst too small");
  if (L.precision == TFKT_FP64)
    return moments_noalloc<double, double>(*p, L, pops, field_mask, dst, (cudaStream_t)stream);
  if (L.precision == TFKT_FP32)
    return moments_noalloc<float, float>(*p, L, pops, field_mask, dst, (cudaStream_t)stream);
  return moments_noalloc<float, __half>(*p, L, pops, field_mask, dst, (cudaStream_t)stream);
}
