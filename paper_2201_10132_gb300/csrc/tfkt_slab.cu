// Domain decomposition of one run in y (tfkt_slab_*).
//
// A slab context holds the owned global rows [y0, y0 + n) and G ghost rows on
// each side; it is an ordinary periodic context of n + 2G rows whose forcing
// and laminar profile follow the global rows (Lattice::y_origin). One step of
// the scheme (Sec. VI: pull-streaming over one node, the mixture velocity with
// the divergence of the stress, central differences of U and psi) reads data
// at most three rows away, so within one step whatever the periodic wrap of the
// extended slab brings into its outermost rows reaches at most three rows in;
// G = 8, one row of the fused path's 32 x 8 tiles, keeps every owned row clear
// of it and, with slabs starting on multiples of 8, keeps the tiles those of
// the whole run (a node on a tile border sums its arrivals in another order
// than an interior node). Every owned row is then computed exactly as in the
// whole run, provided the ghost rows are overwritten with the neighbours'
// current rows (current populations and moment planes) before each step. The
// exchange moves G rows of every plane per side: G rows of a plane are one
// contiguous chunk, and the message is the chunks back to back. Packing and
// unpacking run on the context's stream, as one gather or scatter kernel when
// the message is in device memory and as strided copies when it is on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "tfkt_internal.cuh"

namespace tfkt {
namespace {

constexpr int G = TFKT_SLAB_GHOST;

tfkt_status slab_lattice(const tfkt_params* p, int32_t y0, int32_t ny_local, Lattice* L) {
  tfkt_status s = map_params(p, L);
  if (s != TFKT_OK) return s;
  if (ny_local < G || ny_local > p->ny)
    return fail(TFKT_EINVAL, "ny_local must be in [TFKT_SLAB_GHOST, ny]");
  if (y0 < 0 || y0 >= p->ny) return fail(TFKT_EINVAL, "y0 must be in [0, ny)");
  L->ny_global = p->ny;
  L->y_origin = y0 - G;
  L->ny = ny_local + 2 * G;
  L->plane = (size_t)L->ny * L->pitch;
  return TFKT_OK;
}

struct Blocks {
  // strided blocks of a halo message: base offset in the workspace, plane stride
  // and row length in bytes, number of planes
  size_t off[3], stride[3], bytes_per_row[3];
  int planes[3];
  int n;
};

Blocks halo_blocks(const Ctx* c) {
  const Lattice& L = c->L;
  Blocks b{};
  const size_t es = store_size(L), rs = real_size(L);
  b.off[0] = c->ws.off_pop[c->cur];
  b.stride[0] = L.plane * es;
  b.bytes_per_row[0] = L.pitch * es;
  b.planes[0] = L.npl;
  b.n = 1;
  if (L.precision == TFKT_FP16) {   // the FP32 solvent planes after the FP16 slots
    b.off[1] = c->ws.off_pop[c->cur] + (size_t)L.npl * L.plane * es;
    b.stride[1] = L.plane * sizeof(float);
    b.bytes_per_row[1] = L.pitch * sizeof(float);
    b.planes[1] = 9;
    b.n = 2;
  }
  b.off[b.n] = c->mcur ? c->ws.off_M2 : c->ws.off_M;
  b.stride[b.n] = L.plane * rs;
  b.bytes_per_row[b.n] = L.pitch * rs;
  b.planes[b.n] = L.nm;
  ++b.n;
  return b;
}

// Moves the chunks of a halo message between the workspace and the message
// (pack: workspace -> message) in 16-byte words. Chunk sizes, offsets and plane
// strides are multiples of 16 bytes (rows are padded to 32 elements).
struct ChunkSet {
  size_t off[3], stride[3];   // byte offset of plane 0's chunk, plane stride (bytes)
  uint32_t words[3];          // 16-byte words per chunk
  uint32_t first[3];          // first message word of each block
  uint32_t total;             // words of the message (< 2^31)
  int n;
};

__global__ void __launch_bounds__(256) halo_copy_kernel(int4* __restrict__ ws, int4* __restrict__ msg,
                                                        ChunkSet cs, int pack) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < cs.total; u += gridDim.x * blockDim.x) {
    // the block of word u, selected with constant indices (the arguments stay in
    // the parameter space)
    const bool b2 = cs.n > 2 && u >= cs.first[2];
    const bool b1 = !b2 && cs.n > 1 && u >= cs.first[1];
    const uint32_t first = b2 ? cs.first[2] : (b1 ? cs.first[1] : cs.first[0]);
    const uint32_t words = b2 ? cs.words[2] : (b1 ? cs.words[1] : cs.words[0]);
    const size_t off = b2 ? cs.off[2] : (b1 ? cs.off[1] : cs.off[0]);
    const size_t stride = b2 ? cs.stride[2] : (b1 ? cs.stride[1] : cs.stride[0]);
    const uint32_t v = u - first;
    const uint32_t p = v / words, w = v - p * words;
    int4* cell = ws + (off + (size_t)p * stride) / 16 + w;
    if (pack) msg[u] = *cell;
    else *cell = msg[u];
  }
}

size_t halo_bytes(const Ctx* c) {
  const Blocks b = halo_blocks(c);
  size_t t = 0;
  for (int k = 0; k < b.n; ++k) t += (size_t)b.planes[k] * G * b.bytes_per_row[k];
  return t;
}

tfkt_status check_slab(Ctx* c, int32_t side, const void* buf, size_t bytes) {
  if (!c) return fail(TFKT_EINVAL, "context is NULL");
  if (c->poisoned) return fail(TFKT_ESTATE, "context poisoned by an earlier CUDA error");
  if (c->slab_ny == 0) return fail(TFKT_EINVAL, "not a slab context");
  if (side != TFKT_SLAB_LOW && side != TFKT_SLAB_HIGH) return fail(TFKT_EINVAL, "unknown side");
  if (!buf) return fail(TFKT_EINVAL, "buffer is NULL");
  if (bytes < halo_bytes(c)) return fail(TFKT_EINVAL, "buffer smaller than tfkt_slab_halo_bytes");
  return TFKT_OK;
}

// Copies G rows starting at extended row r0 of every plane of the current state
// to (pack) or from (unpack) a message buffer.
tfkt_status move_rows(Ctx* c, int r0, void* msg, bool pack, bool msg_on_device) {
  const Blocks b = halo_blocks(c);
  // (below 2^31 words, so that the kernel's 32-bit word index cannot wrap)
  if (msg_on_device && halo_bytes(c) / 16 < ((size_t)1 << 31)) {
    ChunkSet cs{};
    cs.n = b.n;
    size_t first = 0;
    for (int k = 0; k < b.n; ++k) {
      const size_t width = (size_t)G * b.bytes_per_row[k];
      cs.off[k] = b.off[k] + (size_t)r0 * b.bytes_per_row[k];
      cs.stride[k] = b.stride[k];
      cs.words[k] = (uint32_t)(width / 16);
      cs.first[k] = (uint32_t)first;
      first += (size_t)b.planes[k] * cs.words[k];
    }
    cs.total = (uint32_t)first;
    if (((uintptr_t)msg & 15) != 0) return fail(TFKT_EINVAL, "device message not 16-byte aligned");
    // a grid-stride loop: eight 256-thread blocks per SM of the 152 fill the GPU
    const int blocks = (int)std::min<size_t>((first + 255) / 256, (size_t)152 * 8);
    halo_copy_kernel<<<blocks, 256, 0, c->stream>>>((int4*)c->ws.base, (int4*)msg, cs, pack ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      c->poisoned = true;
      return fail(TFKT_ECUDA, std::string("halo copy: ") + cudaGetErrorString(e));
    }
    return TFKT_OK;
  }
  char* ws = (char*)c->ws.base;
  char* m = (char*)msg;
  const cudaMemcpyKind kind = msg_on_device ? cudaMemcpyDeviceToDevice
                                            : (pack ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  for (int k = 0; k < b.n; ++k) {
    const size_t width = (size_t)G * b.bytes_per_row[k];
    char* plane0 = ws + b.off[k] + (size_t)r0 * b.bytes_per_row[k];
    cudaError_t e = pack ? cudaMemcpy2DAsync(m, width, plane0, b.stride[k], width, b.planes[k], kind,
                                             c->stream)
                         : cudaMemcpy2DAsync(plane0, b.stride[k], m, width, width, b.planes[k], kind,
                                             c->stream);
    if (e != cudaSuccess) {
      c->poisoned = true;
      return fail(TFKT_ECUDA, std::string("halo copy: ") + cudaGetErrorString(e));
    }
    m += width * b.planes[k];
  }
  if (!msg_on_device) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      c->poisoned = true;
      return fail(TFKT_ECUDA, std::string("halo copy: ") + cudaGetErrorString(e));
    }
  }
  return TFKT_OK;
}

}  // namespace
}  // namespace tfkt

using namespace tfkt;

extern "C" {

tfkt_status tfkt_slab_required_bytes(const tfkt_params* p, int32_t ny_local, size_t* bytes) {
  if (!bytes) return fail(TFKT_EINVAL, "bytes is NULL");
  Lattice L;
  tfkt_status s = slab_lattice(p, 0, ny_local, &L);
  if (s != TFKT_OK) return s;
  *bytes = ctx_layout(L);
  return TFKT_OK;
}

tfkt_status tfkt_slab_create(const tfkt_params* p, int32_t y0, int32_t ny_local,
                             const double* perturb, void* dev_workspace, size_t workspace_bytes,
                             void* stream, tfkt_ctx** out) {
  NvtxRange nvtx_range("tfkt_slab_create");
  if (!out) return fail(TFKT_EINVAL, "out is NULL");
  *out = nullptr;
  Lattice L;
  tfkt_status s = slab_lattice(p, y0, ny_local, &L);
  if (s != TFKT_OK) return s;
  s = ctx_create(L, perturb, dev_workspace, workspace_bytes, stream, out);
  if (s != TFKT_OK) return s;
  Ctx* c = ctx_of(*out);
  c->slab_y0 = y0;
  c->slab_ny = ny_local;
  return TFKT_OK;
}

tfkt_status tfkt_slab_halo_bytes(const tfkt_ctx* cc, size_t* bytes) {
  if (!cc || !bytes) return fail(TFKT_EINVAL, "NULL argument");
  const Ctx* c = ctx_of(const_cast<tfkt_ctx*>(cc));
  if (c->slab_ny == 0) return fail(TFKT_EINVAL, "not a slab context");
  *bytes = halo_bytes(c);
  return TFKT_OK;
}

tfkt_status tfkt_slab_halo_pack(tfkt_ctx* cc, int32_t side, void* dst, size_t bytes,
                                int dst_is_device) {
  NvtxRange nvtx_range("tfkt_slab_halo_pack");
  Ctx* c = ctx_of(cc);
  tfkt_status s = check_slab(c, side, dst, bytes);
  if (s != TFKT_OK) return s;
  // the moment planes travel with the populations; a context that recomputes them
  // each step (two-pass path) forms them now from its current state
  if (!c->m_valid) {
    s = ctx_ensure_moments(c);
    if (s != TFKT_OK) return s;
  }
  const int r0 = side == TFKT_SLAB_LOW ? G : c->slab_ny;
  return move_rows(c, r0, dst, true, dst_is_device != 0);
}

tfkt_status tfkt_slab_halo_unpack(tfkt_ctx* cc, int32_t side, const void* src, size_t bytes,
                                  int src_is_device) {
  NvtxRange nvtx_range("tfkt_slab_halo_unpack");
  Ctx* c = ctx_of(cc);
  tfkt_status s = check_slab(c, side, src, bytes);
  if (s != TFKT_OK) return s;
  const int r0 = side == TFKT_SLAB_LOW ? 0 : c->slab_ny + G;
  return move_rows(c, r0, const_cast<void*>(src), false, src_is_device != 0);
}

tfkt_status tfkt_slab_rows(const tfkt_ctx* cc, int32_t* y0, int32_t* ny_local, int32_t* ghost) {
  if (!cc) return fail(TFKT_EINVAL, "context is NULL");
  const Ctx* c = ctx_of(const_cast<tfkt_ctx*>(cc));
  if (c->slab_ny == 0) return fail(TFKT_EINVAL, "not a slab context");
  if (y0) *y0 = c->slab_y0;
  if (ny_local) *ny_local = c->slab_ny;
  if (ghost) *ghost = G;
  return TFKT_OK;
}

}  // extern "C"
