// Checkpoint and restart of a context (tfkt_save / tfkt_load).
//
// The paper's runs are long (Sec. VII follows the flow to 2000 convective
// times); a checkpoint lets such a run stop and resume. A file holds a fixed
// header (magic, version, the derived lattice parameters that fix the meaning
// of the state, the step count, the payload sizes and a checksum), then the
// raw current population buffer (9 + 25 nq planes of the storage type, row
// pitch included, and under FP16 storage the FP32 solvent planes after them) and, when they are valid, the current moment planes (the
// fused path carries them from step to step). Resuming from the file gives
// the same trajectory bit for bit as the run that was never stopped.
//
// Layout: little-endian, the header written field by field with fixed-width
// types (no struct padding in the file).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"

namespace tfkt {
namespace {

constexpr char kMagic[8] = {'T', 'F', 'K', 'T', 'C', 'K', 'P', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kChunk = (size_t)64 << 20;   // staging buffer (pinned host memory)

// 64-bit hash: four interleaved multiply-xor lanes over 8-byte words (fast
// enough for tens of GB), folded at the end; the same sequence of add() calls
// gives the same value.
struct Hash {
  uint64_t lane[4] = {0x9E3779B97F4A7C15ull, 0xC2B2AE3D27D4EB4Full, 0x165667B19E3779F9ull,
                      0x27D4EB2F165667C5ull};
  uint64_t count = 0;
  void add(const unsigned char* p, size_t n) {
    size_t k = 0;
    for (; k + 8 <= n; k += 8) {
      uint64_t w;
      std::memcpy(&w, p + k, 8);
      uint64_t& h = lane[(count >> 3) & 3];
      h = (h ^ w) * 0x100000001B3ull;
      h ^= h >> 29;
      count += 8;
    }
    for (; k < n; ++k) {
      uint64_t& h = lane[count & 3];
      h = (h ^ p[k]) * 0x100000001B3ull;
      ++count;
    }
  }
  uint64_t value() const {
    uint64_t h = count;
    for (uint64_t l : lane) h = (h ^ l) * 0x9E3779B97F4A7C15ull, h ^= h >> 31;
    return h;
  }
};

// The parameters that give the stored numbers their meaning.
struct Key {
  int32_t ints[9];
  uint64_t sizes[2];
  double reals[12];
};

Key key_of(const Lattice& L) {
  Key k{};
  const int32_t ints[9] = {L.nx, L.ny, L.S, L.nq, L.precision, L.qe_model, L.ic_mode, L.npl, L.nm};
  std::memcpy(k.ints, ints, sizeof ints);
  k.sizes[0] = L.pitch;
  k.sizes[1] = L.plane;
  const double reals[12] = {L.q_radius, L.tau1, L.tau2, L.tau_m, L.H,  L.kappa,
                            L.ell,      L.psi_tot, L.a0, L.kf,   L.u0, L.fene_b};
  std::memcpy(k.reals, reals, sizeof reals);
  return k;
}

bool same_key(const Key& a, const Key& b) {
  return std::memcmp(a.ints, b.ints, sizeof a.ints) == 0 &&
         std::memcmp(a.sizes, b.sizes, sizeof a.sizes) == 0 &&
         std::memcmp(a.reals, b.reals, sizeof a.reals) == 0;   // bit for bit
}

struct Header {
  char magic[8];
  uint32_t version;
  Key key;
  int64_t step;
  int32_t has_m;
  uint64_t pop_bytes, m_bytes, checksum;
};

// Fixed-width field I/O (the header is written member by member).
template <typename T>
bool put(std::FILE* f, const T& v) {
  return std::fwrite(&v, sizeof v, 1, f) == 1;
}
template <typename T>
bool get(std::FILE* f, T& v) {
  return std::fread(&v, sizeof v, 1, f) == 1;
}

bool write_header(std::FILE* f, const Header& hd) {
  bool ok = std::fwrite(hd.magic, 1, 8, f) == 8 && put(f, hd.version);
  for (int32_t v : hd.key.ints) ok = ok && put(f, v);
  for (uint64_t v : hd.key.sizes) ok = ok && put(f, v);
  for (double v : hd.key.reals) ok = ok && put(f, v);
  return ok && put(f, hd.step) && put(f, hd.has_m) && put(f, hd.pop_bytes) && put(f, hd.m_bytes) &&
         put(f, hd.checksum);
}

bool read_header(std::FILE* f, Header& hd) {
  bool ok = std::fread(hd.magic, 1, 8, f) == 8 && get(f, hd.version);
  for (int32_t& v : hd.key.ints) ok = ok && get(f, v);
  for (uint64_t& v : hd.key.sizes) ok = ok && get(f, v);
  for (double& v : hd.key.reals) ok = ok && get(f, v);
  return ok && get(f, hd.step) && get(f, hd.has_m) && get(f, hd.pop_bytes) && get(f, hd.m_bytes) &&
         get(f, hd.checksum);
}

// The checksum covers the payload and then every header field but itself.
uint64_t checksum(Hash h, const Header& hd) {
  h.add((const unsigned char*)hd.magic, 8);
  h.add((const unsigned char*)&hd.version, sizeof hd.version);
  h.add((const unsigned char*)hd.key.ints, sizeof hd.key.ints);
  h.add((const unsigned char*)hd.key.sizes, sizeof hd.key.sizes);
  h.add((const unsigned char*)hd.key.reals, sizeof hd.key.reals);
  h.add((const unsigned char*)&hd.step, sizeof hd.step);
  h.add((const unsigned char*)&hd.has_m, sizeof hd.has_m);
  h.add((const unsigned char*)&hd.pop_bytes, sizeof hd.pop_bytes);
  h.add((const unsigned char*)&hd.m_bytes, sizeof hd.m_bytes);
  return h.value();
}

tfkt_status cuda_error(Ctx* c, cudaError_t e, const char* where) {
  c->poisoned = true;
  return fail(TFKT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

struct File {
  std::FILE* f = nullptr;
  std::string remove_on_exit;   // a partly written file
  ~File() {
    if (f) std::fclose(f);
    if (!remove_on_exit.empty()) std::remove(remove_on_exit.c_str());
  }
};

size_t pop_bytes(const Lattice& L) { return population_bytes(L); }
size_t m_bytes(const Lattice& L) { return (size_t)L.nm * L.plane * real_size(L); }
char* pop_ptr(Ctx* c) { return (char*)c->ws.base + c->ws.off_pop[c->cur]; }
char* m_ptr(Ctx* c) { return (char*)c->ws.base + (c->mcur ? c->ws.off_M2 : c->ws.off_M); }

}  // namespace
}  // namespace tfkt

using namespace tfkt;

extern "C" {

tfkt_status tfkt_save(tfkt_ctx* ctx, const char* path) {
  NvtxRange nvtx_range("tfkt_save");
  if (!ctx || !path) return fail(TFKT_EINVAL, "NULL context or path");
  Ctx* c = ctx_of(ctx);
  if (c->poisoned) return fail(TFKT_ESTATE, "context poisoned by an earlier CUDA error");
  if (c->lpm_pending) {   // a learned block's pending increment is applied first
    tfkt_status s = ctx_lpm_flush(c);
    if (s != TFKT_OK) return s;
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_error(c, e, "save: synchronise");
  const Lattice& L = c->L;
  Header hd{};
  std::memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.key = key_of(L);
  hd.step = c->step;
  hd.has_m = c->m_valid ? 1 : 0;
  hd.pop_bytes = pop_bytes(L);
  hd.m_bytes = hd.has_m ? m_bytes(L) : 0;
  hd.checksum = 0;
  const std::string tmp = std::string(path) + ".part";
  File f;
  f.f = std::fopen(tmp.c_str(), "wb");
  if (!f.f) return fail(TFKT_EIO, std::string("cannot open ") + tmp + " for writing");
  f.remove_on_exit = tmp;
  if (!write_header(f.f, hd)) return fail(TFKT_EIO, "header write failed");
  Pinned stage;
  e = cudaMallocHost(&stage.p, kChunk);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TFKT_ENOMEM, "pinned staging buffer");
  }
  Hash hash;
  auto copy_out = [&](const char* dev, size_t bytes) -> tfkt_status {
    for (size_t o = 0; o < bytes; o += kChunk) {
      const size_t n = std::min(kChunk, bytes - o);
      cudaError_t e2 = cudaMemcpyAsync(stage.p, dev + o, n, cudaMemcpyDeviceToHost, c->stream);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
      if (e2 != cudaSuccess) return cuda_error(c, e2, "save: copy");
      hash.add((const unsigned char*)stage.p, n);
      if (std::fwrite(stage.p, 1, n, f.f) != n) return fail(TFKT_EIO, "payload write failed");
    }
    return TFKT_OK;
  };
  tfkt_status s = copy_out(pop_ptr(c), hd.pop_bytes);
  if (s == TFKT_OK && hd.has_m) s = copy_out(m_ptr(c), hd.m_bytes);
  if (s != TFKT_OK) return s;
  // the checksum is the header's last field
  hd.checksum = checksum(hash, hd);
  if (std::fseek(f.f, 0, SEEK_SET) != 0 || !write_header(f.f, hd))
    return fail(TFKT_EIO, "header rewrite failed");
  const int closed = std::fclose(f.f);
  f.f = nullptr;
  if (closed != 0) return fail(TFKT_EIO, "close failed");
  if (std::rename(tmp.c_str(), path) != 0) return fail(TFKT_EIO, std::string("cannot rename to ") + path);
  f.remove_on_exit.clear();
  return TFKT_OK;
}

tfkt_status tfkt_load(tfkt_ctx* ctx, const char* path) {
  NvtxRange nvtx_range("tfkt_load");
  if (!ctx || !path) return fail(TFKT_EINVAL, "NULL context or path");
  Ctx* c = ctx_of(ctx);
  if (c->poisoned) return fail(TFKT_ESTATE, "context poisoned by an earlier CUDA error");
  if (c->in_batch) return fail(TFKT_EINVAL, "load into a standalone context, not a run of a batch");
  const Lattice& L = c->L;
  File f;
  f.f = std::fopen(path, "rb");
  if (!f.f) return fail(TFKT_EIO, std::string("cannot open ") + path);
  Header hd{};
  if (!read_header(f.f, hd)) return fail(TFKT_EIO, "truncated header");
  if (std::memcmp(hd.magic, kMagic, 8) != 0) return fail(TFKT_EIO, "not a checkpoint file");
  if (hd.version != kVersion) return fail(TFKT_EIO, "unsupported checkpoint version");
  if (!same_key(hd.key, key_of(L)))
    return fail(TFKT_EINVAL, "checkpoint was written for other parameters");
  if (hd.pop_bytes != pop_bytes(L) || (hd.has_m != 0 && hd.has_m != 1) ||
      hd.m_bytes != (hd.has_m ? m_bytes(L) : 0) || hd.step < 0)
    return fail(TFKT_EIO, "inconsistent checkpoint header");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_error(c, e, "load: synchronise");
  Pinned stage;
  e = cudaMallocHost(&stage.p, kChunk);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TFKT_ENOMEM, "pinned staging buffer");
  }
  // From here the device state is being overwritten: a failure resets the
  // context to its initial state (no perturbation).
  auto reset = [&](tfkt_status s, const std::string& msg) {
    std::string m = msg;
    if (ctx_reinit(c, nullptr) != TFKT_OK) return fail(TFKT_ECUDA, m + "; reset failed");
    return fail(s, m + "; the context was reset to its initial state");
  };
  Hash hash;
  auto copy_in = [&](char* dev, size_t bytes) -> bool {
    for (size_t o = 0; o < bytes; o += kChunk) {
      const size_t n = std::min(kChunk, bytes - o);
      if (std::fread(stage.p, 1, n, f.f) != n) return false;
      hash.add((const unsigned char*)stage.p, n);
      cudaError_t e2 = cudaMemcpyAsync(dev + o, stage.p, n, cudaMemcpyHostToDevice, c->stream);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
      if (e2 != cudaSuccess) {
        cuda_error(c, e2, "load: copy");
        return false;
      }
    }
    return true;
  };
  c->lpm_pending = false;
  c->lpm_step = -1;
  bool ok = copy_in(pop_ptr(c), hd.pop_bytes);
  if (ok && hd.has_m) ok = copy_in(m_ptr(c), hd.m_bytes);
  if (c->poisoned) return fail(TFKT_ECUDA, "load: copy failed; context poisoned");
  if (!ok) return reset(TFKT_EIO, "truncated checkpoint payload");
  unsigned char extra;
  if (std::fread(&extra, 1, 1, f.f) != 0) return reset(TFKT_EIO, "trailing bytes after the payload");
  if (checksum(hash, hd) != hd.checksum) return reset(TFKT_EIO, "checksum mismatch");
  c->step = hd.step;
  c->m_valid = hd.has_m != 0;
  return TFKT_OK;
}

}  // extern "C"
