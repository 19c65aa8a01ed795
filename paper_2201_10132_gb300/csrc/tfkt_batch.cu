// Batched ensembles: independent runs advanced together, two steps at a time
// replayed from a CUDA graph, in one of two plans: one launch of the batched
// fused kernel (and one of its border fix-up) over the tiles of all runs, at
// a tile height of 4, 8 or 16 rows of 32 nodes; or every run's own single-run
// kernels as parallel branches of the graph, largest runs first. The plan is
// chosen by timing each candidate on the batch itself before the runs are
// initialised.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"

struct tfkt_batch {
  std::vector<tfkt_ctx*> runs;
  void* ws = nullptr;
  bool owned = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  tfkt::BatchRun<float>* d_runs = nullptr;  // in the workspace
  int* d_tile_start = nullptr;             // in the workspace, n + 1 entries
  int total_tiles = 0, max_nq = 0;
  int parity = 0;                          // buffer parity shared by all runs
  cudaGraphExec_t graph = nullptr;         // two steps: parity 0 then 1
  int64_t step = 0;
  int ty = tfkt::TY;                       // tile height of the launch
  float tune_ms[4] = {NAN, NAN, NAN, NAN}; // timed ms per step: heights 4, 8, 16, per-run plan
  std::vector<tfkt::BatchRun<float>> host; // launch tables of the chosen height
  bool per_run = false;                    // the per-run plan
  std::vector<cudaStream_t> pool;          // its graph branches
  std::vector<cudaEvent_t> join;           // one per branch
  cudaEvent_t fork = nullptr;
  std::vector<int> order;                  // runs, largest first
};

namespace tfkt {
namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

tfkt_status check_runs(const tfkt_params* runs, int32_t n, std::vector<Lattice>& L) {
  if (!runs || n < 1) return fail(TFKT_EINVAL, "a batch needs at least one run");
  L.resize(n);
  for (int32_t i = 0; i < n; ++i) {
    tfkt_status s = map_params(&runs[i], &L[i]);
    if (s != TFKT_OK) return s;
    if (runs[i].precision != TFKT_FP32) return fail(TFKT_EINVAL, "batched runs must use TFKT_FP32");
    if (runs[i].qe_model != TFKT_QE_MOMENTUM)
      return fail(TFKT_EINVAL, "batched runs use the momentum quasi-equilibrium");
    // Every run must take the single-run fused path (8-row tiles): its context
    // then holds the export ring, the second moment buffer and the fused tables
    // that the batch kernels use at any tile height.
    if (!fused_supported(L[i].nx, L[i].ny, L[i].nq, 4, 8))
      return fail(TFKT_EINVAL, "batched runs need nx % 32 == 0 and ny % 8 == 0 (run " +
                                   std::to_string(i) + ")");
  }
  return TFKT_OK;
}

// Workspace: the runs' workspaces one after another, then the launch tables.
size_t batch_layout(const std::vector<Lattice>& L, std::vector<size_t>& off, size_t* off_tab) {
  size_t o = 0;
  off.resize(L.size());
  for (size_t i = 0; i < L.size(); ++i) {
    off[i] = o;
    o = align256(o + ctx_layout(L[i]));
  }
  *off_tab = o;
  o = align256(o + L.size() * sizeof(BatchRun<float>));
  o = align256(o + (L.size() + 1) * sizeof(int));
  return o;
}

void release(tfkt_batch* b) {
  for (tfkt_ctx* c : b->runs)
    if (c) tfkt_destroy(c);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->owned && b->ws) cudaFree(b->ws);
  for (cudaStream_t p : b->pool) cudaStreamDestroy(p);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// The per-run plan: fork from s onto the branch streams, each run's fused step
// and fix-up on branch (position in `order`) mod branches, join back into s.
// Inside a stream capture this records parallel graph branches.
cudaError_t launch_per_run(tfkt_batch* b, int parity, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (size_t k = 0; k < b->pool.size() && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->pool[k], b->fork, 0);
  for (size_t j = 0; j < b->order.size() && e == cudaSuccess; ++j) {
    const int i = b->order[j];
    e = launch_single_fp32(b->host[i].a[parity], b->host[i].f[parity], b->pool[j % b->pool.size()]);
  }
  for (size_t k = 0; k < b->pool.size() && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->pool[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[k], 0);
  }
  return e;
}

// One step of the chosen plan at buffer parity `parity` on stream s.
cudaError_t launch_plan(tfkt_batch* b, int parity, cudaStream_t s) {
  if (b->per_run) return launch_per_run(b, parity, s);
  return launch_batch_step(b->d_runs, b->d_tile_start, (int)b->runs.size(), b->total_tiles,
                           b->max_nq, parity, s, b->ty);
}

// Two steps (parity 0 then 1) of the chosen plan as an instantiated graph.
cudaError_t capture(tfkt_batch* b, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = launch_plan(b, 0, b->stream);
  if (e1 == cudaSuccess) e1 = launch_plan(b, 1, b->stream);
  e = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e1;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

tfkt_status plain_step(tfkt_batch* b) {
  cudaError_t e = launch_plan(b, b->parity, b->stream);
  if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("batch step: ") + cudaGetErrorString(e));
  b->parity ^= 1;
  return TFKT_OK;
}

// Launch tables (ntx, nty per run, prefix sums of the tile counts) for tile height ty.
cudaError_t set_tables(tfkt_batch* b, const std::vector<Lattice>& L, int ty) {
  const int n = (int)b->runs.size();
  std::vector<int> tile_start(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    b->host[i].ntx = L[i].nx / TX;
    b->host[i].nty = L[i].ny / ty;
    tile_start[i + 1] = tile_start[i] + b->host[i].ntx * b->host[i].nty;
  }
  b->total_tiles = tile_start[n];
  b->ty = ty;
  cudaError_t e = cudaMemcpyAsync(b->d_runs, b->host.data(), n * sizeof(BatchRun<float>),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tile_start, tile_start.data(), (n + 1) * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = prepare_batch(b->max_nq, ty);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // host tables are pageable
  return e;
}

// Tile heights every run supports (the grid divides, the tile's shared memory fits).
std::vector<int> candidates(const std::vector<Lattice>& L) {
  std::vector<int> out;
  for (int ty : {4, 8, 16}) {
    bool ok = true;
    for (const Lattice& l : L) ok = ok && fused_supported(l.nx, l.ny, l.nq, 4, ty);
    if (ok) out.push_back(ty);
  }
  return out;
}

// Time each candidate plan on the current states (the runs are initialised
// afterwards, so the states timed here are thrown away): the batched kernel at
// every tile height all runs admit, and the per-run plan; each as its captured
// two-step graph, launched once to warm up and then twice (four steps) between
// events. Keep the fastest. TFKT_BATCH_PER_RUN=1 fixes the per-run plan and
// TFKT_BATCH_TILE_HEIGHT (4, 8 or 16) the batched kernel at that height instead.
tfkt_status autotune(tfkt_batch* b, const std::vector<Lattice>& L) {
  const std::vector<int> cand = candidates(L);
  const char* env_runs = std::getenv("TFKT_BATCH_PER_RUN");
  const char* env = std::getenv("TFKT_BATCH_TILE_HEIGHT");
  const bool force_runs = env_runs && std::atoi(env_runs) == 1;
  const int forced = env ? std::atoi(env) : 0;
  auto use = [&](int ty) -> cudaError_t {   // ty 0: the per-run plan
    b->per_run = ty == 0;
    return set_tables(b, L, ty == 0 ? TY : ty);
  };
  if (force_runs || forced) {
    int pick = -1;
    if (force_runs) pick = 0;
    for (int ty : cand)
      if (!force_runs && ty == forced) pick = ty;
    if (pick < 0) return fail(TFKT_EINVAL, "TFKT_BATCH_TILE_HEIGHT names a height these runs do not support");
    cudaError_t e = use(pick);
    if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("batch tables: ") + cudaGetErrorString(e));
    return TFKT_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(TFKT_ECUDA, "cudaEventCreate");
  }
  std::vector<int> plans(cand);
  plans.push_back(0);
  int best = -1;
  float best_ms = std::numeric_limits<float>::infinity();
  cudaError_t e = cudaSuccess;
  for (int ty : plans) {
    e = use(ty);
    if (e != cudaSuccess) break;
    cudaGraphExec_t g = nullptr;
    e = capture(b, &g);
    if (e == cudaSuccess) e = cudaGraphLaunch(g, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaGraphLaunch(g, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (g) cudaGraphExecDestroy(g);
    if (e != cudaSuccess) break;
    ms /= 4;
    b->tune_ms[ty == 0 ? 3 : (ty == 4 ? 0 : (ty == 8 ? 1 : 2))] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = ty;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess && best >= 0) e = use(best);
  if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
  b->parity = 0;
  return TFKT_OK;
}

}  // namespace
}  // namespace tfkt

using namespace tfkt;

extern "C" {

tfkt_status tfkt_batch_required_bytes(const tfkt_params* runs, int32_t n, size_t* bytes) {
  if (!bytes) return fail(TFKT_EINVAL, "bytes is NULL");
  std::vector<Lattice> L;
  tfkt_status s = check_runs(runs, n, L);
  if (s != TFKT_OK) return s;
  std::vector<size_t> off;
  size_t tab;
  *bytes = batch_layout(L, off, &tab);
  return TFKT_OK;
}

tfkt_status tfkt_batch_create(const tfkt_params* runs, int32_t n, const double* const* perturbs,
                              void* dev_workspace, size_t workspace_bytes, void* stream,
                              tfkt_batch** out) {
  NvtxRange nvtx_range("tfkt_batch_create");
  if (!out) return fail(TFKT_EINVAL, "out is NULL");
  *out = nullptr;
  std::vector<Lattice> L;
  tfkt_status s = check_runs(runs, n, L);
  if (s != TFKT_OK) return s;
  std::vector<size_t> off;
  size_t off_tab;
  const size_t need = batch_layout(L, off, &off_tab);
  tfkt_batch* b = new (std::nothrow) tfkt_batch();
  if (!b) return fail(TFKT_ENOMEM, "host allocation failed");
  if (dev_workspace) {
    if (workspace_bytes < need || ((uintptr_t)dev_workspace) % 256) {
      delete b;
      return fail(TFKT_ENOMEM, "workspace too small or not 256-byte aligned: need " +
                                   std::to_string(need) + " bytes");
    }
    b->ws = dev_workspace;
  } else {
    cudaError_t e = cudaMalloc(&b->ws, need);
    if (e != cudaSuccess) {
      delete b;
      cudaGetLastError();
      return fail(TFKT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->owned = true;
  }
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      release(b);
      return fail(TFKT_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  b->host.resize(n);
  for (int32_t i = 0; i < n; ++i) {
    tfkt_ctx* c = nullptr;
    // rest state first: the tile-height timing below runs on it
    s = tfkt_create(&runs[i], nullptr, (char*)b->ws + off[i], ctx_layout(L[i]), b->stream, &c);
    if (s != TFKT_OK) {
      release(b);
      return s;
    }
    b->runs.push_back(c);
    Ctx* x = ctx_of(c);
    x->in_batch = true;
    for (int p = 0; p < 2; ++p) {
      x->cur = x->mcur = p;
      b->host[i].a[p] = ctx_args<float>(x);
      b->host[i].f[p] = ctx_fused<float>(x);
    }
    x->cur = x->mcur = 0;
    if (L[i].nq > b->max_nq) b->max_nq = L[i].nq;
  }
  b->d_runs = (BatchRun<float>*)((char*)b->ws + off_tab);
  b->d_tile_start = (int*)((char*)b->ws + align256(off_tab + n * sizeof(BatchRun<float>)));
  // the per-run plan's branches (up to 32) and its order, largest runs first
  for (int32_t i = 0; i < n; ++i) b->order.push_back(i);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int u, int v) {
    return (size_t)L[u].nx * L[u].ny > (size_t)L[v].nx * L[v].ny;
  });
  const int nbranch = n < 32 ? n : 32;
  cudaError_t ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < nbranch && ce == cudaSuccess; ++k) {
    cudaStream_t ps = nullptr;
    cudaEvent_t je = nullptr;
    ce = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (ce == cudaSuccess) b->pool.push_back(ps);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&je, cudaEventDisableTiming);
    if (ce == cudaSuccess) b->join.push_back(je);
  }
  if (ce == cudaSuccess) ce = prepare_single_fp32(b->max_nq);
  if (ce != cudaSuccess) {
    release(b);
    return fail(TFKT_ECUDA, std::string("batch streams: ") + cudaGetErrorString(ce));
  }
  if ((s = autotune(b, L)) != TFKT_OK) {
    release(b);
    return s;
  }
  // the runs' initial states (Sec. VI-D), now that the timing steps are done
  for (int32_t i = 0; i < n; ++i) {
    if ((s = ctx_reinit(ctx_of(b->runs[i]), perturbs ? perturbs[i] : nullptr)) != TFKT_OK) {
      release(b);
      return s;
    }
  }
  *out = b;
  return TFKT_OK;
}

tfkt_status tfkt_batch_step(tfkt_batch* b, int64_t n) {
  NvtxRange nvtx_range("tfkt_batch_step");
  if (!b) return fail(TFKT_EINVAL, "batch is NULL");
  if (n < 0) return fail(TFKT_EINVAL, "n must be >= 0");
  tfkt_status s = TFKT_OK;
  int64_t left = n;
  if (left > 0 && b->parity == 1) {
    s = plain_step(b);
    --left;
  }
  if (left >= 2 && !b->graph) {   // capture two steps (parity 0 then 1) once
    cudaError_t e = capture(b, &b->graph);
    if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
  }
  while (s == TFKT_OK && left >= 2) {
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    left -= 2;
  }
  if (s == TFKT_OK && left == 1) s = plain_step(b);
  if (s != TFKT_OK) return s;
  b->step += n;
  // keep every run's view of the state current
  for (tfkt_ctx* c : b->runs) {
    Ctx* x = ctx_of(c);
    x->cur = x->mcur = b->parity;
    x->step = b->step;
  }
  return TFKT_OK;
}

tfkt_status tfkt_batch_run(tfkt_batch* b, int32_t i, tfkt_ctx** run) {
  if (!b || !run || i < 0 || i >= (int32_t)b->runs.size())
    return fail(TFKT_EINVAL, "bad batch, run index or output pointer");
  *run = b->runs[i];
  return TFKT_OK;
}

tfkt_status tfkt_batch_tile_height(const tfkt_batch* b, int32_t* ty, float* ms) {
  if (!b || !ty) return fail(TFKT_EINVAL, "NULL argument");
  *ty = b->ty;
  if (ms)
    for (int k = 0; k < 3; ++k) ms[k] = b->tune_ms[k];
  return TFKT_OK;
}

tfkt_status tfkt_batch_plan(const tfkt_batch* b, int32_t* per_run, int32_t* ty, float* ms) {
  if (!b || !per_run || !ty) return fail(TFKT_EINVAL, "NULL argument");
  *per_run = b->per_run ? 1 : 0;
  *ty = b->ty;
  if (ms)
    for (int k = 0; k < 4; ++k) ms[k] = b->tune_ms[k];
  return TFKT_OK;
}

tfkt_status tfkt_batch_destroy(tfkt_batch* b) {
  if (!b) return TFKT_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  release(b);
  if (e != cudaSuccess) return fail(TFKT_ECUDA, std::string("destroy: ") + cudaGetErrorString(e));
  return TFKT_OK;
}

}  // extern "C"
