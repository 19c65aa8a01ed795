// The learned macro-step's network: forward pass, loss and gradient by
// backpropagation, and Adam, as hand-written kernels (bfloat16 matrices, FP32
// accumulation, on the tensor cores for the forward pass and for the weight
// gradients and propagated errors of the backward pass). Gradients are summed
// per block of 128 samples and the block partials in a fixed order, so results
// are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"
#include "tfkt_mlp.cuh"

namespace tfkt {
namespace {

constexpr int TB = 128;          // samples (threads) per training block

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Inference on raw samples: one warp per TC_ROWS samples, the network on the
// tensor cores (mlp_warp_tc).
__global__ void __launch_bounds__(128) forward_kernel(const float* __restrict__ master,
                                                      const __nv_bfloat16* __restrict__ wmat,
                                                      const float* __restrict__ X, int64_t n,
                                                      float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char fw_smem[];
  MlpTc& s = *reinterpret_cast<MlpTc*>(fw_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* Xw = reinterpret_cast<float*>(fw_smem + ((sizeof(MlpTc) + 15) & ~(size_t)15)) +
              (size_t)warp * TC_WARP_FLOATS;
  float* Ow = Xw + TC_ROWS * TC_XLD;
  mlp_stage_tc(s, master, wmat, threadIdx.x, blockDim.x);
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // warp-uniform pass
  const bool ok = k < n;
  float* xr = Xw + lane * TC_XLD;
#pragma unroll
  for (int i = 0; i < NIN; ++i) xr[i] = ok ? (X[k * NIN + i] - s.mx[i]) * s.rsx[i] : 0.f;
#pragma unroll
  for (int i = NIN; i < TC_K1; ++i) xr[i] = 0.f;
  __syncwarp();
  mlp_warp_tc(s, Xw, Ow, lane);
  __syncwarp();
  if (ok) {
#pragma unroll
    for (int j = 0; j < NOUT; ++j) Y[k * NOUT + j] = Ow[lane * 4 + j] * s.st[j] + s.mt[j];
  }
}

// ---- training: forward and backward on the tensor cores
// Per block TB = 128 samples (4 warps of 32). The forward pass is the inference
// routine's (standardised inputs and GELU activations as bfloat16 high part plus
// remainder, bfloat16 weights, FP32 accumulation), keeping pre-activations and
// activations per sample. Backward: the output layer, the bias sums and the
// GELU derivatives on the CUDA cores; the weight gradients dW2 = dz2^T h1 and
// dW1 = dz1^T x (sums over the block's samples) and the propagated error
// dz2 W2 as mma.sync, both FP32 operands split into high part and remainder
// (three products per pair: high x high, high x remainder, remainder x high).
constexpr int TR_LD = 68;   // FP32 row stride of the per-sample tables (float2-aligned)

struct TrainTc {
  MlpTc net;                         // forward weights ([out][in] bfloat16) and normalisation
  __nv_bfloat16 w2t[NH * TC_W2LD];   // W2 transposed ([in][out]) for the propagated error
  float xs[TB * TC_XLD];             // standardised inputs; columns NIN .. TC_K1 - 1 zero
  float z1[TB * TR_LD], h1[TB * TR_LD], z2[TB * TR_LD], h2[TB * TR_LD];
  float o[TB * 4], dO[TB * 4];
  double lsum[TB];
};

// Fragment pair (p, q) of an FP32 table split into bfloat16 high part and remainder.
__device__ __forceinline__ void tr_split2(const float* p, const float* q, uint32_t& hi, uint32_t& lo) {
  tc_split(*p, *q, hi, lo);
}

// Forward pass of the warp's 32 samples (rows wb .. wb + 31 of the tables).
__device__ __forceinline__ void train_forward_warp(TrainTc& sh, int wb, int lane) {
  const MlpTc& s = sh.net;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int m = 0; m < 2; ++m) {
    const int r0 = wb + 16 * m + g, r1 = r0 + 8;
    const float* x0 = sh.xs + r0 * TC_XLD;
    const float* x1 = sh.xs + r1 * TC_XLD;
    uint32_t ah1[3][4], al1[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c0 = 16 * k + 2 * t;
      tc_split(x0[c0], x0[c0 + 1], ah1[k][0], al1[k][0]);
      tc_split(x1[c0], x1[c0 + 1], ah1[k][1], al1[k][1]);
      tc_split(x0[c0 + 8], x0[c0 + 9], ah1[k][2], al1[k][2]);
      tc_split(x1[c0 + 8], x1[c0 + 9], ah1[k][3], al1[k][3]);
    }
    float c[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      c[n][0] = c[n][2] = s.b1[8 * n + 2 * t];
      c[n][1] = c[n][3] = s.b1[8 * n + 2 * t + 1];
    }
    tc_layer<3, 8, TC_W1LD>(c, ah1, al1, s.w1, g, t);
    uint32_t ah[4][4], al[4][4];
    // keep z1, h1; the next layer's operands from h1
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int col = 8 * n + 2 * t;
      float a[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = gelu(c[n][e]);
      sh.z1[r0 * TR_LD + col] = c[n][0];
      sh.z1[r0 * TR_LD + col + 1] = c[n][1];
      sh.z1[r1 * TR_LD + col] = c[n][2];
      sh.z1[r1 * TR_LD + col + 1] = c[n][3];
      sh.h1[r0 * TR_LD + col] = a[0];
      sh.h1[r0 * TR_LD + col + 1] = a[1];
      sh.h1[r1 * TR_LD + col] = a[2];
      sh.h1[r1 * TR_LD + col + 1] = a[3];
      const int k = n >> 1, half = (n & 1) * 2;
      tc_split(a[0], a[1], ah[k][half], al[k][half]);
      tc_split(a[2], a[3], ah[k][half + 1], al[k][half + 1]);
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      c[n][0] = c[n][2] = s.b2[8 * n + 2 * t];
      c[n][1] = c[n][3] = s.b2[8 * n + 2 * t + 1];
    }
    tc_layer<4, 8, TC_W2LD>(c, ah, al, s.w2, g, t);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int col = 8 * n + 2 * t;
      float a[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = gelu(c[n][e]);
      sh.z2[r0 * TR_LD + col] = c[n][0];
      sh.z2[r0 * TR_LD + col + 1] = c[n][1];
      sh.z2[r1 * TR_LD + col] = c[n][2];
      sh.z2[r1 * TR_LD + col + 1] = c[n][3];
      sh.h2[r0 * TR_LD + col] = a[0];
      sh.h2[r0 * TR_LD + col + 1] = a[1];
      sh.h2[r1 * TR_LD + col] = a[2];
      sh.h2[r1 * TR_LD + col + 1] = a[3];
      const int k = n >> 1, half = (n & 1) * 2;
      tc_split(a[0], a[1], ah[k][half], al[k][half]);
      tc_split(a[2], a[3], ah[k][half + 1], al[k][half + 1]);
    }
    float c3[1][4] = {{s.b3[2 * t], s.b3[2 * t + 1], s.b3[2 * t], s.b3[2 * t + 1]}};
    tc_layer<4, 1, TC_W2LD>(c3, ah, al, s.w3, g, t);
    if (2 * t < NOUT) {
      sh.o[r0 * 4 + 2 * t] = c3[0][0];
      sh.o[r1 * 4 + 2 * t] = c3[0][2];
    }
    if (2 * t + 1 < NOUT) {
      sh.o[r0 * 4 + 2 * t + 1] = c3[0][1];
      sh.o[r1 * 4 + 2 * t + 1] = c3[0][3];
    }
  }
}

// G[o][i] = sum over the block's TB samples s of D[s][o] B[s][i] for o in this
// warp's 16 rows (o0 ..) and i < ni (NN n-tiles of 8), written to P[o * ld + i].
template <int NN>
__device__ __forceinline__ void train_weight_grad(const float* D, const float* B, int bld, int o0,
                                                  int ni, float* P, int ld, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float c[NN][4];
#pragma unroll
  for (int n = 0; n < NN; ++n) c[n][0] = c[n][1] = c[n][2] = c[n][3] = 0.f;
#pragma unroll 1
  for (int k = 0; k < TB / 16; ++k) {
    const int s0 = 16 * k + 2 * t;
    uint32_t ah[4], al[4];
    tr_split2(D + s0 * TR_LD + o0 + g, D + (s0 + 1) * TR_LD + o0 + g, ah[0], al[0]);
    tr_split2(D + s0 * TR_LD + o0 + g + 8, D + (s0 + 1) * TR_LD + o0 + g + 8, ah[1], al[1]);
    tr_split2(D + (s0 + 8) * TR_LD + o0 + g, D + (s0 + 9) * TR_LD + o0 + g, ah[2], al[2]);
    tr_split2(D + (s0 + 8) * TR_LD + o0 + g + 8, D + (s0 + 9) * TR_LD + o0 + g + 8, ah[3], al[3]);
#pragma unroll
    for (int n = 0; n < NN; ++n) {
      const int i = 8 * n + g;
      uint32_t bh0, bl0, bh1, bl1;
      tr_split2(B + s0 * bld + i, B + (s0 + 1) * bld + i, bh0, bl0);
      tr_split2(B + (s0 + 8) * bld + i, B + (s0 + 9) * bld + i, bh1, bl1);
      tc_mma(c[n], ah, bh0, bh1);
      tc_mma(c[n], ah, bl0, bl1);
      tc_mma(c[n], al, bh0, bh1);
    }
  }
#pragma unroll
  for (int n = 0; n < NN; ++n) {
    const int i = 8 * n + 2 * t;
    if (i < ni) {
      P[(o0 + g) * ld + i] = c[n][0];
      P[(o0 + g + 8) * ld + i] = c[n][2];
    }
    if (i + 1 < ni) {
      P[(o0 + g) * ld + i + 1] = c[n][1];
      P[(o0 + g + 8) * ld + i + 1] = c[n][3];
    }
  }
}

// Loss and gradient partials of one block of TB samples; partial[b][NWEIGHTS].
__global__ void __launch_bounds__(TB) loss_grad_kernel(const float* __restrict__ master,
                                                       const __nv_bfloat16* __restrict__ wmat,
                                                       const float* __restrict__ X,
                                                       const float* __restrict__ T, int64_t n,
                                                       float* __restrict__ partial,
                                                       double* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainTc& sh = *reinterpret_cast<TrainTc*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  mlp_stage_tc(sh.net, master, wmat, tid, TB);
  for (int k = tid; k < NH * TC_W2LD; k += TB) {
    const int i = k / TC_W2LD, o = k % TC_W2LD;
    sh.w2t[k] = o < NH ? wmat[NH * NIN + o * NH + i] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  const MlpTc& s = sh.net;
  const int64_t k = (int64_t)blockIdx.x * TB + tid;
  const bool valid = k < n;
  const float inv_n = 1.0f / (float)n;
  // ---- forward, keeping what the backward pass needs
  float* xs = sh.xs + tid * TC_XLD;
#pragma unroll
  for (int i = 0; i < NIN; ++i) xs[i] = valid ? (X[k * NIN + i] - s.mx[i]) * s.rsx[i] : 0.0f;
#pragma unroll
  for (int i = NIN; i < TC_XLD; ++i) xs[i] = 0.0f;
  __syncwarp();
  train_forward_warp(sh, warp * 32, lane);
  __syncwarp();
  double lsq = 0.0;
  for (int j = 0; j < NOUT; ++j) {
    float d = 0.0f;
    if (valid) {
      const float tj = (T[k * NOUT + j] - s.mt[j]) / s.st[j];
      const float r = sh.o[tid * 4 + j] - tj;
      lsq += (double)r * (double)r;
      d = 2.0f * r * inv_n;
    }
    sh.dO[tid * 4 + j] = d;
  }
  sh.lsum[tid] = lsq;
  __syncthreads();
  float* P = partial + (size_t)blockIdx.x * TFKT_MLP_NWEIGHTS;
  // ---- output layer: dW3 = sum_s dO h2^T, db3 = sum_s dO (invalid samples carry dO = 0)
  for (int e = tid; e < NOUT * NH + NOUT; e += TB) {
    float acc = 0.0f;
    if (e < NOUT * NH) {
      const int j = e / NH, i = e % NH;
      for (int r = 0; r < TB; ++r) acc = fmaf(sh.dO[r * 4 + j], sh.h2[r * TR_LD + i], acc);
      P[OW3 + e] = acc;
    } else {
      const int j = e - NOUT * NH;
      for (int r = 0; r < TB; ++r) acc += sh.dO[r * 4 + j];
      P[OB3 + j] = acc;
    }
  }
  // ---- dz2 = (W3^T dO) GELU'(z2) for this thread's sample, in place of z2
  for (int o = 0; o < NH; ++o) {
    float acc = 0.0f;
    for (int j = 0; j < NOUT; ++j)
      acc = fmaf(__bfloat162float(s.w3[j * TC_W2LD + o]), sh.dO[tid * 4 + j], acc);
    sh.z2[tid * TR_LD + o] = acc * gelu_grad(sh.z2[tid * TR_LD + o]);
  }
  __syncthreads();
  // ---- layer 2: dW2 = dz2^T h1 (warp: 16 output rows), db2 = sum_s dz2
  train_weight_grad<8>(sh.z2, sh.h1, TR_LD, 16 * warp, NH, P + OW2, NH, lane);
  if (tid < NH) {
    float acc = 0.0f;
    for (int r = 0; r < TB; ++r) acc += sh.z2[r * TR_LD + tid];
    P[OB2 + tid] = acc;
  }
  // ---- dz1 = (dz2 W2) GELU'(z1) for the warp's 32 samples, in place of z1
  {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int m = 0; m < 2; ++m) {
      const int r0 = warp * 32 + 16 * m + g, r1 = r0 + 8;
      uint32_t ah[4][4], al[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t;
        const float* d0 = sh.z2 + r0 * TR_LD;
        const float* d1 = sh.z2 + r1 * TR_LD;
        tc_split(d0[c0], d0[c0 + 1], ah[kk][0], al[kk][0]);
        tc_split(d1[c0], d1[c0 + 1], ah[kk][1], al[kk][1]);
        tc_split(d0[c0 + 8], d0[c0 + 9], ah[kk][2], al[kk][2]);
        tc_split(d1[c0 + 8], d1[c0 + 9], ah[kk][3], al[kk][3]);
      }
      float c[8][4];
#pragma unroll
      for (int nn = 0; nn < 8; ++nn) c[nn][0] = c[nn][1] = c[nn][2] = c[nn][3] = 0.f;
      tc_layer<4, 8, TC_W2LD>(c, ah, al, sh.w2t, g, t);
#pragma unroll
      for (int nn = 0; nn < 8; ++nn) {
        const int col = 8 * nn + 2 * t;
        float* z0 = sh.z1 + r0 * TR_LD + col;
        float* z1r = sh.z1 + r1 * TR_LD + col;
        z0[0] = c[nn][0] * gelu_grad(z0[0]);
        z0[1] = c[nn][1] * gelu_grad(z0[1]);
        z1r[0] = c[nn][2] * gelu_grad(z1r[0]);
        z1r[1] = c[nn][3] * gelu_grad(z1r[1]);
      }
    }
  }
  __syncthreads();
  // ---- layer 1: dW1 = dz1^T x (warp: 16 output rows, inputs padded to 48), db1 = sum_s dz1
  train_weight_grad<6>(sh.z1, sh.xs, TC_XLD, 16 * warp, NIN, P + OW1, NIN, lane);
  if (tid < NH) {
    float acc = 0.0f;
    for (int r = 0; r < TB; ++r) acc += sh.z1[r * TR_LD + tid];
    P[OB1 + tid] = acc;
  }
  if (tid == 0) {
    double l = 0.0;
    for (int r = 0; r < TB; ++r) l += sh.lsum[r];
    lpart[blockIdx.x] = l;
  }
}

// grad[w] = sum over blocks of partial[b][w], in block order; loss = sum lpart / n.
__global__ void reduce_kernel(const float* __restrict__ partial, int nblocks,
                              float* __restrict__ grad, const double* __restrict__ lpart,
                              double* __restrict__ loss, int64_t n) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < TFKT_MLP_NWEIGHTS) {
    float acc = 0.0f;
    for (int b = 0; b < nblocks; ++b) acc += partial[(size_t)b * TFKT_MLP_NWEIGHTS + w];
    grad[w] = acc;
  }
  if (w == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += lpart[b];
    *loss = l / (double)n;
  }
}

// Adam on the master weights; c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float* __restrict__ master, __nv_bfloat16* __restrict__ wmat,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= TFKT_MLP_NWEIGHTS) return;
  const float g = grad[w];
  const float mw = b1 * m[w] + (1.0f - b1) * g;
  const float vw = b2 * v[w] + (1.0f - b2) * g * g;
  m[w] = mw;
  v[w] = vw;
  const float p = master[w] - lr * (mw * c1) / (sqrtf(vw * c2) + eps);
  master[w] = p;
  int e = -1;
  if (w < OB1) e = w;                                   // W1
  else if (w >= OW2 && w < OB2) e = NH * NIN + (w - OW2);   // W2
  else if (w >= OW3 && w < OB3) e = NH * NIN + NH * NH + (w - OW3);   // W3
  if (e >= 0) wmat[e] = __float2bfloat16_rn(p);
}

__global__ void refresh_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ wmat) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NMAT) return;
  int w;
  if (e < NH * NIN) w = OW1 + e;
  else if (e < NH * NIN + NH * NH) w = OW2 + (e - NH * NIN);
  else w = OW3 + (e - NH * NIN - NH * NH);
  wmat[e] = __float2bfloat16_rn(master[w]);
}

tfkt_status cuda_err(cudaError_t e, const char* what) {
  return fail(TFKT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MLP_CUDA(...)                                          \
  do {                                                         \
    cudaError_t e_ = (__VA_ARGS__);                            \
    if (e_ != cudaSuccess) return cuda_err(e_, #__VA_ARGS__);  \
  } while (0)

tfkt_status ensure_blocks(tfkt_mlp* net, int nblocks) {
  if (nblocks <= net->max_blocks) return TFKT_OK;
  if (net->partial) MLP_CUDA(cudaFree(net->partial));
  if (net->lpart) MLP_CUDA(cudaFree(net->lpart));
  net->partial = nullptr;
  net->lpart = nullptr;
  net->max_blocks = 0;
  MLP_CUDA(cudaMalloc(&net->partial, (size_t)nblocks * TFKT_MLP_NWEIGHTS * sizeof(float)));
  MLP_CUDA(cudaMalloc(&net->lpart, (size_t)nblocks * sizeof(double)));
  net->max_blocks = nblocks;
  return TFKT_OK;
}

}  // namespace

const MlpDev& mlp_dev(const tfkt_mlp* net) { return net->d; }

}  // namespace tfkt

using namespace tfkt;

extern "C" {

tfkt_status tfkt_mlp_create(const float* params, void* stream, tfkt_mlp** out) {
  if (!params || !out) return fail(TFKT_EINVAL, "NULL argument");
  *out = nullptr;
  tfkt_mlp* net = new (std::nothrow) tfkt_mlp();   // nothing may throw across the C interface
  if (!net) return fail(TFKT_ENOMEM, "host allocation failed");
  net->stream = (cudaStream_t)stream;
  auto bad = [&](cudaError_t e, const char* what) {
    tfkt_mlp_destroy(net);
    return cuda_err(e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&net->d.master, TFKT_MLP_NPARAM * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&net->d.wmat, NMAT * sizeof(__nv_bfloat16))) != cudaSuccess ||
      (e = cudaMalloc(&net->m, TFKT_MLP_NWEIGHTS * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&net->v, TFKT_MLP_NWEIGHTS * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&net->grad, TFKT_MLP_NWEIGHTS * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&net->loss_dev, sizeof(double))) != cudaSuccess) {
    tfkt_mlp_destroy(net);
    cudaGetLastError();   // clear the allocation error
    return fail(TFKT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemsetAsync(net->m, 0, TFKT_MLP_NWEIGHTS * sizeof(float), net->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(net->v, 0, TFKT_MLP_NWEIGHTS * sizeof(float), net->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(net->grad, 0, TFKT_MLP_NWEIGHTS * sizeof(float), net->stream)) != cudaSuccess)
    return bad(e, "cudaMemsetAsync");
  tfkt_status s = tfkt_mlp_set(net, params);
  if (s != TFKT_OK) {
    tfkt_mlp_destroy(net);
    return s;
  }
  *out = net;
  return TFKT_OK;
}

tfkt_status tfkt_mlp_destroy(tfkt_mlp* net) {
  if (!net) return TFKT_OK;
  cudaError_t e = cudaStreamSynchronize(net->stream);
  void* ptrs[] = {net->d.master, net->d.wmat, net->m, net->v, net->grad, net->partial, net->lpart,
                  net->loss_dev};
  for (void* p : ptrs)
    if (p) {
      cudaError_t f = cudaFree(p);
      if (e == cudaSuccess) e = f;
    }
  delete net;
  if (e != cudaSuccess) return cuda_err(e, "destroy");
  return TFKT_OK;
}

tfkt_status tfkt_mlp_get(tfkt_mlp* net, float* params) {
  if (!net || !params) return fail(TFKT_EINVAL, "NULL argument");
  MLP_CUDA(cudaMemcpyAsync(params, net->d.master, TFKT_MLP_NPARAM * sizeof(float),
                           cudaMemcpyDeviceToHost, net->stream));
  MLP_CUDA(cudaStreamSynchronize(net->stream));
  return TFKT_OK;
}

tfkt_status tfkt_mlp_set(tfkt_mlp* net, const float* params) {
  if (!net || !params) return fail(TFKT_EINVAL, "NULL argument");
  for (int k = 0; k < NIN; ++k)
    if (!(params[OSX + k] > 0)) return fail(TFKT_EINVAL, "input scales sx must be > 0");
  for (int k = 0; k < NOUT; ++k)
    if (!(params[OST + k] > 0)) return fail(TFKT_EINVAL, "output scales st must be > 0");
  MLP_CUDA(cudaMemcpyAsync(net->d.master, params, TFKT_MLP_NPARAM * sizeof(float),
                           cudaMemcpyHostToDevice, net->stream));
  refresh_kernel<<<(NMAT + 255) / 256, 256, 0, net->stream>>>(net->d.master, net->d.wmat);
  MLP_CUDA(cudaGetLastError());
  // the host vector may be released as soon as this returns
  MLP_CUDA(cudaStreamSynchronize(net->stream));
  return TFKT_OK;
}

tfkt_status tfkt_mlp_forward(tfkt_mlp* net, const float* X, int64_t n, float* Y) {
  NvtxRange nvtx_range("tfkt_mlp_forward");
  if (!net || n < 0 || (n > 0 && (!X || !Y))) return fail(TFKT_EINVAL, "bad argument");
  if (n == 0) return TFKT_OK;
  const int64_t blocks = (n + 127) / 128;
  forward_kernel<<<(unsigned)blocks, 128, tc_smem_bytes(4), net->stream>>>(net->d.master, net->d.wmat,
                                                                          X, n, Y);
  MLP_CUDA(cudaGetLastError());
  return TFKT_OK;
}

tfkt_status tfkt_mlp_loss_grad(tfkt_mlp* net, const float* X, const float* T, int64_t n,
                               double* loss, float* grad) {
  NvtxRange nvtx_range("tfkt_mlp_loss_grad");
  if (!net || n < 1 || !X || !T) return fail(TFKT_EINVAL, "bad argument");
  const int64_t nb = (n + TB - 1) / TB;
  if (nb > (1 << 20)) return fail(TFKT_EINVAL, "batch too large (at most 2^27 samples)");
  tfkt_status s = ensure_blocks(net, (int)nb);
  if (s != TFKT_OK) return s;
  const size_t smem = sizeof(TrainTc);
  MLP_CUDA(cudaFuncSetAttribute(loss_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  loss_grad_kernel<<<(unsigned)nb, TB, smem, net->stream>>>(net->d.master, net->d.wmat, X, T, n,
                                                            net->partial, net->lpart);
  MLP_CUDA(cudaGetLastError());
  reduce_kernel<<<(TFKT_MLP_NWEIGHTS + 255) / 256, 256, 0, net->stream>>>(
      net->partial, (int)nb, net->grad, net->lpart, net->loss_dev, n);
  MLP_CUDA(cudaGetLastError());
  if (grad)
    MLP_CUDA(cudaMemcpyAsync(grad, net->grad, TFKT_MLP_NWEIGHTS * sizeof(float),
                             cudaMemcpyDeviceToDevice, net->stream));
  if (loss) {
    MLP_CUDA(cudaMemcpyAsync(loss, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost,
                             net->stream));
    MLP_CUDA(cudaStreamSynchronize(net->stream));
  }
  return TFKT_OK;
}

tfkt_status tfkt_mlp_adam(tfkt_mlp* net, float lr, float beta1, float beta2, float eps) {
  NvtxRange nvtx_range("tfkt_mlp_adam");
  if (!net) return fail(TFKT_EINVAL, "NULL argument");
  if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(TFKT_EINVAL, "bad Adam hyper-parameters");
  net->t += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)net->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)net->t)));
  adam_kernel<<<(TFKT_MLP_NWEIGHTS + 255) / 256, 256, 0, net->stream>>>(
      net->d.master, net->d.wmat, net->m, net->v, net->grad, lr, beta1, beta2, eps, c1, c2);
  MLP_CUDA(cudaGetLastError());
  return TFKT_OK;
}

}  // extern "C"
