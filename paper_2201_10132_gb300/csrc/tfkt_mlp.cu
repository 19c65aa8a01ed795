// The learned macro-step's network: forward pass, loss and gradient by
// backpropagation, and Adam, as hand-written kernels (bfloat16 matrices, FP32
// accumulation; inference on the tensor cores, training on the CUDA cores in
// FP32). Gradients are summed per block of 128 samples and the block partials
// in a fixed order, so results are reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tfkt_internal.cuh"
#include "tfkt_mlp.cuh"

namespace tfkt {
namespace {

constexpr int TB = 128;          // samples (threads) per training block
constexpr int XS = NIN + 1;      // padded row strides of the per-sample tables
constexpr int HS = NH + 1;

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

struct TrainShared {
  MlpShared net;
  float xs[TB * XS];
  float z1[TB * HS], h1[TB * HS], z2[TB * HS], h2[TB * HS];
  float dO[TB * NOUT];
  double lsum[TB];
};

// Loss and gradient partials of one block of TB samples; partial[b][NWEIGHTS].
__global__ void __launch_bounds__(TB) loss_grad_kernel(const float* __restrict__ master,
                                                       const __nv_bfloat16* __restrict__ wmat,
                                                       const float* __restrict__ X,
                                                       const float* __restrict__ T, int64_t n,
                                                       float* __restrict__ partial,
                                                       double* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainShared& sh = *reinterpret_cast<TrainShared*>(smem_raw);
  const int tid = threadIdx.x;
  mlp_stage(sh.net, master, wmat, tid, TB);
  __syncthreads();
  const MlpShared& s = sh.net;
  const int64_t k = (int64_t)blockIdx.x * TB + tid;
  const bool valid = k < n;
  const float inv_n = 1.0f / (float)n;
  float* xs = sh.xs + tid * XS;
  float* z1 = sh.z1 + tid * HS;
  float* h1 = sh.h1 + tid * HS;
  float* z2 = sh.z2 + tid * HS;
  float* h2 = sh.h2 + tid * HS;
  double lsq = 0.0;
  // ---- forward, keeping what the backward pass needs
  if (valid) {
    for (int i = 0; i < NIN; ++i) xs[i] = (X[k * NIN + i] - s.mx[i]) * s.rsx[i];
    for (int o = 0; o < NH; ++o) {
      float acc = s.b1[o];
      for (int i = 0; i < NIN; ++i) acc = fmaf(s.w1[o * NIN + i], xs[i], acc);
      z1[o] = acc;
      h1[o] = gelu(acc);
    }
    for (int o = 0; o < NH; ++o) {
      float acc = s.b2[o];
      for (int i = 0; i < NH; ++i) acc = fmaf(s.w2[o * NH + i], h1[i], acc);
      z2[o] = acc;
      h2[o] = gelu(acc);
    }
    for (int j = 0; j < NOUT; ++j) {
      float acc = s.b3[j];
      for (int i = 0; i < NH; ++i) acc = fmaf(s.w3[j * NH + i], h2[i], acc);
      const float t = (T[k * NOUT + j] - s.mt[j]) / s.st[j];
      const float r = acc - t;
      lsq += (double)r * (double)r;
      sh.dO[tid * NOUT + j] = 2.0f * r * inv_n;
    }
  } else {
    for (int i = 0; i < NIN; ++i) xs[i] = 0.0f;
    for (int o = 0; o < NH; ++o) z1[o] = h1[o] = z2[o] = h2[o] = 0.0f;
    for (int j = 0; j < NOUT; ++j) sh.dO[tid * NOUT + j] = 0.0f;
  }
  sh.lsum[tid] = lsq;
  __syncthreads();
  float* P = partial + (size_t)blockIdx.x * TFKT_MLP_NWEIGHTS;
  // ---- output layer: dW3 = sum_s dO h2^T, db3 = sum_s dO
  for (int e = tid; e < NOUT * NH + NOUT; e += TB) {
    float acc = 0.0f;
    if (e < NOUT * NH) {
      const int j = e / NH, i = e % NH;
      for (int r = 0; r < TB; ++r) acc = fmaf(sh.dO[r * NOUT + j], sh.h2[r * HS + i], acc);
      P[OW3 + e] = acc;
    } else {
      const int j = e - NOUT * NH;
      for (int r = 0; r < TB; ++r) acc += sh.dO[r * NOUT + j];
      P[OB3 + j] = acc;
    }
  }
  // ---- dz2 = (W3^T dO) * GELU'(z2), in place of z2 (own row)
  for (int o = 0; o < NH; ++o) {
    float acc = 0.0f;
    for (int j = 0; j < NOUT; ++j) acc = fmaf(s.w3[j * NH + o], sh.dO[tid * NOUT + j], acc);
    z2[o] = acc * gelu_grad(z2[o]);
  }
  __syncthreads();
  // ---- layer 2: dW2 = sum_s dz2 h1^T, db2 = sum_s dz2
  for (int e = tid; e < NH * NH + NH; e += TB) {
    float acc = 0.0f;
    if (e < NH * NH) {
      const int o = e / NH, i = e % NH;
      for (int r = 0; r < TB; ++r) acc = fmaf(sh.z2[r * HS + o], sh.h1[r * HS + i], acc);
      P[OW2 + e] = acc;
    } else {
      const int o = e - NH * NH;
      for (int r = 0; r < TB; ++r) acc += sh.z2[r * HS + o];
      P[OB2 + o] = acc;
    }
  }
  // ---- dz1 = (W2^T dz2) * GELU'(z1), in place of z1 (own row)
  for (int i = 0; i < NH; ++i) {
    float acc = 0.0f;
    for (int o = 0; o < NH; ++o) acc = fmaf(s.w2[o * NH + i], z2[o], acc);
    z1[i] = acc * gelu_grad(z1[i]);
  }
  __syncthreads();
  // ---- layer 1: dW1 = sum_s dz1 x^T, db1 = sum_s dz1
  for (int e = tid; e < NH * NIN + NH; e += TB) {
    float acc = 0.0f;
    if (e < NH * NIN) {
      const int o = e / NIN, i = e % NIN;
      for (int r = 0; r < TB; ++r) acc = fmaf(sh.z1[r * HS + o], sh.xs[r * XS + i], acc);
      P[OW1 + e] = acc;
    } else {
      const int o = e - NH * NIN;
      for (int r = 0; r < TB; ++r) acc += sh.z1[r * HS + o];
      P[OB1 + o] = acc;
    }
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
  tfkt_mlp* net = new tfkt_mlp;
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
      (e = cudaMalloc(&net->loss_dev, sizeof(double))) != cudaSuccess)
    return bad(e, "cudaMalloc");
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
  if (!net || n < 1 || !X || !T) return fail(TFKT_EINVAL, "bad argument");
  const int64_t nb = (n + TB - 1) / TB;
  if (nb > (1 << 20)) return fail(TFKT_EINVAL, "batch too large (at most 2^27 samples)");
  tfkt_status s = ensure_blocks(net, (int)nb);
  if (s != TFKT_OK) return s;
  const size_t smem = sizeof(TrainShared);
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
