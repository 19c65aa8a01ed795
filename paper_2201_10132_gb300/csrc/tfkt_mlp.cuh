// The per-node network of the learned macro-step: layout of its parameters
// and the device-side forward pass on weights staged in shared memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tfkt_lpm.h"

namespace tfkt {

constexpr int NIN = TFKT_MLP_IN, NH = TFKT_MLP_HID, NOUT = TFKT_MLP_OUT;
// offsets in the packed parameter vector
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH,
              OW3 = OB2 + NH, OB3 = OW3 + NOUT * NH, OMX = OB3 + NOUT, OSX = OMX + NIN,
              OMT = OSX + NIN, OST = OMT + NOUT;
static_assert(OMX == TFKT_MLP_NWEIGHTS, "parameter layout");
static_assert(OST + NOUT == TFKT_MLP_NPARAM, "parameter layout");
constexpr int NMAT = NH * NIN + NH * NH + NOUT * NH;   // bfloat16 matrix entries

// Device state of a network.
struct MlpDev {
  float* master;            // [NPARAM] FP32 master parameters
  __nv_bfloat16* wmat;      // [NMAT] W1, W2, W3 in bfloat16
};

// Shared-memory copy of everything the forward pass reads, as FP32.
struct MlpShared {
  float w1[NH * NIN], b1[NH], w2[NH * NH], b2[NH], w3[NOUT * NH], b3[NOUT];
  float mx[NIN], rsx[NIN], mt[NOUT], st[NOUT];
};

// Stage the network into shared memory (all threads of the block take part).
__device__ __forceinline__ void mlp_stage(MlpShared& s, const float* master,
                                          const __nv_bfloat16* wmat, int tid, int nthreads) {
  for (int k = tid; k < NH * NIN; k += nthreads) s.w1[k] = __bfloat162float(wmat[k]);
  for (int k = tid; k < NH * NH; k += nthreads) s.w2[k] = __bfloat162float(wmat[NH * NIN + k]);
  for (int k = tid; k < NOUT * NH; k += nthreads)
    s.w3[k] = __bfloat162float(wmat[NH * NIN + NH * NH + k]);
  for (int k = tid; k < NH; k += nthreads) {
    s.b1[k] = master[OB1 + k];
    s.b2[k] = master[OB2 + k];
  }
  for (int k = tid; k < NIN; k += nthreads) {
    s.mx[k] = master[OMX + k];
    s.rsx[k] = 1.0f / master[OSX + k];
  }
  for (int k = tid; k < NOUT; k += nthreads) {
    s.b3[k] = master[OB3 + k];
    s.mt[k] = master[OMT + k];
    s.st[k] = master[OST + k];
  }
}

// GELU(z) = z Phi(z) (Hendrycks & Gimpel 2016), Phi through the library erff.
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// Forward pass of one sample: raw features x[NIN] -> raw outputs y[NOUT].
// Layer 2 feeds layer 3 one unit at a time, so only x, h1 and the outputs are live.
__device__ __forceinline__ void mlp_forward(const MlpShared& s, const float* x, float* y) {
  float xn[NIN];
#pragma unroll
  for (int i = 0; i < NIN; ++i) xn[i] = (x[i] - s.mx[i]) * s.rsx[i];
  float h1[NH];
#pragma unroll
  for (int o = 0; o < NH; ++o) {
    float acc = s.b1[o];
    const float4* w = reinterpret_cast<const float4*>(s.w1 + o * NIN);
#pragma unroll
    for (int i = 0; i < NIN / 4; ++i) {
      const float4 v = w[i];
      acc = fmaf(v.x, xn[4 * i], acc);
      acc = fmaf(v.y, xn[4 * i + 1], acc);
      acc = fmaf(v.z, xn[4 * i + 2], acc);
      acc = fmaf(v.w, xn[4 * i + 3], acc);
    }
    h1[o] = gelu(acc);
  }
  float out[NOUT];
#pragma unroll
  for (int j = 0; j < NOUT; ++j) out[j] = s.b3[j];
#pragma unroll 2
  for (int o = 0; o < NH; ++o) {
    float acc = s.b2[o];
    const float4* w = reinterpret_cast<const float4*>(s.w2 + o * NH);
#pragma unroll
    for (int i = 0; i < NH / 4; ++i) {
      const float4 v = w[i];
      acc = fmaf(v.x, h1[4 * i], acc);
      acc = fmaf(v.y, h1[4 * i + 1], acc);
      acc = fmaf(v.z, h1[4 * i + 2], acc);
      acc = fmaf(v.w, h1[4 * i + 3], acc);
    }
    const float h2 = gelu(acc);
#pragma unroll
    for (int j = 0; j < NOUT; ++j) out[j] = fmaf(s.w3[j * NH + o], h2, out[j]);
  }
#pragma unroll
  for (int j = 0; j < NOUT; ++j) y[j] = out[j] * s.st[j] + s.mt[j];
}

}  // namespace tfkt

// The network object behind the C-ABI handle.
struct tfkt_mlp {
  tfkt::MlpDev d{};
  float* m = nullptr;         // [NWEIGHTS] Adam first moments
  float* v = nullptr;         // [NWEIGHTS] Adam second moments
  float* grad = nullptr;      // [NWEIGHTS] last gradient
  float* partial = nullptr;   // [max_blocks][NWEIGHTS] per-block gradient partials
  double* lpart = nullptr;    // [max_blocks] per-block loss partials
  double* loss_dev = nullptr;
  int max_blocks = 0;
  int64_t t = 0;              // Adam steps taken
  cudaStream_t stream = nullptr;
};
