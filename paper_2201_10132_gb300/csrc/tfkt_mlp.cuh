// The per-node network of the learned macro-step: layout of its parameters
// and the device-side forward pass (tensor cores) on weights staged in shared memory.
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

// GELU(z) = z Phi(z) (Hendrycks & Gimpel 2016), Phi through the library erff.
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// ---- Tensor-core forward pass: mma.sync m16n8k16, bfloat16 operands, FP32
// accumulation. One warp takes TC_ROWS samples (two 16-row tiles). Activations
// (standardised inputs, hidden units after GELU) are FP32 values split into a
// bfloat16 high part and a bfloat16 remainder, each multiplied by the bfloat16
// weights into the same FP32 accumulator, so the products keep about 16 bits of
// the activation (a single bfloat16 operand keeps 8). A layer's accumulator
// fragments are, after GELU, the next layer's operand fragments in registers.
constexpr int TC_ROWS = 32;                 // samples per warp pass
constexpr int TC_K1 = 48;                   // layer-1 inner size, NIN padded to 3 steps of 16
constexpr int TC_W1LD = 56, TC_W2LD = 72;   // bfloat16 row strides (padded against bank conflicts)
constexpr int TC_XLD = 52;                  // FP32 row stride of a warp's standardised samples
static_assert(NIN <= TC_K1 && NH == 64 && NOUT <= 8, "tensor-core tiling of the network");

struct MlpTc {
  __nv_bfloat16 w1[NH * TC_W1LD];      // [out][in], in >= NIN zero
  __nv_bfloat16 w2[NH * TC_W2LD];      // [out][in]
  __nv_bfloat16 w3[8 * TC_W2LD];       // [out][in], out >= NOUT zero
  float b1[NH], b2[NH], b3[8];
  float mx[NIN], rsx[NIN], mt[NOUT], st[NOUT];
};
// per-warp scratch: TC_ROWS rows of TC_XLD standardised inputs, then TC_ROWS x 4 outputs
constexpr int TC_WARP_FLOATS = TC_ROWS * TC_XLD + TC_ROWS * 4;
constexpr size_t tc_smem_bytes(int warps) {
  return ((sizeof(MlpTc) + 15) & ~(size_t)15) + sizeof(float) * (size_t)TC_WARP_FLOATS * warps;
}

__device__ __forceinline__ void mlp_stage_tc(MlpTc& s, const float* master,
                                             const __nv_bfloat16* wmat, int tid, int nthreads) {
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k = tid; k < NH * TC_W1LD; k += nthreads) {
    const int o = k / TC_W1LD, i = k % TC_W1LD;
    s.w1[k] = i < NIN ? wmat[o * NIN + i] : zero;
  }
  for (int k = tid; k < NH * TC_W2LD; k += nthreads) {
    const int o = k / TC_W2LD, i = k % TC_W2LD;
    s.w2[k] = i < NH ? wmat[NH * NIN + o * NH + i] : zero;
  }
  for (int k = tid; k < 8 * TC_W2LD; k += nthreads) {
    const int o = k / TC_W2LD, i = k % TC_W2LD;
    s.w3[k] = (o < NOUT && i < NH) ? wmat[NH * NIN + NH * NH + o * NH + i] : zero;
  }
  for (int k = tid; k < NH; k += nthreads) {
    s.b1[k] = master[OB1 + k];
    s.b2[k] = master[OB2 + k];
  }
  for (int k = tid; k < 8; k += nthreads) s.b3[k] = k < NOUT ? master[OB3 + k] : 0.0f;
  for (int k = tid; k < NIN; k += nthreads) {
    s.mx[k] = master[OMX + k];
    s.rsx[k] = 1.0f / master[OSX + k];
  }
  for (int k = tid; k < NOUT; k += nthreads) {
    s.mt[k] = master[OMT + k];
    s.st[k] = master[OST + k];
  }
}

// bfloat16 high part and remainder of the pair (a, b), lower column in the low half.
__device__ __forceinline__ void tc_split(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D = A B + D for a 16 x 16 bfloat16 A (row fragments), 16 x 8 bfloat16 B (column
// fragments) and a 16 x 8 FP32 accumulator.
__device__ __forceinline__ void tc_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t tc_ld2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// One layer's MMAs for a 16-row tile: c[n] += A(k-steps) W^T over NK k-steps of
// 16 and NN n-tiles of 8, A given as high/remainder fragment pairs.
template <int NK, int NN, int LD>
__device__ __forceinline__ void tc_layer(float (&c)[NN][4], const uint32_t (&ah)[NK][4],
                                         const uint32_t (&al)[NK][4], const __nv_bfloat16* w,
                                         int g, int t) {
#pragma unroll
  for (int n = 0; n < NN; ++n)
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const __nv_bfloat16* wr = w + (8 * n + g) * LD + 16 * k + 2 * t;
      const uint32_t b0 = tc_ld2(wr), b1 = tc_ld2(wr + 8);
      tc_mma(c[n], ah[k], b0, b1);
      tc_mma(c[n], al[k], b0, b1);
    }
}

// Operand fragments of the next layer from this layer's accumulators (GELU
// applied): k-step k of the next layer is n-tiles 2k and 2k + 1 of this one.
template <int NK>
__device__ __forceinline__ void tc_gelu_operands(const float (&c)[2 * NK][4], uint32_t (&ah)[NK][4],
                                                 uint32_t (&al)[NK][4]) {
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    tc_split(gelu(c[2 * k][0]), gelu(c[2 * k][1]), ah[k][0], al[k][0]);
    tc_split(gelu(c[2 * k][2]), gelu(c[2 * k][3]), ah[k][1], al[k][1]);
    tc_split(gelu(c[2 * k + 1][0]), gelu(c[2 * k + 1][1]), ah[k][2], al[k][2]);
    tc_split(gelu(c[2 * k + 1][2]), gelu(c[2 * k + 1][3]), ah[k][3], al[k][3]);
  }
}

// Forward pass of one warp's TC_ROWS standardised samples X [TC_ROWS][TC_XLD]
// (columns NIN .. TC_K1 - 1 zero) into the raw outputs O [TC_ROWS][4] (columns
// 0 .. NOUT - 1; the caller applies (st, mt)). All 32 lanes must call it.
__device__ __forceinline__ void mlp_warp_tc(const MlpTc& s, const float* X, float* O, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int m = 0; m < TC_ROWS / 16; ++m) {
    const float* x0 = X + (16 * m + g) * TC_XLD;
    const float* x1 = x0 + 8 * TC_XLD;
    uint32_t ah1[3][4], al1[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c0 = 16 * k + 2 * t;
      const float2 v0 = *reinterpret_cast<const float2*>(x0 + c0);
      const float2 v1 = *reinterpret_cast<const float2*>(x1 + c0);
      const float2 v2 = *reinterpret_cast<const float2*>(x0 + c0 + 8);
      const float2 v3 = *reinterpret_cast<const float2*>(x1 + c0 + 8);
      tc_split(v0.x, v0.y, ah1[k][0], al1[k][0]);
      tc_split(v1.x, v1.y, ah1[k][1], al1[k][1]);
      tc_split(v2.x, v2.y, ah1[k][2], al1[k][2]);
      tc_split(v3.x, v3.y, ah1[k][3], al1[k][3]);
    }
    float c1[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      c1[n][0] = c1[n][2] = s.b1[8 * n + 2 * t];
      c1[n][1] = c1[n][3] = s.b1[8 * n + 2 * t + 1];
    }
    tc_layer<3, 8, TC_W1LD>(c1, ah1, al1, s.w1, g, t);
    uint32_t ah2[4][4], al2[4][4];
    tc_gelu_operands<4>(c1, ah2, al2);
    float c2[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      c2[n][0] = c2[n][2] = s.b2[8 * n + 2 * t];
      c2[n][1] = c2[n][3] = s.b2[8 * n + 2 * t + 1];
    }
    tc_layer<4, 8, TC_W2LD>(c2, ah2, al2, s.w2, g, t);
    uint32_t ah3[4][4], al3[4][4];
    tc_gelu_operands<4>(c2, ah3, al3);
    float c3[1][4] = {{s.b3[2 * t], s.b3[2 * t + 1], s.b3[2 * t], s.b3[2 * t + 1]}};
    tc_layer<4, 1, TC_W2LD>(c3, ah3, al3, s.w3, g, t);
    if (2 * t < NOUT) {
      O[(16 * m + g) * 4 + 2 * t] = c3[0][0];
      O[(16 * m + g + 8) * 4 + 2 * t] = c3[0][2];
    }
    if (2 * t + 1 < NOUT) {
      O[(16 * m + g) * 4 + 2 * t + 1] = c3[0][1];
      O[(16 * m + g + 8) * 4 + 2 * t + 1] = c3[0][3];
    }
  }
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
