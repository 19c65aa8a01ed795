/*
 * Learned polymer macro-step of libtfkt (extension of tfkt.h).
 *
 * The paper has no learned component; this one is built on its scheme
 * (arXiv 2201.10132, Sec. VI). A block advances a context by 1 + K lattice
 * steps:
 *  1. one plain step of the scheme (tfkt_step);
 *  2. a small network predicts the conformation C = ell^2 <QQ> (r-lengths^2)
 *     of every node K steps later from the conformation of the parcel that
 *     arrives there (C interpolated at r - K U) and the velocity-gradient
 *     stencil; the plain step's own rate of change of C, carried over the K
 *     steps, checks it tile by tile, and a tile whose largest disagreement
 *     exceeds the threshold keeps the plain step's conformation instead;
 *  3. K solvent-only steps under the polymer stress (H/2) psi_tot C of the
 *     conformation interpolated linearly in time (Sec. III, Eq. IDef), the
 *     polymer momentum slaved to psi_tot U + tau2 E + (its offset in the plain
 *     state of step 1);
 *  4. the polymer populations are moved to the predicted conformation by an
 *     equilibrium-shaped increment (mass and momentum unchanged).
 * The K solvent sub-steps never touch the polymer populations, which hold
 * 98.9% of the state at N_Q = 32, so a block moves a fraction of the bytes of
 * 1 + K plain steps.
 *
 * Network: inputs (40) = (C_dep - c_e I)/c_e (xx, xy, yy; c_e the lattice
 * equilibrium C_xx), K dU_b/dr_a on the 3 x 3 stencil around the node (order
 * dy = -1..1, dx = -1..1, then dU_x/dx, dU_y/dx, dU_x/dy, dU_y/dy), K/lambda_H;
 * standardised by (mx, sx); two hidden layers of 64 with GELU; 3 outputs
 * rescaled by (st, mt) to (C_new - C_dep)/c_e. Matrices are used in bfloat16,
 * everything else in FP32, accumulation in FP32.
 *
 * Packed parameter vector (TFKT_MLP_NPARAM floats, FP32):
 *   W1[64][40], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]   (trainable)
 *   mx[40], sx[40], mt[3], st[3]                                (fixed)
 *
 * All device arrays are row-major float32 on the context's / network's device;
 * n samples of X are [n][40], of targets and outputs [n][3].
 */
#ifndef TFKT_LPM_H
#define TFKT_LPM_H

#include "tfkt.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TFKT_MLP_IN 40
#define TFKT_MLP_HID 64
#define TFKT_MLP_OUT 3
#define TFKT_MLP_NWEIGHTS (64 * 40 + 64 + 64 * 64 + 64 + 3 * 64 + 3)
#define TFKT_MLP_NPARAM (TFKT_MLP_NWEIGHTS + 40 + 40 + 3 + 3)

typedef struct tfkt_mlp tfkt_mlp;

/* A network on the current device from a host parameter vector (copied).
   stream: the stream its kernels run on (NULL: the legacy default stream).
   Errors (all network calls): TFKT_EINVAL for NULL arguments, n out of range,
   non-positive scales sx, st or bad Adam hyper-parameters (nothing launched);
   TFKT_ENOMEM if an allocation fails; TFKT_ECUDA if a CUDA call fails. */
tfkt_status tfkt_mlp_create(const float* params, void* stream, tfkt_mlp** out);
/* Free the network's device memory; NULL is accepted. */
tfkt_status tfkt_mlp_destroy(tfkt_mlp* net);
/* Copy the FP32 master parameters to / from a host vector of TFKT_MLP_NPARAM. */
tfkt_status tfkt_mlp_get(tfkt_mlp* net, float* params);
tfkt_status tfkt_mlp_set(tfkt_mlp* net, const float* params);

/* Y = network(X) for n >= 0 samples (raw inputs, raw outputs). Runs on the
   tensor cores: bfloat16 weights, each FP32 activation as a bfloat16 high part
   plus a bfloat16 remainder, FP32 accumulation (within about 1e-5 of the FP32
   forward pass). */
tfkt_status tfkt_mlp_forward(tfkt_mlp* net, const float* X, int64_t n, float* Y);

/* Loss L = (1/n) sum_n sum_j (o_nj - (t_nj - mt_j)/st_j)^2 of n >= 1 samples, o the
   standardised outputs, and its gradient with respect to the trainable
   parameters (evaluated with the bfloat16 matrices, on the tensor cores with
   FP32 accumulation and activations split into bfloat16 high part and
   remainder; within about 1e-5 of FP32 arithmetic). loss: host double (may be
   NULL); grad: device float[TFKT_MLP_NWEIGHTS] (may be NULL; the gradient is
   also kept for tfkt_mlp_adam). Deterministic: fixed reduction order. */
tfkt_status tfkt_mlp_loss_grad(tfkt_mlp* net, const float* X, const float* T, int64_t n,
                               double* loss, float* grad);

/* One Adam step (Kingma & Ba 2015) on the FP32 master weights with the last
   gradient; the bfloat16 matrices are refreshed (round to nearest even). */
tfkt_status tfkt_mlp_adam(tfkt_mlp* net, float lr, float beta1, float beta2, float eps);

/* Options of the learned block. */
typedef struct {
  int32_t K;          /* solvent sub-steps per block: even, 2 <= K <= 64 */
  int32_t tile;       /* side of the check's tiles, 1 <= tile <= 64 */
  float threshold;    /* largest |C_net - C_plain| / c_e a tile may show */
  int32_t mode;       /* TFKT_LPM_NET, or TFKT_LPM_FROZEN: every tile keeps the plain
                         step's conformation (the block without the network) */
  int32_t inject_wait_timeout; /* fault injection for tests, normally 0: nonzero makes
                         the network kernel issue no tensor-core work, so that its
                         waits for it run out after a few polls (TFKT_ETIMEOUT) */
} tfkt_lpm_opts;
enum { TFKT_LPM_NET = 0, TFKT_LPM_FROZEN = 1 };

/* Run nblocks >= 0 blocks on the context's stream and synchronise it at the
   end. The context must be FP32, Hookean (fene_b = 0), with polymer, and on
   the fused path (nx a multiple of 32, ny of 8); net may be NULL in
   TFKT_LPM_FROZEN mode. flagged: host int64, if not NULL receives the number
   of tiles that fell back, summed over the blocks. Scratch (about 18 planes of
   ny * pitch floats) is allocated on first use and freed with the context.
   Errors: EINVAL for unsupported contexts or options; ETIMEOUT when a wait of
   the network kernel for its tensor-core work ran out (bounded; the tiles
   concerned fell back to the plain step, so the state is that of a valid
   block and the context stays usable); ECUDA if a launch fails. */
tfkt_status tfkt_lpm_run(tfkt_ctx* c, const tfkt_mlp* net, const tfkt_lpm_opts* opts,
                         int64_t nblocks, int64_t* flagged);

/* Training data from the current (plain) state of c: the features X [nx*ny][40]
   of a block starting now (node order y-major) and the parcels' departure
   conformations C_dep [nx*ny][3]; after K plain steps, tfkt_lpm_targets writes
   T = (C - C_dep) / c_e [nx*ny][3]. Same context requirements as tfkt_lpm_run. */
tfkt_status tfkt_lpm_features(tfkt_ctx* c, int32_t K, float* X, float* C_dep);
tfkt_status tfkt_lpm_targets(tfkt_ctx* c, const float* C_dep, float* T);

#ifdef __cplusplus
}
#endif
#endif
