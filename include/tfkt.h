/*
 * tfkt — two-fluid kinetic step for dilute polymer solutions on one GB300 GPU.
 *
 * C-ABI of the library libtfkt.so. It advances the discrete two-fluid kinetic
 * scheme of Singh, Subramanian & Ansumali, "Two-fluid kinetic theory for
 * dilute polymer solutions" (arXiv 2201.10132):
 *   - solvent: D2Q9 populations with the two-relaxation (tau1 / tau2)
 *     quasi-equilibrium collision about the solvent velocity u_S and the
 *     mixture velocity U (Sec. VI-A, Eq. dis_sol, Eq. dis_eq);
 *   - polymer dumbbells: D4Q25 populations on the 4-D (r_x, r_y, Q_x, Q_y)
 *     hyper-lattice (Sec. VI-B, Table dis_vel) with linear equilibria about
 *     the imposed velocities of Eq. poly_imposed_vel (Eqs. feq_rq_space,
 *     fstar_rq_space), bounce-back at the edge of the Q-disk (Sec. VI-D);
 *   - time stepping by the trapezoidal rule made explicit through the
 *     auxiliary population g = f - (dt/2) Omega (Sec. VI-C, Eqs. eq1, aux);
 *   - the Kolmogorov body force of Sec. VII, a0 sin(2 pi k_periods y / ny).
 * Lattice units: dt = dr = 1, c_s^2 = 1/3 on both lattices.
 *
 * Conventions shared by every call:
 *   - All functions return tfkt_status; nothing throws across the ABI.
 *   - A context owns one CUDA stream (the caller's, or the legacy default
 *     stream when NULL is passed); all device work of the context is
 *     enqueued on it. A context is not thread-safe.
 *   - After a CUDA error the context is poisoned: every later call except
 *     tfkt_destroy returns TFKT_ESTATE. tfkt_last_error() gives the text.
 *   - Grids are periodic, node (x, y) at row-major index y * nx + x.
 *   - Q-nodes: the S x S cell-centred grid Q = (i - (S-1)/2, j - (S-1)/2)
 *     (Q lattice units), keeping |Q| <= R, numbered row-major over (j, i).
 */
#ifndef TFKT_H
#define TFKT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TFKT_OK = 0,
  TFKT_EINVAL = 1,  /* invalid argument; nothing was allocated or launched */
  TFKT_ENOMEM = 2,  /* device allocation failed, or the workspace is too small */
  TFKT_ECUDA = 3,   /* a CUDA call failed; the context is now poisoned */
  TFKT_ENAN = 4,    /* diagnostics found a non-finite value; state kept */
  TFKT_ESTATE = 5,  /* the context was poisoned by an earlier CUDA error */
  TFKT_EIO = 6,     /* a checkpoint file could not be written or read, or is corrupt */
  TFKT_ETIMEOUT = 7 /* a bounded wait inside a kernel ran out; the kernel gave up cleanly,
                       the affected work took its documented fallback, state kept */
} tfkt_status;

typedef enum {
  TFKT_FP64 = 0,    /* populations stored and updated in double */
  TFKT_FP32 = 1,    /* populations stored as float deviations from rest, updated in float */
  TFKT_FP16 = 2     /* polymer populations stored as half deviations from rest (rounded to
                       nearest, scaled by a power of two), solvent populations as float
                       deviations; updated in float; moment planes in float */
} tfkt_precision;

/* Quasi-equilibrium of the collision (Sec. V): which variables the fast
   relaxation keeps. */
typedef enum {
  TFKT_QE_MOMENTUM = 0,  /* component momenta (Eq. quasieq1): the stress relaxes at tau1,
                            the momenta at tau2 (Schmidt numbers up to Sc*) */
  TFKT_QE_STRESS = 1     /* component stresses (Eq. quasieq2): the momenta relax at tau1,
                            the stress at tau2 (Schmidt numbers from Sc* up) */
} tfkt_qe_model;

/* Physical description of one Kolmogorov run (Sec. VII definitions:
   Re = U0 l / nu, Wi = U0 lambda_H / l, beta = eta_s / (eta_s + eta_p),
   l = ny / (2 pi k_periods), forcing amplitude nu U0 / l^2). */
typedef struct {
  int32_t nx, ny;        /* r-grid, periodic; 1 <= nx, ny */
  int32_t q_side;        /* S: Q-grid side, 1 <= S <= 64 */
  double q_radius;       /* R: disk radius in Q lattice units, > 0 */
  double re, wi, beta;   /* Re > 0; Wi >= 0 (Wi = 0 only with beta = 1); 0 < beta <= 1 */
  double u0;             /* laminar peak velocity, 0 < u0 <= 0.2 */
  int32_t k_periods;     /* forcing periods across ny, >= 1 */
  double tau2;           /* momentum relaxation time tau_m (drag, bead diffusion, Q-drift);
                            <= 0 selects the stress relaxation time 3 beta nu; the momentum
                            model needs tau_m >= 3 beta nu, the stress model tau_m <= 3 beta nu */
  double ell;            /* Q-lattice spacing in r-lengths; <= 0 selects sqrt(2) */
  int32_t ic_mode;       /* 0: start from rest; 1: start from the laminar profile */
  int32_t precision;     /* tfkt_precision */
  double fene_b;         /* 0: Hookean springs; > 0: FENE springs of extensibility b
                            (Sec. VI-D), force H Q / (1 - Q^2/Q0^2) with Q0^2 = b kT/H;
                            every Q-node must lie inside Q0 (q_radius^2 < b sigma_q2,
                            else EINVAL). The drift of a Q-node grows as 1/(1 - Q^2/Q0^2):
                            nodes where kappa |Q| / (1 - Q^2/Q0^2) exceeds about 1, or
                            where the bead-force flux makes the node strongly
                            anti-diffusive in r, make the step unstable; keep the disk
                            well inside Q0. */
  int32_t qe_model;      /* tfkt_qe_model: which variables the collision holds
                            quasi-conserved (Sec. V); both models take the fused
                            kernel on grids of 32 x 8 tiles */
} tfkt_params;

/* Derived lattice parameters and layout of a context. */
typedef struct {
  int32_t nx, ny, nq, precision;
  double tau1, tau2;     /* fast and slow relaxation times of the update (momentum model:
                            stress, momentum; stress model: momentum, stress) */
  double H, kappa;       /* spring constant; Q-drift rate kappa = 2 H tau2 */
  double ell, psi_tot;   /* Q spacing; sum_q psi per r-node (psi counts beads) */
  double sigma_q2;       /* variance of the initial Gaussian in Q (Q lattice units) */
  double a0, kf;         /* forcing amplitude and wavenumber */
  double nu, nu_s, eta_p, lambda_h;
  int64_t step;          /* steps taken since tfkt_create */
  size_t workspace_bytes;
  size_t pitch;          /* elements per stored row (>= nx, multiple of 32) */
  size_t bytes_per_node_step; /* algorithmic HBM bytes of one node update, fused model */
  double fene_b;         /* 0 for Hookean springs */
  int32_t qe_model;
} tfkt_info;

typedef struct tfkt_ctx tfkt_ctx;

/* Kernels timed by tfkt_step_profiled. */
enum {
  TFKT_K_MOMENTS = 0,  /* pull-read of all populations -> moment planes */
  TFKT_K_STEP,         /* two-pass path: pull, collide and write of all populations */
  TFKT_K_FUSED,        /* fused path: pull, collide, write and next-step moments */
  TFKT_K_FIXUP,        /* fused path: completion of the tiles' border moments */
  TFKT_NKERNELS
};

/* Macroscopic fields for tfkt_moments (bit i of the mask selects field i;
   fields are written in increasing bit order, ny * nx doubles each). */
enum {
  TFKT_F_RHO_S = 0,   /* solvent density */
  TFKT_F_PSI_TOT,     /* sum_q psi */
  TFKT_F_UX, TFKT_F_UY,          /* mixture velocity U of f (Sec. VI-C) */
  TFKT_F_CXX, TFKT_F_CXY, TFKT_F_CYY,   /* conformation ell^2 sum psi QQ / psi_tot */
  TFKT_F_THXX, TFKT_F_THXY, TFKT_F_THYY, /* stress (ell^2 / 2) sum psi Q F(Q) */
  TFKT_F_QRMS,        /* sqrt(<psi Q^2> / <psi>) in r-lengths (Sec. VII) */
  TFKT_F_VORT,        /* d_x U_y - d_y U_x, central differences */
  TFKT_NFIELDS
};

/* Global diagnostics of tfkt_diagnostics. MASS_S..EY2 are FP64 sums over all
   r-nodes (QRMS_MEAN the mean); the last two are maxima over the r-nodes:
   TFKT_D_U2_MAX holds max |u| (its square is what is reduced), a guard on the
   low-Mach condition |u| << c_s = 1/sqrt(3) under which the D2Q9 equilibrium
   of Sec. VI A holds, and TFKT_D_QRMS_MAX the largest local Q_rms (Sec. VII).
   A maximum meets a NaN node as NaN. */
enum {
  TFKT_D_MASS_S = 0, TFKT_D_MASS_P, TFKT_D_PX, TFKT_D_PY, TFKT_D_KE,
  TFKT_D_ENSTROPHY, TFKT_D_QRMS_MEAN, TFKT_D_EY2, TFKT_D_U2_MAX, TFKT_D_QRMS_MAX,
  TFKT_NDIAG
};

/* Device bytes that tfkt_create needs for these parameters (two population
   buffers, the moment fields, scratch). EINVAL for invalid parameters. */
tfkt_status tfkt_required_bytes(const tfkt_params* p, size_t* bytes);

/* Create a context and its initial state (Sec. VI-D initial condition: psi is
   the equilibrium of the spring, the Gaussian for Hookean dumbbells or
   (1 - Q^2/Q0^2)^(b/2) for FENE ones, discretely normalised; g = f^eq).
   perturb: host array [2][ny][nx] of the initial velocity perturbation
            (u'_x plane then u'_y plane), or NULL; copied during the call.
   dev_workspace: device memory of at least tfkt_required_bytes bytes, owned
            by the caller and kept alive until tfkt_destroy; or NULL, and the
            library allocates (and frees in tfkt_destroy).
   stream:  cudaStream_t for all work of the context, or NULL.
   On success *out is the new context; on failure *out is NULL. */
tfkt_status tfkt_create(const tfkt_params* p, const double* perturb, void* dev_workspace,
                        size_t workspace_bytes, void* stream, tfkt_ctx** out);

/* Advance n >= 0 time steps. One step is the scheme of Sec. VI: pull-stream
   both lattices (Sec. VI-A, VI-B, bounce-back at the Q-disk, Sec. VI-D), take
   the moments, form the mixture velocity and the imposed velocities, convert g
   to f (Sec. VI-C), collide with the two-relaxation update and the body force
   of Sec. VII, and write the post-collision populations to the other buffer.
   Asynchronous on the context stream. Errors: TFKT_EINVAL if n < 0 (nothing
   launched); TFKT_ESTATE on a poisoned context; TFKT_ECUDA if a launch fails
   (the context is then poisoned). A NaN in the state is not an error here;
   tfkt_diagnostics reports it. */
tfkt_status tfkt_step(tfkt_ctx* ctx, int64_t n);

/* Same as tfkt_step, with CUDA events recorded on the context stream around
   every kernel launch; adds the elapsed time of each kernel kind, in
   milliseconds, to kernel_ms[TFKT_NKERNELS] (host) and the launch counts to
   launches[TFKT_NKERNELS] (host, may be NULL). The launches are queued without
   waiting in between; the host waits for the events once every 64 launches
   and at the end, so the call returns with the stream idle. */
tfkt_status tfkt_step_profiled(tfkt_ctx* ctx, int64_t n, double* kernel_ms, int64_t* launches);

/* Macroscopic fields of the current state (see TFKT_F_*: the moments of
   Sec. VI-A and VI-B, the mixture velocity of f of Sec. VI-C, the
   conformation and Q_rms of Sec. VII, the vorticity), as doubles, layout
   [field][ny][nx] in increasing bit order of field_mask. dst: device pointer
   if dst_is_device, else host pointer, owned by the caller; bytes is its size
   and must hold popcount(field_mask) * ny * nx doubles. Synchronises the
   stream when dst is host memory. Errors: TFKT_EINVAL for a NULL dst, an
   empty or out-of-range mask, or dst too small; TFKT_ESTATE / TFKT_ECUDA as
   for tfkt_step. */
tfkt_status tfkt_moments(tfkt_ctx* ctx, uint32_t field_mask, double* dst, size_t bytes,
                         int dst_is_device);

/* psi(x, q) = sum_i g_i(x, q) of the current state (Sec. VI-B, the
   conformation density on the Q-grid) as doubles, layout [ny][nx][nq]; dst
   and bytes as for tfkt_moments (nq * ny * nx doubles), same errors. */
tfkt_status tfkt_psi(tfkt_ctx* ctx, double* dst, size_t bytes, int dst_is_device);

/* Global diagnostics into host out[TFKT_NDIAG]; synchronises. TFKT_ENAN if
   any is not finite: out still holds all values, tfkt_last_error names the
   first non-finite one and the step, and the context stays usable (the state
   is neither changed nor reset). */
tfkt_status tfkt_diagnostics(tfkt_ctx* ctx, double* out);

/* The stored (post-collision, not yet streamed) populations g' of Sec. VI-C
   as doubles in host memory owned by the caller, layout [plane][ny][nx]:
   planes 0..8 solvent (tfkt_lattice order), then plane 9 + 25 q + i for the
   polymer; the storage shift (w_i for the solvent, w_i psi0(q) for the
   polymer) is added back. bytes must hold (9 + 25 nq) * ny * nx doubles.
   Allocates a temporary device buffer of that size. Synchronises. Errors:
   TFKT_EINVAL for a NULL or too small dst; TFKT_ESTATE / TFKT_ECUDA as for
   tfkt_step. */
tfkt_status tfkt_populations(tfkt_ctx* ctx, double* host_dst, size_t bytes);

/* Macroscopic fields without any device allocation. The paper has no
   counterpart of this call; it exists for callers that may not allocate GPU
   memory at the point where they need the fields: code inside a fixed-size
   memory arena or pool whose budget is already spoken for, or a host
   framework that forbids entering the allocator from that point. It computes
   the same fields as tfkt_moments from a population buffer the caller
   passes; its scratch (moment planes, velocity planes, lattice tables) is one
   static device array of TFKT_NOALLOC_SCRATCH_BYTES that every GPU loading
   the library holds until the process exits.
   p:      the run's parameters (as given to tfkt_create).
   pops:   device pointer to a population buffer in a context's storage
           layout. A context created on workspace W keeps its state, after
           n steps, at W + (n mod 2) * B with B = the population bytes
           rounded up to 256, but never less than TFKT_NFIELDS * ny * nx * 8
           bytes. After a learned block (tfkt_lpm_run) that buffer lacks the
           block's polymer increment, which waits for the context's next
           step; tfkt_populations and tfkt_save add it to the buffer. Until
           then this call gives the fields without the increment, where
           tfkt_moments gives them with it. The population bytes are (9 + 25 nq) * ny * pitch * e (nq,
           pitch from tfkt_get_info; e = 8 for TFKT_FP64, 4 for TFKT_FP32,
           2 for TFKT_FP16): planes 0..8 the solvent, 9 + 25 q + i the
           polymer; under TFKT_FP16 planes 0..8 are unused and the nine
           solvent planes follow as floats, 9 * ny * pitch * 4 bytes more.
   dst:    device pointer, popcount(field_mask) * ny * nx doubles; bytes is
           its size.
   stream: cudaStream_t or NULL. The kernels run asynchronously on the
           stream. The lattice tables are kept in the array with the
           parameters they belong to: the first call on a device, and a call
           whose parameters differ from those of the last upload, copies them
           from host memory and synchronises the stream before queuing the
           kernels; a call with the same parameters as the last upload only
           queues the kernels.
   Errors: TFKT_EINVAL for invalid parameters, pointers or mask, and when the
           grid needs more scratch than TFKT_NOALLOC_SCRATCH_BYTES (the
           message gives both sizes); TFKT_ECUDA if a CUDA call fails.
   The first call on a device looks up the address of the static array on
   that device (with the device current); make that first call before any
   stream capture. All calls share the one array, which keeps what the last
   call left in it; every moment and velocity value a call reads from it is
   written by the same call first, and the tables are re-uploaded whenever
   the parameters change, so nothing needs clearing. Calls whose work
   overlaps on the GPU (other streams, other threads) race on the array. */
#define TFKT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
tfkt_status tfkt_moments_noalloc(const tfkt_params* p, const void* pops, uint32_t field_mask,
                                 double* dst, size_t bytes, void* stream);

tfkt_status tfkt_get_info(const tfkt_ctx* ctx, tfkt_info* info);

/* Velocity ordering of the library: c9[9][2] (D2Q9), c25[25][4] (D4Q25 on
   r_x, r_y, Q_x, Q_y). Either pointer may be NULL. */
tfkt_status tfkt_lattice(int32_t* c9, int32_t* c25);

/* Wait for all work of the context. */
tfkt_status tfkt_sync(tfkt_ctx* ctx);

/* Checkpoint and restart. tfkt_save writes the current state to the file
   `path` (through `path`.part, renamed when complete): a header (the lattice
   parameters the state belongs to, the step count, sizes, a 64-bit checksum)
   and the raw current populations plus, where valid, the current moment
   planes. A pending learned-block increment is applied first. The file is
   about the size of one population buffer (54 GB at 4096^2, N_Q = 32, FP32).
   Synchronises. Allowed on a run of a batch.
   tfkt_load reads such a file into a context created with the same
   parameters (TFKT_EINVAL otherwise, nothing changed) and sets its step count;
   stepping on gives the trajectory of the run that was saved, bit for bit.
   TFKT_EIO: unreadable, not a checkpoint, truncated, trailing bytes or a
   checksum mismatch; if the payload was already being copied, the context is
   reset to its initial state (without perturbation). Not allowed on a run of
   a batch (TFKT_EINVAL). Synchronises. */
tfkt_status tfkt_save(tfkt_ctx* ctx, const char* path);
tfkt_status tfkt_load(tfkt_ctx* ctx, const char* path);

/* Release the context (and the workspace if the library allocated it).
   Synchronises first. NULL is accepted. */
tfkt_status tfkt_destroy(tfkt_ctx* ctx);

/* ---- Batched ensembles -------------------------------------------------
   Many independent Kolmogorov runs (their own grid size, Re, Wi, beta,
   forcing and seed) advanced together, replayed from a CUDA graph two steps at
   a time, in one of two plans: one launch of the batched fused kernel over the
   tiles of all runs plus one launch of its border fix-up per step; or each
   run's own single-run kernels as parallel branches of the graph (largest runs
   first, up to 32 branches). The paper runs one case at a time; batching is
   this library's addition. Requirements: every run uses TFKT_FP32 and has nx a
   multiple of 32 and ny a multiple of 8 (the fused path); otherwise
   TFKT_EINVAL. Under the per-run plan a run of the batch is bit-identical to
   the same run stepped alone; under the batched kernel it matches up to float
   rounding (that kernel sums some moments in another order). */
typedef struct tfkt_batch tfkt_batch;

/* Device bytes for the batch (the runs' workspaces and the launch tables). */
tfkt_status tfkt_batch_required_bytes(const tfkt_params* runs, int32_t n, size_t* bytes);

/* Create n runs. perturbs: n host pointers to [2][ny][nx] perturbations (or
   NULL entries, or perturbs NULL). dev_workspace/bytes as in tfkt_create. The
   batch uses the caller's stream if it is not NULL, else one it creates (a CUDA
   graph cannot capture the legacy default stream). Before the runs are
   initialised, the batch times four steps of each candidate plan (the batched
   kernel at each tile height, 4, 8 or 16 rows of 32 nodes, that every run
   supports, and the per-run plan), each as its captured graph, and keeps the
   fastest. The environment variable TFKT_BATCH_PER_RUN=1 fixes the per-run
   plan, and TFKT_BATCH_TILE_HEIGHT (4, 8 or 16) the batched kernel at that
   height (EINVAL if a run does not support it), instead of the timing. */
tfkt_status tfkt_batch_create(const tfkt_params* runs, int32_t n, const double* const* perturbs,
                              void* dev_workspace, size_t workspace_bytes, void* stream,
                              tfkt_batch** out);

/* Advance every run by n >= 0 steps of the scheme of tfkt_step
   (asynchronous on the batch stream). Errors: TFKT_EINVAL for a NULL batch or
   n < 0; TFKT_ECUDA if a launch or a graph launch fails. */
tfkt_status tfkt_batch_step(tfkt_batch* b, int64_t n);

/* The context of run i (0 <= i < n), for tfkt_moments, tfkt_diagnostics,
   tfkt_psi, tfkt_populations and tfkt_get_info; owned by the batch: do not
   call tfkt_step or tfkt_destroy on it. */
tfkt_status tfkt_batch_run(tfkt_batch* b, int32_t i, tfkt_ctx** run);

/* The batch's tile height (8 under the per-run plan, the single-run tile), and
   (ms: float[3] or NULL) the timed milliseconds per step of the batched kernel
   at heights 4, 8 and 16 (NaN where not timed). */
tfkt_status tfkt_batch_tile_height(const tfkt_batch* b, int32_t* ty, float* ms);

/* The chosen plan: *per_run 1 for each run's own kernels, 0 for the batched
   kernel at tile height *ty; ms (float[4] or NULL): the timed milliseconds per
   step at heights 4, 8, 16 and of the per-run plan (NaN where not timed). */
tfkt_status tfkt_batch_plan(const tfkt_batch* b, int32_t* per_run, int32_t* ty, float* ms);

/* Release the batch, its runs, streams and graph (and the workspace if the
   library allocated it). Synchronises first; NULL is accepted. */
tfkt_status tfkt_batch_destroy(tfkt_batch* b);

/* ---- Domain decomposition in y (slabs) ---------------------------------
   One run split into horizontal slabs, for example one per process or GPU.
   The paper runs one domain; the split is this library's addition. A slab
   context owns the global rows [y0, y0 + ny_local) of the run described by the
   params (which name the WHOLE run: its nx, ny, forcing and parameters) and
   computes TFKT_SLAB_GHOST ghost rows more on each side; it is an ordinary
   context of ny_local + 2 TFKT_SLAB_GHOST rows (tfkt_step, tfkt_moments,
   tfkt_psi, tfkt_populations, tfkt_diagnostics, tfkt_get_info and the
   checkpoint calls act on all of them, local row j holding global row
   (y0 - TFKT_SLAB_GHOST + j) mod ny), whose forcing and laminar profile are
   those of the global rows. One step of the scheme (Sec. VI) reads data at
   most three rows away, so the owned rows advance exactly as in the single-
   domain run as long as, before every step and after tfkt_slab_create, each
   side's ghost rows are replaced with the neighbour's current rows: pack the
   side on the neighbour, unpack it here. Slab k's TFKT_SLAB_HIGH pack goes to
   slab k+1's TFKT_SLAB_LOW unpack and slab k's TFKT_SLAB_LOW pack to slab
   k-1's TFKT_SLAB_HIGH unpack (periodic: the last slab's high neighbour is
   the first slab). The ghost width is one row of the fused path's 32 x 8
   tiles: with y0 and ny_local multiples of 8 (and nx of 32) every slab takes
   the fused path on tiles that are the single-domain run's tiles, so every
   owned node sums its arrivals in the same order and the owned rows are bit-
   identical to the single-domain run (the two-pass path is bit-identical for
   any split). The learned block does not run on a slab context (EINVAL). */
#define TFKT_SLAB_GHOST 8
enum { TFKT_SLAB_LOW = 0, TFKT_SLAB_HIGH = 1 };

/* Device bytes of a slab context with ny_local owned rows of the run p.
   EINVAL for invalid params or ny_local outside [TFKT_SLAB_GHOST, ny]. */
tfkt_status tfkt_slab_required_bytes(const tfkt_params* p, int32_t ny_local, size_t* bytes);

/* Create the slab of rows [y0, y0 + ny_local) of the run p (0 <= y0 < ny) and
   its initial state (as tfkt_create). perturb: host [2][ny_local + 2G][nx] (G =
   TFKT_SLAB_GHOST) of the whole run's perturbation at the global rows
   y0 - G ... y0 + ny_local + G - 1 (mod ny), or NULL; dev_workspace, bytes,
   stream and the errors as for tfkt_create. */
tfkt_status tfkt_slab_create(const tfkt_params* p, int32_t y0, int32_t ny_local,
                             const double* perturb, void* dev_workspace, size_t workspace_bytes,
                             void* stream, tfkt_ctx** out);

/* Bytes of one side's halo message: TFKT_SLAB_GHOST rows of every population
   plane (storage type; under FP16 storage also the FP32 solvent planes) and of
   every moment plane, packed plane after plane. EINVAL on a context that is
   not a slab. */
tfkt_status tfkt_slab_halo_bytes(const tfkt_ctx* ctx, size_t* bytes);

/* Copy the TFKT_SLAB_GHOST owned rows next to `side` of the current state into
   dst (bytes >= tfkt_slab_halo_bytes; device memory if dst_is_device, 16-byte
   aligned, else host memory; owned by the caller). A device message is written
   by one kernel queued on the context stream; host copies synchronise it.
   Errors: EINVAL for a non-slab context, an unknown side, NULL or too small dst,
   or a device dst that is not 16-byte aligned; ECUDA (context poisoned) if a
   copy fails. */
tfkt_status tfkt_slab_halo_pack(tfkt_ctx* ctx, int32_t side, void* dst, size_t bytes,
                                int dst_is_device);

/* Overwrite the TFKT_SLAB_GHOST ghost rows on `side` of the current state with
   a neighbour's packed rows (src, bytes, src_is_device as for the pack). The
   neighbour's pack must be complete (the same stream, an event, or a host
   buffer). Errors as for tfkt_slab_halo_pack. */
tfkt_status tfkt_slab_halo_unpack(tfkt_ctx* ctx, int32_t side, const void* src, size_t bytes,
                                  int src_is_device);

/* The slab's first owned global row, owned rows and ghost rows per side (any
   pointer may be NULL); EINVAL for a context that is not a slab. */
tfkt_status tfkt_slab_rows(const tfkt_ctx* ctx, int32_t* y0, int32_t* ny_local, int32_t* ghost);

/* Static one-line description of a status code ("ok", "invalid argument",
   ...; "unknown status" for other values); never NULL. */
const char* tfkt_status_string(tfkt_status s);
/* Text of the last error seen by this thread ("" if none). */
const char* tfkt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
