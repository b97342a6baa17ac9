/*
 * mc.h - C ABI of the GB300 filament-fluid step library (libmc.so).
 *
 * The library advances "worlds" of the Microcosmos model (arXiv 2607.02954):
 * elastic bead chains (filaments) immersed in a 2D periodic viscous fluid.
 * One time step (Methods and Fields sections, Fluid-filament Interaction):
 *   a1 rest-angle drive      theta_rest,j(t) = theta0_j + A_j sin(2 pi (freq_j t + phase_j))
 *   a2 cell / bin indexing   counting sort of beads by 8x8-cell bin (row-major)
 *   a3 PBD                   n_pbd x (bending pass Eq. 1, position pass Eqs. 2-4);
 *                            elastic force F_el = kappa (x_hat - X) / dt
 *   a4 steric deposit        rho_s(c) = sum_i delta_h(c - X_i)
 *   a5 Gaussian filter       rho_bar = G_sigma * rho_s (periodic, separable)
 *   a6 force + spread        F_s,i = -k_rep sum_c delta_h(c - X_i) grad rho_bar(c)
 *                            F(c)  = sum_i delta_h(c - X_i) (F_el,i + F_s,i)
 *   a7 D2Q9 TRT LBM          collide (Guo forcing) + periodic streaming -> f, u
 *   a8 IB interpolation      U_i = sum_c delta_h(c - X_i) u(c);  X += dt U (wrapped)
 * delta_h is Peskin's 4-point kernel.  All device arithmetic is FP32.
 *
 * Conventions shared by every call:
 *  - Every function returns mc_status.  MC_OK = 0.  On failure nothing is
 *    enqueued and mc_last_error() describes the problem (thread-local text).
 *    Nothing aborts the process.
 *  - Streams are CUDA streams (cudaStream_t, passed as void*); NULL means the
 *    legacy default stream.  Calls that take a stream are asynchronous on it
 *    unless stated otherwise.
 *  - Arrays passed in are copied; the caller keeps ownership.  mem_kind says
 *    whether a pointer argument is host (MC_MEM_HOST) or device (MC_MEM_DEVICE)
 *    memory.  Host input arrays may be reused as soon as the call returns.
 *  - Grids are row-major [y][x] with W cells per row; population arrays are
 *    [9][H][W] in the D2Q9 order c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),
 *    (-1,1),(-1,-1),(1,-1).
 *  - Filaments are linear chains: filament f owns beads fil_off[f] ..
 *    fil_off[f+1]-1 (2 to 3072 beads); it owns B_f - 1 edges and B_f - 2
 *    joints, numbered consecutively across filaments (edge e joins beads
 *    (a, a+1) of one filament; joint j sits between two consecutive edges).
 *    N = fil_off[n_fil], E = N - n_fil, J = N - 2 n_fil.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_ABI_VERSION 7

typedef enum mc_status {
  MC_OK = 0,
  MC_ERR_INVALID_ARG = 1,  /* a size, pointer or value failed validation */
  MC_ERR_OOM = 2,          /* device or host allocation failed */
  MC_ERR_CUDA = 3,         /* a CUDA runtime call failed (text in mc_last_error) */
  MC_ERR_TIMEOUT = 4,      /* a bounded wait gave up */
  MC_ERR_UNSTABLE = 5,     /* the velocity watchdog tripped (|U| too large or not finite) */
  MC_ERR_BUSY = 6,         /* result not ready yet / queue full */
  MC_ERR_NOT_FOUND = 7,    /* unknown ticket or handle */
  MC_ERR_CANCELLED = 8     /* the rollout was cancelled (mc_serve_cancel) */
} mc_status;

typedef enum mc_mem_kind { MC_MEM_HOST = 0, MC_MEM_DEVICE = 1 } mc_mem_kind;

/* World constants.  The paper names these quantities (Methods: k_bend,
 * k_shear, k_stretch per Eqs. 1-4; Fields: LBM relaxation tau, Gaussian
 * filter of the steric density) but fixes none of their values.
 *   nu       kinematic viscosity, tau+ = 3 nu + 1/2 (must give tau+ > 1/2)
 *   dt       bead advance step (the lattice time step is 1)
 *   Lambda   TRT magic parameter, tau- = 1/2 + Lambda / (tau+ - 1/2)
 *   kappa    penalty stiffness turning the PBD correction into a force
 *   k_bend, k_stretch, k_shear   PBD stiffnesses (Eqs. 1-4), in [0, 1]
 *   k_rep    steric repulsion strength
 *   sigma    Gaussian filter width in cells, 0 < sigma <= 2 (taps R = ceil(4 sigma))
 *   orient   1: the position pass also turns the edge frame toward the edge
 *            (Gauss-Newton step on |v - L d(theta)|^2); 0: positions only
 *   n_pbd    PBD iterations per step, 0 <= n_pbd <= 64
 *   pbd_order  0: Jacobi passes (every correction of a pass from the state
 *            before it); 1: red-black passes (within each pass the joints or
 *            edges of even index in their filament first, then the odd ones
 *            from the updated state: a two-colour Gauss-Seidel sweep).  The
 *            reverse mode supports both.
 *   layers   1: the beads are the immersed-boundary points; 2: two-layer
 *            filament (Fluid-filament Interaction): each bead couples to the
 *            fluid at X +- layer_half n (n the filament's unit normal at the
 *            bead), spreading half its force at each point and moving with
 *            the mean of the two interpolated velocities; 0 < layer_half <= 2
 *            cells.  The steric field stays on the beads.  The reverse mode
 *            supports both.
 *   ib       immersed-boundary coupling (Fluid-filament Interaction).
 *            0: penalty, F_el = kappa (x_hat - X)/dt spread as a force and
 *            the beads move with the interpolated fluid velocity.
 *            1: direct forcing with multi-direct-forcing (MDF) passes: the
 *            steric force acts on the fluid, the fluid velocity before the
 *            filament's forcing u* = (sum_i c_i f_i + F_s/2)/rho carries the
 *            beads to X~ = X + dt I[u*](X), PBD from X~ gives x_hat, and each
 *            bead takes the velocity U_s = I[u*](X) + (x_hat - X~)/dt; then
 *            mdf_iters passes force the fluid to follow it (per bead
 *            dF = 2 I[rho](X) (U_s - I[u](X)), F += S[dF], u += S[dF]/(2 rho)),
 *            the LBM steps with the total force and X^{n+1} = X + dt U_s.
 *            kappa is unused; needs layers = 1.  The reverse mode supports
 *            it (the passes, the drag and the moments reversed).
 *   mdf_iters  MDF passes per step with ib = 1, 0 <= mdf_iters <= 64 (0: the
 *            filament does not force the fluid). */
typedef struct mc_params {
  float nu, dt, Lambda, kappa, k_bend, k_stretch, k_shear, k_rep, sigma, orient;
  int n_pbd;
  int pbd_order;
  int layers;
  float layer_half;
  int ib;
  int mdf_iters;
} mc_params;

/* The paper's statement of one world (Methods: filaments as graphs with
 * per-edge orientation, rest length and rest angle; Fields: the grid).
 *   H, W        grid size, multiples of 8, 8 <= H, W <= 8192
 *   n_fil       number of filaments (>= 0), fil_off [n_fil + 1]
 *   x, y        [N] bead positions (any finite value; wrapped into the box)
 *   theta       [E] edge orientation angles (radians, not wrapped)
 *   L_rest      [E] rest lengths (> 0)
 *   theta0      [J] static part of the rest angles
 *   drive_amp, drive_freq, drive_phase  [J] rest-angle drive: amplitude
 *               (rad), frequency (cycles per step), phase (cycles)
 *   f0          [9][H][W] initial populations minus the rest weights w_i
 *               (pre-collision, as returned by mc_world_get_state); NULL =
 *               fluid at rest (f = w_i)
 *   t0          initial step counter (0 <= t0 < 2^24)
 *   p           constants
 *   mem_kind    where the array pointers live (fil_off always host memory)
 * Optional, NULL = absent (the Neuroevolution and QD Search experiments):
 *   len_amp, len_freq, len_phase  [E] rest-length drive, all three or none:
 *               L_rest(t) = L_rest (1 + len_amp sin(2 pi (len_freq t +
 *               len_phase))), the controller's rest-length output; |len_amp| < 1
 *   energy      [H][W] persistent scalar energy field (Gaussian packets in the
 *               paper), sampled at every bead each step with the
 *               interpolation kernel
 *   observe     1: accumulate the behaviour descriptors and the collected
 *               energy every step (see mc_world_get_observables); 0: off */
typedef struct mc_world_desc {
  int H, W;
  int n_fil;
  const int* fil_off;
  const float* x;
  const float* y;
  const float* theta;
  const float* L_rest;
  const float* theta0;
  const float* drive_amp;
  const float* drive_freq;
  const float* drive_phase;
  const float* f0;
  int64_t t0;
  mc_params p;
  int mem_kind;
  const float* len_amp;
  const float* len_freq;
  const float* len_phase;
  const float* energy;
  int observe;
} mc_world_desc;

typedef struct mc_world mc_world;

typedef struct mc_world_info {
  int H, W, n_fil, N, E, J;
  int bin_edge, n_bins;  /* bin edge in cells (8) and number of bins (H W / 64) */
  int64_t t;             /* step counter after all enqueued steps */
  size_t device_bytes;   /* device memory held by the world */
} mc_world_info;

/* Fills p with the library's default constants. */
mc_status mc_params_default(mc_params* p);

/* Creates a world: validates the description, allocates its device memory
 * (one stream-ordered allocation on `stream`, freed by mc_world_destroy),
 * copies the inputs and enqueues the set-up kernels on `stream`.
 * Errors: MC_ERR_INVALID_ARG (sizes, non-finite values, filaments with fewer
 * than 2 beads, tau+ <= 1/2), MC_ERR_OOM, MC_ERR_CUDA. */
mc_status mc_world_create(const mc_world_desc* desc, void* stream, mc_world** out);

/* Releases a world.  Work already enqueued on the world must be complete or
 * ordered before the stream the world was created on. */
mc_status mc_world_destroy(mc_world* w);

/* Checkpoint and resume (a library service; the paper has no counterpart).
 * mc_world_save writes an image of the world after the work enqueued on
 * `stream` (every field of its state: beads, angles, drives, populations,
 * bins, step counter, observables, optional fields) into a host buffer of
 * at least mc_world_save_size bytes, and synchronizes `stream`.  The image
 * holds no recorded rollout (mc_rollout_forward's checkpoints).
 * mc_world_load creates a world from such an image (its memory allocated on
 * `stream`, which it synchronizes before returning); stepping it continues
 * the saved world bitwise.  Errors: MC_ERR_INVALID_ARG (NULL, a buffer too
 * small, an image that is corrupt or from another C ABI version),
 * MC_ERR_OOM, MC_ERR_CUDA. */
mc_status mc_world_save_size(const mc_world* w, size_t* bytes);
mc_status mc_world_save(const mc_world* w, void* buf, size_t bytes, void* stream);
mc_status mc_world_load(const void* buf, size_t bytes, void* stream, mc_world** out);

mc_status mc_world_info_get(const mc_world* w, mc_world_info* out);

/* Advances one world by n_steps >= 0 time steps (a1..a8 each), enqueued on
 * `stream`.  Steps are replayed from a captured CUDA graph.  Asynchronous:
 * the velocity watchdog result is read with mc_world_check. */
mc_status mc_step(mc_world* w, int n_steps, void* stream);

/* Advances n_worlds distinct worlds of any sizes by n_steps each, every
 * kernel covering all worlds at once (one launch per stage per step).
 * Results are bitwise identical to advancing each world alone with mc_step.
 * worlds is a host array of n_worlds distinct handles. */
mc_status mc_step_batched(mc_world* const* worlds, int n_worlds, int n_steps, void* stream);

/* ---- Launch configuration and autotuner -----------------------------------
 * The steps of a plan (one world, or one batch of worlds as passed to
 * mc_step_batched) can run in several launch configurations, all of which
 * advance the worlds bitwise the same:
 *   persistent    0: the stage kernels (one launch per stage per step,
 *                 covering every world), replayed from a captured CUDA
 *                 graph of 16 steps; 3 or 4: one persistent cooperative
 *                 launch per run of steps with that many blocks per SM, the
 *                 stages separated by grid-wide barriers (plans without
 *                 direct forcing or two layers, filaments of at most 64
 *                 beads, sigma in (0.75, 1]).  Each barrier wait is bounded
 *                 (1 s); when it runs out the kernel ends and the worlds'
 *                 check reports MC_ERR_TIMEOUT (their state is then
 *                 unspecified).
 *   pbd_warps     most filaments per block of the PBD kernels: 8, 4 or 2
 *   scan_kernels  0: one bin-offset kernel when every world's bins fit one
 *                 scan block (1024 bins), else two; 2: always two
 *   force_kernel  0: the fused force + LBM kernel with one 32x32 tile per
 *                 block; 1: its warp-specialised persistent form (half of
 *                 each block's warps run a tile's force phase while the
 *                 other half collide the previous tile; worlds without two
 *                 layers)
 * The autotuner measures the candidates on device copies of the plan's
 * worlds (the worlds do not move) and caches its choice per class of plan
 * (world count, sizes, tile and bead counts) for the life of the process.
 * By default the first mc_step / mc_step_batched of at least 16 steps of a
 * plan looks the class up and, when it is not cached yet, tunes it then,
 * which synchronizes `stream` (single worlds below 2^20 cells and 2^18 beads
 * keep the defaults unless tuned explicitly; nothing is measured while
 * `stream` is being captured).  The plan of a batch is the one
 * mc_step_batched caches for that exact list of handles. */
typedef struct mc_launch_config {
  int persistent;     /* 0, 3 or 4 */
  int pbd_warps;      /* 8, 4 or 2 */
  int scan_kernels;   /* 0 or 2 */
  int force_kernel;   /* 0 or 1 */
} mc_launch_config;

/* Tunes the plan of worlds[0..n_worlds) now (or takes its class's cached
 * choice) and returns the configuration in *chosen (may be NULL).
 * Synchronizes `stream`; needs device memory for a copy of the worlds (if
 * it cannot get it, the defaults stay).  Errors: MC_ERR_INVALID_ARG. */
mc_status mc_autotune(mc_world* const* worlds, int n_worlds, void* stream, mc_launch_config* chosen);

/* The configuration the plan of worlds[0..n_worlds) runs with. */
mc_status mc_launch_config_get(mc_world* const* worlds, int n_worlds, mc_launch_config* out);

/* Pins the configuration of the plan of worlds[0..n_worlds) (no tuning
 * afterwards).  Errors: MC_ERR_INVALID_ARG for a value out of range or a
 * persistent step on a plan it does not support. */
mc_status mc_launch_config_set(mc_world* const* worlds, int n_worlds, const mc_launch_config* cfg);

/* 1 (default): the first run of at least 16 steps of an untuned plan tunes
 * it as described above; 0: plans keep the defaults unless mc_autotune is
 * called.  Process-wide. */
mc_status mc_autotune_mode(int mode);

/* Test support for the bounded barrier of the persistent step (process-wide;
 * defaults 0 and 1 s): each barrier waits for extra_arrivals (0 or 1) more
 * blocks than the launch has, and gives up after timeout_ns (1e3 to 1e10).
 * With 1 no barrier completes, so a persistent run ends at its first
 * barrier with the timeout reported; nothing else changes. */
mc_status mc_debug_barrier_test(unsigned extra_arrivals, int64_t timeout_ns);

/* Enqueues one stage of the next step on `stream` (for per-stage timing).
 * Stages: 0 drive + PBD + elastic force + bin histogram (a1-a3), 1 bin
 * offsets (one kernel, or two when the bins span several scan blocks),
 * 2 bin scatter (a2), 3 steric deposit + x pass of
 * the Gaussian filter (a4, a5), 7 y pass + steric force + spread + LBM
 * (a5-a7, one kernel, the force density handed to the collision in shared
 * memory), 6 interpolation + advance (a8).  Enqueuing stages 0, 1, 2, 3, 7, 6
 * in that order is exactly one mc_step(w, 1) without the graph.  Stages 4
 * (y pass + steric force + spread, writes F) and 5 (LBM, reads F) are stage 7
 * split in two kernels with F through device memory; 0, 1, 2, 3, 4, 5, 6
 * give the same step bitwise.  Any other use leaves the world in an
 * unspecified state.  The step counter advances with stage 6.  Errors:
 * MC_ERR_INVALID_ARG for an unknown stage or a world with ib = 1 (its
 * step has more stages; mc_step runs them). */
mc_status mc_step_stage(mc_world* w, int stage, void* stream);
#define MC_N_STAGES 8

/* Copies the state after the enqueued steps.  Any output may be NULL.
 *   x, y      [N] wrapped bead positions
 *   theta     [E] edge angles
 *   disp      [2N] interleaved (dx, dy) unwrapped displacement since creation
 *   fdev      [9][H][W] pre-collision populations minus the rest weights w_i
 * Outputs live in mem_kind memory.  With MC_MEM_HOST the call synchronizes
 * `stream` before returning. */
mc_status mc_world_get_state(const mc_world* w, float* x, float* y, float* theta, float* disp,
                             float* fdev, int mem_kind, void* stream);

/* Allocation-free read-out of the bead positions into host memory.
 * The paper has no counterpart: this is a library service.  It returns the
 * same x, y as mc_world_get_state, for callers that cannot allocate device
 * memory while reading results (mc_world_get_state allocates a device
 * staging buffer per call): processes whose device memory is fully reserved
 * by another allocator or capped by a fixed budget, and latency-critical
 * loops where cudaMalloc / cudaFree may synchronize the device.
 *   x, y    [N] host buffers (pageable or pinned) receiving wrapped positions
 *   stream  the call enqueues a kernel and two copies on it, then
 *           synchronizes it before returning
 * Staging uses a file-scope device array sized for 2^20 beads (8 MiB) that
 * every GPU loading the library holds until the process exits.  The first
 * call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream
 * capture.  All calls share the array: calls whose GPU work overlaps (for
 * example on different streams) race on it.
 * Errors: MC_ERR_INVALID_ARG for NULL arguments or a world with more than
 * 2^20 beads (nothing is enqueued), MC_ERR_CUDA for a failed CUDA call. */
mc_status mc_world_get_positions_noalloc(const mc_world* w, float* x, float* y, void* stream);

/* Fields of the last completed step, for inspection and parity tests. */
typedef enum mc_field {
  MC_FIELD_FEL = 0,      /* [2N] elastic force per bead (a3); with ib = 1 the summed MDF force per bead */
  MC_FIELD_FS = 1,       /* [2N] steric force per bead (a6) */
  MC_FIELD_UBEAD = 2,    /* [2N] interpolated velocity per bead (a8); with ib = 1 the bead velocity U_s */
  MC_FIELD_RHO_S = 3,    /* [H*W] deposited steric density (a4), recomputed on request */
  MC_FIELD_RHO_BAR = 4,  /* [H*W] filtered density (a5), recomputed on request */
  MC_FIELD_FORCE = 5,    /* [2*H*W] interleaved (Fx, Fy) spread force density (a6), recomputed on request
                            (with ib = 1 the step's total force, steric spread plus MDF passes) */
  MC_FIELD_U = 6,        /* [2*H*W] interleaved (ux, uy) fluid velocity (a7) */
  MC_FIELD_CELL = 7,     /* [N] int32 cell index (floor(y) mod H) W + (floor(x) mod W) (a2) */
  MC_FIELD_BIN = 8,      /* [N] int32 bin index (floor(y)/8) (W/8) + floor(x)/8 of each bead (a2) */
  MC_FIELD_BIN_OFF = 9,  /* [n_bins + 1] int32 exclusive prefix sum of beads per bin (a2) */
  MC_FIELD_BIN_BEADS = 10, /* [N] int32 bead ids in bin order (order inside a bin unspecified) */
  MC_FIELD_EBEAD = 11    /* [N] energy sampled at each bead in the last step (observe and energy set) */
} mc_field;

/* Copies one field (see mc_field for its size and type) into `out`. */
mc_status mc_world_get_field(const mc_world* w, int field, void* out, int mem_kind, void* stream);

/* Synchronizes `stream` and reads the world's watchdog: MC_OK, or
 * MC_ERR_UNSTABLE when some step saw a non-finite or too large bead velocity
 * (the flag stays set until mc_world_clear_flags). */
mc_status mc_world_check(const mc_world* w, void* stream);
mc_status mc_world_clear_flags(mc_world* w, void* stream);

/* Search-side observables accumulated since creation (worlds created with
 * observe = 1; zeros otherwise), QD Search and Neuroevolution experiments:
 *   out[0] E_bend = sum over steps t >= 1 and joints of (theta_rest(t-1) -
 *          theta_rest(t))^2  (Eq. 5)
 *   out[1] E_pos  = sum over steps t >= 1 and edges of (L_rest(t-1) -
 *          L_rest(t))^2  (Eq. 6; zero without a rest-length drive)
 *   out[2] energy collected = sum over steps and beads of the energy field
 *          at the bead's position at the start of the step
 * t is the world's step counter when the step starts.  The sums are kept in
 * 64-bit fixed point: each warp's per-step partial sum (32 beads, or one
 * filament's joints and edges) is rounded to 2^-24, so the totals are
 * bitwise the same alone, batched or served, and exact while below 5.5e11.
 * out: 3 host doubles; the call synchronizes `stream`. */
mc_status mc_world_get_observables(const mc_world* w, double* out, void* stream);

/* ---- Reverse mode ----------------------------------------------------------
 * The Filament Folding experiment (Experiments section) optimises rest
 * angles by gradients that flow through the whole simulation.  Here the
 * gradient of a loss on the final unwrapped bead positions with respect to
 * theta0 (the static rest angles) is computed by a hand-written adjoint of
 * every stage, with checkpoint-and-recompute: the forward stores the state
 * every ckpt_every steps, the backward re-runs one segment at a time from
 * its checkpoint and reverses it step by step.  Device memory: one state
 * record (16 N + 4 E + 36 H W bytes) per checkpoint and per step of one
 * segment, plus adjoint buffers of about 150 bytes per cell; with direct
 * forcing each step of the segment also keeps 8 H W bytes per MDF pass,
 * 4 H W and 8 N, and the adjoint about 60 bytes more per cell. */

/* Advances the world n_steps >= 1 steps (like mc_step) recording
 * checkpoints every ckpt_every >= 1 steps.  Errors: MC_ERR_INVALID_ARG,
 * MC_ERR_OOM, MC_ERR_CUDA. */
mc_status mc_rollout_forward(mc_world* w, int n_steps, int ckpt_every, void* stream);

/* Advances the world n_steps >= 1 steps like mc_rollout_forward and stores
 * every step's record (its start state and the intermediates the reverse
 * mode reads), so the next mc_rollout_backward reverses the steps without
 * re-running any of them: memory for compute.  The steps run the unfused
 * stages (the same results bitwise).  Device memory per step: 32 N + 4 E
 * + 56 H W bytes (+ 8 N with two layers; with direct forcing + 8 H W per MDF
 * pass (at least one), 4 H W and 8 N), plus two state records.
 * mc_rollout_rewind, mc_world_set_rest and both backward calls work as
 * after mc_rollout_forward.  Errors: MC_ERR_INVALID_ARG (n_steps < 1, the
 * step counter would reach 2^24), MC_ERR_OOM, MC_ERR_CUDA. */
mc_status mc_rollout_forward_stored(mc_world* w, int n_steps, void* stream);

/* Returns the world to the start of the last mc_rollout_forward (its first
 * checkpoint, displacement, observables and step counter), so an
 * optimisation loop can re-run the same rollout with new parameters on the
 * same world: its buffers and its captured reverse sweep are reused.  The
 * recorded rollout stays; a backward needs a new forward first.  Errors:
 * MC_ERR_INVALID_ARG when no rollout was recorded. */
mc_status mc_rollout_rewind(mc_world* w, void* stream);

/* Replaces the static rest angles theta0 [J] and/or the rest lengths L_rest
 * [E] (the quantities the folding optimisation and the searches change);
 * either may be NULL.  Arrays in mem_kind memory; host arrays are checked
 * (finite, L_rest > 0) and the call synchronizes `stream`; device arrays are
 * used as given.  With a rest-length drive the new L_rest is its L0. */
mc_status mc_world_set_rest(mc_world* w, const float* theta0, const float* L_rest, int mem_kind, void* stream);

/* Reverse sweep of the last mc_rollout_forward.  dL_dx, dL_dy: [N] device
 * arrays, the loss gradient with respect to the final unwrapped positions
 * (creation position + displacement).  Writes dL_dtheta0 [J] (device).
 * The world ends in the final state of the rollout.  The sweep is captured
 * as a CUDA graph on first use and replayed while the rollout length,
 * checkpoint spacing, start step and buffers stay the same.  Errors:
 * MC_ERR_INVALID_ARG when no rollout was recorded or the world was stepped
 * since, or when filaments are too long for the adjoint kernel. */
mc_status mc_rollout_backward(mc_world* w, const float* dL_dx, const float* dL_dy, float* dL_dtheta0, void* stream);

/* As mc_rollout_backward, and also the gradients with respect to the
 * physical parameters the paper's searches act on (Methods, Filaments:
 * rest lengths and stiffnesses; the CPPN of the Neuroevolution experiment
 * outputs L_rest):
 *   dL_dL_rest [E] (device, may be NULL): with respect to each edge's rest
 *              length;
 *   dL_dk      [3] (device, may be NULL): with respect to k_bend,
 *              k_stretch, k_shear of the world.
 * The stiffness gradients are sums over all edges, joints, passes and steps,
 * added per filament and then over filaments in a fixed order.  Every
 * gradient of the reverse mode is bitwise repeatable: its scatters sum in
 * 64-bit fixed point.  Errors as mc_rollout_backward. */
mc_status mc_rollout_backward_params(mc_world* w, const float* dL_dx, const float* dL_dy, float* dL_dtheta0,
                                     float* dL_dL_rest, float* dL_dk, void* stream);

/* Folding loss with a polyline target (device arrays): loss[0] = mean over
 * beads of the squared distance from the unwrapped position to the nearest
 * segment of the polyline poly_xy [n_vertices][2]; dL_dx, dL_dy [N] its
 * gradient.  loss is one device float (written; summed in a fixed order, so
 * bitwise repeatable). */
mc_status mc_loss_polyline(mc_world* w, const float* poly_xy, int n_vertices, float* loss, float* dL_dx,
                           float* dL_dy, void* stream);

/* The paper's folding loss (Filament Folding experiment): mean squared
 * error between the Gaussian-splatted bead density of the world's current
 * positions and target [R][R] (device, row-major, row = y), an image of
 * R x R pixels covering the periodic domain.  Pixel (px, py) is centred at
 * ((px + 1/2) W/R, (py + 1/2) H/R); a bead at image coordinates
 * u = (X R/W, Y R/H) adds exp(-|c - u|^2 / (2 sigma^2)) (sigma in pixels) to
 * the pixels c with px in floor(u_x) - K .. floor(u_x) + K and likewise py,
 * periodic, K = ceil(4 sigma); no normalisation.  loss: one device float;
 * dL_dx, dL_dy [N] (device): its gradient with respect to the positions,
 * the input of mc_rollout_backward.  The image is accumulated in 64-bit
 * fixed point, so the loss is bitwise repeatable.  8 <= R <= 1024,
 * 0 < sigma <= 4.  Allocates R^2 * 12 bytes of scratch for the call. */
mc_status mc_loss_splat(mc_world* w, const float* target, int R, float sigma, float* loss, float* dL_dx,
                        float* dL_dy, void* stream);

/* ---- Rollout serving: continuous batching ---------------------------------
 * Search loops (the paper's Neuroevolution and QD Search experiments,
 * Experiments section) request rollouts as they go and read back a fitness,
 * the mean displacement of the world's beads.  A server owns a scheduler
 * thread and two CUDA streams (steps, world creation) on the device current
 * at creation.  Requests wait in a queue until a slot is free and their
 * device footprint fits the budget (a lone request larger than the budget is
 * still admitted when nothing else runs); all admitted worlds advance
 * together through the batched kernels, steps_per_tick steps at a time (one
 * tick); a finished world leaves the batch at once and is published, and its
 * memory released, when its last tick has completed on the device, which
 * admits waiting requests.  The scheduler enqueues up to two ticks ahead of
 * the device.  Results are bitwise the same as running the world alone. */
typedef struct mc_server mc_server;

typedef struct mc_server_cfg {
  size_t hbm_budget_bytes;  /* device memory the admitted worlds may hold */
  int max_slots;            /* most worlds advanced at once (>= 1) */
  int steps_per_tick;       /* steps between admission / retirement points (>= 1) */
  int max_pending;          /* queue capacity; submit returns MC_ERR_BUSY beyond it */
} mc_server_cfg;

typedef struct mc_result {
  double com_disp[2];       /* mean unwrapped bead displacement after n_steps */
  double e_bend, e_pos;     /* behaviour descriptors over the rollout (Eqs. 5, 6; observe set) */
  double energy;            /* energy collected over the rollout (observe and energy set) */
  int status;               /* MC_OK, MC_ERR_UNSTABLE, or the world's creation error */
  int n_steps;
  int64_t t_submit_ns;      /* steady-clock times of submit, admission, completion */
  int64_t t_admit_ns;
  int64_t t_done_ns;
} mc_result;

typedef struct mc_server_stats {
  int64_t submitted, completed, steps_run, ticks, pending;
} mc_server_stats;

/* Starts a server (thread + stream).  Errors: MC_ERR_INVALID_ARG for
 * non-positive settings, MC_ERR_CUDA. */
mc_status mc_server_create(const mc_server_cfg* cfg, mc_server** out);

/* Queues one rollout of n_steps >= 1 steps of the described world.  The
 * description's arrays are copied before the call returns (device arrays
 * with a synchronous copy).  Validation of sizes happens here
 * (MC_ERR_INVALID_ARG); value checks happen at admission and show up in the
 * result's status.  MC_ERR_BUSY when the queue is full. */
mc_status mc_serve_submit(mc_server* s, const mc_world_desc* desc, int n_steps, uint64_t* ticket);

/* Non-blocking: MC_OK and the result (once; the ticket is then forgotten),
 * MC_ERR_BUSY while pending or running, MC_ERR_NOT_FOUND otherwise. */
mc_status mc_serve_poll(mc_server* s, uint64_t ticket, mc_result* out);

/* Blocks up to timeout_ms: MC_OK, MC_ERR_TIMEOUT or MC_ERR_NOT_FOUND. */
mc_status mc_serve_wait(mc_server* s, uint64_t ticket, int timeout_ms, mc_result* out);

mc_status mc_server_stats_get(mc_server* s, mc_server_stats* out);

/* Cancels a rollout that is queued or running.  A queued request leaves the
 * queue at once; a running one leaves the batch at the scheduler's next
 * tick (its world is freed once the device has finished the ticks that used
 * it), so the rollouts around it continue unchanged.  Its result is then
 * published with status MC_ERR_CANCELLED (collect it with poll or wait;
 * com_disp and the observables are zero), unless the rollout completed in
 * a tick the scheduler had already enqueued, in which case its normal
 * result stands.  Returns MC_OK when the ticket was queued or running,
 * MC_ERR_NOT_FOUND when it is unknown, finished (its result stays
 * collectable) or collected. */
mc_status mc_serve_cancel(mc_server* s, uint64_t ticket);

/* Test support for the allocation-failure path (host side only; nothing is
 * done on the device).  Arms a fake of the world allocation: the nth world
 * allocation from now (1 = the next; mc_world_create's arena, including the
 * worlds a server's scheduler creates) reports an out-of-memory failure as
 * cudaMallocAsync would, without calling it, and that creation returns
 * MC_ERR_OOM (a served request reports it in its result's status).  Other
 * allocations are real.  0 disarms.  Process-wide.  Errors:
 * MC_ERR_INVALID_ARG for nth < 0. */
mc_status mc_inject_world_alloc_failure(int nth);

/* Stops the scheduler, drops queued requests and frees everything.  No
 * other call on this server may run concurrently or afterwards. */
mc_status mc_server_destroy(mc_server* s);

/* Thread-local description of the last error of this thread. */
const char* mc_last_error(void);
int mc_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
