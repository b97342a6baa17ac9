// Internal types and device helpers of libmc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mc.h"

namespace mc {

// Beads are counting-sorted by 8x8-cell bins (row-major over the bin grid);
// the steric kernels work on 32x32-cell tiles.  Grid sizes are multiples of
// 8, so bins are never ragged and ragged last tiles are at least 8 cells
// wide.
constexpr int kBin = 8;
constexpr int kTile = 32;
constexpr int kScanChunk = 1024;    // bins per block of the offset scan
constexpr int kMaxR = 8;            // Gaussian half width ceil(4 sigma) <= 8
constexpr int kBeadChunk = 256;     // beads per block of the bead-parallel kernels
constexpr int kCellChunk = 256;     // cells per block of the LBM kernel
constexpr int kMaxNpbd = 64;

// Deposition accumulates in int32 fixed point in shared memory: integer adds
// commute, so every deposited field is bitwise independent of the order in
// which beads arrive (alone, batched or served).  Each tile picks a
// power-of-two scale 2^k from a bound B on its largest cell sum of |terms|
// (B 2^k < 2^30, k in [8, 40]), so no sum can overflow; the bound and hence
// the scale depend only on the data.

enum : unsigned {
  kFlagUnstable = 1u,   // the velocity watchdog tripped
  kFlagTimeout = 2u     // a grid barrier of the persistent step, or a wait for bulk copies, ran out of time
};

// Everything the kernels need to know about one world.  Lives in device
// memory as one entry of a world table; all pointers are device pointers.
struct WorldDev {
  int H, W, N, E, J, n_fil;
  int nbx, nby, n_bins;             // 8x8 bins
  int ntx, nty, n_tiles;            // 32x32 tiles
  int n_chunks;                     // scan blocks over the bins
  int R, n_pbd, pbd_order;
  float dt, kappa_dt, k_bend, k_st, k_sh, k_rep, orient;
  float om_p, om_m, src_p, src_m;   // 1/tau+-, 1 - 1/(2 tau+-)
  float u_max;                      // watchdog threshold on |U|
  float taps[2 * kMaxR + 1];
  const int* fil_off;     // [n_fil + 1]
  float4* pos;            // [N]  (frac x, frac y, int cell x, int cell y)
  float2* disp;           // [N]
  float2* pos0;           // [N] positions at creation (unwrapped position = pos0 + disp)
  float* theta;           // [E]
  const float* L_rest;    // [E]
  const float4* drive;    // [J]  (theta0, amp, freq, phase)
  float2* fel;            // [N]
  float2* fs;             // [N]
  float2* ubead;          // [N]
  int* bead_bin;          // [N]
  int* bin_count;         // [n_bins]
  int* bin_off;           // [n_bins + 1]
  int* bin_cursor;        // [n_bins]
  int* chunk_sum;         // [n_chunks]
  float4* spos;           // [N] positions in bin order
  float4* srec;           // [N] per bead in bin order: F_el (x, y), bead id (int bits), 0
  float* g[2];            // [9 * H * W] post-collision population deviations (ping-pong)
  float2* F;              // [H * W]
  float2* u;              // [H * W]
  float* rho_s;           // [H * W] (written only on request)
  float* rho_x;           // [H * W] x-filtered density
  float* rho_b;           // [H * W] (written only on request)
  float* tile_rho_max;    // [n_tiles] bound of each tile's rho_s (largest deposited sum + its rounding; 0 iff no bead reaches the tile)
  long long* t;           // step counter
  unsigned* fel_max;      // [2] largest |F_el| component of the step, by step parity (float bits)
  unsigned* flags;        // watchdog flags
  // optional inputs and search-side observables
  int has_ldrive, has_energy, observe;
  int layers;             // 1 or 2 (two-layer filament)
  float layer_half;       // half distance between the layers (cells)
  int ib, mdf_iters;      // coupling (0 penalty, 1 direct forcing) and MDF passes per step
  float* mrho;            // [H * W] fluid density of the step (ib == 1)
  int* bead_slot;         // [N] slot of each bead in the bin-ordered arrays (ib == 1, else nullptr)
  float2* u2;             // [H * W] second velocity buffer: MDF passes alternate u -> u2 -> u (ib == 1)
  float2* sus;            // [N] U_s in bin order (ib == 1)
  float2* nrm;            // [N] filament unit normal at each bead (layers == 2)
  unsigned long long* facc;  // [2 H W] fixed-point spread of the layer points (layers == 2)
  const float4* ldrive;   // [E] (L0, amp, freq, phase) rest-length drive, or nullptr (static L_rest)
  const float* energy;    // [H * W] energy field, or nullptr
  float* ebead;           // [N] energy sampled at each bead (observe and energy)
  unsigned long long* obs;  // [3] E_bend, E_pos, energy collected, fixed point 2^-24 (two's complement)
  // reverse mode: where an unfused PBD records the positions and edge angles
  // it starts from (nullptr outside the reverse sweep's recompute)
  float4* rec_pos;        // [N]
  float* rec_theta;       // [E]
};

// Fixed-point scale of the observable sums (units of 2^-24): a warp's
// per-step sum is rounded to the unit, and a world's total stays exact
// while below 2^63 units (5.5e11).
constexpr float kObsScale = 16777216.0f;

// Adjoint buffers of one world (reverse-mode sweep), all device pointers.
struct AdjDev {
  float2* adjX;            // [N] adjoint of the bead positions
  float* adjTh;            // [E] adjoint of the edge angles
  float* gth0;             // [J] accumulated gradient with respect to theta0
  float* gL;               // [E] accumulated gradient with respect to L_rest
  float* gk;               // [3] accumulated gradient with respect to k_bend, k_stretch, k_shear
  const float* adjG_next;  // [9 H W] adjoint of the populations after the step
  float* adjG_cur;         // [9 H W] adjoint of the populations before it
  unsigned long long* ubar;  // [2 H W] adjoint of the fluid velocity, 64-bit fixed point (x, y interleaved)
  float2* Fbar;            // [H W] adjoint of the force density
  unsigned long long* Q;   // [2 H W] spread of the steric-force adjoint, 64-bit fixed point
  float* rsb;              // [H W] adjoint of rho_s
  float2* fbt;             // [N] adjoint of F_el + F_s per bead
  float2* dbar;            // [N] adjoint of the PBD correction
  const float* theta_n;    // [E] edge angles at the start of the step
  float2* nbar;            // [N] adjoint of the filament normal at each bead (two-layer worlds)
  const float2* nrm;       // [N] the step's filament normals (two-layer worlds)
  unsigned* amax;          // [3] bounds of the fixed-point sums (float bits): max |dt X_bar| by step
                           // parity (slots 0, 1), max |F_bar| (slot 2)
  float* gkf;              // [3 n_fil] per-filament sums of the stiffness gradients
  int par;                 // parity of the step being reversed (the slot of amax its u_bar reads)
  const float4* xt;        // [N] direct forcing: the positions the PBD started from (X~); NULL: X^n
  float2* xtb;             // [N] direct forcing: the PBD's adjoint of X~ through its edge vectors
  long long t_step;        // the reversed step's counter value (read instead of the world's when setup != 0)
  int setup;               // 1: k_adj_spread_u clears this step's bound slots, k_adj_pbd reads t_step
};

// Reverse-mode buffers of a direct-forcing step (k_adj_mdf.cu): the step's
// record (the passes' input velocities, the density, U_s) and the pass
// adjoints.
struct AdjMdf {
  int m;                       // MDF passes per step
  const float2* mu;            // [max(m, 1) H W] input velocity of pass k (u_0 = u* of the moments)
  const float* rho;            // [H W] density of the moments
  const float2* Us;            // [N] the beads' velocity U_s
  float2* Gbar;                // [H W] adjoint of a pass's spread S[dF]
  float2* ubf;                 // [H W] adjoint of the next pass's input velocity
  float* rhob;                 // [H W] adjoint of rho, from the passes
  unsigned long long* su;      // [2 H W] S of a pass's velocity adjoints (64-bit fixed point)
  unsigned long long* sr;      // [H W] S of a pass's density adjoints
  unsigned long long* ss;      // [2 H W] S of the drag velocity's adjoint
  float2* usb;                 // [N] adjoint of U_s
  float2* iub;                 // [N] adjoint of I[u_k] of a pass
  float* rbb;                  // [N] adjoint of I[rho] of a pass
  float4* xt;                  // [N] X~ = X + dt I[u_0](X)
  float2* xtb;                 // [N] the PBD's adjoint of X~
  float2* ust;                 // [N] adjoint of the drag velocity U* = I[u_0](X)
  unsigned* bnd;               // [5] bounds (float bits): su by pass parity (0, 1), sr (2, 3), ss (4)
};

// Exponent k of a 64-bit fixed-point scale 2^k for sums of terms whose
// total magnitude is below `bound` (bound 2^k < 2^62; k in [-64, 120]).
__device__ __forceinline__ int fix_exponent64(float bound) {
  if (!(bound > 0.0f)) return 62;
  if (!(bound < 3.0e38f)) return -64;
  const int e = ((__float_as_int(bound) >> 23) & 255) - 126;
  const int k = 62 - e;
  return k < -64 ? -64 : (k > 120 ? 120 : k);
}

// Launch configuration of a plan's steps.  Every choice advances the worlds
// bitwise the same; the autotuner (mc_tune.cu) picks the fastest one for
// each class of plan.
struct LaunchCfg {
  int persistent = 0;     // 3 or 4: one cooperative launch per run of steps with that many blocks per SM (k_persist.cu)
  int pbd_warps = 8;      // most filaments (warps) per block of the PBD kernels: 8, 4 or 2
  int scan_kernels = 0;   // 0: one scan kernel when every world fits one scan block; 2: always two
  int force_ws = 0;       // 1: the warp-specialised persistent force + LBM kernel (worlds without two layers)
};

// A set of worlds advanced together, with the work items of each stage.
struct Plan {
  int n_worlds = 0;
  // A plan of one world lets the step's kernels take each block's work item
  // from the block index instead of the item list.  The tile kernels, the
  // bin scatter and the scans also take the world's descriptor as a
  // __grid_constant__ parameter, so their blocks start without a dependent
  // load; the PBD and advance kernels keep reading it from the table (their
  // arithmetic then compiles exactly as in a batch, and a world stepped alone
  // stays bitwise equal to the same world batched, as measured).
  WorldDev h_world0{};
  int max_B = 2;
  int max_R = 4;                 // largest Gaussian half width among the worlds
  bool any_layered = false;      // some world is a two-layer filament world
  bool any_mdf = false;          // some world couples by direct forcing (ib == 1)
  int max_mdf = 0;               // most MDF passes of a world
  bool any_ext = false;          // some world has two layers, observables, a rest-length drive or direct forcing
  bool one_chunk = false;        // every world's bins fit one scan block (its offsets need no block sums)
  int n_fil_items = 0, n_bead_items = 0, n_tile_items = 0, n_cell_items = 0, n_scan_items = 0;
  WorldDev* d_worlds = nullptr;  // [n_worlds]
  int2* d_fil_items = nullptr;   // (world, filament)
  int2* d_bead_items = nullptr;  // (world, first bead)
  int2* d_tile_items = nullptr;  // (world, tx | ty << 16), row-major over the tiles
  int2* d_cell_items = nullptr;  // (world, first cell)
  int2* d_scan_items = nullptr;  // (world, scan chunk)
  void* d_mem = nullptr;
  unsigned* d_persist_bar = nullptr;   // [3] barrier words and status of the persistent step
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  LaunchCfg cfg;
  bool tuned = false;                  // cfg has been looked up or measured for this plan
};

// --- persistent batched step (k_persist.cu) ---------------------------------
bool persistent_supported(const Plan& p);
cudaError_t launch_persistent(const Plan& p, int n, cudaStream_t s);
void persistent_setup();   // host set-up (occupancy queries) outside any stream capture
void persistent_test_settings(unsigned extra_arrivals, unsigned long long timeout_ns);
void steric_setup(int sms);   // host set-up of the tile kernels (k_steric.cu), outside any stream capture

// --- stage launchers (one launch covers every world of the plan) ---------
void launch_pbd(const Plan& p, cudaStream_t s);
void launch_bin_scan(const Plan& p, cudaStream_t s, int inc_t = 0);      // one kernel when every world fits one scan block, else two
void launch_bin_scatter(const Plan& p, cudaStream_t s);
// a4 + x pass of a5; store_fields also writes rho_s of each tile
void launch_deposit_x(const Plan& p, cudaStream_t s, int store_fields);
// y pass of a5 + a6; store_fields also writes rho_bar of each tile;
// after_step = 1 when re-run after the step that produced the binned beads
void launch_force_spread(const Plan& p, cudaStream_t s, int store_fields, int after_step = 0);
void launch_lbm(const Plan& p, cudaStream_t s, int layered_only = 0);   // layered_only: two-layer worlds only
void launch_layer_spread(const Plan& p, cudaStream_t s);   // two-layer worlds: F from the layer points
void launch_force_lbm(const Plan& p, cudaStream_t s);   // y pass of a5 + a6 + a7 in one kernel
void launch_interp_advance(const Plan& p, cudaStream_t s);
// direct forcing (ib == 1 worlds; the others return at once): bins and a
// zero F_el before the steric spread, then u*, the predicted PBD and the
// MDF passes after it
void launch_mdf_bins(const Plan& p, cudaStream_t s);
void launch_mdf(const Plan& p, cudaStream_t s);
cudaError_t launch_mdf_recorded(const Plan& p, const WorldDev& h, float2* mu, cudaStream_t s);   // one world, passes' inputs kept
void launch_mdf_pass(const Plan& p, cudaStream_t s, int pass);   // k_steric.cu: one MDF pass (tile kernel)
void enqueue_step(const Plan& p, cudaStream_t s);
void enqueue_steps(const Plan& p, int n, cudaStream_t s);   // n steps, fused bead stages where possible
void launch_advance_pbd(const Plan& p, cudaStream_t s);
constexpr int kKernelsPerStep = 8;

// --- adjoint (one world) ----------------------------------------------------
void launch_adj_step(const Plan& p, const WorldDev& h, AdjDev a, const AdjMdf* m, int src_parity, cudaStream_t s);
// direct forcing (k_adj_mdf.cu): the passes reversed and X~ with the PBD's
// d_bar; then, after the PBD's reverse, the drag and the moments reversed
void launch_adj_mdf_passes(const WorldDev& h, const WorldDev* wd, const AdjDev& a, const AdjMdf& m, cudaStream_t s);
void launch_adj_mdf_moments(const WorldDev& h, const WorldDev* wd, const AdjDev& a, const AdjMdf& m, cudaStream_t s);
void launch_adj_gk_reduce(const AdjDev& a, int n_fil, cudaStream_t s);   // gk = sum over filaments of gkf
size_t adj_pbd_smem_per_filament(int maxB, int n_pbd, int order);
void adj_setup(const Plan& p, const WorldDev& h);   // host set-up of the adjoint kernels (before capture)
void launch_set_rest(const WorldDev& h, const float* theta0, const float* L_rest, cudaStream_t s);
// Launches kernel k, with programmatic stream serialization (see pdl_wait)
// unless the stream is being captured into a graph.  Direct launches (server
// ticks, short runs) gain from it; in a replayed graph, programmatic edges
// measured slower than plain ones.
template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cfg.attrs = at;
  cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}
void kernel_setup();   // one-time host set-up of the kernels' shared-memory limits
void launch_loss_splat(const Plan& p, const WorldDev& h, const float* target, int R, float sigma,
                       unsigned long long* acc, float* diff, float* loss, float* gx, float* gy, cudaStream_t s);
void launch_loss_polyline(const Plan& p, const WorldDev& h, const float2* pos0, const float2* poly, int nv,
                          float* loss, float* gx, float* gy, cudaStream_t s);
void launch_set_counter(const WorldDev& h, long long t, cudaStream_t s);

// --- set-up / read-out kernels (one world) --------------------------------
void launch_unstream_in(const float* f0dev, float* g_dst, int H, int W, cudaStream_t s);
void launch_stream_out(const float* g_src, float* out, int H, int W, cudaStream_t s);
void launch_positions_out(const WorldDev& w, float* x, float* y, cudaStream_t s);
// positions, creation positions, drive and rest-length drive records from the
// raw device arrays x, y [N], theta0, amp, freq, phase [J], len_amp,
// len_freq, len_phase [E] (the last three may be null)
void launch_world_init(const WorldDev& w, const float* const raw[9], cudaStream_t s);
void launch_cells_out(const WorldDev& w, int* cell, cudaStream_t s);

// --- world life cycle and plans (host, mc_api.cu) -------------------------
void world_sizes(WorldDev& h, int H, int W, int n_fil, int N);
size_t world_layout(WorldDev& h, void* arena);
mc_status plan_build(mc_world* const* ws, int n, cudaStream_t s, Plan& out);
mc_status plan_run(Plan& p, int n_steps, cudaStream_t s);
void plan_free(Plan& p, cudaStream_t s);
void plan_set_cfg(Plan& p, const LaunchCfg& c);   // drops the captured graph when the configuration changes
// A device copy of a world (same state, its own arena; no plan of its own)
// made on stream s, or nullptr when its memory cannot be allocated.
mc_world* world_clone(const mc_world* w, cudaStream_t s);

// --- autotuner (mc_tune.cu) -------------------------------------------------
// Looks up, or measures on device copies of the worlds, the launch
// configuration of plan p of worlds ws[0..n) (see mc_autotune); with
// `automatic`, only for plans large enough to repay the measurement and only
// when the tuner is enabled.
mc_status plan_tune(mc_world* const* ws, int n, Plan& p, cudaStream_t s, bool automatic);

// --- host accessors for code outside the ABI translation unit ------------
const WorldDev& world_dev(const mc_world* w);
void set_last_error(const char* msg);

// --- device helpers -------------------------------------------------------
__device__ __forceinline__ int wrap_once(int v, int n) {
  // v in [-n, 2n): one conditional correction maps it into [0, n)
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

__device__ __forceinline__ int wrap_mod(int v, int n) {
  const int r = v % n;
  return r < 0 ? r + n : r;
}

// Peskin's 4-point kernel phi at the four cells floor(X)-1 .. floor(X)+2
// for fractional part a in [0, 1).  With s = sqrt(1 + 4a - 4a^2):
//   phi(1+a) = (3 - 2a - s)/8, phi(a) = (3 - 2a + s)/8,
//   phi(1-a) = (1 + 2a + s)/8, phi(2-a) = (1 + 2a - s)/8.
__device__ __forceinline__ void peskin4(float a, float w[4]) {
  const float s = sqrtf(fmaf(-4.0f * a, a, fmaf(4.0f, a, 1.0f)));
  const float p = 3.0f - 2.0f * a, q = 1.0f + 2.0f * a;
  w[0] = (p - s) * 0.125f;
  w[1] = (p + s) * 0.125f;
  w[2] = (q + s) * 0.125f;
  w[3] = (q - s) * 0.125f;
}

// One cell of a7 (D2Q9 TRT with Guo forcing, shifted populations d = f - w):
// pulls the nine populations of cell c = r0 + x from its neighbours in
// `src` (rows r0, rm = row above in pull order y - 1, rp = y + 1; columns
// x, xm = x - 1, xp = x + 1, all wrapped), collides with force density F,
// stores the post-collision populations of c in `dst` (SoA, plane stride
// HW) and returns the velocity u = (sum c_i f_i + F/2) / rho.
struct LbmConst {
  float om_p, om_m, src_p, src_m;   // 1/tau+-, 1 - 1/(2 tau+-)
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// Two opposite pairs (i, opp(i)) at once in packed FP32x2 arithmetic (one
// pair per component): with d+ = (d_i + d_opp)/2, d- = (d_i - d_opp)/2,
//   e+ = w (drho + rho (4.5 (c.u)^2 - 1.5 u.u)),  e- = 3 w rho c.u,
//   S+ = w (9 (c.u)(c.F) - 3 u.F),               S- = 3 w c.F,
//   d*_i = d_i + even + odd,  d*_opp = d_opp + even - odd,
//   even = -(d+ - e+)/tau+ + (1 - 1/(2 tau+)) S+,  odd = -(d- - e-)/tau- + (1 - 1/(2 tau-)) S-.
__device__ __forceinline__ void trt_pairs(float2 di, float2 dib, float wi, float2 cu, float2 cF, float drho,
                                          float rho, float uu, float uF, const LbmConst& k, float2& a, float2& b) {
  const float2 c2 = __fmul2_rn(cu, cu);
  const float2 t1 = __ffma2_rn(c2, f2(4.5f), f2(-1.5f * uu));
  const float2 ep = __fmul2_rn(f2(wi), __ffma2_rn(f2(rho), t1, f2(drho)));
  const float2 em = __fmul2_rn(f2(3.0f * wi * rho), cu);
  const float2 sp = __ffma2_rn(__fmul2_rn(f2(9.0f * wi), cu), cF, f2(-3.0f * wi * uF));
  const float2 sm = __fmul2_rn(f2(3.0f * wi), cF);
  const float2 s = __fadd2_rn(di, dib);
  const float2 d = __ffma2_rn(dib, f2(-1.0f), di);
  const float2 even = __ffma2_rn(s, f2(-0.5f * k.om_p), __ffma2_rn(ep, f2(k.om_p), __fmul2_rn(f2(k.src_p), sp)));
  const float2 odd = __ffma2_rn(d, f2(-0.5f * k.om_m), __ffma2_rn(em, f2(k.om_m), __fmul2_rn(f2(k.src_m), sm)));
  a = __fadd2_rn(__fadd2_rn(di, even), odd);
  b = __ffma2_rn(odd, f2(-1.0f), __fadd2_rn(dib, even));
}

// The nine pulled populations of cell (x, y) (see lbm_cell).
struct LbmPull {
  float d[9];
};

__device__ __forceinline__ void lbm_pull(const float* __restrict__ src, int HW, int r0, int rm, int rp, int x, int xm,
                                         int xp, LbmPull& q) {
  q.d[0] = src[r0 + x];
  q.d[1] = src[1 * HW + r0 + xm];   // c = ( 1, 0) pulls from (x-1, y)
  q.d[2] = src[2 * HW + rm + x];    // ( 0, 1) from (x, y-1)
  q.d[3] = src[3 * HW + r0 + xp];   // (-1, 0) from (x+1, y)
  q.d[4] = src[4 * HW + rp + x];    // ( 0,-1) from (x, y+1)
  q.d[5] = src[5 * HW + rm + xm];   // ( 1, 1) from (x-1, y-1)
  q.d[6] = src[6 * HW + rm + xp];   // (-1, 1) from (x+1, y-1)
  q.d[7] = src[7 * HW + rp + xp];   // (-1,-1) from (x+1, y+1)
  q.d[8] = src[8 * HW + rp + xm];   // ( 1,-1) from (x-1, y+1)
}

// Collision of cell c from its pulled populations: stores the post-collision
// populations of c in `dst` and returns u.
__device__ __forceinline__ float2 lbm_collide(const LbmPull& q, float* __restrict__ dst, int HW, int c, float2 F,
                                              const LbmConst& k) {
  const float d0 = q.d[0], d1 = q.d[1], d2 = q.d[2], d3 = q.d[3], d4 = q.d[4];
  const float d5 = q.d[5], d6 = q.d[6], d7 = q.d[7], d8 = q.d[8];
  const float drho = ((d0 + (d1 + d3)) + (d2 + d4)) + ((d5 + d7) + (d6 + d8));
  const float rho = 1.0f + drho;
  const float jx = (d1 - d3) + (d5 - d7) + (d8 - d6);
  const float jy = (d2 - d4) + (d5 - d7) + (d6 - d8);
  const float inv = __frcp_rn(rho);
  const float ux = (jx + 0.5f * F.x) * inv;
  const float uy = (jy + 0.5f * F.y) * inv;
  const float uu = ux * ux + uy * uy;
  const float uF = ux * F.x + uy * F.y;
  constexpr float w0 = 4.0f / 9.0f, w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
  const float e0 = w0 * (drho - 1.5f * rho * uu);
  const float s0 = w0 * (-3.0f * uF);
  dst[c] = d0 - k.om_p * (d0 - e0) + k.src_p * s0;
  float2 a, b;
  // pairs (1, 3) and (2, 4): c = (1, 0), (0, 1)
  trt_pairs(make_float2(d1, d2), make_float2(d3, d4), w1, make_float2(ux, uy), F, drho, rho, uu, uF, k, a, b);
  dst[1 * HW + c] = a.x;
  dst[2 * HW + c] = a.y;
  dst[3 * HW + c] = b.x;
  dst[4 * HW + c] = b.y;
  // pairs (5, 7) and (6, 8): c = (1, 1), (-1, 1)
  trt_pairs(make_float2(d5, d6), make_float2(d7, d8), w5, make_float2(ux + uy, uy - ux),
            make_float2(F.x + F.y, F.y - F.x), drho, rho, uu, uF, k, a, b);
  dst[5 * HW + c] = a.x;
  dst[6 * HW + c] = a.y;
  dst[7 * HW + c] = b.x;
  dst[8 * HW + c] = b.y;
  return make_float2(ux, uy);
}

__device__ __forceinline__ float2 lbm_cell(const float* __restrict__ src, float* __restrict__ dst, int HW, int r0,
                                           int rm, int rp, int x, int xm, int xp, float2 F, const LbmConst& k) {
  LbmPull q;
  lbm_pull(src, HW, r0, rm, rp, x, xm, xp, q);
  return lbm_collide(q, dst, HW, r0 + x, F, k);
}

// sin(2 pi (freq t + phase)), phase in cycles, reduced exactly: hi + lo =
// freq * t (two-product via FMA) and only the fractional parts are added,
// so the angle keeps full precision at large t (t < 2^24 converts to float
// exactly).
__device__ __forceinline__ float drive_sin(float freq, float phase, long long t) {
  const float tf = (float)t;
  const float hi = freq * tf;
  const float lo = fmaf(freq, tf, -hi);
  float fr = (hi - rintf(hi)) + lo + phase;
  fr -= rintf(fr);
  return sinpif(2.0f * fr);
}

// a1: theta_rest = theta0 + A sin(2 pi (freq t + phase)), d = (theta0, A, freq, phase).
__device__ __forceinline__ float drive_angle(const float4 d, long long t) { return d.x + d.y * drive_sin(d.z, d.w, t); }

// Rest-length drive: L_rest = L0 (1 + A sin(2 pi (freq t + phase))), d = (L0, A, freq, phase).
__device__ __forceinline__ float drive_length(const float4 d, long long t) {
  return d.x * (1.0f + d.y * drive_sin(d.z, d.w, t));
}

// Rest length of edge e (global index) at step t.
__device__ __forceinline__ float rest_length(const WorldDev& w, int e, long long t) {
  return w.ldrive ? drive_length(w.ldrive[e], t) : w.L_rest[e];
}

// Programmatic dependent launch.  The step's kernels may be launched so that
// a kernel's blocks are scheduled while its predecessor drains:
// pdl_trigger lets the next kernel launch once every block of this one has
// started, and pdl_wait blocks until every prerequisite grid has completed
// and its memory operations are visible (it returns at once in a kernel
// launched without the attribute).  Every kernel of the step files calls
// both first, before it touches device memory.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A contribution to an observable in its fixed point (2^-24 resolution).
__device__ __forceinline__ long long obs_q(float v) { return __float2ll_rn(v * kObsScale); }

// Adds a warp's sum of fixed-point contributions to an observable.  Integer
// sums are exact, so the total does not depend on how contributions are
// grouped into lanes, warps or launches.  Every lane calls.
__device__ __forceinline__ void obs_add_warp(unsigned long long* acc, long long q) {
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0 && q != 0) atomicAdd(acc, (unsigned long long)q);
}

__device__ __forceinline__ int cell_x(const float4& p) { return __float_as_int(p.z); }
__device__ __forceinline__ int cell_y(const float4& p) { return __float_as_int(p.w); }

// Cell and fraction of the point X + d n for X = (cell, fraction) in p.
__device__ __forceinline__ void layer_cell(const float4 p, float2 n, float d, int W, int H, int& cx, int& cy,
                                           float& fx, float& fy) {
  fx = p.x + d * n.x;
  fy = p.y + d * n.y;
  const float kx = floorf(fx), ky = floorf(fy);
  fx -= kx;
  fy -= ky;
  cx = cell_x(p) + (int)kx;
  cy = cell_y(p) + (int)ky;
  if (fx >= 1.0f) { fx = 0.0f; cx += 1; }
  if (fy >= 1.0f) { fy = 0.0f; cy += 1; }
  cx = wrap_once(cx, W);   // |d| <= 2 keeps the offset within one period (W, H >= 8)
  cy = wrap_once(cy, H);
}

// Exponent k of the per-tile fixed-point scale for a bound on |cell sums|:
// the largest k in [8, 40] with bound * 2^k < 2^30.  With bound = m 2^e,
// m in [0.5, 1), k = 30 - e; e is read from the exponent bits (a subnormal
// bound gives e = -126 and k clamps to 40 as it would anyway).
__device__ __forceinline__ int fix_exponent(float bound) {
  if (!(bound > 0.0f)) return 40;
  if (!(bound < 1.0e30f)) return 8;
  const int e = ((__float_as_int(bound) >> 23) & 255) - 126;
  const int k = 30 - e;
  return k < 8 ? 8 : (k > 40 ? 40 : k);
}

// 2^k for k in [-126, 127] (exact, from the exponent bits).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

}  // namespace mc

// One world: its device descriptor, its arena and host-side bookkeeping.
// What a captured reverse sweep depends on (mc_rollout_backward caches one per world).
struct BwdKey {
  int n = 0, K = 0;
  int64_t t0 = -1;
  void* tape = nullptr;
  void* adj = nullptr;
  bool stored = false;
  bool operator==(const BwdKey& o) const {
    return n == o.n && K == o.K && t0 == o.t0 && tape == o.tape && adj == o.adj && stored == o.stored;
  }
};

struct mc_world {
  mc::WorldDev h{};               // device descriptor (host copy)
  void* arena = nullptr;          // one allocation holding every device array
  size_t bytes = 0;
  cudaStream_t stream = nullptr;  // creation stream; the arena is freed on it
  int64_t t = 0;                  // step counter after all enqueued steps
  int max_B = 2;
  std::vector<int> fil_off;
  mc::Plan plan;                  // single-world plan
  mc_params params{};
  // reverse-mode state (mc_rollout_forward / mc_rollout_backward)
  void* tape = nullptr;           // checkpoints + final state
  size_t tape_bytes = 0;
  int tape_steps = 0, tape_every = 0;
  int64_t tape_t0 = 0;
  bool tape_stored = false;       // the tape holds every step's record (mc_rollout_forward_stored)
  void* adj = nullptr;            // adjoint buffers + per-segment step tape
  size_t adj_bytes = 0;
  cudaGraphExec_t bwd_exec = nullptr;   // captured reverse sweep
  BwdKey bwd_key;
};
