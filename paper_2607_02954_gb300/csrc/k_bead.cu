// Bead-parallel stages of one time step: drive + PBD + elastic force + bin
// histogram (a1-a3), bin scatter (a2), IB interpolation + advance (a8), and
// the per-world set-up / read-out kernels.
#include <mutex>

#include "bead_dev.cuh"

namespace mc {

// One warp per filament (a1 + a3 + the a2 histogram).  Bead positions enter
// as edge vectors v0 = min_image(X_b - X_a) plus the accumulated corrections,
// so the corrections keep full FP32 precision whatever the magnitude of the
// coordinates.  Filaments of at most 64 beads run in registers; longer ones
// in the warp's slice of dynamic shared memory (maxB floats per array; zero
// when no filament of the launch is longer than 64 beads).
template <bool kExt, int kMode, bool kSingle>
__global__ void __launch_bounds__(256, 4) k_pbd(const WorldDev* __restrict__ worlds,
                                             const int2* __restrict__ items, int n_items, int maxB) {
  pdl_trigger();
  pdl_wait();
  pbd_body<kExt, kMode, kSingle>(worlds, items, n_items, maxB, blockIdx.x);
}

// a2: scatter bead records into bin order.  Lanes of one warp that share a
// bin take consecutive slots from one atomic.
template <bool kSingle>
__global__ void __launch_bounds__(kBeadChunk) k_bin_scatter(const WorldDev* __restrict__ worlds,
                                                            const int2* __restrict__ items,
                                                            const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  bin_scatter_body<kSingle>(worlds, items, w1, blockIdx.x);
}

// Spread of half of F_el + F_s at each layer point of every bead of
// two-layer worlds, in 64-bit fixed point (bitwise independent of order).
// Beads are read through the step's binned records, so the positions are
// those at the start of the step even when the spread is re-run later.
__global__ void __launch_bounds__(kBeadChunk) k_layer_spread(const WorldDev* __restrict__ worlds,
                                                             const int2* __restrict__ items) {
  pdl_trigger();
  pdl_wait();
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.layers != 2) return;
  const int slot = it.y + threadIdx.x;
  if (slot >= w.N) return;
  const int W = w.W, H = w.H;
  const float4 rec = w.srec[slot];
  const int i = __float_as_int(rec.z);
  const float4 p = w.spos[slot];
  const float2 n = w.nrm[i], fe = make_float2(rec.x, rec.y), fs = w.fs[i];
  const float hx = 0.5f * (fe.x + fs.x), hy = 0.5f * (fe.y + fs.y);
  for (int side = 0; side < 2; ++side) {
    int cx, cy;
    float fx, fy;
    layer_cell(p, n, side ? -w.layer_half : w.layer_half, W, H, cx, cy, fx, fy);
    float wx[4], wy[4];
    peskin4(fx, wx);
    peskin4(fy, wy);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      unsigned long long* row = w.facc + 2 * (size_t)wrap_once(cy - 1 + b, H) * W;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float g = wx[a] * wy[b];
        unsigned long long* c = row + 2 * wrap_once(cx - 1 + a, W);
        atomicAdd(c, (unsigned long long)__double2ll_rn((double)(g * hx) * kLayerScale));
        atomicAdd(c + 1, (unsigned long long)__double2ll_rn((double)(g * hy) * kLayerScale));
      }
    }
  }
}

// F = the layer spread, and the accumulator cleared for the next step.
__global__ void __launch_bounds__(kCellChunk) k_layer_finish(const WorldDev* __restrict__ worlds,
                                                             const int2* __restrict__ items) {
  pdl_trigger();
  pdl_wait();
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.layers != 2) return;
  const int c = it.y + threadIdx.x;
  if (c >= w.H * w.W) return;
  const long long ax = (long long)w.facc[2 * c], ay = (long long)w.facc[2 * c + 1];
  w.F[c] = make_float2((float)((double)ax / kLayerScale), (float)((double)ay / kLayerScale));
  w.facc[2 * c] = 0ull;
  w.facc[2 * c + 1] = 0ull;
}

// a8: U_i = sum_c delta_h(c - X_i) u(c) over the 4x4 stencil, then the
// inertia-free advance X += dt U (cell index + fraction, wrapped) and the
// unwrapped displacement D += dt U.  Thread 0 of each world's first block
// advances the world's step counter (no other stage kernel reads it).
template <bool kExt, bool kSingle>
__global__ void __launch_bounds__(kBeadChunk) k_interp_advance(const WorldDev* __restrict__ worlds,
                                                               const int2* __restrict__ items) {
  pdl_trigger();
  pdl_wait();
  interp_advance_body<kExt, kSingle>(worlds, items, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Set-up and read-out (one world).
// ---------------------------------------------------------------------------
__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// The stored state is post-collision (the LBM pulls on read).  Given
// pre-collision populations f0, store g_i(c) = f0_i(c + c_i) so that pulling
// g_i(c - c_i) returns f0_i(c).
__global__ void k_unstream_in(const float* __restrict__ f0, float* __restrict__ g, int H, int W) {
  pdl_trigger();
  pdl_wait();
  const int HW = H * W;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 9 * HW) return;
  const int i = idx / HW, c = idx - i * HW;
  const int y = c / W, x = c - y * W;
  const int sx = wrap_once(x + kCx[i], W), sy = wrap_once(y + kCy[i], H);
  g[idx] = f0[i * HW + sy * W + sx];
}

__global__ void k_stream_out(const float* __restrict__ g, float* __restrict__ out, int H, int W) {
  pdl_trigger();
  pdl_wait();
  const int HW = H * W;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 9 * HW) return;
  const int i = idx / HW, c = idx - i * HW;
  const int y = c / W, x = c - y * W;
  const int sx = wrap_once(x - kCx[i], W), sy = wrap_once(y - kCy[i], H);
  out[idx] = g[i * HW + sy * W + sx];
}

// A world's set-up from its raw inputs: each position wrapped into the box
// in double precision (fmod is exact) and split into cell index + fraction,
// the creation positions, the drive records (theta0, A, freq, phase) and the
// rest-length drive records (L0 = L_rest, amp, freq, phase).
__global__ void k_world_init(WorldDev h, const float* x, const float* y, const float* t0, const float* amp,
                             const float* frq, const float* phs, const float* la, const float* lf,
                             const float* lp) {
  pdl_trigger();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < h.N) {
    const double xd = fmod((double)x[i], (double)h.W), yd = fmod((double)y[i], (double)h.H);
    float xw = (float)(xd < 0 ? xd + h.W : xd), yw = (float)(yd < 0 ? yd + h.H : yd);
    if (xw >= (float)h.W) xw = 0.0f;
    if (yw >= (float)h.H) yw = 0.0f;
    const float cx = floorf(xw), cy = floorf(yw);
    h.pos0[i] = make_float2(xw, yw);
    h.pos[i] = make_float4(xw - cx, yw - cy, __int_as_float((int)cx), __int_as_float((int)cy));
  }
  if (i < h.J) const_cast<float4*>(h.drive)[i] = make_float4(t0[i], amp[i], frq[i], phs[i]);
  if (la && i < h.E) const_cast<float4*>(h.ldrive)[i] = make_float4(h.L_rest[i], la[i], lf[i], lp[i]);
}

__global__ void k_positions_out(const float4* __restrict__ pos, int N, float* x, float* y) {
  pdl_trigger();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = pos[i];
  if (x) x[i] = (float)cell_x(p) + p.x;
  if (y) y[i] = (float)cell_y(p) + p.y;
}

__global__ void k_cells_out(const float4* __restrict__ pos, int N, int W, int* cell) {
  pdl_trigger();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = pos[i];
  cell[i] = cell_y(p) * W + cell_x(p);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
// Warps (filaments) per block: at most 8, at most what 48 KB of shared
// memory holds, and few enough that a small launch still spreads over every
// SM (each warp's filament is a serial chain; warps sharing an SM's
// schedulers only delay one another).
static int num_sms() {
  // first asked by kernel_setup, outside any stream capture
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

static int pbd_warps_per_block(int maxB, int n_items, int most) {
  const int sms = num_sms();
  const int per_warp = maxB * kPbdFloatsPerBead * (int)sizeof(float);
  int wpb = (48 * 1024) / per_warp;
  if (wpb > most) wpb = most;
  const int spread = (n_items + sms - 1) / sms;
  if (wpb > spread) wpb = spread;
  if (wpb < 1) wpb = 1;
  return wpb;
}

void launch_pbd(const Plan& p, cudaStream_t s) {
  if (p.n_fil_items == 0) return;
  const int mb = (p.max_B + 3) & ~3;
  const int wpb = pbd_warps_per_block(mb, p.n_fil_items, p.cfg.pbd_warps);
  // filaments of at most 64 beads need no shared memory
  const size_t smem = p.max_B <= 64 ? 0 : (size_t)wpb * mb * kPbdFloatsPerBead * sizeof(float);
  const int grid = (p.n_fil_items + wpb - 1) / wpb;
  // worlds with a rest-length drive, observables or two layers need the
  // extended kernel; it computes every other world exactly as the plain one
  const bool one = p.n_worlds == 1;
  auto kern = p.any_ext ? (one ? k_pbd<true, 0, true> : k_pbd<true, 0, false>)
                        : (one ? k_pbd<false, 0, true> : k_pbd<false, 0, false>);
  launch_pdl(kern, grid, wpb * 32, smem, s, p.d_worlds, p.d_fil_items, p.n_fil_items, mb);
}

// The PBD of direct-forcing worlds (from the positions the fluid carries
// the beads to; the others return at once).
void launch_pbd_mdf(const Plan& p, cudaStream_t s) {
  if (p.n_fil_items == 0) return;
  const int mb = (p.max_B + 3) & ~3;
  const int wpb = pbd_warps_per_block(mb, p.n_fil_items, p.cfg.pbd_warps);
  const size_t smem = p.max_B <= 64 ? 0 : (size_t)wpb * mb * kPbdFloatsPerBead * sizeof(float);
  const int grid = (p.n_fil_items + wpb - 1) / wpb;
  auto kern = p.n_worlds == 1 ? k_pbd<true, 2, true> : k_pbd<true, 2, false>;
  launch_pdl(kern, grid, wpb * 32, smem, s, p.d_worlds, p.d_fil_items, p.n_fil_items, mb);
}

// a8 of the previous step fused with this step's a1-a3 (plans without
// direct-forcing worlds): the counter is advanced by this step's scan.
void launch_advance_pbd(const Plan& p, cudaStream_t s) {
  if (p.n_fil_items == 0) return;
  const int mb = (p.max_B + 3) & ~3;
  const int wpb = pbd_warps_per_block(mb, p.n_fil_items, p.cfg.pbd_warps);
  const size_t smem = p.max_B <= 64 ? 0 : (size_t)wpb * mb * kPbdFloatsPerBead * sizeof(float);
  const int grid = (p.n_fil_items + wpb - 1) / wpb;
  const bool one = p.n_worlds == 1;
  auto kern = p.any_ext ? (one ? k_pbd<true, 1, true> : k_pbd<true, 1, false>)
                        : (one ? k_pbd<false, 1, true> : k_pbd<false, 1, false>);
  launch_pdl(kern, grid, wpb * 32, smem, s, p.d_worlds, p.d_fil_items, p.n_fil_items, mb);
}

// Shared-memory limits set once per process, outside any stream capture: the
// PBD kernel stages up to 8 warps' filaments of at most 3072 beads.
void kernel_setup() {
  static std::once_flag once;
  std::call_once(once, [] {
    steric_setup(num_sms());
    persistent_setup();
    const int most = 227 * 1024;
    for (auto f : {k_pbd<false, 0, false>, k_pbd<true, 0, false>, k_pbd<false, 1, false>, k_pbd<true, 1, false>,
                   k_pbd<true, 2, false>, k_pbd<false, 0, true>, k_pbd<true, 0, true>, k_pbd<false, 1, true>,
                   k_pbd<true, 1, true>, k_pbd<true, 2, true>})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  });
}

void launch_bin_scatter(const Plan& p, cudaStream_t s) {
  // (data moves only: the single-world path cannot change a result)
  if (p.n_worlds == 1) launch_pdl(k_bin_scatter<true>, p.n_bead_items, kBeadChunk, 0, s, p.d_worlds, p.d_bead_items, p.h_world0);
  else launch_pdl(k_bin_scatter<false>, p.n_bead_items, kBeadChunk, 0, s, p.d_worlds, p.d_bead_items, p.h_world0);
}

void launch_layer_spread(const Plan& p, cudaStream_t s) {
  if (!p.any_layered) return;
  k_layer_spread<<<p.n_bead_items, kBeadChunk, 0, s>>>(p.d_worlds, p.d_bead_items);
  if (p.n_cell_items) k_layer_finish<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items);
}

void launch_interp_advance(const Plan& p, cudaStream_t s) {
  const bool one = p.n_worlds == 1;
  auto kern = p.any_ext ? (one ? k_interp_advance<true, true> : k_interp_advance<true, false>)
                        : (one ? k_interp_advance<false, true> : k_interp_advance<false, false>);
  launch_pdl(kern, p.n_bead_items, kBeadChunk, 0, s, p.d_worlds, p.d_bead_items);
}

void launch_unstream_in(const float* f0dev, float* g_dst, int H, int W, cudaStream_t s) {
  const int n = 9 * H * W;
  k_unstream_in<<<(n + 255) / 256, 256, 0, s>>>(f0dev, g_dst, H, W);
}

void launch_stream_out(const float* g_src, float* out, int H, int W, cudaStream_t s) {
  const int n = 9 * H * W;
  k_stream_out<<<(n + 255) / 256, 256, 0, s>>>(g_src, out, H, W);
}

void launch_world_init(const WorldDev& w, const float* const raw[9], cudaStream_t s) {
  if (w.N == 0) return;
  k_world_init<<<(w.N + 255) / 256, 256, 0, s>>>(w, raw[0], raw[1], raw[2], raw[3], raw[4], raw[5], raw[6], raw[7],
                                                 raw[8]);
}

void launch_positions_out(const WorldDev& w, float* x, float* y, cudaStream_t s) {
  if (w.N == 0) return;
  k_positions_out<<<(w.N + 255) / 256, 256, 0, s>>>(w.pos, w.N, x, y);
}

void launch_cells_out(const WorldDev& w, int* cell, cudaStream_t s) {
  if (w.N == 0) return;
  k_cells_out<<<(w.N + 255) / 256, 256, 0, s>>>(w.pos, w.N, w.W, cell);
}

}  // namespace mc
