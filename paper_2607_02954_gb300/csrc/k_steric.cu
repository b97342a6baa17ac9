// a4-a6: steric deposit, Gaussian filter, steric force and immersed-boundary
// force spread, in tile kernels (one 32x32 tile of cells per block).
//
//   rho_s(c)  = sum_i delta_h(c - X_i)                        (a4, Fields)
//   rho_bar   = G_sigma * rho_s, periodic, x pass then y pass  (a5, Fields)
//   F_s,i     = -k_rep sum_c delta_h(c - X_i) grad rho_bar(c)  (a6, central differences)
//   F(c)      = sum_i delta_h(c - X_i) (F_el,i + F_s,i)       (a6, Fluid-filament Interaction)
//
// k_deposit_x    deposits rho_s on the tile plus R columns on each side in
//                shared memory, applies the x pass of the filter and writes
//                the x-filtered density rho_x of the tile (4 B per cell) and
//                a bound of the tile's rho_s (its largest deposited sum plus
//                the rounding the fixed point can hide).
// k_force_spread loads rho_x on the tile plus 4 + R rows and 4 columns,
//                applies the y pass (rho_bar on the tile plus 4 cells),
//                gathers the steric force of every bead whose stencil touches
//                the tile, spreads F_el + F_s into the tile and writes F.
// k_force_lbm    does the same and then the LBM step (a7) of the tile's
//                cells with F taken from shared memory: the step's path.
//
// Beads are sorted by 8x8-cell bins in row-major order, so the beads that
// can reach a tile lie in a few contiguous segments of the sorted arrays,
// one per bin row (two where the row range wraps around the periodic edge).
// The force kernel stages grid windows and bead records in shared memory
// with cp.async, every copy in flight at once, and lists the staged beads
// whose stencil reaches the tile first (a block-wide compaction), so its
// per-bead arithmetic runs on full warps.  The deposit, whose per-bead work
// is 16 atomics, reads each record straight into registers and lets the
// beads that miss the region drop out.
//
// Both kernels are compiled for each filter half width R (1..8) so that the
// filter loops unroll with the taps in registers; a launch uses the largest R
// of its worlds, and a world with a smaller R sees its taps padded with zeros
// (which leaves every sum unchanged).  Everything that decides a result (the
// bead ranges, the fixed-point scales) uses the world's own R.
//
// Stencil cells are accumulated in a halo-extended buffer (3 cells on each
// side of the tile), so no per-cell wrap or bounds test is needed; cells
// outside the tile belong to a neighbouring tile and are dropped, except on
// an axis that one tile covers whole, where they are folded back
// periodically before use.
//
// Periodic images: with several tiles on an axis a bead is taken at the one
// image of it that can reach the tile (the reachable range is shorter than
// the axis); with one tile the tile is the whole axis.
#include <algorithm>

#include "steric_dev.cuh"

namespace mc {

template <int R, bool kSingle>
__global__ void __launch_bounds__(kThreads, 8) k_deposit_x(const WorldDev* __restrict__ worlds,
                                                        const int2* __restrict__ items, int store_fields,
                                                        const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) DepositSmem<R> sm;
  deposit_x_body<R, kSingle>(worlds, items, store_fields, w1, blockIdx.x, sm);
}

// y pass of a5 + a6: writes F.
template <int R>
__global__ void __launch_bounds__(kThreads) k_force_spread(const WorldDev* __restrict__ worlds,
                                                           const int2* __restrict__ items, int store_fields,
                                                           int after_step) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) ForceSmem<R> sm;
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const TileBox tb = tile_box(w, it.y);
  float2* __restrict__ F_out = w.F;
  const int W = w.W;
  const int k = force_tile<R>(sm, w, (tb.y0 / kTile) * w.ntx + tb.x0 / kTile, tb, store_fields, after_step);
  __syncthreads();
  force_fold(sm.wk, tb, w.ntx, w.nty);
  const float inv = pow2f(-k);
  const int lane = threadIdx.x & 31;
  // a direct-forcing world's F holds the step's total force (steric spread
  // plus MDF passes): a re-run for the density fields leaves it
  if (store_fields && w.ib == 1) return;
  for (int ly = threadIdx.x >> 5; ly < tb.th; ly += kWarps) {
    if (lane < tb.tw) {
      const int s = (ly + 3) * kAx + lane + 3;
      F_out[(size_t)(tb.y0 + ly) * W + tb.x0 + lane] = make_float2((float)sm.wk.accx[s] * inv, (float)sm.wk.accy[s] * inv);
    }
  }
}

template <int R, bool kSingle>
__global__ void __launch_bounds__(kThreads, 4) k_force_lbm(const WorldDev* __restrict__ worlds,
                                                           const int2* __restrict__ items,
                                                           const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) ForceSmem<R> sm;
  // tiles in reverse order: the first rows' velocities, written last, are
  // still in L2 when the next PBD (filaments in index order) interpolates
  // them, and the last rows' x-filtered densities, which the deposit wrote
  // last, are read first
  force_lbm_body<R, kSingle>(worlds, items, w1, gridDim.x - 1 - blockIdx.x, sm);
}

// y pass of a5 + a6 + a7, warp-specialised and persistent: each block walks
// the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; warps 0-3 run the force
// phase of a tile (staging, y pass, steric gather, spread) while warps 4-7
// collide the previous tile, so the collision's memory traffic overlaps the
// force phase's arithmetic.  The force warps hand the tile's F over in a
// shared buffer: they fill it once the collision warps have released it
// (named barrier 4) and signal it full (named barrier 3); each tile's F and
// collision are computed exactly as in k_force_lbm (bitwise the same
// results).  Worlds without two layers only.
constexpr int kWsForce = kThreads / 2;   // threads of the force group
constexpr int kWsLbmWarps = (kThreads - kWsForce) / 32;

template <int R>
struct WsSmem {
  ForceSmem<R> f;
  float2 Fh[kTile * kTile];   // the hand-off buffer: F of the tile being collided
};

__device__ __forceinline__ void ws_bar_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kThreads) : "memory"); }
__device__ __forceinline__ void ws_bar_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "n"(kThreads) : "memory");
}
constexpr int kWsFull = 3, kWsEmpty = 4;

template <int R, bool kSingle>
__global__ void __launch_bounds__(kThreads, 4) k_force_lbm_ws(const WorldDev* __restrict__ worlds,
                                                              const int2* __restrict__ items, int n_items,
                                                              const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char ws_raw[];
  WsSmem<R>& sm = *reinterpret_cast<WsSmem<R>*>(ws_raw);
  const bool force_group = threadIdx.x < kWsForce;
  int done = 0;   // tiles of this block handed over so far
  for (int i = blockIdx.x; i < n_items; i += gridDim.x, ++done) {
    const int2 it = kSingle ? single_tile_item(w1, (unsigned)i) : items[i];
    const WorldDev& w = kSingle ? w1 : worlds[it.x];
    const TileBox tb = tile_box(w, it.y);
    if (force_group) {
      prefetch_populations<kWsForce>(w, tb);
      const int tile = (tb.y0 / kTile) * w.ntx + tb.x0 / kTile;
      int k = 40;
      if (!kSingle && w.tile_rho_max[tile] == 0.0f) {
        tile_clear<kWsForce>(sm.f.wk);   // no bead reaches the tile: F = 0 (see k_force_lbm)
      } else {
        k = force_tile<R, kWsForce>(sm.f, w, tile, tb, 0, 0);
      }
      force_sync<kWsForce>();
      force_fold<TileWork, kWsForce>(sm.f.wk, tb, w.ntx, w.nty);
      if (done > 0) ws_bar_sync(kWsEmpty);   // the collision warps are done with the previous F
      const float inv = pow2f(-k);
      for (int c = threadIdx.x; c < kTile * kTile; c += kWsForce) {
        const int s = ((c >> 5) + 3) * kAx + (c & 31) + 3;
        sm.Fh[c] = make_float2((float)sm.f.wk.accx[s] * inv, (float)sm.f.wk.accy[s] * inv);
      }
      force_sync<kWsForce>();   // the accumulators are read: the next tile may clear them
      ws_bar_arrive(kWsFull);
    } else {
      const int W = w.W, H = w.H, HW = H * W;
      const long long t = *w.t;
      const float* __restrict__ src = w.g[t & 1];
      float* __restrict__ dst = w.g[(t + 1) & 1];
      float2* __restrict__ u_out = w.u;
      const LbmConst kc{w.om_p, w.om_m, w.src_p, w.src_m};
      const int lane = threadIdx.x & 31, lw = (threadIdx.x - kWsForce) >> 5;
      const bool active = lane < tb.tw && lw < tb.th;
      const int x = tb.x0 + lane;
      const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
      LbmPull q;
      int y = tb.y0 + lw;
      // the first row's populations are pulled while the force warps finish
      if (active) lbm_pull(src, HW, y * W, (y == 0 ? H - 1 : y - 1) * W, (y == H - 1 ? 0 : y + 1) * W, x, xm, xp, q);
      ws_bar_sync(kWsFull);
      if (active) {
        for (int ly = lw; ly < tb.th; ly += kWsLbmWarps) {
          if (ly != lw)
            lbm_pull(src, HW, y * W, (y == 0 ? H - 1 : y - 1) * W, (y == H - 1 ? 0 : y + 1) * W, x, xm, xp, q);
          u_out[(size_t)y * W + x] = lbm_collide(q, dst, HW, y * W + x, sm.Fh[ly * kTile + lane], kc);
          y += kWsLbmWarps;
        }
      }
      ws_bar_arrive(kWsEmpty);
    }
  }
  if (force_group && done > 0) ws_bar_sync(kWsEmpty);   // the last F has been read
}

// One MDF pass of the direct-forcing worlds on one tile, Jacobi in u.  Every
// bead whose stencil reaches the tile gets
//   dF_i = 2 I[rho](X_i) (U_s,i - I[u](X_i))
// from the pass's input velocity (u for even passes, u2 for odd ones) and
// rho, both staged with a 3-cell halo; then the tile's cells get
// F += S[dF] and u' = u + S[dF] / (2 rho) in the other velocity buffer, and
// the tile that holds a bead adds its dF to F_el.  A bead near a tile edge
// is evaluated by each tile its stencil reaches, from the same inputs in the
// same order, so every tile uses the same dF bitwise.  The spread is in
// int32 fixed point with the scale from the largest |dF| component among
// the tile's beads times the tile's largest rho_s (the sum of the spread
// weights of a cell): bitwise independent of order.  The dF of a tile's
// beads are kept in shared memory when they fit one staging pass, and are
// evaluated again in a second sweep otherwise.
constexpr int kMwy = kTile + 6;   // window rows: the tile and 3 cells a side
constexpr int kMwx = kTile + 8;   // window columns: the tile and 4 cells a side (16-byte chunks)

struct MdfSmem {
  float4 sp[kForceCap];   // staged bead records
  float2 su[kForceCap];   // their U_s
  float2 df[kForceCap];   // their dF (one-pass tiles)
  int si[kForceCap];      // their bead indices
  float2 uw[kMwy * kMwx];   // input velocity window
  float rw[kMwy * kMwx];    // density window
  int accx[kAx * kAx];    // spread accumulators
  int accy[kAx * kAx];
  int list[kForceCap];
  int s_cnt;
  int s_start[kMaxSeg], s_pre[kMaxSeg + 1];
  float red[kWarps];
};

// dF of the staged bead v whose tile-relative cell is (rx, ry) in [-2, tw] x
// [-2, th]: its stencil cells sit at window rows ry + 2 .. ry + 5 and
// columns rx + 3 .. rx + 6.
__device__ __forceinline__ float2 mdf_bead_force(const MdfSmem& sm, int v, int rx, int ry) {
  const float4 p = sm.sp[v];
  float wx[4], wy[4];
  peskin4(p.x, wx);
  peskin4(p.y, wy);
  float Ux = 0.0f, Uy = 0.0f, r = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int row = (ry + 2 + b) * kMwx + rx + 3;
    float ax = 0.0f, ay = 0.0f, ar = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 v2 = sm.uw[row + a];
      ax = fmaf(wx[a], v2.x, ax);
      ay = fmaf(wx[a], v2.y, ay);
      ar = fmaf(wx[a], sm.rw[row + a], ar);
    }
    Ux = fmaf(wy[b], ax, Ux);
    Uy = fmaf(wy[b], ay, Uy);
    r = fmaf(wy[b], ar, r);
  }
  const float2 Us = sm.su[v];
  return make_float2(2.0f * r * (Us.x - Ux), 2.0f * r * (Us.y - Uy));
}

// Stages chunk c0 of the tile's bead segments and lists the beads whose
// stencil reaches the tile (the block synchronises inside).
__device__ __forceinline__ int mdf_stage_chunk(MdfSmem& sm, const WorldDev& w, const TileBox& tb, int c0, int total) {
  const int tid = threadIdx.x;
  const int W = w.W, H = w.H, ntx = w.ntx, nty = w.nty;
  const int n = min(kForceCap, total - c0);
  for (int v = tid; v < n; v += kThreads) {
    const int slot = seg_slot(c0 + v, sm.s_start, sm.s_pre);
    cp_async16(&sm.sp[v], &w.spos[slot]);
    cp_async8(&sm.su[v], &w.sus[slot]);
    cp_async4(&sm.si[v], reinterpret_cast<const int*>(&w.srec[slot]) + 2);   // the record's id
  }
  cp_async_wait_all();
  if (tid == 0) sm.s_cnt = 0;
  __syncthreads();
  for (int v0 = 0; v0 < n; v0 += kThreads) {
    const int v = v0 + tid;
    bool keep = false;
    int rx = 0, ry = 0;
    if (v < n) {
      const float4 p = sm.sp[v];
      rx = cell_x(p) - tb.x0;
      ry = cell_y(p) - tb.y0;
      keep = true;
      if (ntx > 1) {
        rx = image_lo(rx, W, 2);
        keep = rx <= tb.tw;
      }
      if (nty > 1) {
        ry = image_lo(ry, H, 2);
        keep = keep && ry <= tb.th;
      }
    }
    list_push(keep, pack_code(v, rx, ry), sm.list, &sm.s_cnt);
  }
  __syncthreads();
  return sm.s_cnt;
}

__global__ void __launch_bounds__(kThreads) k_mdf_pass(const WorldDev* __restrict__ worlds,
                                                       const int2* __restrict__ items, int pass) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) MdfSmem sm;
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1 || pass >= w.mdf_iters) return;
  const TileBox tb = tile_box(w, it.y);
  const int W = w.W, H = w.H, ntx = w.ntx, nty = w.nty;
  const int tile = (tb.y0 / kTile) * ntx + tb.x0 / kTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2* __restrict__ u_in = (pass & 1) ? w.u2 : w.u;
  float2* __restrict__ u_out = (pass & 1) ? w.u : w.u2;
  if (warp == 0) build_segments(w, tb.x0 - 2, tb.x0 + tb.tw, tb.y0 - 2, tb.y0 + tb.th, sm.s_start, sm.s_pre, nullptr);
  // the velocity and density windows, rows y0 - 3 .. y0 + th + 2 and
  // columns x0 - 4 .. x0 + tw + 3, periodic (W, H >= 8: one wrap at most),
  // in 16-byte chunks (2 velocities or 4 densities; x0 and W are multiples
  // of 8, so a chunk never straddles the periodic edge)
  const bool full = tb.tw == kTile;   // full tile: constant divisors
  const int nu = full ? kMwx / 2 : (tb.tw + 8) >> 1, nr = full ? kMwx / 4 : (tb.tw + 8) >> 2, wh = tb.th + 6;
  for (int c = tid; c < wh * nu; c += kThreads) {
    const int i = full ? c / (kMwx / 2) : c / nu, j = 2 * (c - i * nu);
    const size_t g = (size_t)wrap_once(tb.y0 - 3 + i, H) * W + wrap_once(tb.x0 - 4 + j, W);
    cp_async16(&sm.uw[i * kMwx + j], &u_in[g]);
  }
  for (int c = tid; c < wh * nr; c += kThreads) {
    const int i = full ? c / (kMwx / 4) : c / nr, j = 4 * (c - i * nr);
    const size_t g = (size_t)wrap_once(tb.y0 - 3 + i, H) * W + wrap_once(tb.x0 - 4 + j, W);
    cp_async16(&sm.rw[i * kMwx + j], &w.mrho[g]);
  }
  for (int c = tid; c < kAx * kAx / 4; c += kThreads) {
    reinterpret_cast<int4*>(sm.accx)[c] = make_int4(0, 0, 0, 0);
    reinterpret_cast<int4*>(sm.accy)[c] = make_int4(0, 0, 0, 0);
  }
  __syncthreads();   // segments visible (the windows land with the first chunk's wait)
  const int total = sm.s_pre[kMaxSeg];
  const bool one_pass = total <= kForceCap;
  // sweep 1: dF of every listed bead and their largest component
  float m = 0.0f;
  for (int c0 = 0; c0 < total; c0 += kForceCap) {
    if (c0 > 0) __syncthreads();   // the previous chunk is no longer read
    const int cnt = mdf_stage_chunk(sm, w, tb, c0, total);
    for (int q = tid; q < cnt; q += kThreads) {
      const int code = sm.list[q];
      const int v = code_slot(code);
      const float2 dF = mdf_bead_force(sm, v, code_rx(code), code_ry(code));
      if (one_pass) sm.df[v] = dF;
      m = fmaxf(m, fmaxf(fabsf(dF.x), fabsf(dF.y)));
    }
  }
  if (total == 0) cp_async_wait_all();
  m = block_max(m, sm.red);   // also orders the df writes before sweep 2
  const int k = fix_exponent(m * w.tile_rho_max[tile] * 1.0001f + 1e-30f);
  const float scale = pow2f(k);
  // sweep 2: the spread, and F_el += dF on the bead's own tile
  float2* __restrict__ fel = w.fel;
  for (int c0 = 0; c0 < total; c0 += kForceCap) {
    int cnt = sm.s_cnt;
    if (!one_pass) {
      __syncthreads();
      cnt = mdf_stage_chunk(sm, w, tb, c0, total);
    }
    for (int q = tid; q < cnt; q += kThreads) {
      const int code = sm.list[q];
      const int v = code_slot(code), rx = code_rx(code), ry = code_ry(code);
      const float2 dF = one_pass ? sm.df[v] : mdf_bead_force(sm, v, rx, ry);
      if (rx >= 0 && rx < tb.tw && ry >= 0 && ry < tb.th) {
        // the bead's own tile is its one writer in this pass: the adds
        // need no return value and leave the same bits in any order
        const int i = sm.si[v];
        atomicAdd(&fel[i].x, dF.x);
        atomicAdd(&fel[i].y, dF.y);
      }
      const float4 p = sm.sp[v];
      float wx[4], wy[4];
      peskin4(p.x, wx);
      peskin4(p.y, wy);
      const float Fx = dF.x * scale, Fy = dF.y * scale;
      int* bx = sm.accx + (ry + 2) * kAx + rx + 2;
      int* by = sm.accy + (ry + 2) * kAx + rx + 2;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float g = wx[a] * wy[b];
          atomicAdd(bx + b * kAx + a, __float2int_rn(g * Fx));
          atomicAdd(by + b * kAx + a, __float2int_rn(g * Fy));
        }
      }
    }
  }
  __syncthreads();
  force_fold(sm, tb, ntx, nty);
  const float inv = pow2f(-k);
  // the warp's rows warp, warp + 8, ...: every F load in flight at once
  float2* __restrict__ Fg = w.F;
  constexpr int kRows = kTile / kWarps;
  float2 Fv[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int ly = warp + r * kWarps;
    if (ly < tb.th && lane < tb.tw) Fv[r] = Fg[(size_t)(tb.y0 + ly) * W + tb.x0 + lane];
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int ly = warp + r * kWarps;
    if (ly < tb.th && lane < tb.tw) {
      const int sidx = (ly + 3) * kAx + lane + 3;
      const int widx = (ly + 3) * kMwx + lane + 4;
      const size_t c = (size_t)(tb.y0 + ly) * W + tb.x0 + lane;
      const float Gx = (float)sm.accx[sidx] * inv, Gy = (float)sm.accy[sidx] * inv;
      Fg[c] = make_float2(Fv[r].x + Gx, Fv[r].y + Gy);
      const float ih = __frcp_rn(2.0f * sm.rw[widx]);   // 1 / (2 rho), correctly rounded
      const float2 u = sm.uw[widx];
      u_out[c] = make_float2(fmaf(Gx, ih, u.x), fmaf(Gy, ih, u.y));
    }
  }
}

namespace {

// Blocks of the warp-specialised force + LBM kernel: as many as fit on every
// SM at once (set up outside any stream capture by steric_setup).
int g_ws_grid[kMaxR + 1] = {};

template <int R>
int ws_grid() {
  return g_ws_grid[R] > 0 ? g_ws_grid[R] : 1;
}

template <int R>
void ws_setup(int sms) {
  const int bytes = (int)sizeof(WsSmem<R>);
  cudaFuncSetAttribute(k_force_lbm_ws<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_force_lbm_ws<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_force_lbm_ws<R, false>, kThreads, bytes);
  g_ws_grid[R] = (per > 0 ? per : 1) * sms;
}

template <int R>
void launch_steric(const Plan& p, cudaStream_t s, int which, int store_fields, int after_step) {
  if (which == 0) {
    if (p.n_worlds == 1)
      launch_pdl(k_deposit_x<R, true>, p.n_tile_items, kThreads, 0, s, p.d_worlds, p.d_tile_items, store_fields, p.h_world0);
    else
      launch_pdl(k_deposit_x<R, false>, p.n_tile_items, kThreads, 0, s, p.d_worlds, p.d_tile_items, store_fields, p.h_world0);
  } else if (which == 1) {
    k_force_spread<R><<<p.n_tile_items, kThreads, 0, s>>>(p.d_worlds, p.d_tile_items, store_fields, after_step);
  } else if (p.cfg.force_ws && !p.any_layered) {
    const int grid = std::min(p.n_tile_items, ws_grid<R>());
    if (p.n_worlds == 1)
      launch_pdl(k_force_lbm_ws<R, true>, grid, kThreads, sizeof(WsSmem<R>), s, p.d_worlds, p.d_tile_items,
                 p.n_tile_items, p.h_world0);
    else
      launch_pdl(k_force_lbm_ws<R, false>, grid, kThreads, sizeof(WsSmem<R>), s, p.d_worlds, p.d_tile_items,
                 p.n_tile_items, p.h_world0);
  } else {
    if (p.n_worlds == 1)
      launch_pdl(k_force_lbm<R, true>, p.n_tile_items, kThreads, 0, s, p.d_worlds, p.d_tile_items, p.h_world0);
    else
      launch_pdl(k_force_lbm<R, false>, p.n_tile_items, kThreads, 0, s, p.d_worlds, p.d_tile_items, p.h_world0);
  }
}

void dispatch_steric(const Plan& p, cudaStream_t s, int which, int store_fields, int after_step) {
  if (!p.n_tile_items) return;
  switch (p.max_R) {
    case 1: launch_steric<1>(p, s, which, store_fields, after_step); break;
    case 2: launch_steric<2>(p, s, which, store_fields, after_step); break;
    case 3: launch_steric<3>(p, s, which, store_fields, after_step); break;
    case 4: launch_steric<4>(p, s, which, store_fields, after_step); break;
    case 5: launch_steric<5>(p, s, which, store_fields, after_step); break;
    case 6: launch_steric<6>(p, s, which, store_fields, after_step); break;
    case 7: launch_steric<7>(p, s, which, store_fields, after_step); break;
    default: launch_steric<kMaxR>(p, s, which, store_fields, after_step); break;
  }
}

}  // namespace

void steric_setup(int sms) {
  ws_setup<1>(sms);
  ws_setup<2>(sms);
  ws_setup<3>(sms);
  ws_setup<4>(sms);
  ws_setup<5>(sms);
  ws_setup<6>(sms);
  ws_setup<7>(sms);
  ws_setup<8>(sms);
}

void launch_deposit_x(const Plan& p, cudaStream_t s, int store_fields) { dispatch_steric(p, s, 0, store_fields, 0); }

// Two-layer worlds get F from their layer points after the tile pass.
void launch_force_spread(const Plan& p, cudaStream_t s, int store_fields, int after_step) {
  dispatch_steric(p, s, 1, store_fields, after_step);
  launch_layer_spread(p, s);
}

void launch_mdf_pass(const Plan& p, cudaStream_t s, int pass) {
  if (p.n_tile_items) k_mdf_pass<<<p.n_tile_items, kThreads, 0, s>>>(p.d_worlds, p.d_tile_items, pass);
}

void launch_force_lbm(const Plan& p, cudaStream_t s) {
  dispatch_steric(p, s, 2, 0, 0);
  if (p.any_layered) {
    launch_layer_spread(p, s);
    launch_lbm(p, s, 1);
  }
}

}  // namespace mc
