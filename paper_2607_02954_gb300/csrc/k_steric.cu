// a4-a6: steric deposit, Gaussian filter, steric force and immersed-boundary
// force spread, in two tile kernels (one 32x32 tile of cells per block).
//
//   rho_s(c)  = sum_i delta_h(c - X_i)                        (a4, Fields)
//   rho_bar   = G_sigma * rho_s, periodic, x pass then y pass  (a5, Fields)
//   F_s,i     = -k_rep sum_c delta_h(c - X_i) grad rho_bar(c)  (a6, central differences)
//   F(c)      = sum_i delta_h(c - X_i) (F_el,i + F_s,i)       (a6, Fluid-filament Interaction)
//
// k_deposit_x    deposits rho_s on the tile plus R columns on each side in
//                shared memory, applies the x pass of the filter and writes
//                the x-filtered density rho_x of the tile (4 B per cell) and
//                the tile's largest rho_s.
// k_force_spread loads rho_x on the tile plus 4 + R rows and 4 columns,
//                applies the y pass (rho_bar on the tile plus 4 cells),
//                gathers the steric force of every bead whose stencil touches
//                the tile, spreads F_el + F_s into the tile and writes F.
//
// Beads are sorted by 8x8-cell bins in row-major order, so the beads that
// can reach a tile lie in a few contiguous segments of the sorted arrays,
// one per bin row (two where the row range wraps around the periodic edge).
// Grid windows and bead records are staged in shared memory with cp.async,
// every copy in flight at once, and all arithmetic reads shared memory.
//
// Periodic images: with several tiles on an axis a bead is taken at its
// image in [-2, n - 2) relative to the tile origin; with one tile the tile is
// the whole axis.  In both cases the tile column of stencil cell a is
// wrap(rx - 1 + a) and it lies in the tile iff it is below the tile width.
#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr int kMaxSeg = 32;
constexpr int kRegX = kTile + 2 * kMaxR;   // deposit region columns (max)
constexpr int kWin = kTile + 8;            // rho_bar window edge
constexpr int kLoadRows = kTile + 8 + 2 * kMaxR;
constexpr int kWarps = 8;
constexpr int kDepCap = 1024;              // bead records staged per pass (deposit)
constexpr int kForceCap = 640;             // bead records staged per pass (force)

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((b - 1 - a) / b); }

// Bead segments of the bins whose cells reach the cell box
// [x_lo, x_hi] x [y_lo, y_hi] (inclusive, unwrapped coordinates), built by
// one warp: lane 2r + q handles part q of bin row r (a row's column range is
// split in two where it wraps), so all bin offsets load in one round trip.
// Fills s_start[32] and s_pre[33] (prefix of segment lengths; empty
// segments have length 0).  With max_count non-null, also returns the
// largest bead count of a single bin in the box.
__device__ void build_segments(const WorldDev& w, int x_lo, int x_hi, int y_lo, int y_hi, int* s_start,
                               int* s_pre, int* max_count) {
  const int lane = threadIdx.x & 31;
  const int nbx = w.nbx, nby = w.nby;
  int bx0 = floor_div(x_lo, kBin), bx1 = floor_div(x_hi, kBin);
  int by0 = floor_div(y_lo, kBin), by1 = floor_div(y_hi, kBin);
  if (bx1 - bx0 + 1 >= nbx) { bx0 = 0; bx1 = nbx - 1; }
  if (by1 - by0 + 1 >= nby) { by0 = 0; by1 = nby - 1; }
  const int r = lane >> 1, q = lane & 1;
  int lo, hi;
  bool split;
  if (bx0 < 0) {
    split = true;
    lo = q == 0 ? bx0 + nbx : 0;
    hi = q == 0 ? nbx - 1 : bx1;
  } else if (bx1 >= nbx) {
    split = true;
    lo = q == 0 ? bx0 : 0;
    hi = q == 0 ? nbx - 1 : bx1 - nbx;
  } else {
    split = false;
    lo = bx0;
    hi = bx1;
  }
  const bool valid = by0 + r <= by1 && (split || q == 0);
  int s0 = 0, len = 0;
  if (valid) {
    const int row = wrap_once(by0 + r, nby) * nbx;
    s0 = w.bin_off[row + lo];
    len = w.bin_off[row + hi + 1] - s0;
  }
  int incl = len;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  s_start[lane] = s0;
  s_pre[lane + 1] = incl;
  if (lane == 0) s_pre[0] = 0;
  if (max_count) {
    int m = 0;
    const int ncol = bx1 - bx0 + 1, nrow = by1 - by0 + 1;
    for (int k = lane; k < ncol * nrow; k += 32) {
      const int rr = k / ncol, cc = k - rr * ncol;
      const int bin = wrap_once(by0 + rr, nby) * nbx + wrap_once(bx0 + cc, nbx);
      m = max(m, w.bin_off[bin + 1] - w.bin_off[bin]);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) *max_count = m;
  }
}

__device__ __forceinline__ int seg_slot(int v, const int* s_start, const int* s_pre) {
  int j = 0;
  while (v >= s_pre[j + 1]) ++j;
  return s_start[j] + v - s_pre[j];
}

// Periodic image of d in [-2, n - 2).
__device__ __forceinline__ int image(int d, int n) {
  if (d < -2) d += n;
  else if (d >= n - 2) d -= n;
  return d;
}

__device__ __forceinline__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = red[0];
  for (int k = 1; k < kWarps; ++k) m = fmaxf(m, red[k]);
  __syncthreads();
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// a4 + the x pass of a5.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_deposit_x(const WorldDev* __restrict__ worlds,
                                                   const int2* __restrict__ items, int store_fields) {
  __shared__ int acc[kTile * kRegX];
  __shared__ float rsf[kTile * kRegX];
  __shared__ float4 sp[kDepCap];
  __shared__ float taps[2 * kMaxR + 1];
  __shared__ int s_start[kMaxSeg], s_pre[kMaxSeg + 1], s_maxc;
  __shared__ float red[kWarps];
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const int W = w.W, H = w.H, R = w.R, ntx = w.ntx;
  const int tx = it.y % ntx, ty = it.y / ntx;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int tw = min(kTile, W - x0), th = min(kTile, H - y0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // x: region = tile +- R columns, or the whole periodic axis when it is short
  const bool full_x = W < tw + 2 * R + 3;
  const int ox = full_x ? 0 : x0 - R;
  const int extx = full_x ? W : tw + 2 * R;
  const bool full_y = w.nty == 1;
  if (warp == 0) build_segments(w, x0 - R - 2, x0 + tw + R, y0 - 2, y0 + th, s_start, s_pre, &s_maxc);
  if (warp == 1 && lane <= 2 * R) taps[lane] = w.taps[lane];
  for (int c = threadIdx.x; c < th * kRegX; c += blockDim.x) acc[c] = 0;
  __syncthreads();
  const int total = s_pre[kMaxSeg];
  // a cell's 4x4 stencil neighbourhood overlaps at most 2x2 bins and each
  // bead adds at most 1/4: the cell sum is below the largest bin count
  const int k = fix_exponent((float)s_maxc + 1.0f);
  const float scale = ldexpf(1.0f, k);
  for (int c0 = 0; c0 < total; c0 += kDepCap) {
    const int n = min(kDepCap, total - c0);
    for (int v = threadIdx.x; v < n; v += blockDim.x) cp_async16(&sp[v], &w.spos[seg_slot(c0 + v, s_start, s_pre)]);
    cp_async_wait_all();
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const float4 p = sp[v];
      int rx = cell_x(p) - ox, ry = cell_y(p) - y0;
      if (!full_x) {
        rx = image(rx, W);
        if (rx > extx) continue;
      }
      if (!full_y) {
        ry = image(ry, H);
        if (ry > th) continue;
      }
      float wx[4], wy[4];
      peskin4(p.x, wx);
      peskin4(p.y, wy);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int row = wrap_once(ry - 1 + b, H);
        if (row >= th) continue;
        const float sy = wy[b] * scale;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int col = full_x ? wrap_once(rx - 1 + a, W) : rx - 1 + a;
          if ((unsigned)col >= (unsigned)extx) continue;
          atomicAdd(&acc[row * kRegX + col], __float2int_rn(wx[a] * sy));
        }
      }
    }
    __syncthreads();
  }
  const float inv = ldexpf(1.0f, -k);
  const int cbase = full_x ? x0 : R;   // region column of tile column 0
  float vmax = 0.0f;
  for (int row = warp; row < th; row += kWarps) {
    for (int col = lane; col < extx; col += 32) {
      const float v = (float)acc[row * kRegX + col] * inv;
      rsf[row * kRegX + col] = v;
      const int lx = col - cbase;
      if (lx >= 0 && lx < tw) {
        vmax = fmaxf(vmax, v);
        if (store_fields) w.rho_s[(y0 + row) * W + x0 + lx] = v;
      }
    }
  }
  vmax = block_max(vmax, red);   // includes the barrier the x pass needs
  if (threadIdx.x == 0) w.tile_rho_max[it.y] = vmax;
  for (int row = warp; row < th; row += kWarps) {
    const float* r = rsf + row * kRegX;
    if (lane < tw) {
      float s = 0.0f;
      if (full_x) {
        for (int m = 0; m <= 2 * R; ++m) s = fmaf(taps[m], r[wrap_mod(x0 + lane - R + m, W)], s);
      } else {
        for (int m = 0; m <= 2 * R; ++m) s = fmaf(taps[m], r[lane + m], s);
      }
      w.rho_x[(y0 + row) * W + x0 + lane] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// The y pass of a5, and a6.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_force_spread(const WorldDev* __restrict__ worlds,
                                                      const int2* __restrict__ items, int store_fields,
                                                      int after_step) {
  __shared__ float xb[kLoadRows * kWin];
  __shared__ float win[kWin * kWin];
  __shared__ int accx[kTile * kTile], accy[kTile * kTile];
  __shared__ float4 sp[kForceCap];
  __shared__ float2 sf[kForceCap];
  __shared__ int si[kForceCap];
  __shared__ float taps[2 * kMaxR + 1];
  __shared__ int s_start[kMaxSeg], s_pre[kMaxSeg + 1];
  __shared__ float red[16];
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const int W = w.W, H = w.H, R = w.R, ntx = w.ntx, nty = w.nty;
  const int tx = it.y % ntx, ty = it.y / ntx;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int tw = min(kTile, W - x0), th = min(kTile, H - y0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ww = tw + 8, wh = th + 8, lh = wh + 2 * R;
  // 1. bead segments (one round trip), then every other load in one batch
  if (warp == 0) build_segments(w, x0 - 2, x0 + tw, y0 - 2, y0 + th, s_start, s_pre, nullptr);
  __syncthreads();
  const int total = s_pre[kMaxSeg];
  {
    // rho_x rows [y0 - 4 - R, y0 + th + 4 + R) x columns [x0 - 4, x0 + tw + 4), wrapped
    // offsets reach at most 4 + R <= 12 cells outside the axis: one
    // conditional correction suffices unless the axis is shorter than that
    const int gx0 = W >= 16 ? wrap_once(x0 - 4 + lane, W) : wrap_mod(x0 - 4 + lane, W);
    const int gx1 = W >= 44 ? wrap_once(x0 + 28 + lane, W) : wrap_mod(x0 + 28 + lane, W);
    for (int i = warp; i < lh; i += kWarps) {
      const int gy = y0 - 4 - R + i;
      const float* src = w.rho_x + (size_t)(H >= 2 * kMaxR + 8 ? wrap_once(gy, H) : wrap_mod(gy, H)) * W;
      if (lane < ww) cp_async4(&xb[i * kWin + lane], src + gx0);
      if (lane + 32 < ww) cp_async4(&xb[i * kWin + 32 + lane], src + gx1);
    }
  }
  const int n0 = min(kForceCap, total);
  for (int v = threadIdx.x; v < n0; v += blockDim.x) {
    const int slot = seg_slot(v, s_start, s_pre);
    cp_async16(&sp[v], &w.spos[slot]);
    cp_async8(&sf[v], &w.sfel[slot]);
    cp_async4(&si[v], &w.sid[slot]);
  }
  if (warp == 1 && lane <= 2 * R) taps[lane] = w.taps[lane];
  // bound of the cell sums of weight * |F_el + F_s|:
  //   |F_s| <= k_rep/2 max|rho_bar(c+1) - rho_bar(c-1)| <= k_rep/2 max rho_bar
  //        <= k_rep/2 max rho_s over the 3x3 tiles around this one,
  // times max rho_s of this tile (the sum of the spread weights of a cell)
  if (warp == 2 && lane < 9) {
    const int ty2 = wrap_once(ty + lane / 3 - 1, nty), tx2 = wrap_once(tx + lane % 3 - 1, ntx);
    red[lane] = w.tile_rho_max[ty2 * ntx + tx2];
  }
  for (int c = threadIdx.x; c < kTile * kTile; c += blockDim.x) {
    accx[c] = 0;
    accy[c] = 0;
  }
  const long long t = *w.t - after_step;
  const float fmax_el = __uint_as_float(w.fel_max[t & 1]);
  const float rho_max = w.tile_rho_max[it.y];
  cp_async_wait_all();
  __syncthreads();
  float rho_nb = red[0];
  for (int k2 = 1; k2 < 9; ++k2) rho_nb = fmaxf(rho_nb, red[k2]);
  const float k_rep = w.k_rep;
  const int k = fix_exponent((fmax_el + 0.5f * k_rep * rho_nb) * rho_max * 1.0001f + 1e-30f);
  const float scale = ldexpf(1.0f, k);
  for (int i = warp; i < wh; i += kWarps) {
    for (int j = lane; j < ww; j += 32) {
      float s = 0.0f;
      for (int m = 0; m <= 2 * R; ++m) s = fmaf(taps[m], xb[(i + m) * kWin + j], s);
      win[i * kWin + j] = s;
      if (store_fields && i >= 4 && i < th + 4 && j >= 4 && j < tw + 4) w.rho_b[(y0 + i - 4) * W + x0 + j - 4] = s;
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < total; c0 += kForceCap) {
    const int n = min(kForceCap, total - c0);
    if (c0 > 0) {   // the first chunk was staged with the window
      for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int slot = seg_slot(c0 + v, s_start, s_pre);
        cp_async16(&sp[v], &w.spos[slot]);
        cp_async8(&sf[v], &w.sfel[slot]);
        cp_async4(&si[v], &w.sid[slot]);
      }
      cp_async_wait_all();
      __syncthreads();
    }
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const float4 p = sp[v];
      const int cx = cell_x(p), cy = cell_y(p);
      int rx = cx - x0, ry = cy - y0;
      if (ntx > 1) {
        rx = image(rx, W);
        if (rx < -2 || rx > tw) continue;
      }
      if (nty > 1) {
        ry = image(ry, H);
        if (ry < -2 || ry > th) continue;
      }
      float wx[4], wy[4];
      peskin4(p.x, wx);
      peskin4(p.y, wy);
      // stencil cell a sits at window column rx + 3 + a; the central
      // differences read one cell further on each side
      const float* base = win + (ry + 2) * kWin + rx + 2;
      float gsx = 0.0f, gsy = 0.0f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float* rowm = base + b * kWin;
        const float* row0 = rowm + kWin;
        const float* rowp = row0 + kWin;
        float sx = 0.0f, sy = 0.0f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          sx = fmaf(wx[a], row0[a + 2] - row0[a], sx);
          sy = fmaf(wx[a], rowp[a + 1] - rowm[a + 1], sy);
        }
        gsx = fmaf(wy[b], sx, gsx);
        gsy = fmaf(wy[b], sy, gsy);
      }
      const float Fsx = -0.5f * k_rep * gsx, Fsy = -0.5f * k_rep * gsy;
      if (cx >= x0 && cx < x0 + tw && cy >= y0 && cy < y0 + th) w.fs[si[v]] = make_float2(Fsx, Fsy);
      const float2 fe = sf[v];
      const float Fx = (fe.x + Fsx) * scale, Fy = (fe.y + Fsy) * scale;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int ly = wrap_once(ry - 1 + b, H);
        if (ly >= th) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int lx = wrap_once(rx - 1 + a, W);
          if (lx >= tw) continue;
          const float wgt = wx[a] * wy[b];
          atomicAdd(&accx[ly * kTile + lx], __float2int_rn(wgt * Fx));
          atomicAdd(&accy[ly * kTile + lx], __float2int_rn(wgt * Fy));
        }
      }
    }
    __syncthreads();
  }
  const float inv = ldexpf(1.0f, -k);
  for (int ly = warp; ly < th; ly += kWarps) {
    if (lane < tw) {
      const int s = ly * kTile + lane;
      w.F[(y0 + ly) * W + x0 + lane] = make_float2((float)accx[s] * inv, (float)accy[s] * inv);
    }
  }
}

void launch_deposit_x(const Plan& p, cudaStream_t s, int store_fields) {
  if (p.n_tile_items) k_deposit_x<<<p.n_tile_items, 256, 0, s>>>(p.d_worlds, p.d_tile_items, store_fields);
}

void launch_force_spread(const Plan& p, cudaStream_t s, int store_fields, int after_step) {
  if (p.n_tile_items)
    k_force_spread<<<p.n_tile_items, 256, 0, s>>>(p.d_worlds, p.d_tile_items, store_fields, after_step);
}

}  // namespace mc
