// Grid-side stages of one time step: bin offsets (a2), binned steric
// deposit (a4), Gaussian filter (a5), steric force + IB force spread (a6) and
// the fused D2Q9 TRT collide + stream (a7).
#include "mc_internal.cuh"

namespace mc {

// ---------------------------------------------------------------------------
// a2: exclusive prefix sum of the per-bin counts, one block per world.  Also
// resets the counts for the next step and primes the scatter cursors.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bin_scan(const WorldDev* __restrict__ worlds) {
  const WorldDev& w = worlds[blockIdx.x];
  __shared__ int warp_tot[32];
  __shared__ int carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = w.n_bins;
  int carry = 0;
  for (int base = 0; base < n; base += 1024) {
    const int k = base + tid;
    const int v = k < n ? w.bin_count[k] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const int warp_base = wid > 0 ? warp_tot[wid - 1] : 0;
    const int excl = carry + warp_base + incl - v;
    if (k < n) {
      w.bin_off[k] = excl;
      w.bin_cursor[k] = excl;
      w.bin_count[k] = 0;
    }
    if (tid == 1023) carry_s = carry + warp_tot[31];
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
  if (tid == 0) w.bin_off[n] = carry;
}

// ---------------------------------------------------------------------------
// Tile geometry shared by the tile kernels.  A tile is a kTile x kTile block
// of cells (ragged at the high edges); its beads are the beads of its bin.
// ---------------------------------------------------------------------------
struct TileGeom {
  int tx, ty, x0, y0, tw, th;
  int dx_lo, dx_hi, dy_lo, dy_hi;   // neighbour bin offsets, each bin once
};

__device__ __forceinline__ void nb_range(int nt, int& lo, int& hi) {
  if (nt == 1) { lo = 0; hi = 0; }
  else if (nt == 2) { lo = 0; hi = 1; }
  else { lo = -1; hi = 1; }
}

__device__ __forceinline__ TileGeom tile_geom(const WorldDev& w, int tile) {
  TileGeom g;
  g.tx = tile % w.ntx;
  g.ty = tile / w.ntx;
  g.x0 = g.tx * w.tile;
  g.y0 = g.ty * w.tile;
  g.tw = min(w.tile, w.W - g.x0);
  g.th = min(w.tile, w.H - g.y0);
  nb_range(w.ntx, g.dx_lo, g.dx_hi);
  nb_range(w.nty, g.dy_lo, g.dy_hi);
  return g;
}

__device__ __forceinline__ int nb_bin(const WorldDev& w, const TileGeom& g, int ddx, int ddy) {
  return wrap_once(g.ty + ddy, w.nty) * w.ntx + wrap_once(g.tx + ddx, w.ntx);
}

// Local tile coordinate of the four stencil cells c-1 .. c+2 along one axis,
// or -1 for cells outside the tile.  c in [0, n), o in [0, n).
__device__ __forceinline__ bool stencil_in_tile(int c, int o, int tw, int n, int l[4]) {
  bool any = false;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int v = wrap_once(c - 1 + a - o, n);
    l[a] = v < tw ? v : -1;
    any |= v < tw;
  }
  return any;
}

// ---------------------------------------------------------------------------
// a4: rho_s(c) = sum_i delta_h(c - X_i).  One block per tile gathers the
// beads of its 3x3 bin neighbourhood, accumulates the stencil weights that
// fall inside the tile in shared memory (64-bit fixed point), and writes
// every cell of the tile once.  No global atomics and no zeroing pass.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_deposit(const WorldDev* __restrict__ worlds,
                                                 const int2* __restrict__ items) {
  __shared__ unsigned long long acc[kTile * kTile];
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const TileGeom g = tile_geom(w, it.y);
  for (int c = threadIdx.x; c < kTile * kTile; c += blockDim.x) acc[c] = 0ull;
  __syncthreads();
  for (int ddy = g.dy_lo; ddy <= g.dy_hi; ++ddy)
    for (int ddx = g.dx_lo; ddx <= g.dx_hi; ++ddx) {
      const int nb = nb_bin(w, g, ddx, ddy);
      const int k1 = w.bin_off[nb + 1];
      for (int k = w.bin_off[nb] + threadIdx.x; k < k1; k += blockDim.x) {
        const float4 p = w.spos[k];
        int lx[4], ly[4];
        if (!stencil_in_tile(cell_x(p), g.x0, g.tw, w.W, lx)) continue;
        if (!stencil_in_tile(cell_y(p), g.y0, g.th, w.H, ly)) continue;
        float wx[4], wy[4];
        peskin4(p.x, wx);
        peskin4(p.y, wy);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (ly[b] < 0) continue;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (lx[a] < 0) continue;
            atomicAdd(&acc[ly[b] * kTile + lx[a]], (unsigned long long)to_fix(wx[a] * wy[b]));
          }
        }
      }
    }
  __syncthreads();
  for (int c = threadIdx.x; c < g.tw * g.th; c += blockDim.x) {
    const int ly = c / g.tw, lx = c - ly * g.tw;
    w.rho_s[(g.y0 + ly) * w.W + g.x0 + lx] = from_fix((long long)acc[ly * kTile + lx]);
  }
}

// ---------------------------------------------------------------------------
// a5: rho_bar = sum_m g_m rho_s(. - m e_x), then along y; periodic, taps
// normalised and truncated at R.  One block per tile with an R-cell halo.
// ---------------------------------------------------------------------------
constexpr int kBlurIn = kTile + 2 * kMaxR;

__global__ void __launch_bounds__(256) k_blur(const WorldDev* __restrict__ worlds,
                                              const int2* __restrict__ items) {
  __shared__ float in[kBlurIn * kBlurIn];
  __shared__ float mid[kBlurIn * kTile];
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const TileGeom g = tile_geom(w, it.y);
  const int R = w.R;
  const int iw = g.tw + 2 * R, ih = g.th + 2 * R;
  for (int c = threadIdx.x; c < iw * ih; c += blockDim.x) {
    const int ly = c / iw, lx = c - ly * iw;
    const int gy = wrap_once(g.y0 - R + ly, w.H), gx = wrap_once(g.x0 - R + lx, w.W);
    in[ly * kBlurIn + lx] = w.rho_s[gy * w.W + gx];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < g.tw * ih; c += blockDim.x) {
    const int ly = c / g.tw, lx = c - ly * g.tw;
    float s = 0.0f;
    for (int m = 0; m <= 2 * R; ++m) s = fmaf(w.taps[m], in[ly * kBlurIn + lx + m], s);
    mid[ly * kTile + lx] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < g.tw * g.th; c += blockDim.x) {
    const int ly = c / g.tw, lx = c - ly * g.tw;
    float s = 0.0f;
    for (int m = 0; m <= 2 * R; ++m) s = fmaf(w.taps[m], mid[(ly + m) * kTile + lx], s);
    w.rho_b[(g.y0 + ly) * w.W + g.x0 + lx] = s;
  }
}

// ---------------------------------------------------------------------------
// a6: steric force F_s,i = -k_rep sum_c delta_h(c - X_i) grad rho_bar(c) with
// central differences, then the IB spread F(c) = sum_i delta_h(c - X_i)
// (F_el,i + F_s,i).  One block per tile: the tile's rho_bar window (4-cell
// halo) is staged in shared memory; every bead of the 3x3 bin neighbourhood
// whose stencil touches the tile gets its steric force from the window and is
// spread into the tile (64-bit fixed point).  Beads of the tile's own bin also
// store their steric force.  Each cell of the tile is written once.
// ---------------------------------------------------------------------------
constexpr int kWin = kTile + 8;

__global__ void __launch_bounds__(256) k_force_spread(const WorldDev* __restrict__ worlds,
                                                      const int2* __restrict__ items) {
  __shared__ float win[kWin * kWin];
  __shared__ unsigned long long accx[kTile * kTile];
  __shared__ unsigned long long accy[kTile * kTile];
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const TileGeom g = tile_geom(w, it.y);
  const int ww = g.tw + 8, wh = g.th + 8;
  for (int c = threadIdx.x; c < ww * wh; c += blockDim.x) {
    const int ly = c / ww, lx = c - ly * ww;
    const int gy = wrap_once(g.y0 - 4 + ly, w.H), gx = wrap_once(g.x0 - 4 + lx, w.W);
    win[ly * kWin + lx] = w.rho_b[gy * w.W + gx];
  }
  for (int c = threadIdx.x; c < kTile * kTile; c += blockDim.x) {
    accx[c] = 0ull;
    accy[c] = 0ull;
  }
  __syncthreads();
  const float k_rep = w.k_rep;
  for (int ddy = g.dy_lo; ddy <= g.dy_hi; ++ddy)
    for (int ddx = g.dx_lo; ddx <= g.dx_hi; ++ddx) {
      const int nb = nb_bin(w, g, ddx, ddy);
      const bool own = nb == it.y;
      const int k1 = w.bin_off[nb + 1];
      for (int k = w.bin_off[nb] + threadIdx.x; k < k1; k += blockDim.x) {
        const float4 p = w.spos[k];
        const int cx = cell_x(p), cy = cell_y(p);
        int lx[4], ly[4];
        if (!stencil_in_tile(cx, g.x0, g.tw, w.W, lx)) continue;
        if (!stencil_in_tile(cy, g.y0, g.th, w.H, ly)) continue;
        // window coordinates: with several tiles on an axis pick the
        // periodic image of the bead next to this tile; with one tile the
        // window spans the whole axis plus a 4-cell margin.
        int rx = cx - g.x0, ry = cy - g.y0;
        if (w.ntx > 1) { if (rx < -4) rx += w.W; else if (rx > g.tw + 3) rx -= w.W; }
        if (w.nty > 1) { if (ry < -4) ry += w.H; else if (ry > g.th + 3) ry -= w.H; }
        float wx[4], wy[4];
        peskin4(p.x, wx);
        peskin4(p.y, wy);
        float gsx = 0.0f, gsy = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int ky = ry + 3 + b;
          float rx_s = 0.0f, ry_s = 0.0f;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int kx = rx + 3 + a;
            const float gx = 0.5f * (win[ky * kWin + kx + 1] - win[ky * kWin + kx - 1]);
            const float gy = 0.5f * (win[(ky + 1) * kWin + kx] - win[(ky - 1) * kWin + kx]);
            rx_s = fmaf(wx[a], gx, rx_s);
            ry_s = fmaf(wx[a], gy, ry_s);
          }
          gsx = fmaf(wy[b], rx_s, gsx);
          gsy = fmaf(wy[b], ry_s, gsy);
        }
        const float2 Fs = make_float2(-k_rep * gsx, -k_rep * gsy);
        if (own) w.fs[w.sid[k]] = Fs;
        const float2 fe = w.sfel[k];
        const float Fx = fe.x + Fs.x, Fy = fe.y + Fs.y;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (ly[b] < 0) continue;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (lx[a] < 0) continue;
            const float wgt = wx[a] * wy[b];
            const int c = ly[b] * kTile + lx[a];
            atomicAdd(&accx[c], (unsigned long long)to_fix(wgt * Fx));
            atomicAdd(&accy[c], (unsigned long long)to_fix(wgt * Fy));
          }
        }
      }
    }
  __syncthreads();
  for (int c = threadIdx.x; c < g.tw * g.th; c += blockDim.x) {
    const int ly = c / g.tw, lx = c - ly * g.tw;
    const int s = ly * kTile + lx;
    w.F[(g.y0 + ly) * w.W + g.x0 + lx] =
        make_float2(from_fix((long long)accx[s]), from_fix((long long)accy[s]));
  }
}

// ---------------------------------------------------------------------------
// a7: D2Q9 lattice Boltzmann, TRT collision with Guo forcing, periodic
// streaming, fused in one pass per cell.  The state is the post-collision
// population minus the rest weight w_i (shifted storage keeps FP32 precision
// on the small deviations); a cell pulls f_i(c) = g_i(c - c_i), collides and
// stores its own post-collision populations.  With d_i = f_i - w_i:
//   rho = 1 + sum d_i,  u = (sum c_i d_i + F/2) / rho
//   feq_i - w_i = w_i [delta_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]
//   S_i = w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]
//   d*_i = d_i - (d+ - e+)/tau+ - (d- - e-)/tau- + (1 - 1/(2tau+)) S+ + (1 - 1/(2tau-)) S-
// evaluated per opposite pair (i, opp(i)) from the even and odd parts.
// ---------------------------------------------------------------------------
struct PairOut {
  float a, b;
};

__device__ __forceinline__ PairOut trt_pair(float di, float dib, float wi, float cu, float cF, float drho,
                                            float rho, float uu, float uF, const WorldDev& w) {
  const float ep = wi * (drho + rho * (4.5f * cu * cu - 1.5f * uu));
  const float em = wi * rho * 3.0f * cu;
  const float sp = wi * (9.0f * cu * cF - 3.0f * uF);
  const float sm = wi * 3.0f * cF;
  const float dp = 0.5f * (di + dib), dm = 0.5f * (di - dib);
  const float even = -w.om_p * (dp - ep) + w.src_p * sp;
  const float odd = -w.om_m * (dm - em) + w.src_m * sm;
  PairOut o;
  o.a = di + even + odd;
  o.b = dib + even - odd;
  return o;
}

__global__ void __launch_bounds__(kCellChunk) k_lbm(const WorldDev* __restrict__ worlds,
                                                    const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  const int W = w.W, H = w.H, HW = H * W;
  const int c = it.y + threadIdx.x;
  if (c >= HW) return;
  const int y = c / W, x = c - y * W;
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
  const long long t = *w.t;
  const float* __restrict__ src = w.g[t & 1];
  float* __restrict__ dst = w.g[(t + 1) & 1];
  const int r0 = y * W, rm = ym * W, rp = yp * W;
  const float d0 = src[c];
  const float d1 = src[1 * HW + r0 + xm];   // c = ( 1, 0) pulls from (x-1, y)
  const float d2 = src[2 * HW + rm + x];    // ( 0, 1) from (x, y-1)
  const float d3 = src[3 * HW + r0 + xp];   // (-1, 0) from (x+1, y)
  const float d4 = src[4 * HW + rp + x];    // ( 0,-1) from (x, y+1)
  const float d5 = src[5 * HW + rm + xm];   // ( 1, 1) from (x-1, y-1)
  const float d6 = src[6 * HW + rm + xp];   // (-1, 1) from (x+1, y-1)
  const float d7 = src[7 * HW + rp + xp];   // (-1,-1) from (x+1, y+1)
  const float d8 = src[8 * HW + rp + xm];   // ( 1,-1) from (x-1, y+1)
  const float2 F = w.F[c];

  const float drho = ((d0 + (d1 + d3)) + (d2 + d4)) + ((d5 + d7) + (d6 + d8));
  const float rho = 1.0f + drho;
  const float jx = (d1 - d3) + (d5 - d7) + (d8 - d6);
  const float jy = (d2 - d4) + (d5 - d7) + (d6 - d8);
  const float inv = 1.0f / rho;
  const float ux = (jx + 0.5f * F.x) * inv;
  const float uy = (jy + 0.5f * F.y) * inv;
  const float uu = ux * ux + uy * uy;
  const float uF = ux * F.x + uy * F.y;

  constexpr float w0 = 4.0f / 9.0f, w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
  const float e0 = w0 * (drho - 1.5f * rho * uu);
  const float s0 = w0 * (-3.0f * uF);
  dst[c] = d0 - w.om_p * (d0 - e0) + w.src_p * s0;
  const PairOut p13 = trt_pair(d1, d3, w1, ux, F.x, drho, rho, uu, uF, w);
  const PairOut p24 = trt_pair(d2, d4, w1, uy, F.y, drho, rho, uu, uF, w);
  const PairOut p57 = trt_pair(d5, d7, w5, ux + uy, F.x + F.y, drho, rho, uu, uF, w);
  const PairOut p68 = trt_pair(d6, d8, w5, uy - ux, F.y - F.x, drho, rho, uu, uF, w);
  dst[1 * HW + c] = p13.a;
  dst[3 * HW + c] = p13.b;
  dst[2 * HW + c] = p24.a;
  dst[4 * HW + c] = p24.b;
  dst[5 * HW + c] = p57.a;
  dst[7 * HW + c] = p57.b;
  dst[6 * HW + c] = p68.a;
  dst[8 * HW + c] = p68.b;
  w.u[c] = make_float2(ux, uy);
}

// ---------------------------------------------------------------------------
// Launchers and the step sequence.
// ---------------------------------------------------------------------------
void launch_bin_scan(const Plan& p, cudaStream_t s) {
  k_bin_scan<<<p.n_worlds, 1024, 0, s>>>(p.d_worlds);
}

void launch_deposit(const Plan& p, cudaStream_t s) {
  if (p.n_tile_items) k_deposit<<<p.n_tile_items, 256, 0, s>>>(p.d_worlds, p.d_tile_items);
}

void launch_blur(const Plan& p, cudaStream_t s) {
  if (p.n_tile_items) k_blur<<<p.n_tile_items, 256, 0, s>>>(p.d_worlds, p.d_tile_items);
}

void launch_force_spread(const Plan& p, cudaStream_t s) {
  if (p.n_tile_items) k_force_spread<<<p.n_tile_items, 256, 0, s>>>(p.d_worlds, p.d_tile_items);
}

void launch_lbm(const Plan& p, cudaStream_t s) {
  if (p.n_cell_items) k_lbm<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items);
}

void enqueue_step(const Plan& p, cudaStream_t s) {
  launch_pbd(p, s);             // a1 + a3 + a2 histogram
  launch_bin_scan(p, s);        // a2 offsets
  launch_bin_scatter(p, s);     // a2 scatter
  launch_deposit(p, s);         // a4
  launch_blur(p, s);            // a5
  launch_force_spread(p, s);    // a6
  launch_lbm(p, s);             // a7
  launch_interp_advance(p, s);  // a8
}

}  // namespace mc
