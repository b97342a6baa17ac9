// Direct forcing with multi-direct-forcing (MDF) passes (Fluid-filament
// Interaction: the nodes sample the fluid velocity for their drag, the
// filament broadcasts its own velocity back onto the grid, MDF of Wang et
// al. 2008 against leakage).  For worlds with ib == 1 a step runs
//
//   k_mdf_bins      bins of X (a2) and F_el = 0, so the steric spread that
//                   follows puts only F_s on the grid;
//   (bins, deposit, steric spread: the penalty path's kernels)
//   k_mdf_moments   u* = (sum_i c_i f_i + F/2) / rho and rho of every cell
//                   (the fluid before the filament's forcing, in u);
//   k_pbd<.., 2>    X~ = X + dt I[u*](X), PBD from X~, and each bead's
//                   velocity U_s = I[u*](X) + (x_hat - X~)/dt (in ubead);
//   m passes of     k_mdf_force:  dF_i = 2 I[rho](X_i) (U_s,i - I[u](X_i)),
//                                 added to F_el,i and spread in 64-bit
//                                 fixed point (bitwise independent of order);
//                   k_mdf_update: F += S[dF], u += S[dF] / (2 rho);
//   (LBM with the total F, then X^{n+1} = X + dt U_s: the penalty path's
//   kernels, the advance reading U_s).
// Every kernel returns at once for the worlds of a batch that couple by
// the penalty force (and for a world's passes beyond its own m).
#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr double kMdfScale = 1099511627776.0;   // 2^40: fixed point of the MDF spread

// a2 for a direct-forcing world: the bin of every bead from X (its PBD runs
// after the steric spread), one histogram atomic per group of lanes sharing
// a bin, and F_el = 0 (the MDF passes accumulate the bead forces in it).
__global__ void __launch_bounds__(kBeadChunk) k_mdf_bins(const WorldDev* __restrict__ worlds,
                                                         const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1) return;
  const int i = it.y + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int bin = -1 - lane;
  if (i < w.N) {
    const float4 p = w.pos[i];
    bin = (cell_y(p) / kBin) * w.nbx + cell_x(p) / kBin;
    w.bead_bin[i] = bin;
    w.fel[i] = make_float2(0.0f, 0.0f);
  }
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if (i < w.N && (__ffs(peers) - 1) == lane) atomicAdd(&w.bin_count[bin], __popc(peers));
}

// u* and rho of every cell from the pulled populations and the steric F.
__global__ void __launch_bounds__(kCellChunk) k_mdf_moments(const WorldDev* __restrict__ worlds,
                                                            const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1) return;
  const int W = w.W, H = w.H, HW = H * W;
  const int c = it.y + threadIdx.x;
  if (c >= HW) return;
  const int y = c / W, x = c - y * W;
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
  LbmPull q;
  lbm_pull(w.g[*w.t & 1], HW, y * W, ym * W, yp * W, x, xm, xp, q);
  const float* d = q.d;
  const float drho = ((d[0] + (d[1] + d[3])) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  const float rho = 1.0f + drho;
  const float jx = (d[1] - d[3]) + (d[5] - d[7]) + (d[8] - d[6]);
  const float jy = (d[2] - d[4]) + (d[5] - d[7]) + (d[6] - d[8]);
  const float inv = __frcp_rn(rho);
  const float2 F = w.F[c];
  w.u[c] = make_float2((jx + 0.5f * F.x) * inv, (jy + 0.5f * F.y) * inv);
  w.mrho[c] = rho;
}

// Pass `pass` of a direct-forcing world: the force that makes the fluid at
// each bead move with U_s, and its spread.
__global__ void __launch_bounds__(kBeadChunk) k_mdf_force(const WorldDev* __restrict__ worlds,
                                                          const int2* __restrict__ items, int pass) {
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1 || pass >= w.mdf_iters) return;
  const int i = it.y + threadIdx.x;
  if (i >= w.N) return;
  const int W = w.W, H = w.H;
  const float4 p = w.pos[i];
  const int cx = cell_x(p), cy = cell_y(p);
  float wx[4], wy[4];
  peskin4(p.x, wx);
  peskin4(p.y, wy);
  int ix[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) ix[a] = wrap_once(cx - 1 + a, W);
  int iy[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) iy[b] = wrap_once(cy - 1 + b, H);
  float Ux = 0.0f, Uy = 0.0f, r = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float2* row = w.u + (size_t)iy[b] * W;
    const float* rrow = w.mrho + (size_t)iy[b] * W;
    float rx = 0.0f, ry = 0.0f, rr = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 v = row[ix[a]];
      rx = fmaf(wx[a], v.x, rx);
      ry = fmaf(wx[a], v.y, ry);
      rr = fmaf(wx[a], rrow[ix[a]], rr);
    }
    Ux = fmaf(wy[b], rx, Ux);
    Uy = fmaf(wy[b], ry, Uy);
    r = fmaf(wy[b], rr, r);
  }
  const float2 Us = w.ubead[i];
  const float dFx = 2.0f * r * (Us.x - Ux), dFy = 2.0f * r * (Us.y - Uy);
  float2 fe = w.fel[i];
  fe.x += dFx;
  fe.y += dFy;
  w.fel[i] = fe;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    unsigned long long* row = w.facc + 2 * (size_t)iy[b] * W;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float g = wx[a] * wy[b];
      unsigned long long* c = row + 2 * ix[a];
      atomicAdd(c, (unsigned long long)__double2ll_rn((double)(g * dFx) * kMdfScale));
      atomicAdd(c + 1, (unsigned long long)__double2ll_rn((double)(g * dFy) * kMdfScale));
    }
  }
}

// F += S[dF], u += S[dF] / (2 rho), and the accumulator cleared.
__global__ void __launch_bounds__(kCellChunk) k_mdf_update(const WorldDev* __restrict__ worlds,
                                                           const int2* __restrict__ items, int pass) {
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1 || pass >= w.mdf_iters) return;
  const int c = it.y + threadIdx.x;
  if (c >= w.H * w.W) return;
  const long long ax = (long long)w.facc[2 * c], ay = (long long)w.facc[2 * c + 1];
  const float Gx = (float)((double)ax / kMdfScale), Gy = (float)((double)ay / kMdfScale);
  float2 F = w.F[c];
  F.x += Gx;
  F.y += Gy;
  w.F[c] = F;
  const float h = 2.0f * w.mrho[c];
  float2 u = w.u[c];
  u.x += Gx / h;
  u.y += Gy / h;
  w.u[c] = u;
  w.facc[2 * c] = 0ull;
  w.facc[2 * c + 1] = 0ull;
}

}  // namespace

void launch_pbd_mdf(const Plan& p, cudaStream_t s);   // k_bead.cu

void launch_mdf_bins(const Plan& p, cudaStream_t s) {
  if (!p.any_mdf) return;
  k_mdf_bins<<<p.n_bead_items, kBeadChunk, 0, s>>>(p.d_worlds, p.d_bead_items);
}

void launch_mdf(const Plan& p, cudaStream_t s) {
  if (!p.any_mdf) return;
  if (p.n_cell_items) k_mdf_moments<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items);
  launch_pbd_mdf(p, s);
  for (int k = 0; k < p.max_mdf; ++k) {
    k_mdf_force<<<p.n_bead_items, kBeadChunk, 0, s>>>(p.d_worlds, p.d_bead_items, k);
    if (p.n_cell_items) k_mdf_update<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items, k);
  }
}

}  // namespace mc
