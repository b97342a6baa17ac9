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
//                                 added to F_el,i and written to the bead's
//                                 slot of the bin-ordered records;
//                   k_mdf_spread: per 32x32 tile (k_steric.cu) the spread
//                                 S[dF] in int32 fixed point (bitwise
//                                 independent of order), then F += S[dF],
//                                 u += S[dF] / (2 rho) on the tile's cells;
//   (LBM with the total F, then X^{n+1} = X + dt U_s: the penalty path's
//   kernels, the advance reading U_s).
// Every kernel returns at once for the worlds of a batch that couple by
// the penalty force (and for a world's passes beyond its own m).
#include "mc_internal.cuh"

namespace mc {

namespace {

// a2 for a direct-forcing world: the bin of every bead from X (its PBD runs
// after the steric spread), one histogram atomic per group of lanes sharing
// a bin, and F_el = 0 (the MDF passes accumulate the bead forces in it).
__global__ void __launch_bounds__(kBeadChunk) k_mdf_bins(const WorldDev* __restrict__ worlds,
                                                         const int2* __restrict__ items) {
  pdl_trigger();
  pdl_wait();
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
  pdl_trigger();
  pdl_wait();
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
  if (c == 0) {
    w.mdf_max[0] = 0u;
    w.mdf_max[1] = 0u;
  }
}

// Pass `pass` of a direct-forcing world: the force that makes the fluid at
// each bead move with U_s, into F_el and the bead's bin-ordered slot, and
// the pass's largest component (bounds the spread's fixed-point scale).
__global__ void __launch_bounds__(kBeadChunk) k_mdf_force(const WorldDev* __restrict__ worlds,
                                                          const int2* __restrict__ items, int pass) {
  pdl_trigger();
  pdl_wait();
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (w.ib != 1 || pass >= w.mdf_iters) return;
  const int i = it.y + threadIdx.x;
  float m = 0.0f;
  if (i < w.N) {
    const int W = w.W, H = w.H;
    const float4 p = w.pos[i];
    const int cx = cell_x(p), cy = cell_y(p);
    float wx[4], wy[4];
    peskin4(p.x, wx);
    peskin4(p.y, wy);
    int ix[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ix[a] = wrap_once(cx - 1 + a, W);
    float Ux = 0.0f, Uy = 0.0f, r = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const size_t row = (size_t)wrap_once(cy - 1 + b, H) * W;
      float rx = 0.0f, ry = 0.0f, rr = 0.0f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float2 v = w.u[row + ix[a]];
        rx = fmaf(wx[a], v.x, rx);
        ry = fmaf(wx[a], v.y, ry);
        rr = fmaf(wx[a], w.mrho[row + ix[a]], rr);
      }
      Ux = fmaf(wy[b], rx, Ux);
      Uy = fmaf(wy[b], ry, Uy);
      r = fmaf(wy[b], rr, r);
    }
    const float2 Us = w.ubead[i];
    const float2 dF = make_float2(2.0f * r * (Us.x - Ux), 2.0f * r * (Us.y - Uy));
    float2 fe = w.fel[i];
    fe.x += dF.x;
    fe.y += dF.y;
    w.fel[i] = fe;
    w.sfel[w.bead_slot[i]] = dF;
    m = fmaxf(fabsf(dF.x), fabsf(dF.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&w.mdf_max[pass & 1], __float_as_uint(m));
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
    launch_mdf_spread(p, s, k);
  }
}

}  // namespace mc
