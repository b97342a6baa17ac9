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
//                   velocity U_s = I[u*](X) + (x_hat - X~)/dt (in ubead,
//                   and in bin order in sus);
//   m passes of     k_mdf_pass (k_steric.cu), one per 32x32 tile, Jacobi in
//                   u (u -> u2 -> u ...): dF_i = 2 I[rho](X_i) (U_s,i -
//                   I[u](X_i)) for every bead whose stencil reaches the
//                   tile, the spread S[dF] in int32 fixed point (bitwise
//                   independent of order), F += S[dF] and
//                   u' = u + S[dF] / (2 rho) on the tile's cells, and
//                   F_el += dF on the bead's own tile;
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
  for (int k = 0; k < p.max_mdf; ++k) launch_mdf_pass(p, s, k);
}

// launch_mdf for the one world h of plan p, keeping u_0 (the drag's
// velocity) and each pass's input velocity (u_0 .. u_{m-1}, m =
// h.mdf_iters) in mu[k H W ..] for the reverse mode.
cudaError_t launch_mdf_recorded(const Plan& p, const WorldDev& h, float2* mu, cudaStream_t s) {
  const size_t bytes = (size_t)h.H * h.W * sizeof(float2);
  if (p.n_cell_items) k_mdf_moments<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items);
  cudaError_t e = cudaSuccess;
  e = cudaMemcpyAsync(mu, h.u, bytes, cudaMemcpyDeviceToDevice, s);
  launch_pbd_mdf(p, s);
  for (int k = 0; k < h.mdf_iters && e == cudaSuccess; ++k) {
    launch_mdf_pass(p, s, k);
    // pass k writes u2 (k even) or u (k odd)
    if (k + 1 < h.mdf_iters)
      e = cudaMemcpyAsync(reinterpret_cast<char*>(mu) + (k + 1) * bytes, (k & 1) ? h.u : h.u2, bytes,
                          cudaMemcpyDeviceToDevice, s);
  }
  return e;
}

}  // namespace mc
