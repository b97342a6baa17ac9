// Grid-side stages of one time step: bin offsets (a2) and the fused D2Q9 TRT
// collide + stream (a7).  The steric and spread stages (a4-a6) are in
// k_steric.cu, the bead stages in k_bead.cu.
#include "grid_dev.cuh"

namespace mc {

template <bool kSingle>
__global__ void __launch_bounds__(256) k_scan_sums(const WorldDev* __restrict__ worlds,
                                                   const int2* __restrict__ items, int inc_t,
                                                   const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  __shared__ ScanSmem sm;
  scan_sums_body<kSingle>(worlds, items, inc_t, w1, blockIdx.x, sm);
}

template <bool kSingle>
__global__ void __launch_bounds__(256) k_scan_apply(const WorldDev* __restrict__ worlds,
                                                    const int2* __restrict__ items, int book, int inc_t,
                                                    const __grid_constant__ WorldDev w1) {
  pdl_trigger();
  pdl_wait();
  __shared__ ScanSmem sm;
  scan_apply_body<kSingle>(worlds, items, book, inc_t, w1, blockIdx.x, sm);
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
__global__ void __launch_bounds__(kCellChunk) k_lbm(const WorldDev* __restrict__ worlds,
                                                    const int2* __restrict__ items, int layered_only) {
  pdl_trigger();
  pdl_wait();
  const int2 it = items[blockIdx.x];
  const WorldDev& w = worlds[it.x];
  if (layered_only && w.layers != 2) return;
  const int W = w.W, H = w.H, HW = H * W;
  const int c = it.y + threadIdx.x;
  if (c >= HW) return;
  const int y = c / W, x = c - y * W;
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
  const long long t = *w.t;
  const LbmConst k{w.om_p, w.om_m, w.src_p, w.src_m};
  w.u[c] = lbm_cell(w.g[t & 1], w.g[(t + 1) & 1], HW, y * W, ym * W, yp * W, x, xm, xp, w.F[c], k);
}

// ---------------------------------------------------------------------------
// Launchers and the step sequence.
// ---------------------------------------------------------------------------
void launch_bin_scan(const Plan& p, cudaStream_t s, int inc_t) {
  // worlds of one scan block each need no block sums: one kernel (unless
  // the launch configuration asks for two)
  const int book = p.one_chunk && p.cfg.scan_kernels != 2 ? 1 : 0;
  if (p.n_worlds == 1) {   // integer work only: the single-world path cannot change a result
    if (!book) launch_pdl(k_scan_sums<true>, p.n_scan_items, 256, 0, s, p.d_worlds, p.d_scan_items, inc_t, p.h_world0);
    launch_pdl(k_scan_apply<true>, p.n_scan_items, 256, 0, s, p.d_worlds, p.d_scan_items, book, inc_t, p.h_world0);
  } else {
    if (!book) launch_pdl(k_scan_sums<false>, p.n_scan_items, 256, 0, s, p.d_worlds, p.d_scan_items, inc_t, p.h_world0);
    launch_pdl(k_scan_apply<false>, p.n_scan_items, 256, 0, s, p.d_worlds, p.d_scan_items, book, inc_t, p.h_world0);
  }
}

void launch_lbm(const Plan& p, cudaStream_t s, int layered_only) {
  if (p.n_cell_items) k_lbm<<<p.n_cell_items, kCellChunk, 0, s>>>(p.d_worlds, p.d_cell_items, layered_only);
}

// n steps; in plans without direct-forcing worlds every step after the
// first runs its PBD fused with the previous step's advance (the same
// arithmetic, one kernel and one position round trip fewer).
void enqueue_steps(const Plan& p, int n, cudaStream_t s) {
  if (p.any_mdf || n < 2) {
    for (int k = 0; k < n; ++k) enqueue_step(p, s);
    return;
  }
  for (int k = 0; k < n; ++k) {
    if (k == 0) launch_pbd(p, s);
    else launch_advance_pbd(p, s);   // a8 of step k - 1 + a1-a3 of step k
    launch_bin_scan(p, s, k > 0);
    launch_bin_scatter(p, s);
    launch_deposit_x(p, s, 0);
    launch_force_lbm(p, s);
  }
  launch_interp_advance(p, s);
}

void enqueue_step(const Plan& p, cudaStream_t s) {
  if (p.any_mdf) {
    // direct forcing: the steric spread and the MDF passes write F to device
    // memory before the LBM (the other worlds of the plan take the same
    // unfused sequence, which gives their step bitwise)
    launch_pbd(p, s);
    launch_mdf_bins(p, s);
    launch_bin_scan(p, s);
    launch_bin_scatter(p, s);
    launch_deposit_x(p, s, 0);
    launch_force_spread(p, s, 0);
    launch_mdf(p, s);
    launch_lbm(p, s);
    launch_interp_advance(p, s);
    return;
  }
  launch_pbd(p, s);              // a1 + a3 + a2 histogram
  launch_bin_scan(p, s);         // a2 offsets (one or two kernels)
  launch_bin_scatter(p, s);      // a2 scatter
  launch_deposit_x(p, s, 0);     // a4 + x pass of a5
  launch_force_lbm(p, s);        // y pass of a5 + a6 + a7
  launch_interp_advance(p, s);   // a8
}

}  // namespace mc
