// Reverse-mode (adjoint) kernels of one time step, and the folding loss.
//
// The paper differentiates its simulator end to end with automatic
// differentiation (Filament Folding experiment); these kernels are the
// hand-written transpose of each forward stage, applied in reverse order:
//   a8  X^{n+1} = X^n + dt U,  U_i = sum_c w(c - X_i) u(c)
//   a7  per cell (g^{n+1}, u) = collide(pull(g^n), F)
//   a6  F(c) = sum_i w(c - X_i) Ftot_i,  F_s,i = -k_rep sum_c w(c - X_i) grad rho_bar(c)
//   a5  rho_bar = G rho_s (G symmetric)
//   a4  rho_s(c) = sum_i w(c - X_i)
//   a3  F_el = kappa/dt (x_hat - X) with (x_hat, theta^{n+1}) = PBD(X^n, theta^n, theta_rest)
//   a1  theta_rest = theta0 + drive(t)
// w(c - X) = phi(c_x - X_x) phi(c_y - X_y) (Peskin 4-point); its gradient
// with respect to X uses phi' at the same four cells per axis.  The adjoint
// scatters (transposed gathers) accumulate in 64-bit fixed point: each term
// is rounded once to a scale 2^k with N max|term| 2^k < 2^62, the bound
// taken from the largest term's factor (a grid-wide maximum, which does not
// depend on order), so the integer sums, and every gradient, are bitwise
// repeatable.  The stiffness gradients are summed per filament and then
// over filaments in a fixed order.
#include <algorithm>

#include "adj_dev.cuh"

namespace mc {

// ---------------------------------------------------------------------------
// a8 transposed: u_bar(c) += sum_i w(c - X_i) dt X_bar_i, fixed point with
// the bound N max|dt X_bar| (slot a.par of amax, written by the kernel that
// produced X_bar).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ubar_exponent(const WorldDev& w, const AdjDev& a) {
  return fix_exponent64((float)w.N * __uint_as_float(a.amax[a.par]));
}

__global__ void __launch_bounds__(256) k_adj_spread_u(const WorldDev* __restrict__ wd, AdjDev a) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (a.setup && i == 0) {
    // the bounds this step's kernels produce: of Q (k_adj_lbm) and of the
    // next reversed step's u_bar (k_adj_pbd; this step's u_bar reads slot
    // a.par).  (The step's counter comes with a.t_step: the world's own
    // counter belongs to a recompute that may run meanwhile.)
    a.amax[2] = 0u;
    a.amax[a.par ^ 1] = 0u;
  }
  if (i >= w.N) return;
  const float scale = pow2f(ubar_exponent(w, a));
  const float2 xb = a.adjX[i];
  const float ux = w.dt * xb.x * scale, uy = w.dt * xb.y * scale;
  auto spread = [&](const Stencil& s, float h) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float wgt = s.wx[c] * s.wy[b] * h;
        unsigned long long* g = &a.ubar[2 * (s.iy[b] + s.ix[c])];
        atomicAdd(g, fx64(wgt * ux));
        atomicAdd(g + 1, fx64(wgt * uy));
      }
  };
  if (w.layers == 2) {
    // U = (I[u](X + d n) + I[u](X - d n)) / 2
    const float4 p = w.pos[i];
    const float2 n = a.nrm[i];
    spread(make_layer_stencil(p, n, w.layer_half, w.W, w.H), 0.5f);
    spread(make_layer_stencil(p, n, -w.layer_half, w.W, w.H), 0.5f);
  } else {
    spread(make_stencil(w.pos[i], w.W, w.H), 1.0f);
  }
}

// ---------------------------------------------------------------------------
// a7 transposed, per cell.  Forward (shifted populations d = f - w, pulled):
//   drho = sum d, rho = 1 + drho, j = sum c d, u = (j + F/2)/rho,
//   pair (i, opp): cu = c.u, cF = c.F, uu = u.u, uF = u.F,
//     ep = w (drho + rho (4.5 cu^2 - 1.5 uu)), em = 3 w rho cu,
//     sp = w (9 cu cF - 3 uF), sm = 3 w cF, dp = (d_i + d_o)/2, dm = (d_i - d_o)/2,
//     even = -wp (dp - ep) + ap sp, odd = -wm (dm - em) + am sm,
//     out_i = d_i + even + odd, out_o = d_o + even - odd;
//   rest: e0 = w0 (drho - 1.5 rho uu), s0 = -3 w0 uF,
//     out_0 = d_0 - wp (d_0 - e0) + ap s0.
// Given out_bar (next step's population adjoint at this cell) and u_bar,
// returns d_bar and F_bar; d_bar_i is pushed to the cell the population was
// pulled from, so every adjoint population is written once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 adj_lbm_cell(const WorldDev& w, const AdjDev& a, int src_parity, int c);

__global__ void __launch_bounds__(256) k_adj_lbm(const WorldDev* __restrict__ wd, AdjDev a, int src_parity) {
  const WorldDev& w = *wd;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.0f;
  if (c < w.H * w.W) {
    const float2 fb = adj_lbm_cell(w, a, src_parity, c);
    m = fmaxf(fabsf(fb.x), fabsf(fb.y));
    // u_bar is read, and the previous reversed step's Q is dead: both start
    // the next reversed step at zero
    a.ubar[2 * c] = 0ull;
    a.ubar[2 * c + 1] = 0ull;
    a.Q[2 * c] = 0ull;
    a.Q[2 * c + 1] = 0ull;
  }
  warp_max_abs(&a.amax[2], m);   // the bound of the steric spread Q (k_adj_bead_a)
}

// One cell of k_adj_lbm: writes the population adjoints and F_bar, returns F_bar.
__device__ __forceinline__ float2 adj_lbm_cell(const WorldDev& w, const AdjDev& a, int src_parity, int c) {
  const int W = w.W, H = w.H, HW = H * W;
  const int y = c / W, x = c - y * W;
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
  const int r0 = y * W, rm = ym * W, rp = yp * W;
  // pull sources of populations 0..8 (same order as the forward kernel)
  const int src[9] = {c, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
  const float* g = w.g[src_parity];
  float d[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = g[i * HW + src[i]];
  const float2 F = w.F[c];
  const float drho = ((d[0] + (d[1] + d[3])) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
  const float rho = 1.0f + drho;
  const float jx = (d[1] - d[3]) + (d[5] - d[7]) + (d[8] - d[6]);
  const float jy = (d[2] - d[4]) + (d[5] - d[7]) + (d[6] - d[8]);
  const float inv = 1.0f / rho;
  const float ux = (jx + 0.5f * F.x) * inv, uy = (jy + 0.5f * F.y) * inv;
  const float uu = ux * ux + uy * uy, uF = ux * F.x + uy * F.y;
  const float wp = w.om_p, wm = w.om_m, ap = w.src_p, am = w.src_m;

  float ob[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) ob[i] = a.adjG_next[i * HW + c];
  const float uinv = pow2f(-ubar_exponent(w, a));
  const float2 ubx = make_float2(fx64_value(a.ubar[2 * c], uinv), fx64_value(a.ubar[2 * c + 1], uinv));
  float db[9];
  float drho_b = 0.0f, rho_b = 0.0f, uu_b = 0.0f, uF_b = 0.0f;
  float uxb = ubx.x, uyb = ubx.y, Fxb = 0.0f, Fyb = 0.0f;

  // rest population
  {
    constexpr float w0 = 4.0f / 9.0f;
    db[0] = (1.0f - wp) * ob[0];
    const float e0b = wp * ob[0], s0b = ap * ob[0];
    drho_b += w0 * e0b;
    rho_b += -1.5f * w0 * uu * e0b;
    uu_b += -1.5f * w0 * rho * e0b;
    uF_b += -3.0f * w0 * s0b;
  }
  // opposite pairs (i, o) with lattice velocity (cx, cy)
  constexpr int PI[4] = {1, 2, 5, 6}, PO[4] = {3, 4, 7, 8};
  constexpr float PX[4] = {1.0f, 0.0f, 1.0f, -1.0f}, PY[4] = {0.0f, 1.0f, 1.0f, 1.0f};
  constexpr float PW[4] = {1.0f / 9.0f, 1.0f / 9.0f, 1.0f / 36.0f, 1.0f / 36.0f};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = PI[k], o = PO[k];
    const float cxv = PX[k], cyv = PY[k], wi = PW[k];
    const float cu = cxv * ux + cyv * uy, cF = cxv * F.x + cyv * F.y;
    const float evb = ob[i] + ob[o];
    const float odb = ob[i] - ob[o];
    const float dpb = -wp * evb, epb = wp * evb, spb = ap * evb;
    const float dmb = -wm * odb, emb = wm * odb, smb = am * odb;
    db[i] = ob[i] + 0.5f * dpb + 0.5f * dmb;
    db[o] = ob[o] + 0.5f * dpb - 0.5f * dmb;
    // ep = wi (drho + rho (4.5 cu^2 - 1.5 uu))
    drho_b += wi * epb;
    rho_b += wi * (4.5f * cu * cu - 1.5f * uu) * epb;
    float cub = wi * rho * 9.0f * cu * epb;
    uu_b += -1.5f * wi * rho * epb;
    // em = 3 wi rho cu
    rho_b += 3.0f * wi * cu * emb;
    cub += 3.0f * wi * rho * emb;
    // sp = wi (9 cu cF - 3 uF), sm = 3 wi cF
    cub += 9.0f * wi * cF * spb;
    float cFb = 9.0f * wi * cu * spb + 3.0f * wi * smb;
    uF_b += -3.0f * wi * spb;
    uxb += cxv * cub;
    uyb += cyv * cub;
    Fxb += cxv * cFb;
    Fyb += cyv * cFb;
  }
  // uu = u.u, uF = u.F
  uxb += 2.0f * ux * uu_b + F.x * uF_b;
  uyb += 2.0f * uy * uu_b + F.y * uF_b;
  Fxb += ux * uF_b;
  Fyb += uy * uF_b;
  // u = (j + F/2) / rho
  const float jxb = uxb * inv, jyb = uyb * inv;
  Fxb += 0.5f * jxb;
  Fyb += 0.5f * jyb;
  rho_b += -(uxb * ux + uyb * uy) * inv;
  drho_b += rho_b;
  // drho = sum d, j = sum c d
  constexpr float CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float v = db[i] + drho_b + CX[i] * jxb + CY[i] * jyb;
    a.adjG_cur[i * HW + src[i]] = v;   // adjoint of the pulled post-collision value
  }
  a.Fbar[c] = make_float2(Fxb, Fyb);
  return make_float2(Fxb, Fyb);
}

// ---------------------------------------------------------------------------
// a8 and a6 gathers transposed, per bead:
//   Ftot_bar_i = sum_c w F_bar(c)
//   X_bar_i   += sum_c grad_X w [u(c).U_bar_i + F_bar(c).Ftot_i]
// then Q(c) += w(c - X_i) Ftot_bar_i for the steric chain, fixed point with
// the bound N max|F_bar| (|Ftot_bar_i| <= max|F_bar|: the weights sum to 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int q_exponent(const WorldDev& w, const AdjDev& a) {
  return fix_exponent64((float)w.N * __uint_as_float(a.amax[2]));
}

__global__ void __launch_bounds__(256) k_adj_bead_a(const WorldDev* __restrict__ wd, AdjDev a) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const float qscale = pow2f(q_exponent(w, a));
  const float4 p = w.pos[i];
  const Stencil s = make_stencil(p, w.W, w.H);
  const float2 xb = a.adjX[i];
  // direct forcing: the advance does not read u, and the steric spread
  // carries F_s alone (the MDF passes' own adjoints are k_adj_mdf.cu's)
  const bool df = w.ib == 1;
  const float Ubx = df ? 0.0f : w.dt * xb.x, Uby = df ? 0.0f : w.dt * xb.y;
  const float2 fe = df ? make_float2(0.0f, 0.0f) : w.fel[i], fs = w.fs[i];
  const float Ftx = fe.x + fs.x, Fty = fe.y + fs.y;
  // over the stencil st (weights scaled by h): the force's adjoint and the
  // position gradient of u.U_bar + F_bar.Ftot
  auto gather = [&](const Stencil& st, float h, float& ftbx, float& ftby, float& gx, float& gy) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = st.iy[b] + st.ix[c];
        const float2 u = w.u[k];
        const float2 fb = a.Fbar[k];
        const float wgt = st.wx[c] * st.wy[b] * h;
        ftbx = fmaf(wgt, fb.x, ftbx);
        ftby = fmaf(wgt, fb.y, ftby);
        const float q = (u.x * Ubx + u.y * Uby + fb.x * Ftx + fb.y * Fty) * h;
        gx = fmaf(st.dx[c] * st.wy[b], q, gx);
        gy = fmaf(st.wx[c] * st.dy[b], q, gy);
      }
  };
  float ftbx = 0.0f, ftby = 0.0f, gx = 0.0f, gy = 0.0f;
  if (w.layers == 2) {
    // both layer points take half of the force and half of the velocity;
    // X +- d n moves with X and (by +-d) with the normal
    const float2 n = a.nrm[i];
    float gpx = 0.0f, gpy = 0.0f, gmx = 0.0f, gmy = 0.0f;
    gather(make_layer_stencil(p, n, w.layer_half, w.W, w.H), 0.5f, ftbx, ftby, gpx, gpy);
    gather(make_layer_stencil(p, n, -w.layer_half, w.W, w.H), 0.5f, ftbx, ftby, gmx, gmy);
    gx = gpx + gmx;
    gy = gpy + gmy;
    a.nbar[i] = make_float2(w.layer_half * (gpx - gmx), w.layer_half * (gpy - gmy));
  } else {
    gather(s, 1.0f, ftbx, ftby, gx, gy);
  }
  a.adjX[i] = make_float2(xb.x + gx, xb.y + gy);
  a.fbt[i] = make_float2(ftbx, ftby);
  const float qx = ftbx * qscale, qy = ftby * qscale;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float wgt = s.wx[c] * s.wy[b];
      unsigned long long* q = &a.Q[2 * (s.iy[b] + s.ix[c])];
      atomicAdd(q, fx64(wgt * qx));
      atomicAdd(q + 1, fx64(wgt * qy));
    }
}

// ---------------------------------------------------------------------------
// a6 gradient transposed and a5 transposed, one 32 x 8 strip per block:
//   rho_bar_bar = -k_rep D^T Q with D the central difference,
//     (D^T v)(c) = (v_x(c - e_x) - v_x(c + e_x) + v_y(c - e_y) - v_y(c + e_y))/2,
//   then the periodic separable filter (symmetric), x pass then y pass.
// rho_bar_bar is formed on the strip plus R cells a side from Q staged with
// one more cell, the x pass on the strip's columns over those rows, the y
// pass on the strip; the sums run in the same order as cell-wise passes over
// the whole grid, so the result does not depend on the tiling.
// ---------------------------------------------------------------------------
constexpr int kBlurRows = 8;   // rows of a block's strip (32 columns): more, smaller blocks for small grids

__global__ void __launch_bounds__(256) k_adj_rho_blur(const WorldDev* __restrict__ wd, AdjDev a) {
  constexpr int kE = kTile + 2 * kMaxR;        // column capacity of the rho_bar_bar region
  constexpr int kER = kBlurRows + 2 * kMaxR;   // row capacity
  constexpr int kQ = kE + 2;                   // Q window capacity
  __shared__ float2 q[(kER + 2) * kQ];
  __shared__ float rb[kER * kE];
  __shared__ float tm[kER * kTile];
  const WorldDev& w = *wd;
  const int W = w.W, H = w.H, R = w.R;
  const int ntx = (W + kTile - 1) / kTile;
  const int x0 = (int)(blockIdx.x % ntx) * kTile, y0 = (int)(blockIdx.x / ntx) * kBlurRows;
  const int tw = min(kTile, W - x0), th = min(kBlurRows, H - y0);
  const int ew = tw + 2 * R, eh = th + 2 * R;   // region: rows y0 - R .., columns x0 - R ..
  const int qw = ew + 2, qh = eh + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float qinv = pow2f(-q_exponent(w, a));
  // rows by warp, columns by lane (no divisions); wrap by at most two periods
  for (int i = warp; i < qh; i += nw) {
    int gy = y0 - R - 1 + i;
    while (gy < 0) gy += H;
    while (gy >= H) gy -= H;
    const unsigned long long* __restrict__ row = a.Q + 2 * (size_t)gy * W;
    for (int j = lane; j < qw; j += 32) {
      int gx = x0 - R - 1 + j;
      while (gx < 0) gx += W;
      while (gx >= W) gx -= W;
      q[i * kQ + j] = make_float2(fx64_value(row[2 * gx], qinv), fx64_value(row[2 * gx + 1], qinv));
    }
  }
  __syncthreads();
  const float kq = -0.5f * w.k_rep;
  for (int i = warp; i < eh; i += nw) {
    for (int j = lane; j < ew; j += 32) {
      const float2* r = q + (i + 1) * kQ + j + 1;
      const float v = r[-1].x - r[1].x + r[-kQ].y - r[kQ].y;
      rb[i * kE + j] = kq * v;
    }
  }
  __syncthreads();
  for (int i = warp; i < eh; i += nw) {
    if (lane < tw) {
      const float* r = rb + i * kE + lane;
      float acc = 0.0f;
      for (int m = 0; m <= 2 * R; ++m) acc = fmaf(w.taps[m], r[m], acc);
      tm[i * kTile + lane] = acc;
    }
  }
  __syncthreads();
  for (int i = warp; i < th; i += nw) {
    if (lane < tw) {
      const float* r = tm + i * kTile + lane;
      float acc = 0.0f;
      for (int m = 0; m <= 2 * R; ++m) acc = fmaf(w.taps[m], r[m * kTile], acc);
      a.rsb[(size_t)(y0 + i) * W + x0 + lane] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// a4 and the a6 gather transposed, per bead:
//   X_bar_i += sum_c grad_X w [rho_s_bar(c) - k_rep grad rho_bar(c) . Ftot_bar_i]
// and the elastic-force adjoint d_bar_i = kappa/dt Ftot_bar_i for the PBD.
// ---------------------------------------------------------------------------
// Bead i: adds its a4 / a6-gradient terms to X_bar, returns Ftot_bar_i.
__device__ __forceinline__ float2 adj_bead_b_one(const WorldDev& w, const AdjDev& a, int i) {
  const int W = w.W, H = w.H;
  const float4 p = w.pos[i];
  const Stencil s = make_stencil(p, W, H);
  const float2 fb = a.fbt[i];
  float gx = 0.0f, gy = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int row = s.iy[b];
    const int rowm = wrap_once(cell_y(p) - 2 + b, H) * W, rowp = wrap_once(cell_y(p) + b, H) * W;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = s.ix[c];
      const int colm = wrap_once(cell_x(p) - 2 + c, W), colp = wrap_once(cell_x(p) + c, W);
      const float grx = 0.5f * (w.rho_b[row + colp] - w.rho_b[row + colm]);
      const float gry = 0.5f * (w.rho_b[rowp + col] - w.rho_b[rowm + col]);
      const float q = a.rsb[row + col] - w.k_rep * (grx * fb.x + gry * fb.y);
      gx = fmaf(s.dx[c] * s.wy[b], q, gx);
      gy = fmaf(s.wx[c] * s.dy[b], q, gy);
    }
  }
  const float2 xb = a.adjX[i];
  a.adjX[i] = make_float2(xb.x + gx, xb.y + gy);
  return fb;
}

// (as its own kernel for direct forcing, whose PBD reverse comes before the
// steric chain; the penalty step runs it inside k_adj_pbd)
__global__ void __launch_bounds__(256) k_adj_bead_b(const WorldDev* __restrict__ wd, AdjDev a) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const float2 fb = adj_bead_b_one(w, a, i);
  if (w.ib != 1) a.dbar[i] = make_float2(w.kappa_dt * fb.x, w.kappa_dt * fb.y);
}

// ---------------------------------------------------------------------------
// a3 + a1 transposed, one block of two warps per filament (each thread
// holds at most one edge of a filament of up to 64 beads per loop trip).  The forward Jacobi PBD is
// recomputed from (X^n, theta^n) keeping, per iteration, the frames before
// and after the bending pass and the corrections before the position pass;
// then the iterations are reversed:
//   position pass (per edge, x = v0 + d_{e+1} - d_e, l = |x|, sc = 1 - L/l):
//     D_e = hs [(1 - ksh) sc x + ksh (x - L d(theta))]
//     theta_e += ko (cos y - sin x) / L
//     d_i += D_i - D_{i-1}
//   bending pass: C_j = theta_{j+1} - theta_j - theta_rest_j,
//     theta_e += hb (C_e - C_{e-1})
// Inputs: d_bar (from F_el), theta_bar of theta^{n+1}.  Outputs: X_bar +=
// (through the edge vectors v0), theta_bar of theta^n, theta0_bar +=,
// L_rest_bar += (per edge), and (k_bend, k_stretch, k_shear)_bar += (float
// atomics, one per warp).
// ---------------------------------------------------------------------------
//
// Red-black passes (kRB, pbd_order 1) reverse colour by colour: the tape
// keeps, per pass, theta before the bending pass, after its even joints and
// after it, and the corrections d before the even and before the odd edges
// of the position pass; the reverse runs odd edges, even edges, odd joints,
// even joints, each colour's constraints independent of one another.
// ---------------------------------------------------------------------------
constexpr int kAdjPbdThreads = 64;  // threads per filament
constexpr int kAdjPbdPerBead = 12;   // floats of working arrays per bead slot
constexpr int kAdjTapePerPass = 4;   // Jacobi, per pass: theta before and after the bend pass, d (x, y)
constexpr int kAdjTapePerPassRB = 7; // red-black, per pass: theta x 3, d (x, y) before each edge colour

// The position correction of edge e (Eqs. 2-4) from the edge vector v0 plus
// corrections d, its frame angle th (turned in place): D into (Dx, Dy).
// (the forward kernel's arithmetic: the same fast forms)
__device__ __forceinline__ void adj_edge_forward(float vx, float vy, float L, float& th, float hs, float ksh,
                                                 float ko, float& Dx, float& Dy) {
  const float sc = fmaf(-L, rsqrtf(vx * vx + vy * vy), 1.0f);
  float sn, cs;
  __sincosf(fmaf(-6.28318548f, rintf(th * 0.159154943f), th), &sn, &cs);
  const float csx = sc * vx, csy = sc * vy;
  Dx = hs * (csx + ksh * (vx - L * cs - csx));
  Dy = hs * (csy + ksh * (vy - L * sn - csy));
  th += ko * (cs * vy - sn * vx) * __frcp_rn(L);
}

// The reverse of adj_edge_forward for edge vector (x, y), rest length L,
// forward angle tb, given D_bar and the angle's adjoint thb after it:
// returns the edge vector's adjoint and the angle's adjoint before it, and
// adds the parameter adjoints.
__device__ __forceinline__ void adj_edge_reverse(float x, float y, float L, float tb, float Dbx, float Dby,
                                                 float thb, float hs, float ksh, float ko, float orient,
                                                 float& xbx, float& xby, float& thb_new, float& hsb, float& kshb,
                                                 float& gL) {
  // (hardware reciprocal square root, reciprocal and reduced-angle
  // sine/cosine: the adjoint needs relative accuracy far below its 1e-3
  // budget, not the forward's bits)
  const float r = rsqrtf(x * x + y * y);   // 1 / |x|
  const float iL = __frcp_rn(L);
  const float sc = fmaf(-L, r, 1.0f);      // (|x| - L) / |x|
  float sn, cs;
  __sincosf(fmaf(-6.28318548f, rintf(tb * 0.159154943f), tb), &sn, &cs);
  // D = hs [(1 - ksh) sc x + ksh x - ksh L d]
  const float xd = x * Dbx + y * Dby;
  const float kq = hs * (1.0f - ksh) * (L * r * r * r) * xd;
  xbx = hs * ((1.0f - ksh) * sc + ksh) * Dbx + kq * x;
  xby = hs * ((1.0f - ksh) * sc + ksh) * Dby + kq * y;
  thb_new = thb + (-hs * ksh * L) * (-sn * Dbx + cs * Dby);
  // theta += ko (cs y - sn x) / L
  const float turn = (cs * y - sn * x) * iL;
  thb_new += thb * ko * (-sn * y - cs * x) * iL;
  xbx += thb * ko * (-sn) * iL;
  xby += thb * ko * cs * iL;
  // parameters: D = hs G, ko = orient hs ksh
  const float rx = x - L * cs - sc * x, ry = y - L * sn - sc * y;
  const float Gx = sc * x + ksh * rx, Gy = sc * y + ksh * ry;
  hsb += Gx * Dbx + Gy * Dby + thb * orient * ksh * turn;
  kshb += hs * (rx * Dbx + ry * Dby) + thb * orient * hs * turn;
  gL += hs * (-(1.0f - ksh) * xd * r - ksh * (cs * Dbx + sn * Dby)) - thb * ko * turn * iL;
}

template <bool kRB>
__global__ void __launch_bounds__(kAdjPbdThreads) k_adj_pbd(const WorldDev* __restrict__ wd, AdjDev a,
                                                            const int2* __restrict__ items, int n_items,
                                                            int maxB, int n_pbd) {
  constexpr int kTape = kRB ? kAdjTapePerPassRB : kAdjTapePerPass;
  extern __shared__ __align__(16) float smem[];
  const WorldDev& w = *wd;
  const int tid = threadIdx.x, lane = tid & 31;
  const int item = blockIdx.x;
  if (item >= n_items) return;   // block-uniform
  const int f = items[item].y;
  const int b0 = w.fil_off[f];
  const int B = w.fil_off[f + 1] - b0;
  const int nE = B - 1, nJ = B - 2;
  const int e0 = b0 - f, j0 = b0 - 2 * f;
  float* s = smem;
  float* vx = s;
  float* vy = s + maxB;
  float* th = s + 2 * maxB;
  float* Lr = s + 3 * maxB;
  float* thr = s + 4 * maxB;
  float* dx = s + 5 * maxB;     // corrections d (x); reused as d_bar later
  float* dy = s + 6 * maxB;
  float* Dx = s + 7 * maxB;     // per-edge D (x); reused for adjoint temporaries
  float* Dy = s + 8 * maxB;
  float* Cb = s + 9 * maxB;     // per-joint C / C_bar
  float* thrb = s + 10 * maxB;  // adjoint of theta_rest
  float* gLa = s + 11 * maxB;   // adjoint of L_rest, this step
  float* tape = s + 12 * maxB;  // per pass: theta before bend, theta after bend, d (x), d (y)
  const int W = w.W, H = w.H;
  const long long t = a.setup ? a.t_step : *w.t;
  const float4* __restrict__ P = a.xt ? a.xt : w.pos;   // the PBD's start: X~ with direct forcing
  for (int e = tid; e < nE; e += kAdjPbdThreads) {
    const float4 pa = P[b0 + e], pb = P[b0 + e + 1];
    int dcx = cell_x(pb) - cell_x(pa), dcy = cell_y(pb) - cell_y(pa);
    if (2 * dcx > W) dcx -= W; else if (2 * dcx < -W) dcx += W;
    if (2 * dcy > H) dcy -= H; else if (2 * dcy < -H) dcy += H;
    vx[e] = (float)dcx + (pb.x - pa.x);
    vy[e] = (float)dcy + (pb.y - pa.y);
    th[e] = a.theta_n[e0 + e];
    Lr[e] = rest_length(w, e0 + e, t);
    gLa[e] = 0.0f;
  }
  for (int j = tid; j < nJ; j += kAdjPbdThreads) {
    thr[j] = drive_angle(w.drive[j0 + j], t);
    thrb[j] = 0.0f;
  }
  for (int i = tid; i < B; i += kAdjPbdThreads) {
    dx[i] = 0.0f;
    dy[i] = 0.0f;
  }
  __syncthreads();
  const float hb = 0.5f * w.k_bend, hs = 0.5f * w.k_st, ksh = w.k_sh;
  const float orient = w.orient;
  const float ko = orient * hs * ksh;
  // ---- forward recompute with tape ----
  constexpr int T2 = 2 * kAdjPbdThreads;
  for (int it = 0; kRB && it < n_pbd; ++it) {
    float* tp = tape + it * kTape * maxB;
    for (int e = tid; e < nE; e += kAdjPbdThreads) tp[e] = th[e];
    __syncthreads();
    for (int c = 0; c < 2; ++c) {   // bending pass, even joints then odd ones
      for (int j = 2 * tid + c; j < nJ; j += T2) {
        const float Cj = th[j + 1] - th[j] - thr[j];
        th[j] += hb * Cj;
        th[j + 1] -= hb * Cj;
      }
      __syncthreads();
      for (int e = tid; e < nE; e += kAdjPbdThreads) tp[(c + 1) * maxB + e] = th[e];
      __syncthreads();
    }
    for (int c = 0; c < 2; ++c) {   // position pass, even edges then odd ones
      for (int i = tid; i < B; i += kAdjPbdThreads) {
        tp[(3 + 2 * c) * maxB + i] = dx[i];
        tp[(4 + 2 * c) * maxB + i] = dy[i];
      }
      __syncthreads();
      for (int e = 2 * tid + c; e < nE; e += T2) {
        float Dxe, Dye;
        adj_edge_forward(vx[e] + (dx[e + 1] - dx[e]), vy[e] + (dy[e + 1] - dy[e]), Lr[e], th[e], hs, ksh, ko,
                         Dxe, Dye);
        dx[e] += Dxe;
        dy[e] += Dye;
        dx[e + 1] -= Dxe;
        dy[e + 1] -= Dye;
      }
      __syncthreads();
    }
  }
  for (int it = 0; !kRB && it < n_pbd; ++it) {
    float* tp = tape + it * kTape * maxB;
    for (int e = tid; e < nE; e += kAdjPbdThreads) tp[e] = th[e];
    for (int j = tid; j < nJ; j += kAdjPbdThreads) Cb[j] = th[j + 1] - th[j] - thr[j];
    __syncthreads();
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      const float c1 = e < nJ ? Cb[e] : 0.0f, c0 = e > 0 ? Cb[e - 1] : 0.0f;
      th[e] += hb * (c1 - c0);
    }
    __syncthreads();
    for (int e = tid; e < nE; e += kAdjPbdThreads) tp[maxB + e] = th[e];
    for (int i = tid; i < B; i += kAdjPbdThreads) {
      tp[2 * maxB + i] = dx[i];
      tp[3 * maxB + i] = dy[i];
    }
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      float Dxe, Dye;
      adj_edge_forward(vx[e] + (dx[e + 1] - dx[e]), vy[e] + (dy[e + 1] - dy[e]), Lr[e], th[e], hs, ksh, ko, Dxe, Dye);
      Dx[e] = Dxe;
      Dy[e] = Dye;
    }
    __syncthreads();
    for (int i = tid; i < B; i += kAdjPbdThreads) {
      const float ax = i < nE ? Dx[i] : 0.0f, ay = i < nE ? Dy[i] : 0.0f;
      const float bx = i > 0 ? Dx[i - 1] : 0.0f, by = i > 0 ? Dy[i - 1] : 0.0f;
      dx[i] += ax - bx;
      dy[i] += ay - by;
    }
    __syncthreads();
  }
  // ---- reverse ----
  // adjoint state: d_bar in dx/dy, theta_bar in th, edge-vector adjoint
  // v0_bar after the tape; per-lane sums of the stiffness adjoints
  for (int i = tid; i < B; i += kAdjPbdThreads) {
    float2 db;
    if (a.xt) {   // direct forcing: d_bar from the bead velocities' adjoint
      db = a.dbar[b0 + i];
    } else {      // penalty: a4 and the a6 gradient of the bead first, d_bar = kappa/dt Ftot_bar
      const float2 fb = adj_bead_b_one(w, a, b0 + i);
      db = make_float2(w.kappa_dt * fb.x, w.kappa_dt * fb.y);
    }
    dx[i] = db.x;
    dy[i] = db.y;
  }
  for (int e = tid; e < nE; e += kAdjPbdThreads) th[e] = a.adjTh[e0 + e];
  float* v0bx = tape + n_pbd * kTape * maxB;
  float* v0by = v0bx + maxB;
  if (w.layers == 2) {
    // the two-layer normals n = (-t_y, t_x), t = s/|s|, s = out + in (the
    // unit vectors of the bead's edges at X^n; a folded chain takes out, or
    // in at the last bead): per bead the adjoints of its out and in unit
    // vectors (Dx: out, Dy: in, as 2 floats each in Dx/Dy pairs of slots)
    for (int i = tid; i < B; i += kAdjPbdThreads) {
      const float2 nb = a.nbar[b0 + i];
      const float tbx = nb.y, tby = -nb.x;
      const bool ho = i < nE, hi = i > 0;
      float ox = 0.0f, oy = 0.0f, ix = 0.0f, iy = 0.0f;
      if (ho) {
        const float r = rsqrtf(vx[i] * vx[i] + vy[i] * vy[i]);
        ox = vx[i] * r;
        oy = vy[i] * r;
      }
      if (hi) {
        const float r = rsqrtf(vx[i - 1] * vx[i - 1] + vy[i - 1] * vy[i - 1]);
        ix = vx[i - 1] * r;
        iy = vy[i - 1] * r;
      }
      const float sx = ox + ix, sy = oy + iy;
      const float ns = sqrtf(sx * sx + sy * sy);
      float obx = 0.0f, oby = 0.0f, ibx = 0.0f, iby = 0.0f;
      if (ns >= 1e-3f) {
        const float tx = sx / ns, ty = sy / ns;
        const float dot = tbx * tx + tby * ty;
        const float sbx = (tbx - dot * tx) / ns, sby = (tby - dot * ty) / ns;
        if (ho) { obx = sbx; oby = sby; }
        if (hi) { ibx = sbx; iby = sby; }
      } else if (ho) {
        obx = tbx;
        oby = tby;
      } else {
        ibx = tbx;
        iby = tby;
      }
      Dx[i] = obx;   // adjoint of the unit vector of edge i (as the bead's out)
      Dy[i] = oby;
      Cb[i] = ibx;   // adjoint of the unit vector of edge i - 1 (as the bead's in)
      thrb[i] = iby;
    }
    __syncthreads();
    // edge e: unit vector u = v/|v| with adjoint ub from bead e (out) and
    // bead e + 1 (in): v_bar = (ub - (ub.u) u)/|v|
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      const float r = rsqrtf(vx[e] * vx[e] + vy[e] * vy[e]);
      const float ux = vx[e] * r, uy = vy[e] * r;
      const float ubx = Dx[e] + Cb[e + 1], uby = Dy[e] + thrb[e + 1];
      const float dot = ubx * ux + uby * uy;
      v0bx[e] = (ubx - dot * ux) * r;
      v0by[e] = (uby - dot * uy) * r;
    }
    __syncthreads();
    for (int j = tid; j < B; j += kAdjPbdThreads) thrb[j] = 0.0f;   // back to the rest-angle adjoint
    __syncthreads();
  } else {
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      v0bx[e] = 0.0f;
      v0by[e] = 0.0f;
    }
  }
  float hbb = 0.0f, hsb = 0.0f, kshb = 0.0f;
  __syncthreads();
  for (int it = n_pbd - 1; kRB && it >= 0; --it) {
    const float* tp = tape + it * kTape * maxB;
    for (int c = 1; c >= 0; --c) {   // position pass: odd edges, then even ones
      const float* dX = tp + (3 + 2 * c) * maxB;
      const float* dY = tp + (4 + 2 * c) * maxB;
      for (int e = tid; e < nE; e += kAdjPbdThreads) {
        if ((e & 1) != c) {   // the other colour's edges add nothing in this phase
          Dx[e] = 0.0f;
          Dy[e] = 0.0f;
          continue;
        }
        float xbx, xby, thb_new;
        adj_edge_reverse(vx[e] + (dX[e + 1] - dX[e]), vy[e] + (dY[e + 1] - dY[e]), Lr[e], tp[2 * maxB + e],
                         dx[e] - dx[e + 1], dy[e] - dy[e + 1], th[e], hs, ksh, ko, orient, xbx, xby, thb_new, hsb,
                         kshb, gLa[e]);
        Dx[e] = xbx;
        Dy[e] = xby;
        th[e] = thb_new;
        v0bx[e] += xbx;
        v0by[e] += xby;
      }
      __syncthreads();
      for (int i = tid; i < B; i += kAdjPbdThreads) {
        const float ax = i < nE ? Dx[i] : 0.0f, ay = i < nE ? Dy[i] : 0.0f;
        const float bx = i > 0 ? Dx[i - 1] : 0.0f, by = i > 0 ? Dy[i - 1] : 0.0f;
        dx[i] += bx - ax;
        dy[i] += by - ay;
      }
      __syncthreads();
    }
    for (int c = 1; c >= 0; --c) {   // bending pass: odd joints, then even ones
      const float* tb = tp + c * maxB;   // angles before this colour
      for (int j = 2 * tid + c; j < nJ; j += T2) {
        const float dth = th[j] - th[j + 1];
        hbb += (tb[j + 1] - tb[j] - thr[j]) * dth;
        const float Cbj = hb * dth;
        th[j] -= Cbj;
        th[j + 1] += Cbj;
        thrb[j] -= Cbj;
      }
      __syncthreads();
    }
  }
  for (int it = n_pbd - 1; !kRB && it >= 0; --it) {
    const float* tp = tape + it * kTape * maxB;
    // position pass reverse: D_bar_e = d_bar_e - d_bar_{e+1}, from theta
    // after the bend pass and the corrections before this pass
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      float xbx, xby, thb_new;
      adj_edge_reverse(vx[e] + (tp[2 * maxB + e + 1] - tp[2 * maxB + e]),
                       vy[e] + (tp[3 * maxB + e + 1] - tp[3 * maxB + e]), Lr[e], tp[maxB + e], dx[e] - dx[e + 1],
                       dy[e] - dy[e + 1], th[e], hs, ksh, ko, orient, xbx, xby, thb_new, hsb, kshb, gLa[e]);
      Dx[e] = xbx;
      Dy[e] = xby;
      th[e] = thb_new;
      v0bx[e] += xbx;
      v0by[e] += xby;
    }
    __syncthreads();
    // x = v0 + d_{e+1} - d_e: d_bar_i += x_bar_{i-1} - x_bar_i
    for (int i = tid; i < B; i += kAdjPbdThreads) {
      const float ax = i < nE ? Dx[i] : 0.0f, ay = i < nE ? Dy[i] : 0.0f;
      const float bx = i > 0 ? Dx[i - 1] : 0.0f, by = i > 0 ? Dy[i - 1] : 0.0f;
      dx[i] += bx - ax;
      dy[i] += by - ay;
    }
    __syncthreads();
    // bending pass reverse: C_bar_j = hb (theta_bar_j - theta_bar_{j+1});
    // d theta_e / d hb = C_e - C_{e-1} with C from the angles before the pass
    for (int j = tid; j < nJ; j += kAdjPbdThreads) {
      const float dth = th[j] - th[j + 1];
      hbb += (tp[j + 1] - tp[j] - thr[j]) * dth;
      Cb[j] = hb * dth;
    }
    __syncthreads();
    for (int e = tid; e < nE; e += kAdjPbdThreads) {
      const float in = e > 0 ? Cb[e - 1] : 0.0f;     // theta_e is theta_{j+1} of joint e-1
      const float out = e < nJ ? Cb[e] : 0.0f;       // ... and theta_j of joint e
      th[e] += in - out;
    }
    for (int j = tid; j < nJ; j += kAdjPbdThreads) thrb[j] -= Cb[j];
    __syncthreads();
  }
  // outputs
  for (int e = tid; e < nE; e += kAdjPbdThreads) {
    a.adjTh[e0 + e] = th[e];
    // with a rest-length drive L(t) = L0 (1 + A s(t)): dL(t)/dL0 = L(t)/L0
    const float dLdL0 = w.ldrive ? 1.0f + w.ldrive[e0 + e].y * drive_sin(w.ldrive[e0 + e].z, w.ldrive[e0 + e].w, t)
                                 : 1.0f;
    a.gL[e0 + e] += gLa[e] * dLdL0;
  }
  for (int j = tid; j < nJ; j += kAdjPbdThreads) a.gth0[j0 + j] += thrb[j];
  // X_bar is final for this step: its largest |dt X_bar| bounds the next
  // reversed step's u_bar (slot par ^ 1; every lane takes part)
  float xm = 0.0f;
  for (int i0 = 0; i0 < B; i0 += kAdjPbdThreads) {
    const int i = i0 + tid;
    if (i < B) {
      const float ax = i < nE ? v0bx[i] : 0.0f, ay = i < nE ? v0by[i] : 0.0f;        // X_i is x_1 of edge i
      const float bx = i > 0 ? v0bx[i - 1] : 0.0f, by = i > 0 ? v0by[i - 1] : 0.0f;  // ... x_2 of edge i-1
      float2 xb = a.adjX[b0 + i];
      xb.x += bx - ax;
      xb.y += by - ay;
      a.adjX[b0 + i] = xb;
      if (a.xtb) a.xtb[b0 + i] = make_float2(bx - ax, by - ay);
      xm = fmaxf(xm, w.dt * fmaxf(fabsf(xb.x), fabsf(xb.y)));
    }
  }
  warp_max_abs(&a.amax[a.par ^ 1], xm);
  // k_bend = 2 hb, k_stretch = 2 hs, k_shear = ksh: the filament's sums
  // (warps reduced in a fixed order) added to its own accumulator
  for (int o = 16; o > 0; o >>= 1) {
    hbb += __shfl_xor_sync(0xffffffffu, hbb, o);
    hsb += __shfl_xor_sync(0xffffffffu, hsb, o);
    kshb += __shfl_xor_sync(0xffffffffu, kshb, o);
  }
  __shared__ float part[3 * (kAdjPbdThreads / 32)];
  if (lane == 0) {
    part[3 * (tid >> 5)] = hbb;
    part[3 * (tid >> 5) + 1] = hsb;
    part[3 * (tid >> 5) + 2] = kshb;
  }
  __syncthreads();
  if (tid == 0) {
    float sb = 0.0f, ss = 0.0f, sk = 0.0f;
    for (int k = 0; k < kAdjPbdThreads / 32; ++k) {
      sb += part[3 * k];
      ss += part[3 * k + 1];
      sk += part[3 * k + 2];
    }
    a.gkf[3 * f] += 0.5f * sb;
    a.gkf[3 * f + 1] += 0.5f * ss;
    a.gkf[3 * f + 2] += sk;
  }
}

// The stiffness gradients: the per-filament sums added over filaments in
// index order (one block).
__global__ void __launch_bounds__(256) k_adj_gk_reduce(const float* __restrict__ gkf, int n_fil, float* gk) {
  __shared__ float red[3][256];
  float s[3] = {0.0f, 0.0f, 0.0f};
  for (int f = threadIdx.x; f < n_fil; f += blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += gkf[3 * f + c];
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) gk[threadIdx.x] = red[threadIdx.x][0];
}

size_t adj_pbd_smem_per_filament(int maxB, int n_pbd, int order) {
  const int per = order == 1 ? kAdjTapePerPassRB : kAdjTapePerPass;
  return (size_t)maxB * (kAdjPbdPerBead + per * n_pbd + 2) * sizeof(float);
}

// ---------------------------------------------------------------------------
// Folding loss (Filament Folding experiment, with a polyline target): mean
// over beads of the squared distance from the unwrapped position
// P_i = X0_i + D_i to the nearest segment of the polyline, and dL/dP_i.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_loss_polyline(const WorldDev* __restrict__ wd, const float2* __restrict__ pos0,
                                                        const float2* __restrict__ poly, int nv, float* loss,
                                                        float* gx, float* gy) {
  // one block: each thread sums its beads in index order, then a fixed tree
  // (the loss is bitwise repeatable)
  const WorldDev& w = *wd;
  __shared__ float red[1024];
  const float invN = 1.0f / (float)max(w.N, 1);
  float l = 0.0f;
  for (int i = threadIdx.x; i < w.N; i += blockDim.x) {
    const float2 d = w.disp[i];
    const float px = pos0[i].x + d.x, py = pos0[i].y + d.y;
    float best = 3.0e38f, qx = px, qy = py;
    for (int k = 0; k + 1 < nv; ++k) {
      const float2 A = poly[k], B = poly[k + 1];
      const float abx = B.x - A.x, aby = B.y - A.y;
      float tt = ((px - A.x) * abx + (py - A.y) * aby) / (abx * abx + aby * aby);
      tt = fminf(fmaxf(tt, 0.0f), 1.0f);
      const float cx = A.x + tt * abx, cy = A.y + tt * aby;
      const float d2 = (px - cx) * (px - cx) + (py - cy) * (py - cy);
      if (d2 < best) {
        best = d2;
        qx = cx;
        qy = cy;
      }
    }
    l += best * invN;
    gx[i] = 2.0f * (px - qx) * invN;
    gy[i] = 2.0f * (py - qy) * invN;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0];
}

__global__ void k_set_counter(long long* t, long long v, unsigned* fel_max) {
  *t = v;
  fel_max[0] = 0u;
  fel_max[1] = 0u;
}

// ---------------------------------------------------------------------------
// Launchers (one world).
// ---------------------------------------------------------------------------
static int blocks(int n) { return (n + 255) / 256; }
// the per-bead adjoint kernels run 64-thread blocks: a few thousand beads
// then spread over several times more SMs
constexpr int kAdjBeadThreads = 64;
static int bead_blocks(int n) { return (n + kAdjBeadThreads - 1) / kAdjBeadThreads; }
static int blur_blocks(const WorldDev& h) { return h.ntx * ((h.H + kBlurRows - 1) / kBlurRows); }

// One reversed step.  Penalty coupling: a8, a7, a6/a4 gathers, a5, a6
// gradient/a4, then a3/a1.  Direct forcing (m != NULL): a7, the MDF passes
// and the drag (k_adj_mdf.cu) around a3/a1, then the steric chain.
void launch_adj_step(const Plan& p, const WorldDev& h, AdjDev a, const AdjMdf* m, int src_parity, cudaStream_t s) {
  const WorldDev* wd = p.d_worlds;
  const int HW = h.H * h.W;
  auto pbd = [&](const AdjDev& ap) {
    if (!p.n_fil_items) return;
    const int mb = (p.max_B + 3) & ~3;
    const size_t smem = adj_pbd_smem_per_filament(mb, h.n_pbd, h.pbd_order);
    if (h.pbd_order == 1)
      k_adj_pbd<true><<<p.n_fil_items, kAdjPbdThreads, smem, s>>>(wd, ap, p.d_fil_items, p.n_fil_items, mb, h.n_pbd);
    else
      k_adj_pbd<false><<<p.n_fil_items, kAdjPbdThreads, smem, s>>>(wd, ap, p.d_fil_items, p.n_fil_items, mb, h.n_pbd);
  };
  // (u_bar and Q are cleared by the caller before each step)
  if (m) {
    k_adj_lbm<<<blocks(HW), 256, 0, s>>>(wd, a, src_parity);
    launch_adj_mdf_passes(h, wd, a, *m, s);
    AdjDev ap = a;
    ap.xt = m->xt;
    ap.xtb = m->xtb;
    pbd(ap);
    launch_adj_mdf_moments(h, wd, a, *m, s);
    if (h.N) k_adj_bead_a<<<bead_blocks(h.N), kAdjBeadThreads, 0, s>>>(wd, a);
    k_adj_rho_blur<<<blur_blocks(h), 256, 0, s>>>(wd, a);
    if (h.N) k_adj_bead_b<<<bead_blocks(h.N), kAdjBeadThreads, 0, s>>>(wd, a);
    return;
  }
  if (h.N || a.setup) k_adj_spread_u<<<std::max(bead_blocks(h.N), 1), kAdjBeadThreads, 0, s>>>(wd, a);
  k_adj_lbm<<<blocks(HW), 256, 0, s>>>(wd, a, src_parity);
  if (h.N) k_adj_bead_a<<<bead_blocks(h.N), kAdjBeadThreads, 0, s>>>(wd, a);
  k_adj_rho_blur<<<blur_blocks(h), 256, 0, s>>>(wd, a);
  pbd(a);   // with a4 and the a6 gradient per bead (k_adj_bead_b's work) first
}

void launch_adj_gk_reduce(const AdjDev& a, int n_fil, cudaStream_t s) {
  k_adj_gk_reduce<<<1, 256, 0, s>>>(a.gkf, n_fil, a.gk);
}

void adj_setup(const Plan& p, const WorldDev& h) {
  const int mb = (p.max_B + 3) & ~3;
  const size_t per = adj_pbd_smem_per_filament(mb, h.n_pbd, h.pbd_order);
  if (per > 48 * 1024) {
    cudaFuncSetAttribute(k_adj_pbd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)per);
    cudaFuncSetAttribute(k_adj_pbd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)per);
  }
}

// theta0 [J] into the drive records' first component, L_rest [E] into the
// rest lengths (and the rest-length drive's L0); either may be NULL.
__global__ void k_set_rest(float4* drive, int J, const float* theta0, float* L_rest, float4* ldrive, int E,
                           const float* L_new) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (theta0 && i < J) drive[i].x = theta0[i];
  if (L_new && i < E) {
    L_rest[i] = L_new[i];
    if (ldrive) ldrive[i].x = L_new[i];
  }
}

void launch_set_rest(const WorldDev& h, const float* theta0, const float* L_rest, cudaStream_t s) {
  const int n = h.J > h.E ? h.J : h.E;
  if (n > 0 && (theta0 || L_rest))
    k_set_rest<<<(n + 255) / 256, 256, 0, s>>>(const_cast<float4*>(h.drive), h.J, theta0,
                                               const_cast<float*>(h.L_rest), const_cast<float4*>(h.ldrive), h.E,
                                               L_rest);
}

// ---------------------------------------------------------------------------
// Folding loss with an image target (Filament Folding experiment): mean
// squared error between the Gaussian-splatted bead density at the final step
// and a target image of R x R pixels covering the periodic domain.  Pixel
// (px, py) has its centre at ((px + 1/2) W/R, (py + 1/2) H/R); a bead at
// image coordinates u = (X R/W, Y R/H) adds exp(-|c - u|^2 / (2 s^2)) to the
// pixels with px in floor(u_x) - K .. floor(u_x) + K (same in y, periodic),
// K = ceil(4 s).  The image accumulates in 64-bit fixed point (2^-32 units),
// so it does not depend on the order of the beads.
// ---------------------------------------------------------------------------
constexpr double kSplatScale = 4294967296.0;   // 2^32

__device__ __forceinline__ float2 image_coords(const float4 p, float sx, float sy) {
  return make_float2(((float)cell_x(p) + p.x) * sx, ((float)cell_y(p) + p.y) * sy);
}

__global__ void __launch_bounds__(256) k_splat_accum(const WorldDev* __restrict__ wd, int R, float sx, float sy,
                                                     float inv2s2, int K, unsigned long long* __restrict__ acc) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const float2 u = image_coords(w.pos[i], sx, sy);
  const int bx = (int)floorf(u.x), by = (int)floorf(u.y);
  for (int b = -K; b <= K; ++b) {
    const float dy = (float)(by + b) + 0.5f - u.y;
    const float gy = expf(-dy * dy * inv2s2);
    const int row = ((by + b) % R + R) % R;
    for (int a = -K; a <= K; ++a) {
      const float dx = (float)(bx + a) + 0.5f - u.x;
      const float g = gy * expf(-dx * dx * inv2s2);
      const int col = ((bx + a) % R + R) % R;
      atomicAdd(&acc[row * R + col], (unsigned long long)__double2ull_rn((double)g * kSplatScale));
    }
  }
}

// One block: diff = I - T per pixel and loss = mean(diff^2), summed in a fixed order.
__global__ void __launch_bounds__(256) k_splat_loss(const unsigned long long* __restrict__ acc,
                                                    const float* __restrict__ target, int RR, float* __restrict__ diff,
                                                    float* loss) {
  __shared__ float red[256];
  float sum = 0.0f;
  for (int q = threadIdx.x; q < RR; q += blockDim.x) {
    const float d = (float)((double)acc[q] / kSplatScale) - target[q];
    diff[q] = d;
    sum = fmaf(d, d, sum);
  }
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = red[0] / (float)RR;
}

// dL/dX_i = (2 / R^2) sum_c diff(c) dG(c - u_i)/du * du/dX, dG/du = G (c - u) / s^2.
__global__ void __launch_bounds__(256) k_splat_grad(const WorldDev* __restrict__ wd, int R, float sx, float sy,
                                                    float inv2s2, int K, const float* __restrict__ diff,
                                                    float* __restrict__ gx, float* __restrict__ gy) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const float2 u = image_coords(w.pos[i], sx, sy);
  const int bx = (int)floorf(u.x), by = (int)floorf(u.y);
  float ax = 0.0f, ay = 0.0f;
  for (int b = -K; b <= K; ++b) {
    const float dy = (float)(by + b) + 0.5f - u.y;
    const float wy = expf(-dy * dy * inv2s2);
    const int row = ((by + b) % R + R) % R;
    for (int a = -K; a <= K; ++a) {
      const float dx = (float)(bx + a) + 0.5f - u.x;
      const float g = wy * expf(-dx * dx * inv2s2) * diff[row * R + ((bx + a) % R + R) % R];
      ax = fmaf(g, dx, ax);
      ay = fmaf(g, dy, ay);
    }
  }
  // dG/du = G (c - u) / s^2 = 2 G (c - u) inv2s2
  const float c = 2.0f / (float)(R * R) * 2.0f * inv2s2;
  gx[i] = c * ax * sx;
  gy[i] = c * ay * sy;
}

void launch_loss_splat(const Plan& p, const WorldDev& h, const float* target, int R, float sigma,
                       unsigned long long* acc, float* diff, float* loss, float* gx, float* gy, cudaStream_t s) {
  const int K = (int)ceilf(4.0f * sigma);
  const float sx = (float)R / (float)h.W, sy = (float)R / (float)h.H;
  const float inv2s2 = 1.0f / (2.0f * sigma * sigma);
  cudaMemsetAsync(acc, 0, (size_t)R * R * sizeof(unsigned long long), s);
  if (h.N) k_splat_accum<<<blocks(h.N), 256, 0, s>>>(p.d_worlds, R, sx, sy, inv2s2, K, acc);
  k_splat_loss<<<1, 256, 0, s>>>(acc, target, R * R, diff, loss);
  if (h.N) k_splat_grad<<<blocks(h.N), 256, 0, s>>>(p.d_worlds, R, sx, sy, inv2s2, K, diff, gx, gy);
}

void launch_loss_polyline(const Plan& p, const WorldDev& h, const float2* pos0, const float2* poly, int nv,
                          float* loss, float* gx, float* gy, cudaStream_t s) {
  if (h.N) k_loss_polyline<<<1, 1024, 0, s>>>(p.d_worlds, pos0, poly, nv, loss, gx, gy);
  else cudaMemsetAsync(loss, 0, sizeof(float), s);
}

void launch_set_counter(const WorldDev& h, long long t, cudaStream_t s) {
  k_set_counter<<<1, 1, 0, s>>>(h.t, t, h.fel_max);
}

}  // namespace mc
