// Reverse mode of a direct-forcing step (ib == 1; Fluid-filament
// Interaction: the nodes move with the fluid, the filament's velocity is
// imposed back on the fluid by multi-direct-forcing passes).  The forward
// step, with stencil weights w(c - X_i) at X = X^n:
//   F0 = S[F_s]                                   the steric force on the fluid
//   rho = sum f, u_0 = (sum c f + F0/2) / rho      the fluid before the filament's forcing
//   U* = I[u_0](X), X~ = X + dt U*                 the fluid carries the beads
//   (x_hat, theta^{n+1}) = PBD(X~, theta^n),  U_s = U* + (x_hat - X~)/dt
//   pass k = 0 .. m-1:  dF_k = 2 I[rho] (U_s - I[u_k]),  G_k = S[dF_k],
//                       F <- F + G_k,  u_{k+1} = u_k + G_k / (2 rho)
//   f' = LBM(f, F_m),  X^{n+1} = X + dt U_s
// Its reverse, from the adjoints of X^{n+1}, theta^{n+1} and f':
//   U_s_bar = dt X_bar;  (f_bar, F_bar) = LBM^T (the LBM's velocity is not
//   read by the beads, so u_bar(m) = 0);  passes k = m-1 .. 0, F_bar the
//   same in every pass:
//     G_bar = F_bar + u_bar_{k+1} / (2 rho),  rho_bar -= u_bar_{k+1} . (u_{k+1} - u_k) / rho,
//     dF_bar = I[G_bar],  r_bar = 2 (U_s - I[u_k]) . dF_bar,  U_s_bar += 2 I[rho] dF_bar,
//     u_bar_k = u_bar_{k+1} + S[-2 I[rho] dF_bar],  rho_bar += S[r_bar],
//     X_bar += sum_c grad w [G_bar . dF + u_k . (-2 I[rho] dF_bar) + rho r_bar];
//   d_bar = U_s_bar / dt for the PBD's reverse from X~, whose edge-vector
//   adjoint x~_bar goes to X_bar (X~ = X + dt U*) and to
//   U*_bar = U_s_bar + dt x~_bar;  X_bar += sum_c grad w u_0 . U*_bar,
//   u_bar_0 += S[U*_bar];  the moments: F0_bar = F_bar + u_bar_0 / (2 rho),
//   rho_bar -= u_bar_0 . u_0 / rho, and each population's adjoint gains
//   rho_bar + c_i . u_bar_0 / rho (at the cell it was pulled from); the
//   steric chain then runs from F0_bar as in the penalty step, with F_s the
//   bead force.
// The transposed interpolations (S of per-bead values) accumulate in 64-bit
// fixed point with grid-wide bounds, so the gradients are bitwise
// repeatable.
#include "adj_dev.cuh"
#include "bead_dev.cuh"

namespace mc {

namespace {

constexpr int kMdfBeadThreads = 64;

__device__ __forceinline__ int scatter_exponent(const WorldDev& w, const unsigned* slot) {
  return fix_exponent64((float)w.N * __uint_as_float(*slot));
}

// S[v] of NC per-bead components into 64-bit fixed-point accumulators
// (interleaved), at the scale of the bound in *slot.
template <int NC>
__device__ __forceinline__ void scatter_fixed(const WorldDev& w, const Stencil& s, const float* v, const unsigned* slot,
                                              unsigned long long* acc) {
  const float scale = pow2f(scatter_exponent(w, slot));
  float sv[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) sv[k] = v[k] * scale;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float g = s.wx[c] * s.wy[b];
      unsigned long long* q = acc + NC * (size_t)(s.iy[b] + s.ix[c]);
#pragma unroll
      for (int k = 0; k < NC; ++k) atomicAdd(q + k, fx64(g * sv[k]));
    }
}

}  // namespace

// Pass k, per cell: u_bar_{k+1} (the previous reversed pass's scatters
// folded in), G_bar, and the density term of the velocity update.
__global__ void __launch_bounds__(256) k_adj_mdf_cell(const WorldDev* __restrict__ wd, AdjMdf m, const float2* Fbar,
                                                      int k) {
  const WorldDev& w = *wd;
  const int HW = w.H * w.W;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) {   // this pass's bounds, which its bead kernel fills next
    m.bnd[k & 1] = 0u;
    m.bnd[2 + (k & 1)] = 0u;
  }
  if (c >= HW) return;
  float2 ub = m.ubf[c];
  float rb = m.rhob[c];
  const float rho = m.rho[c];
  if (k + 1 < m.m) {
    const int q = (k + 1) & 1;
    const float iu = pow2f(-scatter_exponent(w, &m.bnd[q])), ir = pow2f(-scatter_exponent(w, &m.bnd[2 + q]));
    ub.x += fx64_value(m.su[2 * c], iu);
    ub.y += fx64_value(m.su[2 * c + 1], iu);
    rb += fx64_value(m.sr[c], ir);
    m.su[2 * c] = 0ull;
    m.su[2 * c + 1] = 0ull;
    m.sr[c] = 0ull;
    m.ubf[c] = ub;
    const float2 u0 = m.mu[(size_t)k * HW + c], u1 = m.mu[(size_t)(k + 1) * HW + c];
    rb -= (ub.x * (u1.x - u0.x) + ub.y * (u1.y - u0.y)) / rho;
    m.rhob[c] = rb;
  }
  const float2 Fb = Fbar[c];
  const float h = 0.5f / rho;
  m.Gbar[c] = make_float2(fmaf(ub.x, h, Fb.x), fmaf(ub.y, h, Fb.y));
}

// Pass k, per bead: dF_bar = I[G_bar], r_bar, the U_s adjoint, the position
// adjoint of the pass's three interpolations/spreads, and the values the
// scatter kernel spreads (with their grid-wide bounds).
__global__ void __launch_bounds__(kMdfBeadThreads) k_adj_mdf_bead(const WorldDev* __restrict__ wd, AdjDev a,
                                                                  AdjMdf m, int k) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float mu = 0.0f, mr = 0.0f;
  if (i < w.N) {
    const Stencil s = make_stencil(w.pos[i], w.W, w.H);
    const float2* __restrict__ uk = m.mu + (size_t)k * w.H * w.W;
    float gbx = 0.0f, gby = 0.0f, r = 0.0f, Iux = 0.0f, Iuy = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cc = s.iy[b] + s.ix[c];
        const float g = s.wx[c] * s.wy[b];
        const float2 G = m.Gbar[cc], u = uk[cc];
        gbx = fmaf(g, G.x, gbx);
        gby = fmaf(g, G.y, gby);
        r = fmaf(g, m.rho[cc], r);
        Iux = fmaf(g, u.x, Iux);
        Iuy = fmaf(g, u.y, Iuy);
      }
    const float2 Us = m.Us[i];
    const float ex = Us.x - Iux, ey = Us.y - Iuy;
    const float dFx = 2.0f * r * ex, dFy = 2.0f * r * ey;
    const float rbar = 2.0f * (ex * gbx + ey * gby);
    const float ibx = -2.0f * r * gbx, iby = -2.0f * r * gby;
    const float2 xb = a.adjX[i];
    float2 usb = k == m.m - 1 ? make_float2(w.dt * xb.x, w.dt * xb.y) : m.usb[i];
    usb.x -= ibx;
    usb.y -= iby;
    m.usb[i] = usb;
    m.iub[i] = make_float2(ibx, iby);
    m.rbb[i] = rbar;
    float gx = 0.0f, gy = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cc = s.iy[b] + s.ix[c];
        const float2 G = m.Gbar[cc], u = uk[cc];
        const float q = G.x * dFx + G.y * dFy + u.x * ibx + u.y * iby + m.rho[cc] * rbar;
        gx = fmaf(s.dx[c] * s.wy[b], q, gx);
        gy = fmaf(s.wx[c] * s.dy[b], q, gy);
      }
    a.adjX[i] = make_float2(xb.x + gx, xb.y + gy);
    mu = fmaxf(fabsf(ibx), fabsf(iby));
    mr = rbar;
  }
  warp_max_abs(&m.bnd[k & 1], mu);
  warp_max_abs(&m.bnd[2 + (k & 1)], mr);
}

// Pass k: u_bar += S[-2 I[rho] dF_bar], rho_bar += S[r_bar].
__global__ void __launch_bounds__(kMdfBeadThreads) k_adj_mdf_scatter(const WorldDev* __restrict__ wd, AdjMdf m,
                                                                     int k) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const Stencil s = make_stencil(w.pos[i], w.W, w.H);
  const float2 ib = m.iub[i];
  const float vu[2] = {ib.x, ib.y};
  scatter_fixed<2>(w, s, vu, &m.bnd[k & 1], m.su);
  const float vr[1] = {m.rbb[i]};
  scatter_fixed<1>(w, s, vr, &m.bnd[2 + (k & 1)], m.sr);
}

// After the passes, per bead: X~ = X + dt I[u_0](X) as the forward computed
// it (the PBD's start), and the PBD's correction adjoint d_bar = U_s_bar / dt.
__global__ void __launch_bounds__(kMdfBeadThreads) k_adj_mdf_xt(const WorldDev* __restrict__ wd, AdjDev a, AdjMdf m) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) m.bnd[4] = 0u;   // the drag's scatter bound (k_adj_mdf_ustar)
  if (i >= w.N) return;
  const float4 p = w.pos[i];
  const float2 U = interp_field(m.mu, w.W, w.H, p);
  m.xt[i] = advance_pos(w, p, U.x, U.y);
  float2 usb;
  if (m.m > 0) {
    usb = m.usb[i];
  } else {
    const float2 xb = a.adjX[i];
    usb = make_float2(w.dt * xb.x, w.dt * xb.y);
    m.usb[i] = usb;
  }
  a.dbar[i] = make_float2(usb.x / w.dt, usb.y / w.dt);
}

// After the PBD's reverse (which added x~_bar to X_bar and kept it in xtb):
// U*_bar = U_s_bar + dt x~_bar and X_bar += sum_c grad w u_0 . U*_bar.
__global__ void __launch_bounds__(kMdfBeadThreads) k_adj_mdf_ustar(const WorldDev* __restrict__ wd, AdjDev a,
                                                                   AdjMdf m) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) a.amax[2] = 0u;   // the steric spread's bound follows from F0_bar (k_adj_mdf_moments)
  float mx = 0.0f;
  if (i < w.N) {
    const Stencil s = make_stencil(w.pos[i], w.W, w.H);
    const float2 xtb = m.xtb[i], usb = m.usb[i];
    const float sx = fmaf(w.dt, xtb.x, usb.x), sy = fmaf(w.dt, xtb.y, usb.y);
    float gx = 0.0f, gy = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 u = m.mu[s.iy[b] + s.ix[c]];
        const float q = u.x * sx + u.y * sy;
        gx = fmaf(s.dx[c] * s.wy[b], q, gx);
        gy = fmaf(s.wx[c] * s.dy[b], q, gy);
      }
    const float2 xb = a.adjX[i];
    a.adjX[i] = make_float2(xb.x + gx, xb.y + gy);
    m.ust[i] = make_float2(sx, sy);
    mx = fmaxf(fabsf(sx), fabsf(sy));
  }
  warp_max_abs(&m.bnd[4], mx);
}

// u_bar_0 += S[U*_bar].
__global__ void __launch_bounds__(kMdfBeadThreads) k_adj_mdf_ustar_scatter(const WorldDev* __restrict__ wd,
                                                                           AdjMdf m) {
  const WorldDev& w = *wd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w.N) return;
  const float2 v2 = m.ust[i];
  const float v[2] = {v2.x, v2.y};
  scatter_fixed<2>(w, make_stencil(w.pos[i], w.W, w.H), v, &m.bnd[4], m.ss);
}

// The moments reversed, per cell: u_bar_0 (the passes' u_bar plus pass 0's
// and the drag's scatters) and rho_bar, then F0_bar into Fbar (the steric
// chain's input) and the population adjoints at the cells the populations
// were pulled from; the accumulators are cleared for the next reversed step.
__global__ void __launch_bounds__(256) k_adj_mdf_moments(const WorldDev* __restrict__ wd, AdjDev a, AdjMdf m) {
  const WorldDev& w = *wd;
  const int W = w.W, H = w.H, HW = H * W;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  float fm = 0.0f;
  if (c < HW) {
    float2 ub = m.ubf[c];
    float rb = m.rhob[c];
    if (m.m > 0) {
      const float iu = pow2f(-scatter_exponent(w, &m.bnd[0])), ir = pow2f(-scatter_exponent(w, &m.bnd[2]));
      ub.x += fx64_value(m.su[2 * c], iu);
      ub.y += fx64_value(m.su[2 * c + 1], iu);
      rb += fx64_value(m.sr[c], ir);
    }
    const float is = pow2f(-scatter_exponent(w, &m.bnd[4]));
    ub.x += fx64_value(m.ss[2 * c], is);
    ub.y += fx64_value(m.ss[2 * c + 1], is);
    const float rho = m.rho[c];
    const float2 u0 = m.mu[c];
    rb -= (ub.x * u0.x + ub.y * u0.y) / rho;
    const float2 Fb = a.Fbar[c];
    const float h = 0.5f / rho;
    const float2 F0b = make_float2(fmaf(ub.x, h, Fb.x), fmaf(ub.y, h, Fb.y));
    a.Fbar[c] = F0b;
    fm = fmaxf(fabsf(F0b.x), fabsf(F0b.y));
    const float jx = ub.x / rho, jy = ub.y / rho;
    const int y = c / W, x = c - y * W;
    const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
    const int ym = y == 0 ? H - 1 : y - 1, yp = y == H - 1 ? 0 : y + 1;
    const int r0 = y * W, rm = ym * W, rp = yp * W;
    // pull sources of populations 0..8 and their lattice velocities
    const int src[9] = {c, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
    constexpr float CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
    for (int i = 0; i < 9; ++i) a.adjG_cur[i * HW + src[i]] += rb + CX[i] * jx + CY[i] * jy;
    m.ubf[c] = make_float2(0.0f, 0.0f);
    m.rhob[c] = 0.0f;
    m.su[2 * c] = 0ull;
    m.su[2 * c + 1] = 0ull;
    m.sr[c] = 0ull;
    m.ss[2 * c] = 0ull;
    m.ss[2 * c + 1] = 0ull;
  }
  warp_max_abs(&a.amax[2], fm);
}

namespace {
int cell_blocks(int n) { return (n + 255) / 256; }
int bead_blocks_mdf(int n) { return n > 0 ? (n + kMdfBeadThreads - 1) / kMdfBeadThreads : 1; }
}  // namespace

void launch_adj_mdf_passes(const WorldDev& h, const WorldDev* wd, const AdjDev& a, const AdjMdf& m, cudaStream_t s) {
  const int HW = h.H * h.W;
  for (int k = m.m - 1; k >= 0; --k) {
    k_adj_mdf_cell<<<cell_blocks(HW), 256, 0, s>>>(wd, m, a.Fbar, k);
    if (h.N) {
      k_adj_mdf_bead<<<bead_blocks_mdf(h.N), kMdfBeadThreads, 0, s>>>(wd, a, m, k);
      k_adj_mdf_scatter<<<bead_blocks_mdf(h.N), kMdfBeadThreads, 0, s>>>(wd, m, k);
    }
  }
  k_adj_mdf_xt<<<bead_blocks_mdf(h.N), kMdfBeadThreads, 0, s>>>(wd, a, m);
}

void launch_adj_mdf_moments(const WorldDev& h, const WorldDev* wd, const AdjDev& a, const AdjMdf& m, cudaStream_t s) {
  k_adj_mdf_ustar<<<bead_blocks_mdf(h.N), kMdfBeadThreads, 0, s>>>(wd, a, m);
  if (h.N) k_adj_mdf_ustar_scatter<<<bead_blocks_mdf(h.N), kMdfBeadThreads, 0, s>>>(wd, m);
  k_adj_mdf_moments<<<cell_blocks(h.H * h.W), 256, 0, s>>>(wd, a, m);
}

}  // namespace mc
