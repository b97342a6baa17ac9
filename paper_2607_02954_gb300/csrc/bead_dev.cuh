// Device code of the bead-parallel stages (a1-a3 PBD, a2 scatter, a8
// interpolation + advance), shared by the per-stage kernels (k_bead.cu) and
// the persistent batched step (k_persist.cu).
#pragma once

#include "mc_internal.cuh"

namespace mc {

constexpr int kPbdFloatsPerBead = 18;

__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }


// X + dt U in cell + fraction form, wrapped, for X = p.
__device__ __forceinline__ float4 advance_pos(const WorldDev& w, float4 p, float Ux, float Uy) {
  const int W = w.W, H = w.H;
  int cx = cell_x(p), cy = cell_y(p);
  float fx = p.x + w.dt * Ux, fy = p.y + w.dt * Uy;
  const float kx = floorf(fx), ky = floorf(fy);
  fx -= kx;
  fy -= ky;
  cx += (int)kx;
  cy += (int)ky;
  if (fx >= 1.0f) { fx = 0.0f; cx += 1; }   // a tiny negative fraction rounded up to 1
  if (fy >= 1.0f) { fy = 0.0f; cy += 1; }
  cx = wrap_once(cx, W);
  cy = wrap_once(cy, H);
  return make_float4(fx, fy, __int_as_float(cx), __int_as_float(cy));
}

// a8 for one bead at p = X^n with velocity U: the velocity record (kRecord;
// the advance fused into the next step's PBD skips it, since a run of steps
// ends with a standalone advance that writes the last step's), the watchdog
// (|U| > u_max or non-finite: flag the world, keep the bead),
// X^{n+1} = wrap(X^n + dt U) in cell + fraction form, D += dt U.
// Returns X^{n+1} (X^n when the watchdog fired).
template <bool kRecord = true>
__device__ __forceinline__ float4 advance_tail(const WorldDev& w, int i, float4 p, float Ux, float Uy) {
  if (kRecord) w.ubead[i] = make_float2(Ux, Uy);
  const float m2 = Ux * Ux + Uy * Uy;
  if (!(m2 <= w.u_max * w.u_max)) {   // also catches NaN
    atomicOr(w.flags, kFlagUnstable);
    return p;
  }
  const float4 q = advance_pos(w, p, Ux, Uy);
  w.pos[i] = q;
  float2 d = w.disp[i];
  d.x += w.dt * Ux;
  d.y += w.dt * Uy;
  w.disp[i] = d;
  return q;
}

// U_i = sum_c delta_h(c - X_i) u(c) over the 4x4 stencil of p, for the
// velocity field u of a W x H grid.
__device__ __forceinline__ float2 interp_field(const float2* __restrict__ u, int W, int H, const float4 p) {
  const int cx = cell_x(p), cy = cell_y(p);
  float wx[4], wy[4];
  peskin4(p.x, wx);
  peskin4(p.y, wy);
  int ix[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) ix[a] = wrap_once(cx - 1 + a, W);
  float Ux = 0.0f, Uy = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float2* row = u + (size_t)wrap_once(cy - 1 + b, H) * W;
    float rx = 0.0f, ry = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 v = row[ix[a]];
      rx = fmaf(wx[a], v.x, rx);
      ry = fmaf(wx[a], v.y, ry);
    }
    Ux = fmaf(wy[b], rx, Ux);
    Uy = fmaf(wy[b], ry, Uy);
  }
  return make_float2(Ux, Uy);
}

// The world's fluid velocity at bead position p.
__device__ __forceinline__ float2 interp_u(const WorldDev& w, const float4 p) { return interp_field(w.u, w.W, w.H, p); }

// ---------------------------------------------------------------------------
// Two-layer filament (Fluid-filament Interaction): the immersed-boundary
// points of bead i are X_i +- delta n_i.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 layer_velocity(const WorldDev& w, const float4 p, float2 n, float d) {
  int cx, cy;
  float fx, fy;
  layer_cell(p, n, d, w.W, w.H, cx, cy, fx, fy);
  float wx[4], wy[4];
  peskin4(fx, wx);
  peskin4(fy, wy);
  float Ux = 0.0f, Uy = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float2* row = w.u + (size_t)wrap_once(cy - 1 + b, w.H) * w.W;
    float rx = 0.0f, ry = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 v = row[wrap_once(cx - 1 + a, w.W)];
      rx = fmaf(wx[a], v.x, rx);
      ry = fmaf(wx[a], v.y, ry);
    }
    Ux = fmaf(wy[b], rx, Ux);
    Uy = fmaf(wy[b], ry, Uy);
  }
  return make_float2(Ux, Uy);
}

constexpr double kLayerScale = 1099511627776.0;   // 2^40: fixed point of the layer spread

// The energy field sampled at p with the interpolation kernel.
__device__ __forceinline__ float energy_sample(const WorldDev& w, const float4 q) {
  const int W = w.W, H = w.H;
  float ex[4], ey[4];
  peskin4(q.x, ex);
  peskin4(q.y, ey);
  const int qx = cell_x(q), qy = cell_y(q);
  float e = 0.0f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float* row = w.energy + (size_t)wrap_once(qy - 1 + b, H) * W;
    float r = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) r = fmaf(ex[a], row[wrap_once(qx - 1 + a, W)], r);
    e = fmaf(ey[b], r, e);
  }
  return e;
}

// a8's velocity of bead i at p = X^n: the interpolated fluid velocity, or,
// for a two-layer filament, the mean of the velocities at X +- delta n.
// With observables and an energy field (kExt), also the bead's energy
// sample at X^n, stored in ebead and added to q in fixed point.
// The energy bead i collects at p (observables with an energy field): stored
// in ebead and added to q in fixed point.
__device__ __forceinline__ void bead_energy(const WorldDev& w, int i, const float4 p, long long& q) {
  if (w.observe && w.energy) {
    const float e = energy_sample(w, p);
    w.ebead[i] = e;
    q += obs_q(e);
  }
}

template <bool kExt>
__device__ __forceinline__ float2 bead_velocity(const WorldDev& w, int i, const float4 p, long long& q) {
  if (kExt) bead_energy(w, i, p, q);
  if (kExt && w.layers == 2) {
    const float2 n = w.nrm[i];
    const float2 Up = layer_velocity(w, p, n, w.layer_half), Um = layer_velocity(w, p, n, -w.layer_half);
    return make_float2(0.5f * (Up.x + Um.x), 0.5f * (Up.y + Um.y));
  }
  return interp_u(w, p);
}

__device__ __forceinline__ float sq(float v) { return v * v; }

// Constants of the PBD passes, read once per warp.
struct PbdConst {
  float hb, hs, ksh, ko, kappa_dt, dt;
  int n_pbd, order, W, H, nbx;
};

__device__ __forceinline__ PbdConst pbd_const(const WorldDev& w) {
  PbdConst k;
  k.hb = 0.5f * w.k_bend;
  k.hs = 0.5f * w.k_st;
  k.ksh = w.k_sh;
  k.ko = w.orient * k.hs * k.ksh;
  k.kappa_dt = w.kappa_dt;
  k.dt = w.dt;
  k.n_pbd = w.n_pbd;
  k.order = w.pbd_order;
  k.W = w.W;
  k.H = w.H;
  k.nbx = w.nbx;
  return k;
}

// Edge vector min_image(X_b - X_a) from cell indices and fractions.
__device__ __forceinline__ float2 edge_vec(const float4 pa, const float4 pb, int W, int H) {
  int dcx = cell_x(pb) - cell_x(pa), dcy = cell_y(pb) - cell_y(pa);
  if (2 * dcx > W) dcx -= W; else if (2 * dcx < -W) dcx += W;
  if (2 * dcy > H) dcy -= H; else if (2 * dcy < -H) dcy += H;
  return make_float2((float)dcx + (pb.x - pa.x), (float)dcy + (pb.y - pa.y));
}

// The per-edge factors of the position pass: sc = (l - L)/l = 1 - L/l with
// l = |(x, y)| (from the hardware reciprocal square root), and the sine and
// cosine of the frame angle (the hardware's, of the angle reduced to
// [-pi, pi]).  Their errors (a few 1e-7) stay below the step's float32
// resolution of the elastic force.
__device__ __forceinline__ void pbd_edge_terms(float x, float y, float L, float th, float& sc, float& sn, float& cs) {
  sc = fmaf(-L, rsqrtf(x * x + y * y), 1.0f);
  const float tr = fmaf(-6.28318548f, rintf(th * 0.159154943f), th);
  __sincosf(tr, &sn, &cs);
}

// Position pass of one edge (Eqs. 2-4) with current edge vector (x, y),
// rest length L and frame angle th: the correction (ddx, ddy) of its first
// bead (the second gets the opposite), and the frame's turn toward the edge.
__device__ __forceinline__ void edge_correction(float x, float y, float L, float& th, const PbdConst& k, float& ddx,
                                                float& ddy) {
  float sc, sn, cs;
  pbd_edge_terms(x, y, L, th, sc, sn, cs);
  const float csx = sc * x, csy = sc * y;
  ddx = k.hs * (csx + k.ksh * (x - L * cs - csx));
  ddy = k.hs * (csy + k.ksh * (y - L * sn - csy));
  th += k.ko * (cs * y - sn * x) * __frcp_rn(L);   // frame turns toward the edge (orient)
}

// Unit normal of the filament at a bead (two-layer coupling): t is the
// normalised sum of the unit vectors of the bead's outgoing and incoming
// edges; where they nearly cancel (|sum| < 1e-3, a chain folded back) t is
// the outgoing edge, the incoming one at the last bead; n = (-t_y, t_x).
__device__ __forceinline__ float2 unit2(float2 v) {
  const float r = rsqrtf(v.x * v.x + v.y * v.y);
  return make_float2(v.x * r, v.y * r);
}

__device__ __forceinline__ float2 bead_normal(float2 out, bool has_out, float2 in, bool has_in) {
  float sx = 0.0f, sy = 0.0f;
  if (has_out) {
    sx += out.x;
    sy += out.y;
  }
  if (has_in) {
    sx += in.x;
    sy += in.y;
  }
  const float ns = sqrtf(sx * sx + sy * sy);
  float2 t;
  if (ns >= 1e-3f) t = make_float2(sx / ns, sy / ns);
  else t = has_out ? out : in;
  return make_float2(-t.y, t.x);
}

// F_el = kappa (x_hat - X) / dt of one bead, its 8x8 bin (a2) and one
// histogram atomic per group of lanes sharing a bin.  Every lane calls this.
// With direct forcing (kMode 2) the bead's output is instead its velocity
// U_s = U* + dl/dt, U* (the fluid's, stored in ubead by the prediction) plus
// the PBD correction of the carried position.
template <int kMode>
__device__ __forceinline__ void bead_out(const WorldDev& w, const PbdConst& k, bool valid, int b, const float4 P,
                                         float dlx, float dly, float& fmax) {
  if (kMode == 2) {
    if (valid) {
      const float2 U = w.ubead[b];
      const float2 Us = make_float2(U.x + dlx / k.dt, U.y + dly / k.dt);
      w.ubead[b] = Us;
      w.sus[w.bead_slot[b]] = Us;   // the MDF passes read U_s in bin order
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  int bin = -1 - lane;
  if (valid) {
    const float2 fe = make_float2(k.kappa_dt * dlx, k.kappa_dt * dly);
    w.fel[b] = fe;
    fmax = fmaxf(fmax, fmaxf(fabsf(fe.x), fabsf(fe.y)));
    bin = (cell_y(P) / kBin) * k.nbx + cell_x(P) / kBin;
    w.bead_bin[b] = bin;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&w.bin_count[bin], __popc(peers));
}

// Jacobi PBD of a filament of at most 64 beads in registers: lane l holds
// beads, edges and joints 2l and 2l + 1, and reads its neighbours' values by
// warp shuffles.  The same arithmetic, in the same order, as pbd_smem.
template <bool kExt, int kMode>
__device__ __forceinline__ float pbd_regs(const WorldDev& w, const PbdConst& k, int b0, int B, int e0, int j0,
                                          long long t) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nE = B - 1, nJ = B - 2;
  const int i0 = 2 * lane, i1 = i0 + 1;
  const bool hb0 = i0 < B, hb1 = i1 < B, he0 = i0 < nE, he1 = i1 < nE, hj0 = i0 < nJ, hj1 = i1 < nJ;
  const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float4 P0 = hb0 ? w.pos[b0 + i0] : z4;
  float4 P1 = hb1 ? w.pos[b0 + i1] : z4;
  // the filament's own inputs first: their loads and the drive's sines
  // overlap the advance's gathers
  float th0 = he0 ? w.theta[e0 + i0] : 0.0f;
  float th1 = he1 ? w.theta[e0 + i1] : 0.0f;
  const float L0 = he0 ? (kExt ? rest_length(w, e0 + i0, t) : w.L_rest[e0 + i0]) : 1.0f;
  const float L1 = he1 ? (kExt ? rest_length(w, e0 + i1, t) : w.L_rest[e0 + i1]) : 1.0f;
  const float thr0 = hj0 ? drive_angle(w.drive[j0 + i0], t) : 0.0f;
  const float thr1 = hj1 ? drive_angle(w.drive[j0 + i1], t) : 0.0f;
  if (kMode == 1) {
    // a8 of the previous step for the lane's beads, then this step's PBD from X^n
    long long q = 0;
    if (hb0) {
      const float2 U = bead_velocity<kExt>(w, b0 + i0, P0, q);
      P0 = advance_tail<false>(w, b0 + i0, P0, U.x, U.y);
    }
    if (hb1) {
      const float2 U = bead_velocity<kExt>(w, b0 + i1, P1, q);
      P1 = advance_tail<false>(w, b0 + i1, P1, U.x, U.y);
    }
    if (kExt && w.observe && w.energy) obs_add_warp(&w.obs[2], q);
  } else if (kMode == 0 && w.rec_pos) {
    // the step's start, into the reverse mode's record
    if (hb0) w.rec_pos[b0 + i0] = P0;
    if (hb1) w.rec_pos[b0 + i1] = P1;
    if (he0) w.rec_theta[e0 + i0] = th0;
    if (he1) w.rec_theta[e0 + i1] = th1;
  } else if (kMode == 2) {
    // direct forcing: the fluid (u* in u) carries the beads, PBD starts there
    if (hb0) {
      const float2 U = interp_u(w, P0);
      w.ubead[b0 + i0] = U;
      P0 = advance_pos(w, P0, U.x, U.y);
    }
    if (hb1) {
      const float2 U = interp_u(w, P1);
      w.ubead[b0 + i1] = U;
      P1 = advance_pos(w, P1, U.x, U.y);
    }
  }
  float4 Pn;   // bead 2l + 2
  Pn.x = __shfl_down_sync(kAll, P0.x, 1);
  Pn.y = __shfl_down_sync(kAll, P0.y, 1);
  Pn.z = __shfl_down_sync(kAll, P0.z, 1);
  Pn.w = __shfl_down_sync(kAll, P0.w, 1);
  const float2 v0 = edge_vec(P0, P1, k.W, k.H);
  const float2 v1 = edge_vec(P1, Pn, k.W, k.H);
  if (kExt && w.layers == 2) {
    // filament normals at beads 2l, 2l + 1 from X^n
    const float2 z2 = make_float2(0.0f, 0.0f);
    const float2 u0 = he0 ? unit2(v0) : z2, u1 = he1 ? unit2(v1) : z2;
    float2 um;   // edge 2l - 1, incoming at bead 2l
    um.x = __shfl_up_sync(kAll, u1.x, 1);
    um.y = __shfl_up_sync(kAll, u1.y, 1);
    if (hb0) w.nrm[b0 + i0] = bead_normal(u0, he0, um, lane > 0);
    if (hb1) w.nrm[b0 + i1] = bead_normal(u1, he1, u0, true);
  }
  float dlx0 = 0.0f, dly0 = 0.0f, dlx1 = 0.0f, dly1 = 0.0f;
  if (k.order == 1) {
    for (int iter = 0; iter < k.n_pbd; ++iter) {
      // bending pass (Eq. 1), joint 2l of every lane first, then joint 2l + 1
      // from the updated angles: joint j moves theta_j by +h C_j and
      // theta_{j+1} by -h C_j
      const float C0 = hj0 ? th1 - th0 - thr0 : 0.0f;
      if (hj0) {
        th0 += k.hb * C0;
        th1 -= k.hb * C0;
      }
      const float thn = __shfl_down_sync(kAll, th0, 1);   // theta_{2l+2}, updated
      const float C1 = hj1 ? thn - th1 - thr1 : 0.0f;
      if (hj1) th1 += k.hb * C1;
      const float Cm = __shfl_up_sync(kAll, C1, 1);        // joint 2l-1 moves theta_{2l}
      if (lane > 0) th0 -= k.hb * Cm;
      // position pass (Eqs. 2-4), edge 2l first, then edge 2l + 1
      float ddx0 = 0.0f, ddy0 = 0.0f;
      if (he0) {
        edge_correction(v0.x + (dlx1 - dlx0), v0.y + (dly1 - dly0), L0, th0, k, ddx0, ddy0);
        dlx0 += ddx0;
        dly0 += ddy0;
        dlx1 -= ddx0;
        dly1 -= ddy0;
      }
      const float dlxn = __shfl_down_sync(kAll, dlx0, 1), dlyn = __shfl_down_sync(kAll, dly0, 1);
      float ddx1 = 0.0f, ddy1 = 0.0f;
      if (he1) {
        edge_correction(v1.x + (dlxn - dlx1), v1.y + (dlyn - dly1), L1, th1, k, ddx1, ddy1);
        dlx1 += ddx1;
        dly1 += ddy1;
      }
      const float ddxm = __shfl_up_sync(kAll, ddx1, 1), ddym = __shfl_up_sync(kAll, ddy1, 1);
      if (lane > 0) {   // edge 2l-1 moves bead 2l (its second bead)
        dlx0 -= ddxm;
        dly0 -= ddym;
      }
    }
  }
  for (int iter = 0; iter < (k.order == 1 ? 0 : k.n_pbd); ++iter) {
    // bending pass (Eq. 1): C_j = (theta_{j+1} - theta_j) - theta_rest,j
    const float thn = __shfl_down_sync(kAll, th0, 1);
    const float C0 = hj0 ? th1 - th0 - thr0 : 0.0f;
    const float C1 = hj1 ? thn - th1 - thr1 : 0.0f;
    const float Cm = __shfl_up_sync(kAll, C1, 1);   // C_{2l-1}
    if (he0) th0 += k.hb * (C0 - (lane > 0 ? Cm : 0.0f));
    if (he1) th1 += k.hb * (C1 - C0);
    // position pass (Eqs. 2-4) on the updated frames
    const float dlxn = __shfl_down_sync(kAll, dlx0, 1), dlyn = __shfl_down_sync(kAll, dly0, 1);
    float ddx0 = 0.0f, ddy0 = 0.0f, ddx1 = 0.0f, ddy1 = 0.0f;
    if (he0) edge_correction(v0.x + (dlx1 - dlx0), v0.y + (dly1 - dly0), L0, th0, k, ddx0, ddy0);
    if (he1) edge_correction(v1.x + (dlxn - dlx1), v1.y + (dlyn - dly1), L1, th1, k, ddx1, ddy1);
    const float ddxm = __shfl_up_sync(kAll, ddx1, 1), ddym = __shfl_up_sync(kAll, ddy1, 1);
    if (hb0) {
      dlx0 += ddx0 - (lane > 0 ? ddxm : 0.0f);
      dly0 += ddy0 - (lane > 0 ? ddym : 0.0f);
    }
    if (hb1) {
      dlx1 += ddx1 - ddx0;
      dly1 += ddy1 - ddy0;
    }
  }
  if (he0) w.theta[e0 + i0] = th0;
  if (he1) w.theta[e0 + i1] = th1;
  float fmax = 0.0f;
  bead_out<kMode>(w, k, hb0, b0 + i0, P0, dlx0, dly0, fmax);
  bead_out<kMode>(w, k, hb1, b0 + i1, P1, dlx1, dly1, fmax);
  if (kExt && w.observe && t >= 1) {
    // behaviour descriptors (Eqs. 5, 6): squared change of the rest angles
    // and rest lengths from step t - 1 to step t
    float eb = 0.0f, ep = 0.0f;
    if (hj0) eb += sq(drive_angle(w.drive[j0 + i0], t - 1) - thr0);
    if (hj1) eb += sq(drive_angle(w.drive[j0 + i1], t - 1) - thr1);
    if (w.ldrive) {
      if (he0) ep += sq(rest_length(w, e0 + i0, t - 1) - L0);
      if (he1) ep += sq(rest_length(w, e0 + i1, t - 1) - L1);
    }
    obs_add_warp(&w.obs[0], obs_q(eb));
    obs_add_warp(&w.obs[1], obs_q(ep));
  }
  return fmax;
}

// Jacobi PBD of a filament of any length: the filament's edges, joints and
// bead corrections live in a per-warp slice of shared memory; every pass
// reads the slice, then writes corrections, with a warp barrier in between,
// so all corrections of a pass see the state before it.
template <bool kExt, int kMode>
__device__ __forceinline__ float pbd_smem(const WorldDev& w, const PbdConst& k, int b0, int B, int e0, int j0,
                                          long long t, float* s, int maxB) {
  const int lane = threadIdx.x & 31;
  const int nE = B - 1, nJ = B - 2;
  float* vx = s;
  float* vy = s + maxB;
  float* th = s + 2 * maxB;
  float* Lr = s + 3 * maxB;
  float* ddx = s + 4 * maxB;
  float* ddy = s + 5 * maxB;
  float* dlx = s + 6 * maxB;
  float* dly = s + 7 * maxB;
  float* thr = s + 8 * maxB;
  float* C = s + 9 * maxB;
  float4* P = reinterpret_cast<float4*>(s + 10 * maxB);    // bead positions
  float4* D = reinterpret_cast<float4*>(s + 14 * maxB);    // joint drive parameters
  // stage the filament's inputs in shared memory, every copy in flight at once
  if (kMode == 1) {
    // a8 of the previous step, the advanced positions staged directly
    long long q = 0;
    for (int i = lane; i < B; i += 32) {
      const float4 p = w.pos[b0 + i];
      const float2 U = bead_velocity<kExt>(w, b0 + i, p, q);
      P[i] = advance_tail<false>(w, b0 + i, p, U.x, U.y);
    }
    if (kExt && w.observe && w.energy) obs_add_warp(&w.obs[2], q);
  } else if (kMode == 2) {
    // direct forcing: the positions the fluid (u* in u) carries the beads to
    for (int i = lane; i < B; i += 32) {
      const float4 p = w.pos[b0 + i];
      const float2 U = interp_u(w, p);
      w.ubead[b0 + i] = U;
      P[i] = advance_pos(w, p, U.x, U.y);
    }
  } else {
    for (int i = lane; i < B; i += 32) cpa16(&P[i], &w.pos[b0 + i]);
  }
  for (int e = lane; e < nE; e += 32) {
    cpa4(&th[e], &w.theta[e0 + e]);
    if (!kExt || !w.ldrive) cpa4(&Lr[e], &w.L_rest[e0 + e]);
    else Lr[e] = drive_length(w.ldrive[e0 + e], t);
  }
  for (int j = lane; j < nJ; j += 32) cpa16(&D[j], &w.drive[j0 + j]);
  cpa_wait_all();
  __syncwarp();
  if (kMode == 0 && w.rec_pos) {   // the step's start, into the reverse mode's record
    for (int i = lane; i < B; i += 32) w.rec_pos[b0 + i] = P[i];
    for (int e = lane; e < nE; e += 32) w.rec_theta[e0 + e] = th[e];
  }
  for (int e = lane; e < nE; e += 32) {
    const float2 v = edge_vec(P[e], P[e + 1], k.W, k.H);
    vx[e] = v.x;
    vy[e] = v.y;
  }
  for (int j = lane; j < nJ; j += 32) thr[j] = drive_angle(D[j], t);
  for (int i = lane; i < B; i += 32) {
    dlx[i] = 0.0f;
    dly[i] = 0.0f;
  }
  __syncwarp();
  if (kExt && w.layers == 2) {
    for (int i = lane; i < B; i += 32) {
      const float2 z2 = make_float2(0.0f, 0.0f);
      const float2 out = i < nE ? unit2(make_float2(vx[i], vy[i])) : z2;
      const float2 in = i > 0 ? unit2(make_float2(vx[i - 1], vy[i - 1])) : z2;
      w.nrm[b0 + i] = bead_normal(out, i < nE, in, i > 0);
    }
  }
  if (k.order == 1) {
    // red-black passes: within a colour no two joints share an edge and no
    // two edges share a bead, so the lanes update in place
    for (int iter = 0; iter < k.n_pbd; ++iter) {
      for (int c = 0; c < 2; ++c) {
        for (int j = 2 * lane + c; j < nJ; j += 64) {
          const float Cj = th[j + 1] - th[j] - thr[j];
          th[j] += k.hb * Cj;
          th[j + 1] -= k.hb * Cj;
        }
        __syncwarp();
      }
      for (int c = 0; c < 2; ++c) {
        for (int e = 2 * lane + c; e < nE; e += 64) {
          float the = th[e], ddxe, ddye;
          edge_correction(vx[e] + (dlx[e + 1] - dlx[e]), vy[e] + (dly[e + 1] - dly[e]), Lr[e], the, k, ddxe, ddye);
          th[e] = the;
          dlx[e] += ddxe;
          dly[e] += ddye;
          dlx[e + 1] -= ddxe;
          dly[e + 1] -= ddye;
        }
        __syncwarp();
      }
    }
  }
  for (int iter = 0; iter < (k.order == 1 ? 0 : k.n_pbd); ++iter) {
    for (int j = lane; j < nJ; j += 32) C[j] = th[j + 1] - th[j] - thr[j];
    __syncwarp();
    for (int e = lane; e < nE; e += 32) {
      const float c1 = e < nJ ? C[e] : 0.0f;      // edge e is theta_1 of joint e
      const float c0 = e > 0 ? C[e - 1] : 0.0f;   // ... and theta_2 of joint e-1
      th[e] += k.hb * (c1 - c0);
    }
    __syncwarp();
    for (int e = lane; e < nE; e += 32) {
      float the = th[e];
      edge_correction(vx[e] + (dlx[e + 1] - dlx[e]), vy[e] + (dly[e + 1] - dly[e]), Lr[e], the, k, ddx[e], ddy[e]);
      th[e] = the;
    }
    __syncwarp();
    for (int i = lane; i < B; i += 32) {
      const float ax = i < nE ? ddx[i] : 0.0f, ay = i < nE ? ddy[i] : 0.0f;          // x_1 of edge i
      const float bx = i > 0 ? ddx[i - 1] : 0.0f, by = i > 0 ? ddy[i - 1] : 0.0f;    // x_2 of edge i-1
      dlx[i] += ax - bx;
      dly[i] += ay - by;
    }
    __syncwarp();
  }
  for (int e = lane; e < nE; e += 32) w.theta[e0 + e] = th[e];
  float fmax = 0.0f;
  for (int i0 = 0; i0 < B; i0 += 32) {
    const int i = i0 + lane;
    bead_out<kMode>(w, k, i < B, b0 + i, i < B ? P[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f), i < B ? dlx[i] : 0.0f,
                    i < B ? dly[i] : 0.0f, fmax);
  }
  if (kExt && w.observe && t >= 1) {
    float eb = 0.0f, ep = 0.0f;
    for (int j = lane; j < nJ; j += 32) eb += sq(drive_angle(D[j], t - 1) - thr[j]);
    if (w.ldrive)
      for (int e = lane; e < nE; e += 32) ep += sq(drive_length(w.ldrive[e0 + e], t - 1) - Lr[e]);
    obs_add_warp(&w.obs[0], obs_q(eb));
    obs_add_warp(&w.obs[1], obs_q(ep));
  }
  return fmax;
}

// One warp per filament (a1 + a3 + the a2 histogram).  Bead positions enter
// as edge vectors v0 = min_image(X_b - X_a) plus the accumulated corrections,
// so the corrections keep full FP32 precision whatever the magnitude of the
// coordinates.  Filaments of at most 64 beads run in registers; longer ones
// in the warp's slice of dynamic shared memory (maxB floats per array; zero
// when no filament of the launch is longer than 64 beads).
// The block's dynamic shared memory (filaments longer than 64 beads stage
// in per-warp slices of it; maxB is a multiple of 4: float4 slices stay
// aligned).
extern __shared__ __align__(16) float pbd_dyn_smem[];

template <bool kExt, int kMode, bool kSingle>
__device__ __forceinline__ void pbd_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                         int n_items, int maxB, unsigned blk) {
  float* smem = pbd_dyn_smem;
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blk * wpb + warp;
  if (item >= n_items) return;  // warp-uniform exit; the body has no block barrier
  // a single-world launch takes its item from the block index (the world
  // stays in the table: its fields reach the arithmetic exactly as in a batch)
  const int2 it = kSingle ? make_int2(0, item) : items[item];
  const WorldDev& w = worlds[it.x];
  if ((kMode == 2) != (w.ib == 1)) return;   // direct-forcing worlds run their PBD after the steric spread
  const int f = it.y;
  const int b0 = w.fil_off[f];
  const int B = w.fil_off[f + 1] - b0;
  const int e0 = b0 - f, j0 = b0 - 2 * f;
  // with kMode 1 the counter still holds the previous step (the scan of
  // this step advances it)
  const long long t = *w.t + (kMode == 1 ? 1 : 0);
  const PbdConst k = pbd_const(w);
  float fmax = B <= 64 ? pbd_regs<kExt, kMode>(w, k, b0, B, e0, j0, t)
                       : pbd_smem<kExt, kMode>(w, k, b0, B, e0, j0, t,
                                               smem + (size_t)warp * maxB * kPbdFloatsPerBead, maxB);
  if (kMode == 2) return;
  // largest |F_el| component of the world this step (bounds the spread's
  // fixed-point scale); non-negative floats order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
  if (lane == 0) atomicMax(&w.fel_max[t & 1], __float_as_uint(fmax));
}

// a2: scatter bead records into bin order.  Lanes of one warp that share a
// bin take consecutive slots from one atomic.
template <bool kSingle>
__device__ __forceinline__ void bin_scatter_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                                 const WorldDev& w1, unsigned blk) {
  const int2 it = kSingle ? make_int2(0, (int)blk * kBeadChunk) : items[blk];
  const WorldDev& w = kSingle ? w1 : worlds[it.x];
  const int i = it.y + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = i < w.N;
  const int bin = valid ? w.bead_bin[i] : -1 - lane;
  // the record is loaded before the cursor atomic, so its latency overlaps
  const float4 p = valid ? w.pos[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float2 fe = valid ? w.fel[i] : make_float2(0.0f, 0.0f);
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(&w.bin_cursor[bin], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (valid) {
    const int slot = base + __popc(peers & ((1u << lane) - 1u));
    w.spos[slot] = p;
    w.srec[slot] = make_float4(fe.x, fe.y, __int_as_float(i), 0.0f);
    if (w.bead_slot) w.bead_slot[i] = slot;   // direct forcing: U_s goes to the bead's slot
  }
}

// a8: U_i = sum_c delta_h(c - X_i) u(c) over the 4x4 stencil, then the
// inertia-free advance X += dt U (cell index + fraction, wrapped) and the
// unwrapped displacement D += dt U.  Thread 0 of each world's first block
// advances the world's step counter (no other stage kernel reads it).
template <bool kExt, bool kSingle>
__device__ __forceinline__ void interp_advance_body(const WorldDev* __restrict__ worlds,
                                                    const int2* __restrict__ items, unsigned blk) {
  const int2 it = kSingle ? make_int2(0, (int)blk * kBeadChunk) : items[blk];
  const WorldDev& w = worlds[it.x];
  if (it.y == 0 && threadIdx.x == 0) *w.t += 1;
  const int i = it.y + threadIdx.x;
  // the velocity at the bead's position at the start of the step (and, with
  // observables, the energy sampled there; every lane of the block takes
  // part in the warp sum)
  long long q = 0;
  float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float2 U = make_float2(0.0f, 0.0f);
  if (i < w.N) {
    p = w.pos[i];
    if (kExt && w.ib == 1) {
      U = w.ubead[i];   // direct forcing: the bead's own velocity U_s
      bead_energy(w, i, p, q);
    } else {
      U = bead_velocity<kExt>(w, i, p, q);
    }
  }
  if (kExt && w.observe && w.energy) obs_add_warp(&w.obs[2], q);
  if (i >= w.N) return;
  advance_tail(w, i, p, U.x, U.y);
}

}  // namespace mc
