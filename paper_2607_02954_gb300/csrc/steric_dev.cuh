// Device code of the steric tile stages (a4-a6) and the fused force + LBM
// tile (a5-a7), shared by the per-stage kernels (k_steric.cu) and the
// persistent batched step (k_persist.cu).  See k_steric.cu for the design.
#pragma once

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr int kMaxSeg = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kForceCap = 640;             // bead records staged per pass (force)
constexpr int kAx = kTile + 6;             // force accumulator edge: the tile and 3 halo cells a side
constexpr int kWin = kTile + 8;            // rho_bar window edge: the tile and 4 cells a side
__constant__ int kLbmCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};   // D2Q9 lattice velocities, y components

template <int R>
struct Geo {
  static constexpr int kTaps = 2 * R + 1;
  static constexpr int kL4 = (4 + 2 * R + 3) / 4;      // int4 loads per 4-column strip of the x pass
  static constexpr int kDX0 = ((kTile + 2 * R + 11 + 3) / 4) * 4;
  static constexpr int kDX1 = 4 * (kTile / 4 - 1) + 4 + 4 * kL4;
  static constexpr int kDX = kDX0 > kDX1 ? kDX0 : kDX1;   // deposit accumulator row stride (ints)
  static constexpr int kDY = kTile + 6;                    // deposit accumulator rows
  static constexpr int kLoadRows = kWin + 2 * R;           // rho_x rows staged by the force kernel
};

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

// Bulk copies into shared memory completing on an mbarrier (the tile's bead
// records: each bin segment is contiguous in global and in shared memory).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// (before the barrier's memory is re-initialised or used for anything else)
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Copies `bytes` (a multiple of 16; both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_copy_g2s(void* sdst, const void* gsrc, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_addr(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(smem_addr(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier, for at most ~2^22 polls (each
// try_wait itself suspends for a while); a wait that runs out flags the
// world (kFlagTimeout), waits once more as long, and returns.
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned* flags) {
  for (int round = 0; round < 2; ++round) {
    for (int it = 0; it < (1 << 22); ++it)
      if (mbar_try_wait(bar, parity)) return;
    if (round == 0 && flags) atomicOr(flags, kFlagTimeout);
  }
}

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
  const int* bin_off = w.bin_off;
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
  // every load is issued before any is used (one memory round trip)
  int s0 = 0, e1 = 0;
  if (valid) {
    const int row = wrap_once(by0 + r, nby) * nbx;
    s0 = bin_off[row + lo];
    e1 = bin_off[row + hi + 1];
  }
  // the box spans at most 8 bin columns (tile + 2 R + 3 <= 51 cells) and
  // 16 bin rows; lane (rr, cc) = (lane / 8, lane % 8) covers 4 rows per round
  int mlo[4], mhi[4];
  if (max_count) {
    const int ncol = bx1 - bx0 + 1, nrow = by1 - by0 + 1;
    const int cc = lane & 7;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int rr = (lane >> 3) + 4 * k;
      mlo[k] = 0;
      mhi[k] = 0;
      if (rr < nrow && cc < ncol) {
        const int bin = wrap_once(by0 + rr, nby) * nbx + wrap_once(bx0 + cc, nbx);
        mlo[k] = bin_off[bin];
        mhi[k] = bin_off[bin + 1];
      }
    }
  }
  int incl = e1 - s0;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  s_start[lane] = s0;
  s_pre[lane + 1] = incl;
  if (lane == 0) s_pre[0] = 0;
  if (max_count) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) m = max(m, mhi[k] - mlo[k]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) *max_count = m;
  }
}

// Slot of the v-th bead of the concatenated segments: the segment j with
// s_pre[j] <= v < s_pre[j + 1] by binary search over the 33 prefix entries
// (non-decreasing; empty segments repeat a value and are never chosen).
__device__ __forceinline__ int seg_slot(int v, const int* s_start, const int* s_pre) {
  int j = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (v >= s_pre[j + step]) j += step;
  return s_start[j] + v - s_pre[j];
}

// Periodic image of d in (-n, n) taken in [-lo, n - lo).
__device__ __forceinline__ int image_lo(int d, int n, int lo) {
  if (d < -lo) d += n;
  else if (d >= n - lo) d -= n;
  return d;
}

// Appends `code` to the block's list when `keep`; every lane of the warp
// calls this together.  The list order depends on warp timing, which no
// result depends on (the accumulation is in integers).
__device__ __forceinline__ void list_push(bool keep, int code, int* list, int* s_cnt) {
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(s_cnt, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) list[base + __popc(m & ((1u << lane) - 1u))] = code;
}

// list code: staged slot v (10 bits), rx + 16 and ry + 16 (11 bits each)
__device__ __forceinline__ int pack_code(int v, int rx, int ry) { return v | ((rx + 16) << 10) | ((ry + 16) << 21); }
__device__ __forceinline__ int code_slot(int c) { return c & 1023; }
__device__ __forceinline__ int code_rx(int c) { return ((c >> 10) & 2047) - 16; }
__device__ __forceinline__ int code_ry(int c) { return (c >> 21) - 16; }

template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T m = red[0];
  for (int k = 1; k < kWarps; ++k) m = max(m, red[k]);
  __syncthreads();
  return m;
}

// The tile item of this block in a launch over the tiles of one world
// (row-major, as the plan lists them).
__device__ __forceinline__ int2 single_tile_item(const WorldDev& w, unsigned blk) {
  const unsigned ntx = (unsigned)w.ntx;
  return make_int2(0, (int)(blk % ntx) | ((int)(blk / ntx) << 16));
}

// Taps of a world with half width wR laid out for half width R >= wR.
template <int R>
__device__ __forceinline__ float padded_tap(const WorldDev& w, int wR, int m) {
  const int k = m - (R - wR);
  return (k >= 0 && k <= 2 * wR) ? w.taps[k] : 0.0f;
}

}  // namespace

// ---------------------------------------------------------------------------
// a4 + the x pass of a5.
//
// Accumulator: row ly + 3 for tile rows ly in [-3, th + 3); column
// lx + oxe for region columns lx, where the region is the tile plus wR
// columns a side (origin x0, oxe = R + 4, so every 4-column strip of the x
// pass starts on a 16-byte boundary) or, when that would cover the axis
// more than once, the whole axis (origin 0, oxe = 4, folded).
//
// The fixed-point scale 2^k comes from a bound on the cell sums: a cell's
// 4x4 stencil neighbourhood overlaps at most 2x2 bins and each bead adds at
// most 1/4, so a cell sum is below the largest bin count near the tile.
// That bound leaves at least 24 fractional bits up to about one bead per
// cell.  It is loose (a bead adds 1/16 to a cell on average), so a denser
// tile (k < 24) deposits twice: the first pass measures the largest sum of
// the accumulator (plus the rounding its terms can hide), which gives a
// tight scale for the second.
// ---------------------------------------------------------------------------

// Geometry of one deposit tile.
struct DepTile {
  int W, H, wR, x0, y0, tw, th, cx0, oxe, tile, total;
  bool full_x, full_y;
};

// Deposits the tile's beads at scale 2^k into acc (zeroed) and folds the
// wrapped cells.  Ends with the block synchronised.
template <int R>
__device__ __forceinline__ void deposit_accumulate(int* acc, const WorldDev& w, const DepTile& d, int k,
                                                   const int* s_start, const int* s_pre) {
  using G = Geo<R>;
  const int tid = threadIdx.x;
  const int W = d.W, H = d.H, wR = d.wR, x0 = d.x0, y0 = d.y0, tw = d.tw, th = d.th;
  const int cx0 = d.cx0, oxe = d.oxe, total = d.total;
  const bool full_x = d.full_x, full_y = d.full_y;
  const float4* __restrict__ spos = w.spos;
  const float scale = pow2f(k);
  // each thread deposits the beads v = tid, tid + 256, ... of the segments
  // straight from the bin-ordered records, two loads in flight at a time;
  // a bead whose stencil misses the region adds nothing
  auto deposit = [&](const float4 p) {
    int rx = cell_x(p) - cx0, ry = cell_y(p) - y0;
    bool keep = true;
    if (!full_x) {
      rx = image_lo(rx, W, wR + 2);
      keep = rx <= tw + wR;
    }
    if (!full_y) {
      ry = image_lo(ry, H, 2);
      keep = keep && ry <= th;
    }
    if (!keep) return;
    float wx[4], wy[4];
    peskin4(p.x, wx);
    peskin4(p.y, wy);
    int* base = acc + (ry + 2) * G::kDX + rx - 1 + oxe;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float sy = wy[b] * scale;
#pragma unroll
      for (int a = 0; a < 4; ++a) atomicAdd(base + b * G::kDX + a, __float2int_rn(wx[a] * sy));
    }
  };
  for (int v0 = tid; v0 < total; v0 += 2 * kThreads) {
    const int v1 = v0 + kThreads;
    const float4 p0 = spos[seg_slot(v0, s_start, s_pre)];
    float4 p1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (v1 < total) p1 = spos[seg_slot(v1, s_start, s_pre)];
    deposit(p0);
    if (v1 < total) deposit(p1);
  }
  __syncthreads();
  if (full_x || full_y) {
    // fold the stencil cells that wrapped around an axis the region covers whole
    for (int c = tid; c < G::kDY * G::kDX; c += kThreads) {
      const int ly = c / G::kDX - 3, lx = c % G::kDX - oxe;
      const bool out_y = ly < 0 || ly >= th;
      const bool out_x = full_x && (lx < 0 || lx >= W);
      if ((!out_y && !out_x) || (out_y && !full_y)) continue;
      const int v = acc[c];
      if (v == 0) continue;
      const int ly2 = out_y ? wrap_mod(ly, H) : ly;
      const int lx2 = out_x ? wrap_mod(lx, W) : lx;
      atomicAdd(&acc[(ly2 + 3) * G::kDX + lx2 + oxe], v);
    }
    __syncthreads();
  }
}

// The x pass of the accumulated sums at scale 2^k, rho_s when asked for,
// and the tile's bound (see k_deposit_x).
template <int R>
__device__ __forceinline__ void deposit_xpass(const int* acc, const WorldDev& w, const DepTile& d, int k,
                                              const float* tap_s, float* red, int store_fields) {
  using G = Geo<R>;
  const int tid = threadIdx.x;
  const int W = d.W, x0 = d.x0, y0 = d.y0, tw = d.tw, th = d.th, oxe = d.oxe;
  float* __restrict__ rho_x = w.rho_x;
  float* __restrict__ rho_s_out = w.rho_s;
  const float inv = pow2f(-k);
  const int col0 = x0 - d.cx0 + oxe;            // accumulator column of tile column 0
  // the tile's largest rho_s, and rho_s itself when asked for, come with the
  // x pass (the largest converted sum is the converted largest sum: the
  // conversion is monotone, and every sum is non-negative)
  float vmax = 0.0f;
  // x pass with the fixed-point scale folded into the taps (a power of two:
  // the same products as converting first)
  float tp[G::kTaps];
#pragma unroll
  for (int m = 0; m < G::kTaps; ++m) tp[m] = tap_s[m] * inv;
  if (!d.full_x) {
    const int ly = tid >> 3, s = tid & 7;       // row, strip of 4 columns
    if (ly < th && 4 * s < tw) {
      const int4* src = reinterpret_cast<const int4*>(acc + (ly + 3) * G::kDX + 4 * s + oxe - R);
      float v[4 * G::kL4];
#pragma unroll
      for (int q = 0; q < G::kL4; ++q) {
        const int4 t4 = src[q];
        v[4 * q] = (float)t4.x;
        v[4 * q + 1] = (float)t4.y;
        v[4 * q + 2] = (float)t4.z;
        v[4 * q + 3] = (float)t4.w;
      }
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float sacc = 0.0f;
#pragma unroll
        for (int m = 0; m < G::kTaps; ++m) sacc = fmaf(tp[m], v[j + m], sacc);
        o[j] = sacc;
      }
      const size_t c = (size_t)(y0 + ly) * W + x0 + 4 * s;
      *reinterpret_cast<float4*>(rho_x + c) = make_float4(o[0], o[1], o[2], o[3]);
      // the strip's own cells are v[R .. R + 3]
      vmax = fmaxf(fmaxf(v[R], v[R + 1]), fmaxf(v[R + 2], v[R + 3]));
      if (store_fields)
        *reinterpret_cast<float4*>(rho_s_out + c) = make_float4(v[R] * inv, v[R + 1] * inv, v[R + 2] * inv, v[R + 3] * inv);
    }
  } else {
    for (int c = tid; c < th * kTile; c += kThreads) {
      const int ly = c >> 5, lx = c & 31;
      if (lx < tw) {
        const float v = (float)acc[(ly + 3) * G::kDX + col0 + lx];
        vmax = fmaxf(vmax, v);
        if (store_fields) rho_s_out[(size_t)(y0 + ly) * W + x0 + lx] = v * inv;
      }
    }
    for (int c = tid; c < th * tw; c += kThreads) {
      const int ly = c / tw, lx = c - ly * tw;
      const int* r = acc + (ly + 3) * G::kDX + oxe;
      float sacc = 0.0f;
#pragma unroll
      for (int m = 0; m < G::kTaps; ++m) sacc = fmaf(tp[m], (float)r[wrap_mod(x0 + lx - R + m, W)], sacc);
      rho_x[(size_t)(y0 + ly) * W + x0 + lx] = sacc;
    }
  }
  vmax = block_max(vmax, red);
  // Stored bound of the tile's cell sums of the kernel weights, used for
  // the fixed-point scales of the spread: the largest deposited sum plus the
  // largest rounding its terms can hide (half a unit per bead of the
  // covering bins, at most one term per cell each).  It is 0 exactly when
  // the covering bins hold no bead (written by the early exit of
  // k_deposit_x), and then no bead's stencil reaches the tile: the batched
  // force pass skips such a tile with no effect on any result.
  if (tid == 0) w.tile_rho_max[d.tile] = (vmax + 0.5f * (float)d.total) * inv;
}

// Shared memory of the deposit of one tile.
template <int R>
struct DepositSmem {
  int acc[Geo<R>::kDY * Geo<R>::kDX];
  float tap_s[Geo<R>::kTaps];
  int s_start[kMaxSeg], s_pre[kMaxSeg + 1], s_maxc;
  float red[kWarps];
};

// a4 + the x pass of a5 for the tile item of block `blk` (block-uniform
// control flow; the caller's block runs it whole).
template <int R, bool kSingle>
__device__ __forceinline__ void deposit_x_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                               int store_fields, const WorldDev& w1, unsigned blk,
                                               DepositSmem<R>& sm) {
  using G = Geo<R>;
  int* acc = sm.acc;
  float* tap_s = sm.tap_s;
  int* s_start = sm.s_start;
  int* s_pre = sm.s_pre;
  int& s_maxc = sm.s_maxc;
  float* red = sm.red;
  const int2 it = kSingle ? single_tile_item(w1, blk) : items[blk];
  const WorldDev& w = kSingle ? w1 : worlds[it.x];
  DepTile d;
  d.W = w.W;
  d.H = w.H;
  d.wR = w.R;
  const int ntx = w.ntx;
  const int tx = it.y & 0xffff, ty = it.y >> 16;
  d.tile = ty * ntx + tx;
  d.x0 = tx * kTile;
  d.y0 = ty * kTile;
  d.tw = min(kTile, d.W - d.x0);
  d.th = min(kTile, d.H - d.y0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  d.full_x = d.W < d.tw + 2 * d.wR + 3;
  d.full_y = w.nty == 1;
  d.cx0 = d.full_x ? 0 : d.x0;                  // region column origin
  d.oxe = d.full_x ? 4 : R + 4;                 // accumulator column of region column 0
  if (warp == 0)
    build_segments(w, d.x0 - d.wR - 2, d.x0 + d.tw + d.wR, d.y0 - 2, d.y0 + d.th, s_start, s_pre, &s_maxc);
  if (warp == 1 && lane < G::kTaps) tap_s[lane] = padded_tap<R>(w, d.wR, lane);
  for (int c = tid; c < G::kDY * G::kDX / 4; c += kThreads) reinterpret_cast<int4*>(acc)[c] = make_int4(0, 0, 0, 0);
  __syncthreads();
  d.total = s_pre[kMaxSeg];
  if (d.total == 0) {
    // no bead reaches the region: rho_s, rho_x and the tile maximum are zero
    // (what the passes below give for an empty accumulator, bitwise)
    // (tw is a multiple of 8, so each 4-column strip is whole and aligned)
    const int ly = tid >> 3, s = tid & 7;
    if (ly < d.th && 4 * s < d.tw) {
      const size_t c = (size_t)(d.y0 + ly) * d.W + d.x0 + 4 * s;
      const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      *reinterpret_cast<float4*>(w.rho_x + c) = z;
      if (store_fields) *reinterpret_cast<float4*>(w.rho_s + c) = z;
    }
    if (tid == 0) w.tile_rho_max[d.tile] = 0.0f;
    return;
  }
  int k = fix_exponent((float)s_maxc + 1.0f);
  deposit_accumulate<R>(acc, w, d, k, s_start, s_pre);
  if (k < 24) {
    // dense tile: the largest accumulated sum plus the rounding of its terms
    // (half a unit per bead of the covering bins, at most one term per cell
    // each) bounds every sum; deposit again at the scale that bound gives
    int m = 0;
    for (int c = tid; c < G::kDY * G::kDX; c += kThreads) m = max(m, acc[c]);
    m = block_max(m, reinterpret_cast<int*>(red));
    const int k2 = fix_exponent(((float)m + 0.5f * (float)d.total) * pow2f(-k) * 1.0001f);
    if (k2 > k) {
      for (int c = tid; c < G::kDY * G::kDX / 4; c += kThreads) reinterpret_cast<int4*>(acc)[c] = make_int4(0, 0, 0, 0);
      __syncthreads();
      k = k2;
      deposit_accumulate<R>(acc, w, d, k, s_start, s_pre);
    }
  }
  deposit_xpass<R>(acc, w, d, k, tap_s, red, store_fields);
}

// ---------------------------------------------------------------------------
// The y pass of a5, and a6, for one tile; the result stays in shared memory.
//
// Window: rho_x rows [y0 - 4 - R, y0 + th + 4 + R) x columns [x0 - 4,
// x0 + tw + 4), periodic; rho_bar on window rows and columns [0, th + 8) x
// [0, tw + 8) (tile cell (lx, ly) at window (lx + 4, ly + 4)).  Spread
// accumulators: tile cell (lx, ly) at (lx + 3, ly + 3), F = acc 2^-k.
// ---------------------------------------------------------------------------
// Inputs of one tile, staged before its compute (double-buffered by the
// persistent kernel).
template <int R>
struct TileIn {
  float xb[Geo<R>::kLoadRows * kWin];   // rho_x window
  float4 sp[kForceCap];                 // bead positions of the chunk (bin order)
  float4 sr[kForceCap];                 // their F_el (x, y) and bead id (int bits)
  unsigned long long bar;               // completion of the chunk's bulk copies
  int s_start[kMaxSeg], s_pre[kMaxSeg + 1];
  float nbmax[9];                       // largest rho_s of the 3x3 tiles around
  float tap_s[Geo<R>::kTaps];
};

// Working arrays of the tile being computed.
struct TileWork {
  float win[kWin * kWin];               // rho_bar window
  int accx[kAx * kAx];                  // spread accumulators
  int accy[kAx * kAx];
  int list[kForceCap];
  int s_cnt;
};

template <int R>
struct ForceSmem {
  TileIn<R> in;
  TileWork wk;
};

struct TileBox {
  int x0, y0, tw, th;
};

// Barrier of the NT threads that run a tile's force phase: the whole block
// (NT == kThreads), or warps 0 .. NT/32 - 1 on named barrier 1 (the
// warp-specialised kernel, whose other warps collide).
template <int NT>
__device__ __forceinline__ void force_sync() {
  if (NT == kThreads) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Lists the n staged beads whose stencil reaches the tile (image taken on
// axes with several tiles), packed with their tile-relative cell.
template <int R, int NT = kThreads>
__device__ __forceinline__ void force_compact(const TileIn<R>& in, TileWork& wk, int n, const TileBox& tb, int W,
                                              int H, int ntx, int nty) {
  for (int v0 = 0; v0 < n; v0 += NT) {
    const int v = v0 + threadIdx.x;
    bool keep = false;
    int rx = 0, ry = 0;
    if (v < n) {
      const float4 p = in.sp[v];
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
    list_push(keep, pack_code(v, rx, ry), wk.list, &wk.s_cnt);
  }
}

// Stage 1 of a tile: the rho_x window rows [y0 - 4 - R, y0 + th + 4 + R) x
// columns [x0 - 4, x0 + tw + 4) in 16-byte cp.async chunks (independent of
// the beads).  A 4-column chunk never straddles the periodic edge (x0 and W
// are multiples of 8); rows reach at most 4 + R <= 12 cells outside the axis.
template <int R, int NT = kThreads>
__device__ __forceinline__ void tile_stage_window(TileIn<R>& in, const WorldDev& w, const TileBox& tb) {
  const int W = w.W, H = w.H, tid = threadIdx.x;
  const float* __restrict__ rho_x = w.rho_x;
  const int ww = tb.tw + 8, lh = tb.th + 8 + 2 * R;
  const int nq = ww >> 2;
  int rows_per_pass, i0;
  if (nq == kWin / 4) {   // full tile: constant divisor
    rows_per_pass = NT / (kWin / 4);
    i0 = tid / (kWin / 4);
  } else {
    rows_per_pass = NT / nq;
    i0 = tid / nq;
  }
  const int q = tid - i0 * nq;
  if (i0 < rows_per_pass) {
    const int col = wrap_once(tb.x0 - 4 + 4 * q, W);
    for (int i = i0; i < lh; i += rows_per_pass) {
      const int gy = tb.y0 - 4 - R + i;
      const int row = H >= 12 ? wrap_once(gy, H) : wrap_mod(gy, H);
      cp_async16(&in.xb[i * kWin + 4 * q], rho_x + (size_t)row * W + col);
    }
  }
}

// Stage 2 (warps 0-2, plain loads): the bead segments of the bins that reach
// the tile, the filter taps, and the largest rho_s of the 3x3 tiles around.
template <int R>
__device__ __forceinline__ void tile_stage_meta(TileIn<R>& in, const WorldDev& w, const TileBox& tb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) build_segments(w, tb.x0 - 2, tb.x0 + tb.tw, tb.y0 - 2, tb.y0 + tb.th, in.s_start, in.s_pre, nullptr);
  if (warp == 1 && lane < Geo<R>::kTaps) in.tap_s[lane] = padded_tap<R>(w, w.R, lane);
  // bound of the cell sums of weight * |F_el + F_s|:
  //   |F_s| <= k_rep/2 max|rho_bar(c+1) - rho_bar(c-1)| <= k_rep/2 max rho_bar
  //        <= k_rep/2 max rho_s over the 3x3 tiles around this one,
  // times max rho_s of this tile (the sum of the spread weights of a cell)
  if (warp == 2 && lane < 9) {
    const int tx = tb.x0 / kTile, ty = tb.y0 / kTile;
    const int ty2 = wrap_once(ty + lane / 3 - 1, w.nty), tx2 = wrap_once(tx + lane % 3 - 1, w.ntx);
    in.nbmax[lane] = w.tile_rho_max[ty2 * w.ntx + tx2];
  }
}

// Stage 3 (after stage 2 is visible to the block): the bead records c0 ..
// c0 + n - 1 (n > 0, in segment order) as bulk copies, one lane of warp 0
// per segment (a bin segment is contiguous in the bin-ordered arrays and in
// the staging arrays), after lane 0 has announced the bytes on in.bar; the
// block then waits on in.bar.  Positions and (F_el, id) records are 16 bytes
// each, so every copy starts and ends on 16-byte boundaries.
static_assert(kMaxSeg == 32, "one lane of a warp per segment");
template <int R>
__device__ __forceinline__ void tile_stage_records(TileIn<R>& in, const WorldDev& w, int c0, int n) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&in.bar, (unsigned)n * 32u);
  }
  __syncwarp();
  const int lo = max(in.s_pre[lane], c0), hi = min(in.s_pre[lane + 1], c0 + n);
  if (hi > lo) {
    const int src = in.s_start[lane] + (lo - in.s_pre[lane]);
    const unsigned bytes = (unsigned)(hi - lo) * 16u;
    bulk_copy_g2s(&in.sp[lo - c0], &w.spos[src], bytes, &in.bar);
    bulk_copy_g2s(&in.sr[lo - c0], &w.srec[src], bytes, &in.bar);
  }
}

// Zeroes the spread accumulators and the list count (before the barrier
// that precedes tile_compute).
template <int NT = kThreads>
__device__ __forceinline__ void tile_clear(TileWork& wk) {
  for (int c = threadIdx.x; c < kAx * kAx / 4; c += NT) {
    reinterpret_cast<int4*>(wk.accx)[c] = make_int4(0, 0, 0, 0);
    reinterpret_cast<int4*>(wk.accy)[c] = make_int4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) wk.s_cnt = 0;
}

// The y pass of a5 and a6 for one tile whose inputs have landed (all stages
// complete and visible, accumulators cleared).  Returns k: after the caller
// synchronises the block, accx/accy hold the tile's F 2^k (before folding,
// see force_fold).
template <int R, int NT = kThreads>
__device__ __forceinline__ int tile_compute(TileIn<R>& in, TileWork& wk, const WorldDev& w, int tile,
                                            const TileBox& tb, int store_fields, int after_step) {
  using G = Geo<R>;
  const int W = w.W, H = w.H, ntx = w.ntx, nty = w.nty;
  const float4* __restrict__ spos = w.spos;
  float2* __restrict__ fs_out = w.fs;
  float* __restrict__ rho_b = w.rho_b;
  const float k_rep = w.k_rep;
  const float fmax_el = __uint_as_float(w.fel_max[(*w.t - after_step) & 1]);
  const float rho_max = w.tile_rho_max[tile];
  const bool layered = w.layers == 2;
  const int x0 = tb.x0, y0 = tb.y0, tw = tb.tw, th = tb.th;
  const int tid = threadIdx.x;
  const int ww = tw + 8, wh = th + 8;
  const int total = in.s_pre[kMaxSeg];
  const int n0 = min(kForceCap, total);
  float rho_nb = in.nbmax[0];
  for (int k2 = 1; k2 < 9; ++k2) rho_nb = fmaxf(rho_nb, in.nbmax[k2]);
  const int k = fix_exponent((fmax_el + 0.5f * k_rep * rho_nb) * rho_max * 1.0001f + 1e-30f);
  const float scale = pow2f(k);
  // list the first chunk's beads that reach the tile, then the y pass
  force_compact<R, NT>(in, wk, n0, tb, W, H, ntx, nty);
  if (total > 0 || store_fields) {
    // y pass, 8 window rows per thread (only the beads' gradients and the
    // rho_bar field read it)
    float tp[G::kTaps];
#pragma unroll
    for (int m = 0; m < G::kTaps; ++m) tp[m] = in.tap_s[m];
    const int nstrip = wh >> 3;
    for (int c = tid; c < nstrip * ww; c += NT) {
      int s;
      if (ww == kWin) s = c / kWin;   // full tile: constant divisor
      else s = c / ww;
      const int j = c - s * ww;
      const float* src = in.xb + (8 * s) * kWin + j;
      float v[8 + 2 * R];
#pragma unroll
      for (int q = 0; q < 8 + 2 * R; ++q) v[q] = src[q * kWin];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float sacc = 0.0f;
#pragma unroll
        for (int m = 0; m < G::kTaps; ++m) sacc = fmaf(tp[m], v[r + m], sacc);
        const int i = 8 * s + r;
        wk.win[i * kWin + j] = sacc;
        if (store_fields && i >= 4 && i < th + 4 && j >= 4 && j < tw + 4)
          rho_b[(size_t)(y0 + i - 4) * W + x0 + j - 4] = sacc;
      }
    }
  }
  force_sync<NT>();
  for (int c0 = 0;;) {
    const int cnt = wk.s_cnt;
    for (int q = tid; q < cnt; q += NT) {
      const int code = wk.list[q];
      const int v = code_slot(code), rx = code_rx(code), ry = code_ry(code);
      const float4 p = in.sp[v];
      float wx[4], wy[4];
      peskin4(p.x, wx);
      peskin4(p.y, wy);
      // stencil cell a sits at window column rx + 3 + a; the central
      // differences read one cell further on each side
      const float* base = wk.win + (ry + 2) * kWin + rx + 2;
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
      const float4 rec = in.sr[v];
      if (rx >= 0 && rx < tw && ry >= 0 && ry < th) fs_out[__float_as_int(rec.z)] = make_float2(Fsx, Fsy);
      if (layered) continue;   // two-layer worlds spread at their layer points (k_layer_spread)
      const float2 fe = make_float2(rec.x, rec.y);
      const float Fx = (fe.x + Fsx) * scale, Fy = (fe.y + Fsy) * scale;
      float ax[4], ay[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ax[a] = wx[a] * Fx;
        ay[a] = wx[a] * Fy;
      }
      int* bx = wk.accx + (ry + 2) * kAx + rx + 2;
      int* by = wk.accy + (ry + 2) * kAx + rx + 2;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          atomicAdd(bx + b * kAx + a, __float2int_rn(wy[b] * ax[a]));
          atomicAdd(by + b * kAx + a, __float2int_rn(wy[b] * ay[a]));
        }
      }
    }
    c0 += kForceCap;
    if (c0 >= total) break;
    force_sync<NT>();   // every thread is done with this chunk
    if (tid == 0) wk.s_cnt = 0;
    const int n = min(kForceCap, total - c0);
    tile_stage_records(in, w, c0, n);
    mbar_wait_bounded(&in.bar, (unsigned)(c0 / kForceCap) & 1u, w.flags);
    force_sync<NT>();
    force_compact<R, NT>(in, wk, n, tb, W, H, ntx, nty);
    force_sync<NT>();
  }
  return k;   // the caller synchronises before it reads the accumulators
}

// One tile staged and computed (the non-persistent kernels).
template <int R, int NT = kThreads>
__device__ __forceinline__ int force_tile(ForceSmem<R>& sm, const WorldDev& w, int tile, const TileBox& tb,
                                          int store_fields, int after_step) {
  tile_stage_window<R, NT>(sm.in, w, tb);
  tile_stage_meta(sm.in, w, tb);
  tile_clear<NT>(sm.wk);
  if (threadIdx.x == 0) mbar_init(&sm.in.bar);
  force_sync<NT>();
  const int n0 = min(kForceCap, sm.in.s_pre[kMaxSeg]);
  if (n0 > 0) tile_stage_records(sm.in, w, 0, n0);
  cp_async_wait_all();   // the window (cp.async)
  if (n0 > 0) mbar_wait_bounded(&sm.in.bar, 0u, w.flags);
  force_sync<NT>();
  const int k = tile_compute<R, NT>(sm.in, sm.wk, w, tile, tb, store_fields, after_step);
  // every thread is past its last wait on the barrier (tile_compute
  // synchronises after each chunk's wait), so its memory can be released
  if (threadIdx.x == 0) mbar_inval(&sm.in.bar);
  return k;
}

// Folds the stencil cells that wrapped around an axis the tile covers whole
// (one tile on that axis); call after the block has synchronised.
template <class Work, int NT = kThreads>
__device__ __forceinline__ void force_fold(Work& wk, const TileBox& tb, int ntx, int nty) {
  if (ntx > 1 && nty > 1) return;
  const bool fx = ntx == 1, fy = nty == 1;
  for (int c = threadIdx.x; c < kAx * kAx; c += NT) {
    const int ly = c / kAx - 3, lx = c % kAx - 3;
    const bool out_y = ly < 0 || ly >= tb.th, out_x = lx < 0 || lx >= tb.tw;
    if ((!out_y && !out_x) || (out_y && !fy) || (out_x && !fx)) continue;
    const int vx = wk.accx[c], vy = wk.accy[c];
    const int t2 = (wrap_mod(ly, tb.th) + 3) * kAx + wrap_mod(lx, tb.tw) + 3;
    if (vx) atomicAdd(&wk.accx[t2], vx);
    if (vy) atomicAdd(&wk.accy[t2], vy);
  }
  force_sync<NT>();
}

__device__ __forceinline__ TileBox tile_box(const WorldDev& w, int packed) {
  TileBox b;
  const int tx = packed & 0xffff, ty = packed >> 16;
  b.x0 = tx * kTile;
  b.y0 = ty * kTile;
  b.tw = min(kTile, w.W - b.x0);
  b.th = min(kTile, w.H - b.y0);
  return b;
}

// The tile's population rows (plane i, rows y - c_iy, 128-byte segments) to L2.
template <int NT = kThreads>
__device__ __forceinline__ void prefetch_populations(const WorldDev& w, const TileBox& tb) {
  const float* src = w.g[*w.t & 1];
  const int W = w.W, H = w.H;
  const size_t HW = (size_t)H * W;
  for (int c = threadIdx.x; c < 9 * kTile; c += NT) {
    const int i = c >> 5, r = c & (kTile - 1);
    if (r >= tb.th) continue;
    const int y = wrap_once(tb.y0 + r - kLbmCy[i], H);
    const float* a = src + (size_t)i * HW + (size_t)y * W + tb.x0;
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
  }
}

// a7 on the tile's cells with F = acc 2^-k from shared memory.  Each warp
// collides rows warp, warp + 8, ...; the first row's populations are pulled
// before the barrier that completes the spread (pulling one row ahead in the
// loop measured slower: register pressure).
__device__ __forceinline__ void tile_lbm(TileWork& wk, const WorldDev& w, const TileBox& tb, int k) {
  const int W = w.W, H = w.H, HW = H * W;
  const long long t = *w.t;
  const float* __restrict__ src = w.g[t & 1];
  float* __restrict__ dst = w.g[(t + 1) & 1];
  float2* __restrict__ u_out = w.u;
  const LbmConst kc{w.om_p, w.om_m, w.src_p, w.src_m};
  const float inv = pow2f(-k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool active = lane < tb.tw && warp < tb.th;
  const int x = tb.x0 + lane;
  const int xm = x == 0 ? W - 1 : x - 1, xp = x == W - 1 ? 0 : x + 1;
  LbmPull q;
  int y = tb.y0 + warp;
  if (active) lbm_pull(src, HW, y * W, (y == 0 ? H - 1 : y - 1) * W, (y == H - 1 ? 0 : y + 1) * W, x, xm, xp, q);
  __syncthreads();
  force_fold(wk, tb, w.ntx, w.nty);
  if (!active) return;
  for (int ly = warp; ly < tb.th; ly += kWarps) {
    if (ly != warp)
      lbm_pull(src, HW, y * W, (y == 0 ? H - 1 : y - 1) * W, (y == H - 1 ? 0 : y + 1) * W, x, xm, xp, q);
    const int s = (ly + 3) * kAx + lane + 3;
    const float2 F = make_float2((float)wk.accx[s] * inv, (float)wk.accy[s] * inv);
    u_out[(size_t)y * W + x] = lbm_collide(q, dst, HW, y * W + x, F, kc);
    y += kWarps;
  }
}

// y pass of a5 + a6 + a7 on one tile: the force density goes from shared
// memory straight into the collision (the same arithmetic as k_force_spread
// followed by k_lbm, without F's round trip through HBM).  The tile's
// population rows are prefetched into L2 on entry, so their DRAM reads
// overlap the force phase.
template <int R, bool kSingle>
__device__ __forceinline__ void force_lbm_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                               const WorldDev& w1, unsigned blk, ForceSmem<R>& sm) {
  const int2 it = kSingle ? single_tile_item(w1, blk) : items[blk];
  const WorldDev& w = kSingle ? w1 : worlds[it.x];
  const TileBox tb = tile_box(w, it.y);
  const bool layered = w.layers == 2;
  if (!layered) prefetch_populations(w, tb);
  const int tile = (tb.y0 / kTile) * w.ntx + tb.x0 / kTile;
  int k = 40;
  if (!kSingle && !layered && w.tile_rho_max[tile] == 0.0f) {
    // no bead's stencil reaches this tile's cells (the deposit's bound is 0
    // exactly then), so it owns no bead and the spread has no term on it:
    // F = 0, as the force pass would give.  Sparse batched worlds have many
    // such tiles.
    tile_clear(sm.wk);
  } else {
    k = force_tile<R>(sm, w, tile, tb, 0, 0);
  }
  // two-layer worlds: F_s only; their layer spread and collision follow in their own kernels
  if (!layered) tile_lbm(sm.wk, w, tb, k);
}

}  // namespace mc
