// Device code of the bin-offset scan (a2), shared by the per-stage kernels
// (k_grid.cu) and the persistent batched step (k_persist.cu).
#pragma once

#include "mc_internal.cuh"

namespace mc {

// Shared memory of one scan block.
struct ScanSmem {
  int red[9];
  int warp_tot[8];
};

// ---------------------------------------------------------------------------
// a2: exclusive prefix sum of the per-bin bead counts, in blocks of
// kScanChunk bins: k_scan_sums adds up each block, k_scan_apply offsets each
// block by the sum of the world's earlier blocks and scans it.  When every
// world of a plan fits one block, k_scan_apply runs alone (one kernel, no
// block sums), else both run.  Also resets the counts for the next step and
// primes the scatter cursors.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_sum_256(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = threadIdx.x < 8 ? red[threadIdx.x] : 0;
  if (threadIdx.x < 32) {
    for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[8] = t;
  }
  __syncthreads();
  const int r = red[8];
  __syncthreads();
  return r;
}

// The first block of each world also keeps the step counter's bookkeeping:
// with inc_t (the step's PBD ran fused with the previous step's advance,
// which left the counter behind) it advances the counter, and it clears the
// next step's F_el-maximum slot (this step's, written by the PBD, stays
// readable for the spread).
template <bool kSingle>
__device__ __forceinline__ void scan_sums_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                               int inc_t, const WorldDev& w1, unsigned blk, ScanSmem& sm) {
  int* red = sm.red;
  const int2 it = kSingle ? make_int2(0, (int)blk) : items[blk];
  const WorldDev& w = kSingle ? w1 : worlds[it.x];
  if (it.y == 0 && threadIdx.x == 0) {
    const long long t = *w.t + inc_t;
    if (inc_t) *w.t = t;
    w.fel_max[(t + 1) & 1] = 0u;
  }
  const int base = it.y * kScanChunk;
  const int end = min(base + kScanChunk, w.n_bins);
  int s = 0;
  for (int k = base + threadIdx.x; k < end; k += blockDim.x) s += w.bin_count[k];
  s = block_sum_256(s, red);
  if (threadIdx.x == 0) w.chunk_sum[it.y] = s;
}

// With book (plans whose worlds fit one scan block each, where k_scan_sums
// is not launched: a first block has no earlier blocks to add up) it also
// keeps k_scan_sums' step-counter bookkeeping.
template <bool kSingle>
__device__ __forceinline__ void scan_apply_body(const WorldDev* __restrict__ worlds, const int2* __restrict__ items,
                                                int book, int inc_t, const WorldDev& w1, unsigned blk,
                                                ScanSmem& sm) {
  int* red = sm.red;
  int* warp_tot = sm.warp_tot;
  const int2 it = kSingle ? make_int2(0, (int)blk) : items[blk];
  const WorldDev& w = kSingle ? w1 : worlds[it.x];
  if (book && it.y == 0 && threadIdx.x == 0) {
    const long long t = *w.t + inc_t;
    if (inc_t) *w.t = t;
    w.fel_max[(t + 1) & 1] = 0u;
  }
  int pre = 0;
  for (int k = threadIdx.x; k < it.y; k += blockDim.x) pre += w.chunk_sum[k];
  pre = block_sum_256(pre, red);
  const int n = w.n_bins;
  const int base = it.y * kScanChunk + threadIdx.x * 4;
  int v[4];
  int tsum = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? w.bin_count[base + j] : 0;
    tsum += v[j];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  int wbase = 0;
  for (int k = 0; k < wid; ++k) wbase += warp_tot[k];
  int run = pre + wbase + incl - tsum;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = base + j;
    if (k < n) {
      w.bin_off[k] = run;
      w.bin_cursor[k] = run;
      w.bin_count[k] = 0;
      run += v[j];
      if (k == n - 1) w.bin_off[n] = run;
    }
  }
}

}  // namespace mc
