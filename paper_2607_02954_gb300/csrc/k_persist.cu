// Persistent batched step: one cooperative launch advances every world of a
// plan by n steps (a1-a8 each, in the fused order of enqueue_steps), the
// stages separated by grid-wide barriers instead of kernel boundaries.
//
// Every stage runs the same block bodies as the per-stage kernels, over the
// same work items (a block takes items blockIdx.x, blockIdx.x + gridDim.x,
// ...), so the worlds advance bitwise as they do through the per-stage
// graph.  The launch is cooperative (every block resident at once), which
// the barriers need; each barrier wait is bounded in time and, when the
// bound runs out, sets the plan's status word and the worlds' timeout flag
// and ends the kernel (the worlds' state is then unspecified).
//
// Supported plans: penalty coupling, one layer, filaments of at most 64
// beads (register PBD), Gaussian half width 4 (sigma in (0.75, 1]); the
// autotuner offers this path only for such plans.
#include "bead_dev.cuh"
#include "grid_dev.cuh"
#include "steric_dev.cuh"

namespace mc {

namespace {

constexpr int kPersistR = 4;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier on bar[0] (arrivals) and bar[1] (generation), both zero
// at launch.  The last block to arrive resets the count and publishes the
// next generation; the others wait for it with acquire loads (which make
// every write released before the barrier visible), for at most timeout_ns.
// Returns false on every thread of a block whose wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, unsigned target,
                                             unsigned long long timeout_ns, unsigned* status, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();   // this block's writes before its arrival
    const unsigned n = atomicAdd(&bar[0], 1u) + 1u;
    if (n == target) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_gpu(&bar[1]) == gen) {
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(status, 1u);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  gen += 1;
  const bool ok = *s_ok != 0;
  __syncthreads();   // every thread has read the flag before it is reused
  return ok;
}

// Shared memory of the persistent kernel: one stage at a time.
template <int R>
union PersistSmem {
  ForceSmem<R> force;
  DepositSmem<R> deposit;
  ScanSmem scan;
};

}  // namespace

struct PersistArgs {
  const WorldDev* worlds;
  int n_worlds;
  const int2* fil_items;
  int n_pbd_blocks, n_fil_items;
  const int2* bead_items;
  int n_bead_items;
  const int2* tile_items;
  int n_tile_items;
  const int2* scan_items;
  int n_scan_items;
  int one_chunk;
  int n_steps;
  unsigned* bar;       // [2] barrier words, zeroed before the launch
  unsigned* status;    // set to 1 when a barrier wait ran out
  unsigned long long timeout_ns;
  unsigned extra;      // arrivals a barrier waits for beyond the grid (0; tests of the timeout use 1)
};

template <int R, bool kExt, int kBlocks>
__global__ void __launch_bounds__(256, kBlocks) k_step_persistent(const PersistArgs a) {
  __shared__ __align__(16) PersistSmem<R> sm;
  __shared__ int s_ok;
  const WorldDev& w1 = a.worlds[0];   // unused: batched bodies take every world from the table
  unsigned gen = 0;
  const unsigned target = gridDim.x + a.extra;
  auto barrier = [&]() { return grid_barrier(a.bar, gen, target, a.timeout_ns, a.status, &s_ok); };
  bool ok = true;
  for (int s = 0; s < a.n_steps && ok; ++s) {
    // a1-a3 (fused with the previous step's a8 after the first step)
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_pbd_blocks; b += gridDim.x) {
      if (s == 0) pbd_body<kExt, 0, false>(a.worlds, a.fil_items, a.n_fil_items, 0, b);
      else pbd_body<kExt, 1, false>(a.worlds, a.fil_items, a.n_fil_items, 0, b);
    }
    if (!(ok = barrier())) break;
    // a2 bin offsets
    if (!a.one_chunk) {
      for (unsigned b = blockIdx.x; b < (unsigned)a.n_scan_items; b += gridDim.x) {
        __syncthreads();
        scan_sums_body<false>(a.worlds, a.scan_items, s > 0, w1, b, sm.scan);
      }
      if (!(ok = barrier())) break;
    }
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_scan_items; b += gridDim.x) {
      __syncthreads();
      scan_apply_body<false>(a.worlds, a.scan_items, a.one_chunk, s > 0, w1, b, sm.scan);
    }
    if (!(ok = barrier())) break;
    // a2 scatter
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_bead_items; b += gridDim.x)
      bin_scatter_body<false>(a.worlds, a.bead_items, w1, b);
    if (!(ok = barrier())) break;
    // a4 + x pass of a5
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_tile_items; b += gridDim.x) {
      __syncthreads();
      deposit_x_body<R, false>(a.worlds, a.tile_items, 0, w1, b, sm.deposit);
    }
    if (!(ok = barrier())) break;
    // y pass of a5 + a6 + a7
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_tile_items; b += gridDim.x) {
      __syncthreads();
      force_lbm_body<R, false>(a.worlds, a.tile_items, w1, b, sm.force);
    }
    if (!(ok = barrier())) break;
  }
  if (ok) {
    // a8 of the last step
    for (unsigned b = blockIdx.x; b < (unsigned)a.n_bead_items; b += gridDim.x)
      interp_advance_body<kExt, false>(a.worlds, a.bead_items, b);
    return;
  }
  // a barrier wait ran out: flag every world of the plan
  if (threadIdx.x == 0)
    for (int k = blockIdx.x; k < a.n_worlds; k += gridDim.x) atomicOr(a.worlds[k].flags, kFlagTimeout);
}

namespace {

// Blocks of a cooperative launch: every block resident at once.
template <bool kExt, int kBlocks>
int persistent_grid() {
  static int grid = -1;
  if (grid < 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_persistent<kPersistR, kExt, kBlocks>, 256, 0);
    grid = per > 0 ? per * sms : 0;
  }
  return grid;
}

// Test settings of the barrier (process-wide).
unsigned g_extra_arrivals = 0;
unsigned long long g_timeout_ns = 1000000000ull;   // 1 s

}  // namespace

bool persistent_supported(const Plan& p) {
  return p.n_worlds >= 1 && !p.any_mdf && !p.any_layered && p.max_B <= 64 && p.max_R == kPersistR &&
         p.n_tile_items > 0 && p.d_persist_bar != nullptr;
}

void persistent_setup() {
  persistent_grid<false, 3>();
  persistent_grid<true, 3>();
  persistent_grid<false, 4>();
  persistent_grid<true, 4>();
}

void persistent_test_settings(unsigned extra, unsigned long long timeout_ns) {
  g_extra_arrivals = extra;
  g_timeout_ns = timeout_ns;
}

// n steps of the plan in one cooperative launch (the barrier words are
// cleared first, on the same stream), compiled for p.cfg.persistent (3 or
// 4) blocks per SM.
cudaError_t launch_persistent(const Plan& p, int n, cudaStream_t s) {
  const bool ext = p.any_ext, four = p.cfg.persistent == 4;
  const int grid = ext ? (four ? persistent_grid<true, 4>() : persistent_grid<true, 3>())
                       : (four ? persistent_grid<false, 4>() : persistent_grid<false, 3>());
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(p.d_persist_bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  PersistArgs a;
  a.worlds = p.d_worlds;
  a.n_worlds = p.n_worlds;
  a.fil_items = p.d_fil_items;
  a.n_fil_items = p.n_fil_items;
  a.n_pbd_blocks = (p.n_fil_items + 7) / 8;
  a.bead_items = p.d_bead_items;
  a.n_bead_items = p.n_bead_items;
  a.tile_items = p.d_tile_items;
  a.n_tile_items = p.n_tile_items;
  a.scan_items = p.d_scan_items;
  a.n_scan_items = p.n_scan_items;
  a.one_chunk = p.one_chunk && p.cfg.scan_kernels != 2 ? 1 : 0;
  a.n_steps = n;
  a.bar = p.d_persist_bar;
  a.status = p.d_persist_bar + 2;
  a.timeout_ns = g_timeout_ns;
  a.extra = g_extra_arrivals;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (ext) return four ? cudaLaunchKernelEx(&cfg, k_step_persistent<kPersistR, true, 4>, a)
                      : cudaLaunchKernelEx(&cfg, k_step_persistent<kPersistR, true, 3>, a);
  return four ? cudaLaunchKernelEx(&cfg, k_step_persistent<kPersistR, false, 4>, a)
              : cudaLaunchKernelEx(&cfg, k_step_persistent<kPersistR, false, 3>, a);
}

}  // namespace mc
