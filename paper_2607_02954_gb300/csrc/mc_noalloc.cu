// Allocation-free read-out of bead positions into host memory.
//
// mc_world_get_state with host outputs allocates a device staging buffer for
// the positions on every call.  Some callers cannot allocate device memory
// when they read results: processes whose device memory is fully reserved up
// front by another allocator (a framework's caching allocator, or a fixed
// memory budget per tenant), where any further cudaMalloc fails; and
// latency-critical serving or control loops, where cudaMalloc / cudaFree can
// synchronize the whole device and stall unrelated work.  This file gives
// them mc_world_get_positions_noalloc, which stages the positions in a
// file-scope device array instead.
//
// The array is sized for kNoallocMaxBeads beads (2^20 beads, 8 MiB).  Every
// GPU that loads the library holds those 8 MiB until the process exits.
// Every call uses the same array: two calls whose work overlaps on the GPU
// (for example on two streams) race on it.  Each call writes every element
// it later reads, so nothing needs clearing between calls.
#include <mutex>
#include <string>

#include "mc_internal.cuh"

namespace {

constexpr int kNoallocMaxBeads = 1 << 20;
constexpr int kMaxDevices = 64;

// x of bead i at [i], y at [kNoallocMaxBeads + i]
static __device__ __align__(256) float g_noalloc_positions[2 * kNoallocMaxBeads];

std::mutex g_noalloc_mu;
float* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in; the real address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
cudaError_t noalloc_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    float* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_positions);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

__global__ void k_positions_to_static(const float4* __restrict__ pos, int N, float* __restrict__ scratch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = pos[i];
  scratch[i] = (float)mc::cell_x(p) + p.x;
  scratch[kNoallocMaxBeads + i] = (float)mc::cell_y(p) + p.y;
}

mc_status noalloc_fail(mc_status s, const std::string& msg) {
  mc::set_last_error(msg.c_str());
  return s;
}

}  // namespace

extern "C" {

// Allocation-free variant of the position read-out of mc_world_get_state.
// The paper has no counterpart; see include/mc.h for the contract.
mc_status mc_world_get_positions_noalloc(const mc_world* w, float* x, float* y, void* stream) {
  if (!w || !x || !y) return noalloc_fail(MC_ERR_INVALID_ARG, "world, x and y must not be NULL");
  const mc::WorldDev& h = mc::world_dev(w);
  if (h.N > kNoallocMaxBeads)
    return noalloc_fail(MC_ERR_INVALID_ARG, "mc_world_get_positions_noalloc: the world has " + std::to_string(h.N) +
                                                " beads, above the static scratch limit of " +
                                                std::to_string(kNoallocMaxBeads));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* scratch = nullptr;
  cudaError_t e = noalloc_address(&scratch);
  if (e != cudaSuccess)
    return noalloc_fail(MC_ERR_CUDA, std::string("cudaGetSymbolAddress of the read-out scratch: ") +
                                         cudaGetErrorString(e));
  if (h.N == 0) return MC_OK;
  k_positions_to_static<<<(h.N + 255) / 256, 256, 0, s>>>(h.pos, h.N, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(x, scratch, h.N * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(y, scratch + kNoallocMaxBeads, h.N * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return noalloc_fail(MC_ERR_CUDA, std::string("mc_world_get_positions_noalloc: ") + cudaGetErrorString(e));
  return MC_OK;
}

}  // extern "C"
