// Autotuner of the launch configuration of a plan's steps.
//
// A plan (one world, or a batch of worlds advanced by the same launches)
// can run its steps in several configurations that advance the worlds
// bitwise the same (LaunchCfg): the per-stage kernels replayed from a CUDA
// graph or one persistent cooperative launch (3 or 4 blocks per SM), the
// number of filaments per PBD block, one or two bin-offset kernels.  Which
// is fastest depends on the plan's shape (tile and bead counts, world
// sizes).  The tuner measures the candidates on device copies of the plan's
// worlds (the worlds themselves do not move), coordinate by coordinate from
// the default, keeps a candidate only when it is at least 1% faster, and
// caches the choice per class of plan for the life of the process.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "mc_internal.cuh"

namespace mc {

namespace {

std::mutex g_mu;
std::map<std::vector<long long>, LaunchCfg>& tuned() {
  static std::map<std::vector<long long>, LaunchCfg> m;
  return m;
}
bool g_auto = true;

// Class of a plan: what its launches cover.
std::vector<long long> plan_key(mc_world* const* ws, int n, const Plan& p) {
  long long beads = 0, cells = 0;
  std::vector<long long> k = {n, p.max_B, p.max_R, p.any_ext, p.any_mdf, p.any_layered, p.one_chunk,
                              p.n_fil_items, p.n_tile_items, p.n_bead_items};
  for (int i = 0; i < n; ++i) {
    const WorldDev& h = world_dev(ws[i]);
    beads += h.N;
    cells += (long long)h.H * h.W;
  }
  k.push_back(beads);
  k.push_back(cells);
  if (n == 1) {   // a single world's grid shape
    k.push_back(world_dev(ws[0]).H);
    k.push_back(world_dev(ws[0]).W);
  }
  return k;
}

// Milliseconds of `steps` steps of plan p in configuration c (after a warm
// run that also captures the configuration's graph).
float time_cfg(Plan& p, const LaunchCfg& c, int steps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  plan_set_cfg(p, c);
  if (plan_run(p, 16, s) != MC_OK) return -1.0f;
  cudaEventRecord(e0, s);
  if (plan_run(p, steps, s) != MC_OK) return -1.0f;
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
  float ms = -1.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace

mc_status plan_tune(mc_world* const* ws, int n, Plan& p, cudaStream_t s, bool automatic) {
  p.tuned = true;
  const std::vector<long long> key = plan_key(ws, n, p);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = tuned().find(key);
    if (it != tuned().end()) {
      plan_set_cfg(p, it->second);
      return MC_OK;
    }
    if (automatic && !g_auto) return MC_OK;
  }
  long long cells = 0, beads = 0;
  for (int i = 0; i < n; ++i) {
    cells += (long long)world_dev(ws[i]).H * world_dev(ws[i]).W;
    beads += world_dev(ws[i]).N;
  }
  // single small worlds are launch-bound whatever the configuration: not
  // worth a measurement when it would happen on its own
  if (automatic && n == 1 && cells < (1ll << 20) && beads < (1ll << 18)) return MC_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone) return MC_OK;   // no measurement inside a capture
  // device copies of the worlds, and their plan
  std::vector<mc_world*> clones;
  for (int i = 0; i < n; ++i) {
    mc_world* c = world_clone(ws[i], s);
    if (!c) break;
    clones.push_back(c);
  }
  LaunchCfg best;   // the default
  if ((int)clones.size() == n) {
    Plan cp;
    if (plan_build(clones.data(), n, s, cp) == MC_OK) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      // steps per measurement: about 20 ms of work, at least 32 steps
      const int steps = (int)std::min<long long>(512, std::max<long long>(32, (1ll << 28) / (cells + 64 * beads + 1)));
      float t_best = time_cfg(cp, best, steps, s, e0, e1);
      auto consider = [&](LaunchCfg c) {
        const float t = time_cfg(cp, c, steps, s, e0, e1);
        if (t > 0.0f && t_best > 0.0f && t < 0.99f * t_best) {
          t_best = t;
          best = c;
        }
      };
      if (t_best > 0.0f) {
        if (persistent_supported(cp)) {
          for (int b : {4, 3}) {
            LaunchCfg c = best;
            c.persistent = b;
            consider(c);
          }
        }
        if (!cp.any_layered && !best.persistent) {
          LaunchCfg c = best;
          c.force_ws = 1;
          consider(c);
        }
        for (int wp : {4, 2}) {
          LaunchCfg c = best;
          c.pbd_warps = wp;
          consider(c);
        }
        if (cp.one_chunk && !best.persistent) {
          LaunchCfg c = best;
          c.scan_kernels = 2;
          consider(c);
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      plan_free(cp, s);
    }
  }
  for (mc_world* c : clones) mc_world_destroy(c);
  cudaStreamSynchronize(s);
  (void)cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    tuned()[key] = best;
  }
  plan_set_cfg(p, best);
  return MC_OK;
}

}  // namespace mc

extern "C" mc_status mc_autotune_mode(int mode) {
  if (mode != 0 && mode != 1) {
    mc::set_last_error("mode must be 0 or 1");
    return MC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(mc::g_mu);
  mc::g_auto = mode == 1;
  return MC_OK;
}
