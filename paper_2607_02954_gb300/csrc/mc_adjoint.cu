// Reverse mode through a rollout: forward with checkpoints, then the adjoint
// sweep with per-segment recompute (checkpoint-and-recompute every K steps),
// or forward with every step's record kept and a sweep that re-runs nothing.
//
// mc_rollout_forward   advances the world n steps and stores its state (bead
//                      positions, edge angles, populations) every K steps and
//                      at the end.
// mc_rollout_forward_stored
//                      advances n steps writing each step's record (start
//                      state and intermediates) in place.
// mc_rollout_backward  given dL/d(final unwrapped positions), walks the
//                      segments from last to first: re-runs the segment's
//                      forward from its checkpoint keeping every step's
//                      state and intermediates (F_el, F_s, rho_bar, u, F) in
//                      the step's record, then reverses the steps from last
//                      to first, each step's kernels reading its record.
//                      Accumulates the parameter gradients and leaves the
//                      world in its final state.
// Penalty worlds bind each step's fields to its record through a per-step
// world descriptor (bind_step); direct-forcing worlds copy them
// (k_seg_save / k_seg_restore), since their passes alternate two velocity
// buffers whose inputs the record keeps.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "mc_internal.cuh"

namespace {

mc_status afail(mc_status s, const std::string& m) {
  mc::set_last_error(m.c_str());
  return s;
}

#define MC_ACUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return afail(MC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct StateSlot {
  size_t pos, theta, g;   // byte offsets inside one state record
  size_t bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

StateSlot state_slot(const mc::WorldDev& h) {
  StateSlot s;
  s.pos = 0;
  s.theta = align256((size_t)h.N * sizeof(float4));
  s.g = s.theta + align256((size_t)h.E * sizeof(float));
  s.bytes = s.g + align256((size_t)9 * h.H * h.W * sizeof(float));
  return s;
}

// After the n_ck checkpoints and the final state: the final displacement,
// and the start's displacement and observables.
struct TapeTail {
  size_t disp_end, disp0, obs0, end;
};

TapeTail tape_tail(const mc::WorldDev& h, int n_ck, const StateSlot& sl) {
  TapeTail t;
  t.disp_end = (size_t)(n_ck + 1) * sl.bytes;
  t.disp0 = t.disp_end + align256((size_t)h.N * sizeof(float2));
  t.obs0 = t.disp0 + align256((size_t)h.N * sizeof(float2));
  t.end = t.obs0 + 256;
  return t;
}

cudaStream_t adj_capture_stream() {
  thread_local cudaStream_t cs = nullptr;
  if (!cs) cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  return cs;
}

// The second stream of a captured sweep (segment re-runs), joined into the
// capture by an event.
cudaStream_t adj_rerun_stream() {
  thread_local cudaStream_t cs = nullptr;
  if (!cs) cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  return cs;
}

mc_status save_state(const mc::WorldDev& h, int parity, char* rec, const StateSlot& sl, cudaStream_t s) {
  const size_t HW = (size_t)h.H * h.W;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(rec + sl.pos, h.pos, h.N * sizeof(float4), cudaMemcpyDeviceToDevice, s));
  if (h.E) MC_ACUDA(cudaMemcpyAsync(rec + sl.theta, h.theta, h.E * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(rec + sl.g, h.g[parity], 9 * HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MC_OK;
}

mc_status load_state(const mc::WorldDev& h, int parity, const char* rec, const StateSlot& sl, cudaStream_t s) {
  const size_t HW = (size_t)h.H * h.W;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(h.pos, rec + sl.pos, h.N * sizeof(float4), cudaMemcpyDeviceToDevice, s));
  if (h.E) MC_ACUDA(cudaMemcpyAsync(h.theta, rec + sl.theta, h.E * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(h.g[parity], rec + sl.g, 9 * HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MC_OK;
}

// One step of a segment record: the state at the start of the step (as a
// checkpoint) followed by the step's intermediates the adjoint reads.
struct StepSlot {
  StateSlot st;
  size_t fel, fs, rho_b, u, F, nrm;
  size_t mu, mrho, us;   // direct forcing: the MDF passes' input velocities, the density, U_s
  size_t bytes;
};

StepSlot step_slot(const mc::WorldDev& h) {
  StepSlot s;
  s.st = state_slot(h);
  const size_t HW = (size_t)h.H * h.W;
  s.fel = s.st.bytes;
  s.fs = s.fel + align256((size_t)h.N * sizeof(float2));
  s.rho_b = s.fs + align256((size_t)h.N * sizeof(float2));
  s.u = s.rho_b + align256(HW * sizeof(float));
  s.F = s.u + align256(HW * sizeof(float2));
  s.nrm = s.F + align256(HW * sizeof(float2));
  const bool df = h.ib == 1;
  s.mu = s.nrm + align256(h.layers == 2 ? (size_t)h.N * sizeof(float2) : 0);
  s.mrho = s.mu + align256(df ? (size_t)std::max(h.mdf_iters, 1) * HW * sizeof(float2) : 0);   // u_0 at least
  s.us = s.mrho + align256(df ? HW * sizeof(float) : 0);
  s.bytes = s.us + align256(df ? (size_t)h.N * sizeof(float2) : 0);
  return s;
}

// After a recomputed step: its intermediates (F_el, F_s, rho_bar, u, F) into
// `cur`, and, with `next`, the state the next step starts from (positions,
// edge angles, the populations of parity `par`).
__global__ void k_seg_save(const mc::WorldDev* __restrict__ wd, char* cur, char* next, int par, StepSlot sl) {
  const mc::WorldDev& h = *wd;
  const size_t HW = (size_t)h.H * h.W, n9 = 9 * HW;
  const size_t total = n9 > (size_t)h.N ? n9 : (size_t)h.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    if (i < (size_t)h.N) {
      reinterpret_cast<float2*>(cur + sl.fel)[i] = h.fel[i];
      reinterpret_cast<float2*>(cur + sl.fs)[i] = h.fs[i];
      if (h.nrm) reinterpret_cast<float2*>(cur + sl.nrm)[i] = h.nrm[i];
      if (h.ib == 1) reinterpret_cast<float2*>(cur + sl.us)[i] = h.ubead[i];   // U_s (the advance's velocity)
      if (next) reinterpret_cast<float4*>(next + sl.st.pos)[i] = h.pos[i];
    }
    if (next && i < (size_t)h.E) reinterpret_cast<float*>(next + sl.st.theta)[i] = h.theta[i];
    if (i < HW) {
      reinterpret_cast<float*>(cur + sl.rho_b)[i] = h.rho_b[i];
      reinterpret_cast<float2*>(cur + sl.u)[i] = h.u[i];
      reinterpret_cast<float2*>(cur + sl.F)[i] = h.F[i];
      if (h.ib == 1) reinterpret_cast<float*>(cur + sl.mrho)[i] = h.mrho[i];
    }
    if (next && i < n9) reinterpret_cast<float*>(next + sl.st.g)[i] = h.g[par][i];
  }
}

// Before a step's adjoint: the world's positions, populations of parity
// `par` and intermediates from the record, the step counter, and the
// per-step adjoint accumulators (u_bar, Q) cleared.
__global__ void k_seg_restore(const mc::WorldDev* __restrict__ wd, const char* rec, int par, long long t,
                              StepSlot sl, mc::AdjDev a) {
  const mc::WorldDev& h = *wd;
  const size_t HW = (size_t)h.H * h.W, n9 = 9 * HW;
  const size_t total = n9 > (size_t)h.N ? n9 : (size_t)h.N;
  const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i0 == 0) {
    *h.t = t;
    h.fel_max[0] = 0u;
    h.fel_max[1] = 0u;
    // the bounds this step's adjoint kernels produce: of Q, and of the
    // next reversed step's u_bar (this step's u_bar reads slot a.par)
    a.amax[2] = 0u;
    a.amax[a.par ^ 1] = 0u;
  }
  for (size_t i = i0; i < total; i += (size_t)gridDim.x * blockDim.x) {
    if (i < (size_t)h.N) {
      h.pos[i] = reinterpret_cast<const float4*>(rec + sl.st.pos)[i];
      h.fel[i] = reinterpret_cast<const float2*>(rec + sl.fel)[i];
      h.fs[i] = reinterpret_cast<const float2*>(rec + sl.fs)[i];
    }
    if (i < HW) {
      h.rho_b[i] = reinterpret_cast<const float*>(rec + sl.rho_b)[i];
      h.u[i] = reinterpret_cast<const float2*>(rec + sl.u)[i];
      h.F[i] = reinterpret_cast<const float2*>(rec + sl.F)[i];
      a.ubar[2 * i] = 0ull;
      a.ubar[2 * i + 1] = 0ull;
      a.Q[2 * i] = 0ull;
      a.Q[2 * i + 1] = 0ull;
    }
    if (i < n9) h.g[par][i] = reinterpret_cast<const float*>(rec + sl.st.g)[i];
  }
}

// Descriptors of the reverse sweep's steps (penalty coupling), so that
// neither the recompute nor the reverse copies a step's fields: the world's
// own descriptor with the step's fields in its slot q of the segment record.
// Recompute of step q (population parity par): populations in from slot q
// and out to slot q + 1 (the world's own buffer after the last slot), F, u,
// rho_bar, F_el, F_s and the normals written into slot q, and the unfused
// PBD records the positions and edge angles it starts from there.  Reverse
// of step q: the same slot, with the positions read from it.
mc::WorldDev bind_step(const mc::WorldDev& h, char* seg, const StepSlot& ss, int K, int q, int par, bool reverse) {
  mc::WorldDev b = h;
  char* rec = seg + (size_t)q * ss.bytes;
  b.g[par] = reinterpret_cast<float*>(rec + ss.st.g);
  if (q + 1 < K) b.g[par ^ 1] = reinterpret_cast<float*>(seg + (size_t)(q + 1) * ss.bytes + ss.st.g);
  b.F = reinterpret_cast<float2*>(rec + ss.F);
  b.u = reinterpret_cast<float2*>(rec + ss.u);
  b.rho_b = reinterpret_cast<float*>(rec + ss.rho_b);
  b.fel = reinterpret_cast<float2*>(rec + ss.fel);
  b.fs = reinterpret_cast<float2*>(rec + ss.fs);
  if (h.layers == 2) b.nrm = reinterpret_cast<float2*>(rec + ss.nrm);
  if (reverse) {
    b.pos = reinterpret_cast<float4*>(rec + ss.st.pos);
  } else {
    b.rec_pos = reinterpret_cast<float4*>(rec + ss.st.pos);
    b.rec_theta = reinterpret_cast<float*>(rec + ss.st.theta);
  }
  return b;
}

size_t bind_index(int K, int buf, int q, int par, bool reverse) {
  return (((size_t)buf * 2 + (reverse ? 1 : 0)) * 2 + par) * K + q;
}

// A stored rollout's tape: the start and final state records and the tail
// (tape_tail with one checkpoint), then one step record per step, then the
// recorded forward's step descriptors.
struct StoredLayout {
  size_t steps, desc, end;
};

StoredLayout stored_layout(const mc::WorldDev& h, int n) {
  StoredLayout L;
  L.steps = align256(tape_tail(h, 1, state_slot(h)).end);
  L.desc = L.steps + (size_t)n * step_slot(h).bytes;
  L.end = L.desc + align256((size_t)n * sizeof(mc::WorldDev));
  return L;
}

// One step of the penalty path in unfused stages, with p's descriptor
// binding the step's fields to its record (bind_step).
void run_recorded_step(const mc::Plan& p, cudaStream_t s) {
  mc::launch_pbd(p, s);
  mc::launch_bin_scan(p, s);
  mc::launch_bin_scatter(p, s);
  mc::launch_deposit_x(p, s, 0);
  mc::launch_force_spread(p, s, 1, 0);
  mc::launch_lbm(p, s);
  mc::launch_interp_advance(p, s);
}

// One direct-forcing step in unfused stages, recorded: F = S[F_s], then the
// density fields (a re-run that leaves F), the MDF passes keeping their
// input velocities in record q, and afterwards the step's intermediates
// copied into record q and, when q + 1 < steps, the next step's start
// state into record q + 1 (populations of the next step's parity).
mc_status mdf_recorded_step(mc_world* w, char* seg, const StepSlot& ss, int q, int steps, int64_t tk,
                            cudaStream_t s) {
  const mc::WorldDev& h = w->h;
  mc::launch_mdf_bins(w->plan, s);
  mc::launch_bin_scan(w->plan, s);
  mc::launch_bin_scatter(w->plan, s);
  mc::launch_deposit_x(w->plan, s, 0);
  mc::launch_force_spread(w->plan, s, 0, 0);
  mc::launch_force_spread(w->plan, s, 1, 0);
  MC_ACUDA(mc::launch_mdf_recorded(w->plan, h, reinterpret_cast<float2*>(seg + (size_t)q * ss.bytes + ss.mu), s));
  mc::launch_lbm(w->plan, s);
  mc::launch_interp_advance(w->plan, s);
  const size_t total = std::max((size_t)9 * h.H * h.W, (size_t)h.N);
  const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
  char* next = q + 1 < steps ? seg + (size_t)(q + 1) * ss.bytes : nullptr;
  k_seg_save<<<grid, 256, 0, s>>>(w->plan.d_worlds, seg + (size_t)q * ss.bytes, next, (int)((tk + q + 1) & 1), ss);
  MC_ACUDA(cudaGetLastError());
  return MC_OK;
}

// X_bar of the final positions from the caller's gradient, and its largest
// |dt X_bar| (slot 0 of amax, zeroed before: the first reversed step's u_bar
// bound).
__global__ void k_interleave(const float* gx, const float* gy, float2* out, int n, float dt, unsigned* amax0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.0f;
  if (i < n) {
    out[i] = make_float2(gx[i], gy[i]);
    m = dt * fmaxf(fabsf(gx[i]), fabsf(gy[i]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(amax0, __float_as_uint(m));
}

}  // namespace

extern "C" {

mc_status mc_rollout_forward(mc_world* w, int n_steps, int ckpt_every, void* stream) {
  if (!w || n_steps < 1 || ckpt_every < 1) return afail(MC_ERR_INVALID_ARG, "need a world, n_steps >= 1, ckpt_every >= 1");
  if (w->t + n_steps >= (int64_t(1) << 24)) return afail(MC_ERR_INVALID_ARG, "step counter would reach 2^24");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const mc::WorldDev& h = w->h;
  const StateSlot sl = state_slot(h);
  const int n_ck = (n_steps + ckpt_every - 1) / ckpt_every;
  const TapeTail tl = tape_tail(h, n_ck, sl);
  const size_t need = tl.end;
  if (w->tape_bytes < need) {
    if (w->tape) cudaFreeAsync(w->tape, w->stream);
    w->tape = nullptr;
    w->tape_bytes = 0;
    cudaError_t e = cudaMallocAsync(&w->tape, need, s);
    if (e != cudaSuccess) return afail(MC_ERR_OOM, std::string("checkpoint allocation: ") + cudaGetErrorString(e));
    w->tape_bytes = need;
  }
  char* tape = static_cast<char*>(w->tape);
  w->tape_t0 = w->t;
  w->tape_steps = n_steps;
  w->tape_every = ckpt_every;
  w->tape_stored = false;
  // the start's displacement and observables (the checkpoints hold the rest), for mc_rollout_rewind
  if (h.N) MC_ACUDA(cudaMemcpyAsync(tape + tl.disp0, h.disp, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(tape + tl.obs0, h.obs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  int done = 0;
  for (int k = 0; k < n_ck; ++k) {
    mc_status st = save_state(h, (int)(w->t & 1), tape + (size_t)k * sl.bytes, sl, s);
    if (st != MC_OK) return st;
    const int steps = std::min(ckpt_every, n_steps - done);
    st = mc::plan_run(w->plan, steps, s);
    if (st != MC_OK) return st;
    w->t += steps;
    done += steps;
  }
  mc_status st = save_state(h, (int)(w->t & 1), tape + (size_t)n_ck * sl.bytes, sl, s);
  if (st != MC_OK) return st;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(tape + tl.disp_end, h.disp, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  return MC_OK;
}

mc_status mc_rollout_forward_stored(mc_world* w, int n_steps, void* stream) {
  if (!w || n_steps < 1) return afail(MC_ERR_INVALID_ARG, "need a world and n_steps >= 1");
  if (w->t + n_steps >= (int64_t(1) << 24)) return afail(MC_ERR_INVALID_ARG, "step counter would reach 2^24");
  const mc::WorldDev& h = w->h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t HW = (size_t)h.H * h.W;
  const StateSlot sl = state_slot(h);
  const StepSlot ss = step_slot(h);
  const StoredLayout L = stored_layout(h, n_steps);
  if (w->tape_bytes < L.end) {
    if (w->tape) cudaFreeAsync(w->tape, w->stream);
    w->tape = nullptr;
    w->tape_bytes = 0;
    cudaError_t e = cudaMallocAsync(&w->tape, L.end, s);
    if (e != cudaSuccess) return afail(MC_ERR_OOM, std::string("stored rollout allocation: ") + cudaGetErrorString(e));
    w->tape_bytes = L.end;
  }
  char* tape = static_cast<char*>(w->tape);
  char* seg = tape + L.steps;
  const int64_t t0 = w->t;
  w->tape_t0 = t0;
  w->tape_steps = n_steps;
  w->tape_every = n_steps;
  w->tape_stored = true;
  const TapeTail tl = tape_tail(h, 1, sl);
  if (h.N) MC_ACUDA(cudaMemcpyAsync(tape + tl.disp0, h.disp, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(tape + tl.obs0, h.obs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  mc_status st = save_state(h, (int)(t0 & 1), tape, sl, s);   // the start (mc_rollout_rewind)
  if (st != MC_OK) return st;
  if (h.ib == 1) {
    // direct forcing: the world's own buffers step, each step's record is
    // copied out after it (the same path as the sweep's recompute)
    st = save_state(h, (int)(t0 & 1), seg, sl, s);   // step 0's start state
    if (st != MC_OK) return st;
    for (int q = 0; q < n_steps; ++q) {
      st = mdf_recorded_step(w, seg, ss, q, n_steps, t0, s);
      if (st != MC_OK) return st;
    }
    w->t += n_steps;
    st = save_state(h, (int)(w->t & 1), tape + sl.bytes, sl, s);   // the final state
    if (st != MC_OK) return st;
    if (h.N) MC_ACUDA(cudaMemcpyAsync(tape + tl.disp_end, h.disp, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    return MC_OK;
  }
  // step 0 reads its populations from its record
  MC_ACUDA(cudaMemcpyAsync(seg + ss.st.g, h.g[t0 & 1], 9 * HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
  std::vector<mc::WorldDev> desc(n_steps);
  for (int q = 0; q < n_steps; ++q) desc[q] = bind_step(h, seg, ss, n_steps, q, (int)((t0 + q) & 1), false);
  mc::WorldDev* d_desc = reinterpret_cast<mc::WorldDev*>(tape + L.desc);
  MC_ACUDA(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(mc::WorldDev), cudaMemcpyHostToDevice, s));
  for (int q = 0; q < n_steps; ++q) {
    mc::Plan p = w->plan;
    p.d_worlds = d_desc + q;
    p.h_world0 = desc[q];
    run_recorded_step(p, s);
  }
  MC_ACUDA(cudaGetLastError());
  w->t += n_steps;
  // the world's own field buffers get the last step's fields
  char* last = seg + (size_t)(n_steps - 1) * ss.bytes;
  if (h.N) {
    MC_ACUDA(cudaMemcpyAsync(h.fel, last + ss.fel, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MC_ACUDA(cudaMemcpyAsync(h.fs, last + ss.fs, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (h.layers == 2) MC_ACUDA(cudaMemcpyAsync(h.nrm, last + ss.nrm, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  }
  MC_ACUDA(cudaMemcpyAsync(h.u, last + ss.u, HW * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(h.F, last + ss.F, HW * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(h.rho_b, last + ss.rho_b, HW * sizeof(float), cudaMemcpyDeviceToDevice, s));
  st = save_state(h, (int)(w->t & 1), tape + sl.bytes, sl, s);   // the final state
  if (st != MC_OK) return st;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(tape + tl.disp_end, h.disp, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  return MC_OK;   // (a copy from pageable memory returns once it has read the host descriptors)
}

mc_status mc_rollout_rewind(mc_world* w, void* stream) {
  if (!w) return afail(MC_ERR_INVALID_ARG, "world is NULL");
  if (!w->tape || w->tape_steps < 1) return afail(MC_ERR_INVALID_ARG, "no rollout recorded: call mc_rollout_forward first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const mc::WorldDev& h = w->h;
  const StateSlot sl = state_slot(h);
  const int n_ck = (w->tape_steps + w->tape_every - 1) / w->tape_every;
  const TapeTail tl = tape_tail(h, n_ck, sl);
  const char* tape = static_cast<const char*>(w->tape);
  mc_status st = load_state(h, (int)(w->tape_t0 & 1), tape, sl, s);
  if (st != MC_OK) return st;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(h.disp, tape + tl.disp0, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaMemcpyAsync(h.obs, tape + tl.obs0, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  mc::launch_set_counter(h, w->tape_t0, s);
  MC_ACUDA(cudaGetLastError());
  w->t = w->tape_t0;
  return MC_OK;
}

mc_status mc_world_set_rest(mc_world* w, const float* theta0, const float* L_rest, int mem_kind, void* stream) {
  if (!w) return afail(MC_ERR_INVALID_ARG, "world is NULL");
  if (mem_kind != MC_MEM_HOST && mem_kind != MC_MEM_DEVICE) return afail(MC_ERR_INVALID_ARG, "bad mem_kind");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const mc::WorldDev& h = w->h;
  const size_t J = h.J, E = h.E;
  const float* dth = theta0;
  const float* dL = L_rest;
  void* stage = nullptr;
  if (mem_kind == MC_MEM_HOST) {
    for (size_t j = 0; theta0 && j < J; ++j)
      if (!std::isfinite(theta0[j])) return afail(MC_ERR_INVALID_ARG, "non-finite theta0");
    for (size_t e = 0; L_rest && e < E; ++e)
      if (!(std::isfinite(L_rest[e]) && L_rest[e] > 0.0f)) return afail(MC_ERR_INVALID_ARG, "L_rest must be finite and > 0");
    const size_t bytes = ((theta0 ? J : 0) + (L_rest ? E : 0)) * sizeof(float);
    if (bytes) {
      MC_ACUDA(cudaMallocAsync(&stage, bytes, s));
      float* p = static_cast<float*>(stage);
      if (theta0 && J) MC_ACUDA(cudaMemcpyAsync(p, theta0, J * sizeof(float), cudaMemcpyHostToDevice, s));
      if (L_rest && E)
        MC_ACUDA(cudaMemcpyAsync(p + (theta0 ? J : 0), L_rest, E * sizeof(float), cudaMemcpyHostToDevice, s));
      dth = theta0 ? p : nullptr;
      dL = L_rest ? p + (theta0 ? J : 0) : nullptr;
    }
  }
  mc::launch_set_rest(h, dth, dL, s);
  const cudaError_t e = cudaGetLastError();
  if (stage) cudaFreeAsync(stage, s);
  if (mem_kind == MC_MEM_HOST) MC_ACUDA(cudaStreamSynchronize(s));   // the host arrays may go away
  MC_ACUDA(e);
  return MC_OK;
}

}  // extern "C"

namespace {


// The reverse sweep proper (no caller memory: captured into a graph):
// zero the adjoints, re-run each segment from its checkpoint keeping every
// step's state, reverse its steps, and return to the rollout's final state.
// With a second stream and two segment buffers (penalty worlds recorded
// with checkpoints), segment k - 1 is re-run on it into one buffer while
// segment k is reversed from the other: the two chains of small kernels
// overlap.  The re-run of segment k - 1 waits for the reverse of segment
// k + 1 (which read the same buffer); the reverse of a segment waits for its
// re-run.  The reversed steps read their step counter from AdjDev.t_step,
// not from the world, whose counter the concurrent re-run advances.
struct SweepSync {
  cudaStream_t s2 = nullptr;                       // the re-run stream (nullptr: one stream, one buffer)
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t rerun[2] = {nullptr, nullptr};       // a buffer's re-run done
  cudaEvent_t reversed[2] = {nullptr, nullptr};    // a buffer's reverse done
};

mc_status sweep(mc_world* w, mc::AdjDev a, const mc::AdjMdf* mdf, float* const adjG[2], char* obs_keep,
                char* const seg[2], const StateSlot& sl, int n_ck, const mc::WorldDev* bind_h, mc::WorldDev* bind_d,
                bool stored, const SweepSync& sy, cudaStream_t s) {
  const mc::WorldDev& h = w->h;
  const size_t HW = (size_t)h.H * h.W;
  const int K = w->tape_every, n = w->tape_steps;
  char* tape = static_cast<char*>(w->tape);
  const StepSlot ss = step_slot(h);
  const mc::WorldDev* wd = w->plan.d_worlds;
  const size_t total = std::max((size_t)9 * HW, (size_t)h.N);
  const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
  const bool overlap = sy.s2 != nullptr;
  cudaStream_t rs = overlap ? sy.s2 : s;
  // the recompute passes accumulate the observables again: keep the rollout's values
  MC_ACUDA(cudaMemcpyAsync(obs_keep, h.obs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  if (h.E) MC_ACUDA(cudaMemsetAsync(a.adjTh, 0, h.E * sizeof(float), s));
  if (h.J) MC_ACUDA(cudaMemsetAsync(a.gth0, 0, h.J * sizeof(float), s));
  if (h.E) MC_ACUDA(cudaMemsetAsync(a.gL, 0, h.E * sizeof(float), s));
  if (h.n_fil) MC_ACUDA(cudaMemsetAsync(a.gkf, 0, 3 * (size_t)h.n_fil * sizeof(float), s));
  MC_ACUDA(cudaMemsetAsync(adjG[0], 0, 9 * HW * sizeof(float), s));
  MC_ACUDA(cudaMemsetAsync(a.ubar, 0, 2 * HW * sizeof(unsigned long long), s));
  MC_ACUDA(cudaMemsetAsync(a.Q, 0, 2 * HW * sizeof(unsigned long long), s));
  // a step's plan with the step's descriptor (penalty coupling)
  auto step_plan = [&](int buf, int q, int par, bool reverse) {
    mc::Plan p = w->plan;
    const size_t i = bind_index(K, buf, q, par, reverse);
    p.d_worlds = bind_d + i;
    p.h_world0 = bind_h[i];
    return p;
  };
  if (mdf) {   // the pass accumulators (each reversed step leaves them cleared)
    MC_ACUDA(cudaMemsetAsync(mdf->ubf, 0, HW * sizeof(float2), s));
    MC_ACUDA(cudaMemsetAsync(mdf->rhob, 0, HW * sizeof(float), s));
    MC_ACUDA(cudaMemsetAsync(mdf->su, 0, 2 * HW * sizeof(unsigned long long), s));
    MC_ACUDA(cudaMemsetAsync(mdf->sr, 0, HW * sizeof(unsigned long long), s));
    MC_ACUDA(cudaMemsetAsync(mdf->ss, 0, 2 * HW * sizeof(unsigned long long), s));
    MC_ACUDA(cudaMemsetAsync(mdf->bnd, 0, 5 * sizeof(unsigned), s));
  }
  const int64_t t0 = w->tape_t0;
  auto buf_of = [&](int k) { return overlap ? (k & 1) : 0; };
  // segment k's forward, keeping every step's state and intermediates in
  // its buffer (the unfused stages: the same step bitwise, with rho_bar and
  // u in memory), on stream rs
  auto rerun = [&](int k) -> mc_status {
    const int steps = std::min(K, n - k * K);
    const int64_t tk = t0 + (int64_t)k * K;
    const int b = buf_of(k);
    mc_status st = load_state(h, (int)(tk & 1), tape + (size_t)k * sl.bytes, sl, rs);
    if (st != MC_OK) return st;
    mc::launch_set_counter(h, tk, rs);
    st = save_state(h, (int)(tk & 1), seg[b], sl, rs);   // the segment's first state
    if (st != MC_OK) return st;
    for (int q = 0; q < steps; ++q) {
      if (mdf) {
        st = mdf_recorded_step(w, seg[b], ss, q, steps, tk, rs);
        if (st != MC_OK) return st;
      } else {
        run_recorded_step(step_plan(b, q, (int)((tk + q) & 1), false), rs);   // fields straight into the record
      }
    }
    MC_ACUDA(cudaGetLastError());
    return MC_OK;
  };
  int cur = 0;   // adjG[cur] holds the adjoint of the populations after the step being reversed
  // segment k's steps reversed from its buffer, on stream s
  auto reverse = [&](int k) -> mc_status {
    const int steps = std::min(K, n - k * K);
    const int64_t tk = t0 + (int64_t)k * K;
    const int b = buf_of(k);
    for (int q = steps - 1; q >= 0; --q) {
      const int64_t tn = tk + q;
      const int par = (int)(tn & 1);
      const char* rec = seg[b] + (size_t)q * ss.bytes;
      a.adjG_next = adjG[cur];
      a.adjG_cur = adjG[cur ^ 1];
      a.theta_n = reinterpret_cast<const float*>(rec + ss.st.theta);
      a.nrm = reinterpret_cast<const float2*>(rec + ss.nrm);
      a.par = cur;   // reversed steps alternate the u_bar bound slots, the first reads slot 0
      if (mdf) {
        k_seg_restore<<<grid, 256, 0, s>>>(wd, rec, par, (long long)tn, ss, a);
        mc::AdjMdf m = *mdf;
        m.mu = reinterpret_cast<const float2*>(rec + ss.mu);
        m.rho = reinterpret_cast<const float*>(rec + ss.mrho);
        m.Us = reinterpret_cast<const float2*>(rec + ss.us);
        mc::launch_adj_step(w->plan, h, a, &m, par, s);
      } else {
        mc::AdjDev ab = a;
        ab.setup = 1;   // the step's counter and bound slots (fields are read from the record in place)
        ab.t_step = (long long)tn;
        mc::launch_adj_step(step_plan(b, q, par, true), h, ab, nullptr, par, s);
      }
      cur ^= 1;
    }
    MC_ACUDA(cudaGetLastError());
    return MC_OK;
  };
  if (!overlap) {
    for (int k = n_ck - 1; k >= 0; --k) {
      if (!stored) {
        mc_status st = rerun(k);
        if (st != MC_OK) return st;
      }
      mc_status st = reverse(k);
      if (st != MC_OK) return st;
    }
  } else {
    MC_ACUDA(cudaEventRecord(sy.fork, s));
    MC_ACUDA(cudaStreamWaitEvent(rs, sy.fork, 0));
    mc_status st = rerun(n_ck - 1);
    if (st != MC_OK) return st;
    MC_ACUDA(cudaEventRecord(sy.rerun[buf_of(n_ck - 1)], rs));
    for (int k = n_ck - 1; k >= 0; --k) {
      if (k >= 1) {
        // segment k - 1 goes into the buffer segment k + 1 was reversed from
        if (k + 1 <= n_ck - 1) MC_ACUDA(cudaStreamWaitEvent(rs, sy.reversed[buf_of(k + 1)], 0));
        st = rerun(k - 1);
        if (st != MC_OK) return st;
        MC_ACUDA(cudaEventRecord(sy.rerun[buf_of(k - 1)], rs));
      }
      MC_ACUDA(cudaStreamWaitEvent(s, sy.rerun[buf_of(k)], 0));
      st = reverse(k);
      if (st != MC_OK) return st;
      MC_ACUDA(cudaEventRecord(sy.reversed[buf_of(k)], s));
    }
    MC_ACUDA(cudaEventRecord(sy.join, rs));
    MC_ACUDA(cudaStreamWaitEvent(s, sy.join, 0));
  }
  mc::launch_adj_gk_reduce(a, h.n_fil, s);
  // back to the final state of the rollout
  const int64_t tf = t0 + n;
  const TapeTail tl = tape_tail(h, n_ck, sl);
  mc_status st = load_state(h, (int)(tf & 1), tape + (size_t)n_ck * sl.bytes, sl, s);
  if (st != MC_OK) return st;
  if (h.N) MC_ACUDA(cudaMemcpyAsync(h.disp, tape + tl.disp_end, h.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  mc::launch_set_counter(h, tf, s);
  MC_ACUDA(cudaMemcpyAsync(h.obs, obs_keep, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  MC_ACUDA(cudaGetLastError());
  return MC_OK;
}

mc_status backward(mc_world* w, const float* dL_dx, const float* dL_dy, float* dL_dtheta0, float* dL_dL_rest,
                   float* dL_dk, void* stream) {
  if (!w) return afail(MC_ERR_INVALID_ARG, "world is NULL");
  if (!w->tape || w->tape_steps < 1) return afail(MC_ERR_INVALID_ARG, "no rollout recorded: call mc_rollout_forward first");
  if (w->t != w->tape_t0 + w->tape_steps)
    return afail(MC_ERR_INVALID_ARG, "the world was stepped after mc_rollout_forward");
  const mc::WorldDev& h = w->h;
  if ((h.N && (!dL_dx || !dL_dy)) || (h.J && !dL_dtheta0)) return afail(MC_ERR_INVALID_ARG, "NULL gradient pointer");
  const int mb = (w->max_B + 3) & ~3;
  if (mc::adj_pbd_smem_per_filament(mb, h.n_pbd, h.pbd_order) > 220 * 1024)
    return afail(MC_ERR_INVALID_ARG, "filaments too long for the adjoint (reduce beads per filament or n_pbd)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t HW = (size_t)h.H * h.W;
  const StateSlot sl = state_slot(h);
  const int K = w->tape_every, n = w->tape_steps;
  const int n_ck = (n + K - 1) / K;
  // adjoint work memory: buffers + one segment of per-step states
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t o_adjX = take(h.N * sizeof(float2));
  const size_t o_adjTh = take(h.E * sizeof(float));
  const size_t o_gth0 = take(h.J * sizeof(float));
  const size_t o_gL = take(h.E * sizeof(float));
  const size_t o_gk = take(3 * sizeof(float));
  const size_t o_obs = take(3 * sizeof(unsigned long long));
  const size_t o_g0 = take(9 * HW * sizeof(float));
  const size_t o_g1 = take(9 * HW * sizeof(float));
  const size_t o_ub = take(2 * HW * sizeof(unsigned long long));
  const size_t o_Fb = take(HW * sizeof(float2));
  const size_t o_Q = take(2 * HW * sizeof(unsigned long long));
  const size_t o_amax = take(4 * sizeof(unsigned));
  const size_t o_gkf = take(3 * (size_t)h.n_fil * sizeof(float));
  const size_t o_rsb = take(HW * sizeof(float));
  const size_t o_fbt = take(h.N * sizeof(float2));
  const size_t o_dbar = take(h.N * sizeof(float2));
  const size_t o_nbar = take(h.N * sizeof(float2));
  const bool df = h.ib == 1;
  const size_t o_mGb = take(df ? HW * sizeof(float2) : 0);
  const size_t o_mub = take(df ? HW * sizeof(float2) : 0);
  const size_t o_mrb = take(df ? HW * sizeof(float) : 0);
  const size_t o_msu = take(df ? 2 * HW * sizeof(unsigned long long) : 0);
  const size_t o_msr = take(df ? HW * sizeof(unsigned long long) : 0);
  const size_t o_mss = take(df ? 2 * HW * sizeof(unsigned long long) : 0);
  const size_t o_musb = take(df ? h.N * sizeof(float2) : 0);
  const size_t o_miub = take(df ? h.N * sizeof(float2) : 0);
  const size_t o_mrbb = take(df ? h.N * sizeof(float) : 0);
  const size_t o_mxt = take(df ? h.N * sizeof(float4) : 0);
  const size_t o_mxtb = take(df ? h.N * sizeof(float2) : 0);
  const size_t o_must = take(df ? h.N * sizeof(float2) : 0);
  const size_t o_mbnd = take(df ? 8 * sizeof(unsigned) : 0);
  const bool stored = w->tape_stored;
  // penalty worlds recorded with checkpoints re-run a segment while the
  // next one is reversed: two segment buffers
  const bool overlap = !df && !stored;
  const int n_buf = overlap ? 2 : 1;
  const size_t o_bind = take(df ? 0 : 4 * (size_t)n_buf * K * sizeof(mc::WorldDev));
  const size_t o_seg = take(stored ? 0 : (size_t)n_buf * K * step_slot(h).bytes);
  if (w->adj_bytes < off) {
    if (w->adj) cudaFreeAsync(w->adj, w->stream);
    w->adj = nullptr;
    w->adj_bytes = 0;
    cudaError_t e = cudaMallocAsync(&w->adj, off, s);
    if (e != cudaSuccess) return afail(MC_ERR_OOM, std::string("adjoint allocation: ") + cudaGetErrorString(e));
    w->adj_bytes = off;
  }
  char* A = static_cast<char*>(w->adj);
  char* tape = static_cast<char*>(w->tape);
  char* seg[2] = {stored ? tape + stored_layout(h, n).steps : A + o_seg, nullptr};
  if (overlap) seg[1] = A + o_seg + (size_t)K * step_slot(h).bytes;
  mc::AdjDev a{};
  a.adjX = reinterpret_cast<float2*>(A + o_adjX);
  a.adjTh = reinterpret_cast<float*>(A + o_adjTh);
  a.gth0 = reinterpret_cast<float*>(A + o_gth0);
  a.gL = reinterpret_cast<float*>(A + o_gL);
  a.gk = reinterpret_cast<float*>(A + o_gk);
  float* adjG[2] = {reinterpret_cast<float*>(A + o_g0), reinterpret_cast<float*>(A + o_g1)};
  a.ubar = reinterpret_cast<unsigned long long*>(A + o_ub);
  a.Fbar = reinterpret_cast<float2*>(A + o_Fb);
  a.Q = reinterpret_cast<unsigned long long*>(A + o_Q);
  a.amax = reinterpret_cast<unsigned*>(A + o_amax);
  a.gkf = reinterpret_cast<float*>(A + o_gkf);
  a.rsb = reinterpret_cast<float*>(A + o_rsb);
  a.fbt = reinterpret_cast<float2*>(A + o_fbt);
  a.dbar = reinterpret_cast<float2*>(A + o_dbar);
  a.nbar = reinterpret_cast<float2*>(A + o_nbar);
  mc::AdjMdf m{};
  if (df) {
    m.m = h.mdf_iters;
    m.Gbar = reinterpret_cast<float2*>(A + o_mGb);
    m.ubf = reinterpret_cast<float2*>(A + o_mub);
    m.rhob = reinterpret_cast<float*>(A + o_mrb);
    m.su = reinterpret_cast<unsigned long long*>(A + o_msu);
    m.sr = reinterpret_cast<unsigned long long*>(A + o_msr);
    m.ss = reinterpret_cast<unsigned long long*>(A + o_mss);
    m.usb = reinterpret_cast<float2*>(A + o_musb);
    m.iub = reinterpret_cast<float2*>(A + o_miub);
    m.rbb = reinterpret_cast<float*>(A + o_mrbb);
    m.xt = reinterpret_cast<float4*>(A + o_mxt);
    m.xtb = reinterpret_cast<float2*>(A + o_mxtb);
    m.ust = reinterpret_cast<float2*>(A + o_must);
    m.bnd = reinterpret_cast<unsigned*>(A + o_mbnd);
  }

  // inputs (caller memory): outside the cached graph
  MC_ACUDA(cudaMemsetAsync(a.amax, 0, 4 * sizeof(unsigned), s));
  if (h.N) k_interleave<<<(h.N + 255) / 256, 256, 0, s>>>(dL_dx, dL_dy, a.adjX, h.N, h.dt, a.amax);
  MC_ACUDA(cudaGetLastError());
  // the reverse sweep, captured once per (rollout length, checkpoint spacing,
  // start step, buffers) and replayed
  const BwdKey key{n, K, w->tape_t0, w->tape, w->adj, stored};
  if (!w->bwd_exec || !(key == w->bwd_key)) {
    if (w->bwd_exec) cudaGraphExecDestroy(w->bwd_exec);
    w->bwd_exec = nullptr;
    mc::adj_setup(w->plan, h);
    // the per-step descriptors (penalty coupling), uploaded before the capture
    std::vector<mc::WorldDev> bind_h;
    mc::WorldDev* bind_d = reinterpret_cast<mc::WorldDev*>(A + o_bind);
    if (!df) {
      const StepSlot ssl = step_slot(h);
      bind_h.resize(4 * (size_t)n_buf * K);
      for (int b = 0; b < n_buf; ++b)
        for (int rv = 0; rv < 2; ++rv)
          for (int par = 0; par < 2; ++par)
            for (int q = 0; q < K; ++q)
              bind_h[bind_index(K, b, q, par, rv)] = bind_step(h, seg[b], ssl, K, q, par, rv);
      MC_ACUDA(cudaMemcpyAsync(bind_d, bind_h.data(), bind_h.size() * sizeof(mc::WorldDev), cudaMemcpyHostToDevice, s));
      MC_ACUDA(cudaStreamSynchronize(s));
    }
    cudaStream_t cs = adj_capture_stream();
    SweepSync sy;
    if (overlap) {
      sy.s2 = adj_rerun_stream();
      for (cudaEvent_t* e : {&sy.fork, &sy.join, &sy.rerun[0], &sy.rerun[1], &sy.reversed[0], &sy.reversed[1]})
        MC_ACUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    auto drop_events = [&]() {
      for (cudaEvent_t e : {sy.fork, sy.join, sy.rerun[0], sy.rerun[1], sy.reversed[0], sy.reversed[1]})
        if (e) cudaEventDestroy(e);
    };
    MC_ACUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const mc_status st =
        sweep(w, a, df ? &m : nullptr, adjG, A + o_obs, seg, sl, n_ck, bind_h.data(), bind_d, stored, sy, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    drop_events();
    if (st != MC_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    MC_ACUDA(ec);
    const cudaError_t ei = cudaGraphInstantiate(&w->bwd_exec, g, 0);
    cudaGraphDestroy(g);
    MC_ACUDA(ei);
    w->bwd_key = key;
  }
  MC_ACUDA(cudaGraphLaunch(w->bwd_exec, s));
  // outputs (caller memory)
  if (h.J) MC_ACUDA(cudaMemcpyAsync(dL_dtheta0, a.gth0, h.J * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (dL_dL_rest && h.E)
    MC_ACUDA(cudaMemcpyAsync(dL_dL_rest, a.gL, h.E * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (dL_dk) MC_ACUDA(cudaMemcpyAsync(dL_dk, a.gk, 3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return MC_OK;
}

}  // namespace

extern "C" {

mc_status mc_rollout_backward(mc_world* w, const float* dL_dx, const float* dL_dy, float* dL_dtheta0, void* stream) {
  return backward(w, dL_dx, dL_dy, dL_dtheta0, nullptr, nullptr, stream);
}

mc_status mc_rollout_backward_params(mc_world* w, const float* dL_dx, const float* dL_dy, float* dL_dtheta0,
                                     float* dL_dL_rest, float* dL_dk, void* stream) {
  return backward(w, dL_dx, dL_dy, dL_dtheta0, dL_dL_rest, dL_dk, stream);
}

mc_status mc_loss_polyline(mc_world* w, const float* poly_xy, int n_vertices, float* loss, float* dL_dx, float* dL_dy,
                           void* stream) {
  if (!w || !poly_xy || !loss || n_vertices < 2) return afail(MC_ERR_INVALID_ARG, "need a world, >= 2 vertices, outputs");
  const mc::WorldDev& h = w->h;
  if (h.N && (!dL_dx || !dL_dy)) return afail(MC_ERR_INVALID_ARG, "NULL gradient pointer");
  mc::launch_loss_polyline(w->plan, h, h.pos0, reinterpret_cast<const float2*>(poly_xy), n_vertices, loss, dL_dx,
                           dL_dy, static_cast<cudaStream_t>(stream));
  MC_ACUDA(cudaGetLastError());
  return MC_OK;
}

mc_status mc_loss_splat(mc_world* w, const float* target, int R, float sigma, float* loss, float* dL_dx, float* dL_dy,
                        void* stream) {
  if (!w || !target || !loss) return afail(MC_ERR_INVALID_ARG, "need a world, a target image and a loss output");
  if (R < 8 || R > 1024) return afail(MC_ERR_INVALID_ARG, "R must be in [8, 1024]");
  if (!(sigma > 0.0f && sigma <= 4.0f)) return afail(MC_ERR_INVALID_ARG, "sigma must be in (0, 4] pixels");
  const mc::WorldDev& h = w->h;
  if (h.N && (!dL_dx || !dL_dy)) return afail(MC_ERR_INVALID_ARG, "NULL gradient pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t RR = (size_t)R * R;
  void* scratch = nullptr;
  MC_ACUDA(cudaMallocAsync(&scratch, RR * (sizeof(unsigned long long) + sizeof(float)), s));
  auto* acc = static_cast<unsigned long long*>(scratch);
  auto* diff = reinterpret_cast<float*>(acc + RR);
  mc::launch_loss_splat(w->plan, h, target, R, sigma, acc, diff, loss, dL_dx, dL_dy, s);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, s);
  MC_ACUDA(e);
  return MC_OK;
}

}  // extern "C"
