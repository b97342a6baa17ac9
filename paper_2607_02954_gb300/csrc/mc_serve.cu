// Rollout server: continuous batching of independent world rollouts.
//
// Search loops (neuroevolution, MAP-Elites: the paper's Neuroevolution and
// QD Search experiments) submit rollout requests as they go and read back a
// fitness, the centre-of-mass displacement after n steps.  A scheduler
// thread owns one CUDA stream for the steps, one for world creation, and a
// set of active worlds ("slots"):
//   - pending requests are admitted as soon as a slot is free and their
//     device footprint fits the HBM budget;
//   - every tick advances all active worlds together through the batched
//     kernels (one launch per stage for the whole set);
//   - worlds whose rollout is complete are reduced to their mean
//     displacement (fixed-order block reduction) in the same tick, and
//     their result is published, and their memory released, once the
//     tick has finished on the device.
// The host runs at most two ticks ahead of the device: while tick n runs it
// publishes tick n - 1's rollouts, creates the admitted worlds (on the
// creation stream, which the step stream then waits on) and builds the
// plan of tick n + 1, so the device does not idle between ticks.
// Every kernel is deterministic and per world, so a rollout's result is
// bitwise the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mc_internal.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  int n_steps = 0;
  int H = 0, W = 0, n_fil = 0;
  std::vector<int> fil_off;
  std::vector<float> x, y, theta, L_rest, theta0, amp, freq, phase, f0;
  std::vector<float> len_amp, len_freq, len_phase, energy;   // optional (empty = absent)
  int observe = 0;
  int64_t t0 = 0;
  mc_params p{};
  size_t bytes = 0;
  int64_t t_submit = 0;
};

struct Slot {
  mc_world* w = nullptr;
  uint64_t ticket = 0;
  int steps_left = 0;
  int n_steps = 0;
  size_t bytes = 0;
  int64_t t_submit = 0, t_admit = 0;
  int64_t first_tick = 0;   // the first tick that steps the world
};

// The rollouts a tick finished: read back (into output buffer `buf`) by the
// tick itself, published once its event has completed.  Cancelled rollouts
// are released the same way, after the last tick that used their worlds,
// with no read-back.
struct Retire {
  std::vector<Slot> slots;
  int buf = 0;
  bool cancelled = false;
};

constexpr size_t kRec = 40;   // 3 floats (mean displacement, flags) + pad, 3 int64 observables

// Mean displacement of one world, fixed-order reduction (one block).
__global__ void __launch_bounds__(256) k_mean_disp(const float2* __restrict__ disp, int N,
                                                   const unsigned* __restrict__ flags, float* out) {
  __shared__ float sx[256], sy[256];
  float ax = 0.0f, ay = 0.0f;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 d = disp[i];
    ax += d.x;
    ay += d.y;
  }
  sx[threadIdx.x] = ax;
  sy[threadIdx.x] = ay;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sx[threadIdx.x] += sx[threadIdx.x + s];
      sy[threadIdx.x] += sy[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = N > 0 ? sx[0] / (float)N : 0.0f;
    out[1] = N > 0 ? sy[0] / (float)N : 0.0f;
    out[2] = __uint_as_float(*flags);
  }
}

mc_status serve_fail(mc_status s, const std::string& m) {
  mc::set_last_error(m.c_str());
  return s;
}

}  // namespace

struct mc_server {
  mc_server_cfg cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;       // the steps and the read-back
  cudaStream_t adm_stream = nullptr;   // world creation
  cudaEvent_t adm_ev = nullptr;
  cudaEvent_t tick_ev[2] = {nullptr, nullptr};   // end of the last two ticks, by tick parity
  std::thread thread;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, mc_result> done;
  std::unordered_map<uint64_t, int> in_flight;   // ticket -> 1 while pending or active
  std::unordered_set<uint64_t> cancel;           // running rollouts asked to stop
  uint64_t next_ticket = 1;
  bool stop = false;
  // scheduler-thread state
  std::vector<Slot> active;
  size_t bytes_in_use = 0;
  mc::Plan plan;
  bool plan_valid = false;
  // per finished world: kRec bytes (mean displacement, flags, observables),
  // one buffer per tick parity
  char* d_out[2] = {nullptr, nullptr};
  char* h_out[2] = {nullptr, nullptr};
  int out_cap[2] = {0, 0};
  std::deque<Retire> retiring;
  int64_t n_ticks = 0;   // ticks enqueued
  mc_server_stats stats{};
};

namespace {

size_t footprint(int H, int W, int n_fil, int N, bool ldrive, bool energy, int layers) {
  mc::WorldDev h{};
  mc::world_sizes(h, H, W, n_fil, N);
  h.has_ldrive = ldrive;
  h.has_energy = energy;
  h.layers = layers;
  // arena plus this world's share of a plan (work items and table entry)
  const size_t items = (size_t)n_fil + (N / mc::kBeadChunk + 1) + h.n_tiles + (size_t)H * W / mc::kCellChunk + 1 +
                       h.n_chunks;
  return mc::world_layout(h, nullptr) + items * sizeof(int2) + sizeof(mc::WorldDev) + 4096;
}

void publish(mc_server* s, uint64_t ticket, const mc_result& r) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->done[ticket] = r;
  s->in_flight.erase(ticket);
  s->stats.completed += 1;
  s->cv_done.notify_all();
}

// Publishes the rollouts of the oldest retiring tick once its event has
// completed (waiting for it when `block`), releasing their worlds.
// Returns false when it has nothing to publish yet.
bool retire_oldest(mc_server* s, bool block) {
  if (s->retiring.empty()) return false;
  Retire& r = s->retiring.front();
  cudaError_t e = block ? cudaEventSynchronize(s->tick_ev[r.buf]) : cudaEventQuery(s->tick_ev[r.buf]);
  if (e == cudaErrorNotReady) return false;
  const int64_t t = now_ns();
  const char* out = s->h_out[r.buf];
  for (size_t j = 0; j < r.slots.size(); ++j) {
    const Slot& sl = r.slots[j];
    mc_result res{};
    if (r.cancelled) {
      res.status = MC_ERR_CANCELLED;
      res.n_steps = sl.n_steps;
      res.t_submit_ns = sl.t_submit;
      res.t_admit_ns = sl.t_admit;
      res.t_done_ns = t;
      mc_world_destroy(sl.w);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->bytes_in_use -= sl.bytes;
      }
      publish(s, sl.ticket, res);
      continue;
    }
    float rec[3];
    std::memcpy(rec, out + kRec * j, sizeof(rec));
    res.com_disp[0] = rec[0];
    res.com_disp[1] = rec[1];
    unsigned flags;
    std::memcpy(&flags, &rec[2], 4);
    long long obs[3];
    std::memcpy(obs, out + kRec * j + 16, sizeof(obs));
    res.e_bend = (double)obs[0] / (double)mc::kObsScale;
    res.e_pos = (double)obs[1] / (double)mc::kObsScale;
    res.energy = (double)obs[2] / (double)mc::kObsScale;
    res.status = e != cudaSuccess ? MC_ERR_CUDA : ((flags & mc::kFlagUnstable) ? MC_ERR_UNSTABLE : MC_OK);
    res.n_steps = sl.n_steps;
    res.t_submit_ns = sl.t_submit;
    res.t_admit_ns = sl.t_admit;
    res.t_done_ns = t;
    // every use of the world on the step stream has completed
    mc_world_destroy(sl.w);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->bytes_in_use -= sl.bytes;
    }
    publish(s, sl.ticket, res);
  }
  s->retiring.pop_front();
  return true;
}

void scheduler(mc_server* s) {
  cudaSetDevice(s->device);
  bool set_changed = false;
  for (;;) {
    std::vector<Request> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || !s->pending.empty() || !s->active.empty() || !s->retiring.empty();
      });
      if (s->stop) break;
      size_t bytes = s->bytes_in_use;
      while (!s->pending.empty() && (int)(s->active.size() + admit.size()) < s->cfg.max_slots &&
             (bytes + s->pending.front().bytes <= s->cfg.hbm_budget_bytes ||
              (s->active.empty() && admit.empty() && s->retiring.empty()))) {
        bytes += s->pending.front().bytes;
        admit.push_back(std::move(s->pending.front()));
        s->pending.pop_front();
      }
      s->bytes_in_use = bytes;
    }
    bool created = false;
    for (Request& r : admit) {
      mc_world_desc d{};
      d.H = r.H;
      d.W = r.W;
      d.n_fil = r.n_fil;
      d.fil_off = r.fil_off.data();
      d.x = r.x.data();
      d.y = r.y.data();
      d.theta = r.theta.data();
      d.L_rest = r.L_rest.data();
      d.theta0 = r.theta0.data();
      d.drive_amp = r.amp.data();
      d.drive_freq = r.freq.data();
      d.drive_phase = r.phase.data();
      d.f0 = r.f0.empty() ? nullptr : r.f0.data();
      d.len_amp = r.len_amp.empty() ? nullptr : r.len_amp.data();
      d.len_freq = r.len_freq.empty() ? nullptr : r.len_freq.data();
      d.len_phase = r.len_phase.empty() ? nullptr : r.len_phase.data();
      d.energy = r.energy.empty() ? nullptr : r.energy.data();
      d.observe = r.observe;
      d.t0 = r.t0;
      d.p = r.p;
      d.mem_kind = MC_MEM_HOST;
      mc_world* w = nullptr;
      const mc_status st = mc_world_create(&d, s->adm_stream, &w);
      const int64_t t = now_ns();
      if (st != MC_OK) {
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->bytes_in_use -= r.bytes;
        }
        mc_result res{};
        res.status = st;
        res.n_steps = r.n_steps;
        res.t_submit_ns = r.t_submit;
        res.t_admit_ns = t;
        res.t_done_ns = t;
        publish(s, r.ticket, res);
        continue;
      }
      Slot sl;
      sl.w = w;
      sl.ticket = r.ticket;
      sl.steps_left = r.n_steps;
      sl.n_steps = r.n_steps;
      sl.bytes = r.bytes;
      sl.t_submit = r.t_submit;
      sl.t_admit = t;
      sl.first_tick = s->n_ticks;
      s->active.push_back(sl);
      set_changed = true;
      created = true;
    }
    if (created) {
      // the new worlds' set-up precedes their first step
      cudaEventRecord(s->adm_ev, s->adm_stream);
      cudaStreamWaitEvent(s->stream, s->adm_ev, 0);
    }
    // cancelled running rollouts leave the batch before this tick; their
    // worlds are released once the last tick that stepped them is done (at
    // once when none did)
    {
      std::vector<Slot> gone;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->cancel.empty()) {
          for (int i = 0; i < (int)s->active.size();) {
            if (s->cancel.erase(s->active[i].ticket)) {
              gone.push_back(s->active[i]);
              s->active.erase(s->active.begin() + i);
            } else {
              ++i;
            }
          }
          s->cancel.clear();   // tickets no longer running (finished meanwhile)
        }
      }
      if (!gone.empty()) {
        set_changed = true;
        Retire late;
        late.cancelled = true;
        late.buf = (int)((s->n_ticks - 1) & 1);
        for (auto& sl : gone) {
          if (sl.first_tick < s->n_ticks) {
            late.slots.push_back(sl);
            continue;
          }
          // never stepped: only its set-up on the creation stream used it
          cudaStreamSynchronize(s->adm_stream);
          mc_result res{};
          res.status = MC_ERR_CANCELLED;
          res.n_steps = sl.n_steps;
          res.t_submit_ns = sl.t_submit;
          res.t_admit_ns = sl.t_admit;
          res.t_done_ns = now_ns();
          mc_world_destroy(sl.w);
          {
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_in_use -= sl.bytes;
          }
          publish(s, sl.ticket, res);
        }
        // after every tick enqueued so far, on that last tick's event
        if (!late.slots.empty()) s->retiring.push_back(std::move(late));
      }
    }
    while (retire_oldest(s, false)) {
    }
    if (s->active.empty()) {
      // nothing left to enqueue: wait for the ticks still in flight
      while (retire_oldest(s, true)) {
      }
      continue;
    }
    if (set_changed) {
      if (s->plan_valid) mc::plan_free(s->plan, s->stream);
      std::vector<mc_world*> ws;
      for (auto& sl : s->active) ws.push_back(sl.w);
      s->plan_valid = mc::plan_build(ws.data(), (int)ws.size(), s->stream, s->plan) == MC_OK;
      set_changed = false;
      if (!s->plan_valid) {
        // cannot advance this set: fail every active rollout
        cudaStreamSynchronize(s->stream);
        for (auto& sl : s->active) {
          mc_result res{};
          res.status = MC_ERR_OOM;
          res.n_steps = sl.n_steps;
          res.t_submit_ns = sl.t_submit;
          res.t_admit_ns = sl.t_admit;
          res.t_done_ns = now_ns();
          mc_world_destroy(sl.w);
          {
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_in_use -= sl.bytes;
          }
          publish(s, sl.ticket, res);
        }
        s->active.clear();
        continue;
      }
    }
    // the host stays at most two ticks ahead: this tick reuses the event and
    // the output buffer of the tick before the last
    const int b = (int)(s->n_ticks & 1);
    while (!s->retiring.empty() && s->retiring.front().buf == b) retire_oldest(s, true);
    if (s->n_ticks >= 2) cudaEventSynchronize(s->tick_ev[b]);
    int k = s->cfg.steps_per_tick;
    for (auto& sl : s->active) k = std::min(k, sl.steps_left);
    mc::plan_run(s->plan, k, s->stream);
    for (auto& sl : s->active) {
      sl.steps_left -= k;
      sl.w->t += k;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stats.steps_run += k;
      s->stats.ticks += 1;
    }
    // finished rollouts: reduce and read back in this tick
    Retire r;
    r.buf = b;
    for (int i = 0; i < (int)s->active.size();) {
      if (s->active[i].steps_left <= 0) {
        r.slots.push_back(s->active[i]);
        s->active.erase(s->active.begin() + i);
      } else {
        ++i;
      }
    }
    if (!r.slots.empty()) {
      const int nf = (int)r.slots.size();
      if (nf > s->out_cap[b]) {
        // the buffer's last read-back (two ticks ago) has completed
        if (s->d_out[b]) cudaFreeAsync(s->d_out[b], s->stream);
        if (s->h_out[b]) cudaFreeHost(s->h_out[b]);
        s->out_cap[b] = std::max(nf, 2 * s->out_cap[b]);
        cudaMallocAsync(&s->d_out[b], kRec * s->out_cap[b], s->stream);
        cudaMallocHost(&s->h_out[b], kRec * s->out_cap[b]);
      }
      for (int j = 0; j < nf; ++j) {
        const mc::WorldDev& h = r.slots[j].w->h;
        char* o = s->d_out[b] + kRec * j;
        k_mean_disp<<<1, 256, 0, s->stream>>>(h.disp, h.N, h.flags, reinterpret_cast<float*>(o));
        cudaMemcpyAsync(o + 16, h.obs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s->stream);
      }
      cudaMemcpyAsync(s->h_out[b], s->d_out[b], kRec * nf, cudaMemcpyDeviceToHost, s->stream);
      set_changed = true;
    }
    cudaEventRecord(s->tick_ev[b], s->stream);
    s->n_ticks += 1;
    if (!r.slots.empty()) s->retiring.push_back(std::move(r));
  }
  // shutting down: publish what finished, release everything still held
  while (retire_oldest(s, true)) {
  }
  for (auto& sl : s->active) mc_world_destroy(sl.w);
  s->active.clear();
  if (s->plan_valid) mc::plan_free(s->plan, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaStreamSynchronize(s->adm_stream);
}

void release_handles(mc_server* s) {
  for (cudaEvent_t ev : {s->adm_ev, s->tick_ev[0], s->tick_ev[1]})
    if (ev) cudaEventDestroy(ev);
  if (s->adm_stream) cudaStreamDestroy(s->adm_stream);
  if (s->stream) cudaStreamDestroy(s->stream);
}

template <class T>
mc_status copy_in(const T* src, size_t n, int kind, std::vector<T>& out, const char* name) {
  out.resize(n);
  if (n == 0) return MC_OK;
  if (!src) return serve_fail(MC_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (kind == MC_MEM_HOST) {
    std::memcpy(out.data(), src, n * sizeof(T));
  } else {
    const cudaError_t e = cudaMemcpy(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return serve_fail(MC_ERR_CUDA, std::string("copying ") + name + ": " + cudaGetErrorString(e));
  }
  return MC_OK;
}

}  // namespace

extern "C" {

mc_status mc_server_create(const mc_server_cfg* cfg, mc_server** out) {
  if (!cfg || !out) return serve_fail(MC_ERR_INVALID_ARG, "cfg or out is NULL");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->steps_per_tick < 1 || cfg->max_pending < 1 || cfg->hbm_budget_bytes == 0)
    return serve_fail(MC_ERR_INVALID_ARG, "max_slots, steps_per_tick, max_pending and hbm_budget_bytes must be positive");
  mc_server* s = new mc_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->adm_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->adm_ev, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&s->tick_ev[b], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release_handles(s);
    delete s;
    return serve_fail(MC_ERR_CUDA, std::string("server stream: ") + cudaGetErrorString(e));
  }
  s->thread = std::thread(scheduler, s);
  *out = s;
  return MC_OK;
}

mc_status mc_serve_submit(mc_server* s, const mc_world_desc* d, int n_steps, uint64_t* ticket) {
  if (!s || !d || !ticket) return serve_fail(MC_ERR_INVALID_ARG, "NULL argument");
  if (n_steps < 1) return serve_fail(MC_ERR_INVALID_ARG, "n_steps must be >= 1");
  if (d->n_fil < 0 || (d->n_fil > 0 && !d->fil_off)) return serve_fail(MC_ERR_INVALID_ARG, "bad filament table");
  if (d->H < 8 || d->W < 8 || d->H % 8 || d->W % 8 || d->H > 8192 || d->W > 8192)
    return serve_fail(MC_ERR_INVALID_ARG, "H and W must be multiples of 8 in [8, 8192]");
  if (d->mem_kind != MC_MEM_HOST && d->mem_kind != MC_MEM_DEVICE) return serve_fail(MC_ERR_INVALID_ARG, "bad mem_kind");
  Request r;
  r.n_steps = n_steps;
  r.H = d->H;
  r.W = d->W;
  r.n_fil = d->n_fil;
  r.fil_off.assign(d->fil_off, d->fil_off + (d->n_fil > 0 ? d->n_fil + 1 : 0));
  if (r.fil_off.empty()) r.fil_off.push_back(0);
  for (int f = 0; f < d->n_fil; ++f)
    if (r.fil_off[f + 1] - r.fil_off[f] < 2 || r.fil_off[0] != 0)
      return serve_fail(MC_ERR_INVALID_ARG, "every filament needs at least 2 beads and fil_off[0] = 0");
  const int N = r.fil_off.back();
  const int E = N - d->n_fil, J = N - 2 * d->n_fil;
  mc_status st;
  if ((st = copy_in(d->x, N, d->mem_kind, r.x, "x")) || (st = copy_in(d->y, N, d->mem_kind, r.y, "y")) ||
      (st = copy_in(d->theta, E, d->mem_kind, r.theta, "theta")) ||
      (st = copy_in(d->L_rest, E, d->mem_kind, r.L_rest, "L_rest")) ||
      (st = copy_in(d->theta0, J, d->mem_kind, r.theta0, "theta0")) ||
      (st = copy_in(d->drive_amp, J, d->mem_kind, r.amp, "drive_amp")) ||
      (st = copy_in(d->drive_freq, J, d->mem_kind, r.freq, "drive_freq")) ||
      (st = copy_in(d->drive_phase, J, d->mem_kind, r.phase, "drive_phase")))
    return st;
  if (d->f0 && (st = copy_in(d->f0, (size_t)9 * d->H * d->W, d->mem_kind, r.f0, "f0"))) return st;
  if (d->len_amp && (st = copy_in(d->len_amp, E, d->mem_kind, r.len_amp, "len_amp"))) return st;
  if (d->len_freq && (st = copy_in(d->len_freq, E, d->mem_kind, r.len_freq, "len_freq"))) return st;
  if (d->len_phase && (st = copy_in(d->len_phase, E, d->mem_kind, r.len_phase, "len_phase"))) return st;
  if (d->energy && (st = copy_in(d->energy, (size_t)d->H * d->W, d->mem_kind, r.energy, "energy"))) return st;
  r.observe = d->observe;
  r.t0 = d->t0;
  r.p = d->p;
  r.bytes = footprint(d->H, d->W, d->n_fil, N, d->len_amp != nullptr, d->energy != nullptr, d->p.layers);
  r.t_submit = now_ns();
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->pending.size() >= s->cfg.max_pending) return serve_fail(MC_ERR_BUSY, "request queue is full");
  r.ticket = s->next_ticket++;
  *ticket = r.ticket;
  s->in_flight[r.ticket] = 1;
  s->pending.push_back(std::move(r));
  s->stats.submitted += 1;
  s->cv_work.notify_one();
  return MC_OK;
}

mc_status mc_serve_poll(mc_server* s, uint64_t ticket, mc_result* out) {
  if (!s || !out) return serve_fail(MC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *out = it->second;
    s->done.erase(it);
    return MC_OK;
  }
  if (s->in_flight.count(ticket)) return MC_ERR_BUSY;
  return serve_fail(MC_ERR_NOT_FOUND, "unknown or already collected ticket");
}

mc_status mc_serve_wait(mc_server* s, uint64_t ticket, int timeout_ms, mc_result* out) {
  if (!s || !out) return serve_fail(MC_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
  for (;;) {
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
      *out = it->second;
      s->done.erase(it);
      return MC_OK;
    }
    if (!s->in_flight.count(ticket)) return serve_fail(MC_ERR_NOT_FOUND, "unknown or already collected ticket");
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->done.count(ticket))
      return serve_fail(MC_ERR_TIMEOUT, "rollout not finished within the timeout");
  }
}

mc_status mc_server_stats_get(mc_server* s, mc_server_stats* out) {
  if (!s || !out) return serve_fail(MC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->pending = (int64_t)s->pending.size();
  return MC_OK;
}

mc_status mc_serve_cancel(mc_server* s, uint64_t ticket) {
  if (!s) return serve_fail(MC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->in_flight.count(ticket)) return serve_fail(MC_ERR_NOT_FOUND, "ticket is not queued or running");
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    if (it->ticket != ticket) continue;
    mc_result res{};
    res.status = MC_ERR_CANCELLED;
    res.n_steps = it->n_steps;
    res.t_submit_ns = it->t_submit;
    res.t_admit_ns = res.t_done_ns = now_ns();
    s->pending.erase(it);
    s->done[ticket] = res;
    s->in_flight.erase(ticket);
    s->stats.completed += 1;
    s->cv_done.notify_all();
    return MC_OK;
  }
  // admitted: the scheduler takes it out of the batch at its next tick
  s->cancel.insert(ticket);
  s->cv_work.notify_one();
  return MC_OK;
}

mc_status mc_server_destroy(mc_server* s) {
  if (!s) return MC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->thread.joinable()) s->thread.join();
  for (int b = 0; b < 2; ++b) {
    if (s->d_out[b]) cudaFreeAsync(s->d_out[b], s->stream);
    if (s->h_out[b]) cudaFreeHost(s->h_out[b]);
  }
  cudaStreamSynchronize(s->stream);
  release_handles(s);
  delete s;
  return MC_OK;
}

}  // extern "C"
