// C ABI of libmc: world life cycle, plans (world tables + work items), step
// replay through CUDA graphs, and state read-out.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mc_internal.cuh"

using mc::Plan;
using mc::WorldDev;


namespace {

thread_local std::string g_last_error;

mc_status fail(mc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

mc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(MC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MC_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

// Fake of the world allocation for tests of the out-of-memory path: when
// armed with n, the nth world allocation from then on reports
// cudaErrorMemoryAllocation without calling the allocator.
std::atomic<int> g_fail_world_alloc{0};

cudaError_t world_alloc(void** p, size_t bytes, cudaStream_t s) {
  int k = g_fail_world_alloc.load();
  while (k > 0 && !g_fail_world_alloc.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 1) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, s);
}

// Bump allocator inside one arena.
struct Layout {
  size_t off = 0;
  template <class T>
  size_t take(size_t n) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += n * sizeof(T);
    return at;
  }
};

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// Whether ok(a[i]) holds for every i < n; arrays of more than 2^20 values
// are split over up to 8 host threads.
template <class F>
bool all_of(const float* a, size_t n, F ok) {
  const size_t kChunk = size_t(1) << 20;
  const int nt = n <= kChunk ? 1 : (int)std::min<size_t>(8, (n + kChunk - 1) / kChunk);
  auto run = [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i)
      if (!ok(a[i])) return false;
    return true;
  };
  if (nt == 1) return run(0, n);
  std::vector<char> res(nt, 1);
  std::vector<std::thread> th;
  for (int k = 0; k < nt; ++k) th.emplace_back([&, k] { res[k] = run(n * k / nt, n * (k + 1) / nt); });
  for (auto& t : th) t.join();
  return std::all_of(res.begin(), res.end(), [](char r) { return r != 0; });
}

bool finite_all(const float* a, size_t n) {
  return all_of(a, n, [](float v) { return std::isfinite(v); });
}

mc_status validate_params(const mc_params& p) {
  const float v[] = {p.nu, p.dt, p.Lambda, p.kappa, p.k_bend, p.k_stretch, p.k_shear, p.k_rep, p.sigma, p.orient};
  for (float x : v)
    if (!std::isfinite(x)) return fail(MC_ERR_INVALID_ARG, "non-finite constant in mc_params");
  if (!(p.nu > 0.0f)) return fail(MC_ERR_INVALID_ARG, "nu must be > 0 (tau+ > 1/2)");
  if (!(p.Lambda > 0.0f)) return fail(MC_ERR_INVALID_ARG, "Lambda must be > 0");
  if (!(p.dt > 0.0f)) return fail(MC_ERR_INVALID_ARG, "dt must be > 0");
  if (!(p.sigma > 0.0f && p.sigma <= 2.0f)) return fail(MC_ERR_INVALID_ARG, "sigma must be in (0, 2]");
  if (p.n_pbd < 0 || p.n_pbd > mc::kMaxNpbd) return fail(MC_ERR_INVALID_ARG, "n_pbd must be in [0, 64]");
  if (p.pbd_order != 0 && p.pbd_order != 1) return fail(MC_ERR_INVALID_ARG, "pbd_order must be 0 or 1");
  if (p.layers != 1 && p.layers != 2) return fail(MC_ERR_INVALID_ARG, "layers must be 1 or 2");
  if (p.layers == 2 && !(p.layer_half > 0.0f && p.layer_half <= 2.0f))
    return fail(MC_ERR_INVALID_ARG, "layer_half must be in (0, 2] cells");
  if (p.ib != 0 && p.ib != 1) return fail(MC_ERR_INVALID_ARG, "ib must be 0 or 1");
  if (p.ib == 1 && p.layers != 1) return fail(MC_ERR_INVALID_ARG, "direct forcing (ib = 1) needs layers = 1");
  if (p.mdf_iters < 0 || p.mdf_iters > 64) return fail(MC_ERR_INVALID_ARG, "mdf_iters must be in [0, 64]");
  return MC_OK;
}

void fill_constants(WorldDev& h, const mc_params& p) {
  const double tau_p = 3.0 * (double)p.nu + 0.5;
  const double tau_m = 0.5 + (double)p.Lambda / (tau_p - 0.5);
  h.dt = p.dt;
  h.kappa_dt = (float)((double)p.kappa / (double)p.dt);
  h.k_bend = p.k_bend;
  h.k_st = p.k_stretch;
  h.k_sh = p.k_shear;
  h.k_rep = p.k_rep;
  h.orient = p.orient;
  h.n_pbd = p.n_pbd;
  h.pbd_order = p.pbd_order;
  h.layers = p.layers;
  h.layer_half = p.layer_half;
  h.ib = p.ib;
  h.mdf_iters = p.ib == 1 ? p.mdf_iters : 0;
  h.om_p = (float)(1.0 / tau_p);
  h.om_m = (float)(1.0 / tau_m);
  h.src_p = (float)(1.0 - 0.5 / tau_p);
  h.src_m = (float)(1.0 - 0.5 / tau_m);
  h.u_max = 0.5f;
  const int R = (int)std::ceil(4.0 * (double)p.sigma);
  h.R = R;
  double sum = 0.0;
  double g[2 * mc::kMaxR + 1];
  for (int m = -R; m <= R; ++m) {
    g[m + R] = std::exp(-(double)(m * m) / (2.0 * (double)p.sigma * (double)p.sigma));
    sum += g[m + R];
  }
  for (int k = 0; k < 2 * mc::kMaxR + 1; ++k) h.taps[k] = k <= 2 * R ? (float)(g[k] / sum) : 0.0f;
}

void free_plan(Plan& p, cudaStream_t s) {
  if (p.graph) cudaGraphExecDestroy(p.graph);
  if (p.d_mem) cudaFreeAsync(p.d_mem, s);
  p = Plan{};
}

mc_status build_plan(mc_world* const* ws, int n, cudaStream_t s, Plan& out) {
  Plan p;
  p.n_worlds = n;
  mc::kernel_setup();
  p.max_R = 1;
  p.any_layered = false;
  p.any_mdf = false;
  p.max_mdf = 0;
  p.any_ext = false;
  p.one_chunk = true;
  std::vector<int2> fil, bead, tile, cell, scan;
  std::vector<WorldDev> table(n);
  for (int k = 0; k < n; ++k) {
    const mc_world* w = ws[k];
    table[k] = w->h;
    p.max_B = std::max(p.max_B, w->max_B);
    p.max_R = std::max(p.max_R, w->h.R);
    p.any_layered = p.any_layered || w->h.layers == 2;
    p.any_mdf = p.any_mdf || w->h.ib == 1;
    p.max_mdf = std::max(p.max_mdf, w->h.mdf_iters);
    p.any_ext = p.any_ext || w->h.layers == 2 || w->h.observe || w->h.has_ldrive || w->h.ib == 1;
    p.one_chunk = p.one_chunk && w->h.n_chunks <= 1;
    for (int f = 0; f < w->h.n_fil; ++f) fil.push_back(make_int2(k, f));
    const int nb = std::max(w->h.N, 1);
    for (int b = 0; b < nb; b += mc::kBeadChunk) bead.push_back(make_int2(k, b));
    for (int ty = 0; ty < w->h.nty; ++ty)   // tile items carry (tx, ty) packed: tx | ty << 16
      for (int tx = 0; tx < w->h.ntx; ++tx) tile.push_back(make_int2(k, tx | (ty << 16)));
    for (int c = 0; c < w->h.n_chunks; ++c) scan.push_back(make_int2(k, c));
    const int HW = w->h.H * w->h.W;
    for (int c = 0; c < HW; c += mc::kCellChunk) cell.push_back(make_int2(k, c));
  }
  Layout L;
  const size_t o_w = L.take<WorldDev>(n);
  const size_t o_f = L.take<int2>(fil.size());
  const size_t o_b = L.take<int2>(bead.size());
  const size_t o_t = L.take<int2>(tile.size());
  const size_t o_c = L.take<int2>(cell.size());
  const size_t o_s = L.take<int2>(scan.size());
  const size_t o_bar = L.take<unsigned>(4);
  std::vector<char> host(L.off);
  std::memcpy(host.data() + o_w, table.data(), n * sizeof(WorldDev));
  if (!fil.empty()) std::memcpy(host.data() + o_f, fil.data(), fil.size() * sizeof(int2));
  std::memcpy(host.data() + o_b, bead.data(), bead.size() * sizeof(int2));
  if (!tile.empty()) std::memcpy(host.data() + o_t, tile.data(), tile.size() * sizeof(int2));
  std::memcpy(host.data() + o_c, cell.data(), cell.size() * sizeof(int2));
  std::memcpy(host.data() + o_s, scan.data(), scan.size() * sizeof(int2));
  cudaError_t e = cudaMallocAsync(&p.d_mem, L.off, s);
  if (e != cudaSuccess) return fail(MC_ERR_OOM, std::string("plan allocation: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(p.d_mem, host.data(), L.off, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  p.d_worlds = at<WorldDev>(p.d_mem, o_w);
  p.d_fil_items = at<int2>(p.d_mem, o_f);
  p.d_bead_items = at<int2>(p.d_mem, o_b);
  p.d_tile_items = at<int2>(p.d_mem, o_t);
  p.d_cell_items = at<int2>(p.d_mem, o_c);
  p.d_scan_items = at<int2>(p.d_mem, o_s);
  p.d_persist_bar = at<unsigned>(p.d_mem, o_bar);
  p.n_fil_items = (int)fil.size();
  p.n_bead_items = (int)bead.size();
  p.n_tile_items = (int)tile.size();
  p.n_cell_items = (int)cell.size();
  p.n_scan_items = (int)scan.size();
  if (n == 1) p.h_world0 = table[0];
  out = p;
  return MC_OK;
}

constexpr int kGraphSteps = 16;

cudaStream_t capture_stream() {
  thread_local cudaStream_t cs = nullptr;
  if (!cs) cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  return cs;
}

mc_status run_steps(Plan& p, int n, cudaStream_t s) {
  if (p.cfg.persistent && mc::persistent_supported(p)) {
    // one cooperative launch for the whole run
    if (n > 0) MC_CUDA(mc::launch_persistent(p, n, s));
    MC_CUDA(cudaGetLastError());
    return MC_OK;
  }
  if (n >= kGraphSteps) {
    if (!p.graph) {
      cudaStream_t cs = capture_stream();
      MC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      mc::enqueue_steps(p, kGraphSteps, cs);
      cudaGraph_t g = nullptr;
      MC_CUDA(cudaStreamEndCapture(cs, &g));
      cudaError_t e = cudaGraphInstantiate(&p.graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      p.graph_steps = kGraphSteps;
    }
    while (n >= p.graph_steps) {
      MC_CUDA(cudaGraphLaunch(p.graph, s));
      n -= p.graph_steps;
    }
  }
  if (n > 0) mc::enqueue_steps(p, n, s);
  MC_CUDA(cudaGetLastError());
  return MC_OK;
}

// Batched plans are cached by the exact list of world handles.
std::mutex g_plan_mu;
std::map<std::vector<mc_world*>, Plan>& plan_cache() {
  static std::map<std::vector<mc_world*>, Plan> m;
  return m;
}

void drop_plans_with(mc_world* w) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto& m = plan_cache();
  for (auto it = m.begin(); it != m.end();) {
    bool has = false;
    for (auto* x : it->first) has |= (x == w);
    if (has) {
      free_plan(it->second, w->stream);
      it = m.erase(it);
    } else {
      ++it;
    }
  }
}


// The plan of a world (n == 1) or the cached plan of a batch of distinct
// worlds (built on first use).
mc_status find_plan(mc_world* const* ws, int n, cudaStream_t s, Plan** out) {
  if (!ws || n < 1) return fail(MC_ERR_INVALID_ARG, "no worlds");
  for (int k = 0; k < n; ++k) {
    if (!ws[k]) return fail(MC_ERR_INVALID_ARG, "NULL world in batch");
    for (int j = 0; j < k; ++j)
      if (ws[j] == ws[k]) return fail(MC_ERR_INVALID_ARG, "a world appears twice in the batch");
  }
  if (n == 1) {
    *out = &ws[0]->plan;
    return MC_OK;
  }
  std::vector<mc_world*> key(ws, ws + n);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto& m = plan_cache();
  auto it = m.find(key);
  if (it == m.end()) {
    Plan p;
    mc_status st = build_plan(ws, n, s, p);
    if (st != MC_OK) return st;
    it = m.emplace(key, p).first;
  }
  *out = &it->second;
  return MC_OK;
}

}  // namespace

namespace mc {

// Sizes of a world's arrays from its grid and bead counts.
void world_sizes(WorldDev& h, int H, int W, int n_fil, int N) {
  h.H = H;
  h.W = W;
  h.N = N;
  h.n_fil = n_fil;
  h.E = N - n_fil;
  h.J = N - 2 * n_fil;
  h.nbx = W / kBin;
  h.nby = H / kBin;
  h.n_bins = h.nbx * h.nby;
  h.ntx = (W + kTile - 1) / kTile;
  h.nty = (H + kTile - 1) / kTile;
  h.n_tiles = h.ntx * h.nty;
  h.n_chunks = (h.n_bins + kScanChunk - 1) / kScanChunk;
}

// Places every array of a world inside one arena (256-byte aligned slices).
// With A == nullptr only returns the arena size in bytes.
size_t world_layout(WorldDev& h, void* A) {
  Layout L;
  const int N = h.N, E = h.E, J = h.J;
  const size_t HW = (size_t)h.H * h.W;
  const size_t o_fo = L.take<int>(h.n_fil + 1);
  const size_t o_pos = L.take<float4>(N);
  const size_t o_disp = L.take<float2>(N);
  const size_t o_pos0 = L.take<float2>(N);
  const size_t o_th = L.take<float>(E);
  const size_t o_L = L.take<float>(E);
  const size_t o_dr = L.take<float4>(J);
  const size_t o_fel = L.take<float2>(N);
  const size_t o_fs = L.take<float2>(N);
  const size_t o_ub = L.take<float2>(N);
  const size_t o_bb = L.take<int>(N);
  const size_t o_bc = L.take<int>(h.n_bins);
  const size_t o_bo = L.take<int>(h.n_bins + 1);
  const size_t o_bcur = L.take<int>(h.n_bins);
  const size_t o_cs = L.take<int>(h.n_chunks);
  const size_t o_sp = L.take<float4>(N);
  const size_t o_sr = L.take<float4>(N);
  const size_t o_g0 = L.take<float>(9 * HW);
  const size_t o_g1 = L.take<float>(9 * HW);
  const size_t o_F = L.take<float2>(HW);
  const size_t o_u = L.take<float2>(HW);
  const size_t o_rs = L.take<float>(HW);
  const size_t o_rx = L.take<float>(HW);
  const size_t o_rb = L.take<float>(HW);
  const size_t o_trm = L.take<float>(h.n_tiles);
  const size_t o_t = L.take<long long>(1);
  const size_t o_fl = L.take<unsigned>(1);
  const size_t o_fm = L.take<unsigned>(2);
  const size_t o_ld = L.take<float4>(h.has_ldrive ? E : 0);
  const size_t o_en = L.take<float>(h.has_energy ? HW : 0);
  const size_t o_eb = L.take<float>(h.has_energy ? N : 0);
  const size_t o_ob = L.take<unsigned long long>(3);
  const size_t o_nr = L.take<float2>(h.layers == 2 ? N : 0);
  const size_t o_fa = L.take<unsigned long long>(h.layers == 2 ? 2 * HW : 0);
  const bool df = h.ib == 1;
  const size_t o_mr = L.take<float>(df ? HW : 0);
  const size_t o_bs = L.take<int>(df ? N : 0);
  const size_t o_u2 = L.take<float2>(df ? HW : 0);
  const size_t o_su = L.take<float2>(df ? N : 0);
  if (!A) return L.off;
  h.fil_off = at<int>(A, o_fo);
  h.pos = at<float4>(A, o_pos);
  h.disp = at<float2>(A, o_disp);
  h.pos0 = at<float2>(A, o_pos0);
  h.theta = at<float>(A, o_th);
  h.L_rest = at<float>(A, o_L);
  h.drive = at<float4>(A, o_dr);
  h.fel = at<float2>(A, o_fel);
  h.fs = at<float2>(A, o_fs);
  h.ubead = at<float2>(A, o_ub);
  h.bead_bin = at<int>(A, o_bb);
  h.bin_count = at<int>(A, o_bc);
  h.bin_off = at<int>(A, o_bo);
  h.bin_cursor = at<int>(A, o_bcur);
  h.chunk_sum = at<int>(A, o_cs);
  h.spos = at<float4>(A, o_sp);
  h.srec = at<float4>(A, o_sr);
  h.g[0] = at<float>(A, o_g0);
  h.g[1] = at<float>(A, o_g1);
  h.F = at<float2>(A, o_F);
  h.u = at<float2>(A, o_u);
  h.rho_s = at<float>(A, o_rs);
  h.rho_x = at<float>(A, o_rx);
  h.rho_b = at<float>(A, o_rb);
  h.tile_rho_max = at<float>(A, o_trm);
  h.t = at<long long>(A, o_t);
  h.flags = at<unsigned>(A, o_fl);
  h.fel_max = at<unsigned>(A, o_fm);
  h.ldrive = h.has_ldrive ? at<float4>(A, o_ld) : nullptr;
  h.energy = h.has_energy ? at<float>(A, o_en) : nullptr;
  h.ebead = h.has_energy ? at<float>(A, o_eb) : nullptr;
  h.obs = at<unsigned long long>(A, o_ob);
  h.nrm = h.layers == 2 ? at<float2>(A, o_nr) : nullptr;
  h.facc = h.layers == 2 ? at<unsigned long long>(A, o_fa) : nullptr;
  h.mrho = df ? at<float>(A, o_mr) : nullptr;
  h.bead_slot = df ? at<int>(A, o_bs) : nullptr;
  h.u2 = df ? at<float2>(A, o_u2) : nullptr;
  h.sus = df ? at<float2>(A, o_su) : nullptr;
  return L.off;
}

// Plan and step helpers shared with the rollout server.
mc_status plan_build(mc_world* const* ws, int n, cudaStream_t s, Plan& out) { return build_plan(ws, n, s, out); }
void plan_set_cfg(Plan& p, const LaunchCfg& c) {
  if (c.persistent == p.cfg.persistent && c.pbd_warps == p.cfg.pbd_warps && c.scan_kernels == p.cfg.scan_kernels &&
      c.force_ws == p.cfg.force_ws)
    return;
  p.cfg = c;
  if (p.graph) {
    cudaGraphExecDestroy(p.graph);
    p.graph = nullptr;
  }
}

mc_world* world_clone(const mc_world* w, cudaStream_t s) {
  mc_world* c = new mc_world();
  c->h = w->h;
  c->bytes = w->bytes;
  c->stream = s;
  c->t = w->t;
  c->max_B = w->max_B;
  c->fil_off = w->fil_off;
  c->params = w->params;
  if (cudaMallocAsync(&c->arena, c->bytes, s) != cudaSuccess) {
    (void)cudaGetLastError();
    delete c;
    return nullptr;
  }
  if (cudaMemcpyAsync(c->arena, w->arena, c->bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaFreeAsync(c->arena, s);
    delete c;
    return nullptr;
  }
  world_layout(c->h, c->arena);
  return c;   // no plan of its own: a copy is only stepped within the plan it is made for
}
mc_status plan_run(Plan& p, int n_steps, cudaStream_t s) { return run_steps(p, n_steps, s); }
void plan_free(Plan& p, cudaStream_t s) { free_plan(p, s); }

}  // namespace mc

extern "C" {

const char* mc_last_error(void) { return g_last_error.c_str(); }

mc_status mc_inject_world_alloc_failure(int nth) {
  if (nth < 0) return fail(MC_ERR_INVALID_ARG, "nth must be >= 0");
  g_fail_world_alloc.store(nth);
  return MC_OK;
}
int mc_abi_version(void) { return MC_ABI_VERSION; }

mc_status mc_params_default(mc_params* p) {
  if (!p) return fail(MC_ERR_INVALID_ARG, "p is NULL");
  p->nu = 0.1f;
  p->dt = 1.0f;
  p->Lambda = 0.25f;
  p->kappa = 0.05f;
  p->k_bend = 0.5f;
  p->k_stretch = 0.5f;
  p->k_shear = 0.25f;
  p->k_rep = 0.5f;
  p->sigma = 1.0f;
  p->orient = 1.0f;
  p->n_pbd = 4;
  p->pbd_order = 0;
  p->layers = 1;
  p->layer_half = 0.5f;
  p->ib = 0;
  p->mdf_iters = 0;
  return MC_OK;
}

mc_status mc_world_create(const mc_world_desc* d, void* stream, mc_world** out) {
  if (!d || !out) return fail(MC_ERR_INVALID_ARG, "desc or out is NULL");
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int H = d->H, W = d->W;
  if (H < 8 || W < 8 || H % 8 || W % 8 || H > 8192 || W > 8192)
    return fail(MC_ERR_INVALID_ARG, "H and W must be multiples of 8 in [8, 8192]");
  if (d->n_fil < 0) return fail(MC_ERR_INVALID_ARG, "n_fil < 0");
  if (d->mem_kind != MC_MEM_HOST && d->mem_kind != MC_MEM_DEVICE) return fail(MC_ERR_INVALID_ARG, "bad mem_kind");
  if (d->t0 < 0 || d->t0 >= (int64_t(1) << 24)) return fail(MC_ERR_INVALID_ARG, "t0 must be in [0, 2^24)");
  mc_status st = validate_params(d->p);
  if (st != MC_OK) return st;
  if (d->n_fil > 0 && !d->fil_off) return fail(MC_ERR_INVALID_ARG, "fil_off is NULL");
  std::vector<int> fo(d->n_fil + 1, 0);
  int max_B = 2;
  for (int f = 0; f <= d->n_fil; ++f) fo[f] = d->n_fil > 0 ? d->fil_off[f] : 0;
  if (fo[0] != 0) return fail(MC_ERR_INVALID_ARG, "fil_off[0] must be 0");
  for (int f = 0; f < d->n_fil; ++f) {
    const int B = fo[f + 1] - fo[f];
    if (B < 2) return fail(MC_ERR_INVALID_ARG, "every filament needs at least 2 beads");
    max_B = std::max(max_B, B);
  }
  if (max_B > 3072) return fail(MC_ERR_INVALID_ARG, "filaments are limited to 3072 beads");
  const int N = fo[d->n_fil];
  const int E = N - d->n_fil, J = N - 2 * d->n_fil;
  const size_t HW = (size_t)H * W;

  // Inputs: host pointers for validation (the caller's arrays, or host
  // copies of device arrays) and, later, device pointers for the set-up
  // kernel (the caller's device arrays, or a staging buffer the host arrays
  // are uploaded to).
  const bool on_host = d->mem_kind == MC_MEM_HOST;
  std::vector<std::vector<float>> keep;
  auto view = [&](const float* p, size_t n, const char* name, const float*& hv) -> mc_status {
    hv = nullptr;
    if (n == 0) return MC_OK;
    if (!p) return fail(MC_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (on_host) {
      hv = p;
      return MC_OK;
    }
    keep.emplace_back(n);
    MC_CUDA(cudaMemcpy(keep.back().data(), p, n * sizeof(float), cudaMemcpyDeviceToHost));
    hv = keep.back().data();
    return MC_OK;
  };
  auto finite = [](const float* a, size_t n) { return !a || finite_all(a, n); };
  const float *hx, *hy, *hth, *hL, *ht0, *hamp, *hfrq, *hphs;
  const float *hf0 = nullptr, *hla = nullptr, *hlf = nullptr, *hlp = nullptr, *hen = nullptr;
  if ((st = view(d->x, N, "x", hx)) || (st = view(d->y, N, "y", hy)) || (st = view(d->theta, E, "theta", hth)) ||
      (st = view(d->L_rest, E, "L_rest", hL)) || (st = view(d->theta0, J, "theta0", ht0)) ||
      (st = view(d->drive_amp, J, "drive_amp", hamp)) || (st = view(d->drive_freq, J, "drive_freq", hfrq)) ||
      (st = view(d->drive_phase, J, "drive_phase", hphs)))
    return st;
  if (d->f0 && (st = view(d->f0, 9 * HW, "f0", hf0))) return st;
  const int n_len = (d->len_amp != nullptr) + (d->len_freq != nullptr) + (d->len_phase != nullptr);
  if (n_len != 0 && n_len != 3) return fail(MC_ERR_INVALID_ARG, "len_amp, len_freq, len_phase: all three or none");
  if (n_len == 3 && ((st = view(d->len_amp, E, "len_amp", hla)) || (st = view(d->len_freq, E, "len_freq", hlf)) ||
                     (st = view(d->len_phase, E, "len_phase", hlp))))
    return st;
  if (d->energy && (st = view(d->energy, HW, "energy", hen))) return st;
  if (!finite(hla, E) || !finite(hlf, E) || !finite(hlp, E) || !finite(hen, HW))
    return fail(MC_ERR_INVALID_ARG, "non-finite input value");
  if (hla && !all_of(hla, E, [](float v) { return std::fabs(v) < 1.0f; }))
    return fail(MC_ERR_INVALID_ARG, "|len_amp| must be < 1 (rest lengths stay > 0)");
  if (d->observe != 0 && d->observe != 1) return fail(MC_ERR_INVALID_ARG, "observe must be 0 or 1");
  if (!finite(hx, N) || !finite(hy, N) || !finite(hth, E) || !finite(hL, E) || !finite(ht0, J) ||
      !finite(hamp, J) || !finite(hfrq, J) || !finite(hphs, J) || !finite(hf0, 9 * HW))
    return fail(MC_ERR_INVALID_ARG, "non-finite input value");
  if (hL && !all_of(hL, E, [](float v) { return v > 0.0f; })) return fail(MC_ERR_INVALID_ARG, "L_rest must be > 0");

  mc_world* w = new mc_world();
  w->stream = s;
  w->t = d->t0;
  w->max_B = max_B;
  w->fil_off = fo;
  w->params = d->p;
  WorldDev& h = w->h;
  mc::world_sizes(h, H, W, d->n_fil, N);
  fill_constants(h, d->p);
  h.has_ldrive = n_len == 3;
  h.has_energy = d->energy != nullptr;
  h.observe = d->observe;

  w->bytes = mc::world_layout(h, nullptr);
  cudaError_t e = world_alloc(&w->arena, w->bytes, s);
  if (e != cudaSuccess) {
    delete w;
    return fail(MC_ERR_OOM, std::string("world allocation: ") + cudaGetErrorString(e));
  }
  void* A = w->arena;
  mc::world_layout(h, A);

  auto fail_free = [&](mc_status s2) {
    cudaFreeAsync(w->arena, s);
    delete w;
    return s2;
  };
#define MC_CUDA_W(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return fail_free(cuda_fail(e_, #call));       \
  } while (0)
  MC_CUDA_W(cudaMemsetAsync(A, 0, w->bytes, s));
  const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  auto up = [&](void* dst, const void* src, size_t n, cudaMemcpyKind k) {
    return n ? cudaMemcpyAsync(dst, src, n, k, s) : cudaSuccess;
  };
  MC_CUDA_W(up((void*)h.fil_off, fo.data(), fo.size() * sizeof(int), cudaMemcpyHostToDevice));
  MC_CUDA_W(up(h.theta, d->theta, E * sizeof(float), kind));
  MC_CUDA_W(up((void*)h.L_rest, d->L_rest, E * sizeof(float), kind));
  if (h.has_energy) MC_CUDA_W(up((void*)h.energy, d->energy, HW * sizeof(float), kind));
  // raw per-bead, per-joint and per-edge inputs on the device for the set-up
  // kernel (positions wrapped and split into cell + fraction, drive records)
  const float* raw[9] = {d->x, d->y, d->theta0, d->drive_amp, d->drive_freq, d->drive_phase,
                         n_len == 3 ? d->len_amp : nullptr, n_len == 3 ? d->len_freq : nullptr,
                         n_len == 3 ? d->len_phase : nullptr};
  const size_t cnt[9] = {(size_t)N, (size_t)N, (size_t)J, (size_t)J, (size_t)J, (size_t)J,
                         (size_t)E, (size_t)E, (size_t)E};
  float* staging = nullptr;
  if (on_host) {
    size_t tot = 0;
    for (int k = 0; k < 9; ++k) tot += raw[k] ? cnt[k] : 0;
    if (tot) MC_CUDA_W(cudaMallocAsync((void**)&staging, tot * sizeof(float), s));
    size_t off = 0;
    for (int k = 0; k < 9; ++k) {
      if (!raw[k] || !cnt[k]) continue;
      const cudaError_t e2 = up(staging + off, raw[k], cnt[k] * sizeof(float), cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) {
        cudaFreeAsync(staging, s);
        return fail_free(cuda_fail(e2, "input upload"));
      }
      raw[k] = staging + off;
      off += cnt[k];
    }
  }
  mc::launch_world_init(h, raw, s);
  if (staging) cudaFreeAsync(staging, s);
  MC_CUDA_W(cudaGetLastError());
  const long long t0 = d->t0;
  MC_CUDA_W(up(h.t, &t0, sizeof(long long), cudaMemcpyHostToDevice));
  if (d->f0) {
    // stage f0 in the buffer the first step writes, then store its
    // post-collision image in the buffer the first step reads
    float* stage = h.g[(t0 + 1) & 1];
    MC_CUDA_W(up(stage, d->f0, 9 * HW * sizeof(float), kind));
    mc::launch_unstream_in(stage, h.g[t0 & 1], H, W, s);
    MC_CUDA_W(cudaGetLastError());
  }
  // copies from page-locked host memory are still in flight: finish them
  // before returning, so the caller may free or reuse its arrays at once
  if (on_host) {
    bool pinned = false;
    const float* srcs[] = {d->x, d->y, d->theta, d->L_rest, d->theta0, d->drive_amp, d->drive_freq,
                           d->drive_phase, d->len_amp, d->len_freq, d->len_phase, d->energy, d->f0};
    for (const float* p : srcs) {
      if (!p) continue;
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) pinned = true;
      (void)cudaGetLastError();
    }
    if (pinned) MC_CUDA_W(cudaStreamSynchronize(s));
  }
  mc_world* self = w;
  st = build_plan(&self, 1, s, w->plan);
  if (st != MC_OK) return fail_free(st);
#undef MC_CUDA_W
  *out = w;
  return MC_OK;
}

// ---- checkpoint / resume --------------------------------------------------
// Image of a world: a header, the filament offsets, then the device arena
// byte for byte (it holds no pointers: the arrays are placed again from the
// sizes on load).
namespace {
struct SaveHeader {
  char magic[8];          // "MCWORLD1"
  int abi;                // MC_ABI_VERSION of the writer
  int H, W, n_fil, N;
  int has_ldrive, has_energy, observe;
  int max_B;
  long long t;            // step counter (host view; the device one is in the arena)
  unsigned long long arena_bytes;
  mc_params params;
};
constexpr char kSaveMagic[8] = {'M', 'C', 'W', 'O', 'R', 'L', 'D', '1'};

size_t save_size(const mc_world* w) {
  return sizeof(SaveHeader) + (size_t)(w->h.n_fil + 1) * sizeof(int) + w->bytes;
}
}  // namespace

mc_status mc_world_save_size(const mc_world* w, size_t* bytes) {
  if (!w || !bytes) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  *bytes = save_size(w);
  return MC_OK;
}

mc_status mc_world_save(const mc_world* w, void* buf, size_t bytes, void* stream) {
  if (!w || !buf) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  if (bytes < save_size(w)) return fail(MC_ERR_INVALID_ARG, "buffer smaller than mc_world_save_size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SaveHeader hd{};
  std::memcpy(hd.magic, kSaveMagic, 8);
  hd.abi = MC_ABI_VERSION;
  hd.H = w->h.H;
  hd.W = w->h.W;
  hd.n_fil = w->h.n_fil;
  hd.N = w->h.N;
  hd.has_ldrive = w->h.has_ldrive;
  hd.has_energy = w->h.has_energy;
  hd.observe = w->h.observe;
  hd.max_B = w->max_B;
  hd.t = w->t;
  hd.arena_bytes = w->bytes;
  hd.params = w->params;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  std::memcpy(out + sizeof(hd), w->fil_off.data(), (size_t)(w->h.n_fil + 1) * sizeof(int));
  MC_CUDA(cudaMemcpyAsync(out + sizeof(hd) + (size_t)(w->h.n_fil + 1) * sizeof(int), w->arena, w->bytes,
                          cudaMemcpyDeviceToHost, s));
  MC_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

mc_status mc_world_load(const void* buf, size_t bytes, void* stream, mc_world** out) {
  if (!buf || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  SaveHeader hd{};
  if (bytes < sizeof(hd)) return fail(MC_ERR_INVALID_ARG, "buffer too small for a world image");
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kSaveMagic, 8) != 0) return fail(MC_ERR_INVALID_ARG, "not a world image");
  if (hd.abi != MC_ABI_VERSION) return fail(MC_ERR_INVALID_ARG, "world image written by another C ABI version");
  if (hd.H < 8 || hd.W < 8 || hd.H % 8 || hd.W % 8 || hd.H > 8192 || hd.W > 8192 || hd.n_fil < 0 || hd.N < 0 ||
      hd.t < 0 || hd.t >= (int64_t(1) << 24) || hd.max_B < 2 || hd.max_B > 3072)
    return fail(MC_ERR_INVALID_ARG, "corrupt world image header");
  mc_status st = validate_params(hd.params);
  if (st != MC_OK) return st;
  const size_t fo_bytes = (size_t)(hd.n_fil + 1) * sizeof(int);
  if (bytes < sizeof(hd) + fo_bytes) return fail(MC_ERR_INVALID_ARG, "world image truncated");
  std::vector<int> fo(hd.n_fil + 1);
  std::memcpy(fo.data(), static_cast<const char*>(buf) + sizeof(hd), fo_bytes);
  if (fo[0] != 0 || fo[hd.n_fil] != hd.N) return fail(MC_ERR_INVALID_ARG, "corrupt filament table in world image");
  for (int f = 0; f < hd.n_fil; ++f)
    if (fo[f + 1] - fo[f] < 2 || fo[f + 1] - fo[f] > hd.max_B)
      return fail(MC_ERR_INVALID_ARG, "corrupt filament table in world image");
  mc_world* w = new mc_world();
  w->stream = static_cast<cudaStream_t>(stream);
  w->t = hd.t;
  w->max_B = hd.max_B;
  w->fil_off = fo;
  w->params = hd.params;
  WorldDev& h = w->h;
  mc::world_sizes(h, hd.H, hd.W, hd.n_fil, hd.N);
  fill_constants(h, hd.params);
  h.has_ldrive = hd.has_ldrive;
  h.has_energy = hd.has_energy;
  h.observe = hd.observe;
  w->bytes = mc::world_layout(h, nullptr);
  if (w->bytes != hd.arena_bytes || bytes < sizeof(hd) + fo_bytes + w->bytes) {
    delete w;
    return fail(MC_ERR_INVALID_ARG, "world image size does not match its header");
  }
  cudaError_t e = world_alloc(&w->arena, w->bytes, w->stream);
  if (e != cudaSuccess) {
    delete w;
    return fail(MC_ERR_OOM, std::string("world allocation: ") + cudaGetErrorString(e));
  }
  mc::world_layout(h, w->arena);
  e = cudaMemcpyAsync(w->arena, static_cast<const char*>(buf) + sizeof(hd) + fo_bytes, w->bytes,
                      cudaMemcpyHostToDevice, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);   // the caller may reuse the buffer at once
  if (e != cudaSuccess) {
    cudaFreeAsync(w->arena, w->stream);
    delete w;
    return cuda_fail(e, "world image upload");
  }
  mc_world* self = w;
  st = build_plan(&self, 1, w->stream, w->plan);
  if (st != MC_OK) {
    cudaFreeAsync(w->arena, w->stream);
    delete w;
    return st;
  }
  *out = w;
  return MC_OK;
}

mc_status mc_world_destroy(mc_world* w) {
  if (!w) return MC_OK;
  drop_plans_with(w);
  free_plan(w->plan, w->stream);
  if (w->bwd_exec) cudaGraphExecDestroy(w->bwd_exec);
  if (w->tape) cudaFreeAsync(w->tape, w->stream);
  if (w->adj) cudaFreeAsync(w->adj, w->stream);
  cudaFreeAsync(w->arena, w->stream);
  delete w;
  return MC_OK;
}

mc_status mc_world_info_get(const mc_world* w, mc_world_info* out) {
  if (!w || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  out->H = w->h.H;
  out->W = w->h.W;
  out->n_fil = w->h.n_fil;
  out->N = w->h.N;
  out->E = w->h.E;
  out->J = w->h.J;
  out->bin_edge = mc::kBin;
  out->n_bins = w->h.n_bins;
  out->t = w->t;
  out->device_bytes = w->bytes;
  return MC_OK;
}

mc_status mc_step(mc_world* w, int n_steps, void* stream) {
  if (!w || n_steps < 0) return fail(MC_ERR_INVALID_ARG, "bad world or n_steps");
  if (w->t + n_steps >= (int64_t(1) << 24)) return fail(MC_ERR_INVALID_ARG, "step counter would reach 2^24");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!w->plan.tuned && n_steps >= kGraphSteps) {
    mc_world* self = w;
    mc_status st = mc::plan_tune(&self, 1, w->plan, s, true);
    if (st != MC_OK) return st;
  }
  mc_status st = run_steps(w->plan, n_steps, s);
  if (st == MC_OK) w->t += n_steps;
  return st;
}

mc_status mc_step_batched(mc_world* const* ws, int n, int n_steps, void* stream) {
  if (!ws || n < 0 || n_steps < 0) return fail(MC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0 || n_steps == 0) return MC_OK;
  for (int k = 0; k < n; ++k)
    if (ws[k] && ws[k]->t + n_steps >= (int64_t(1) << 24))
      return fail(MC_ERR_INVALID_ARG, "step counter would reach 2^24");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan* plan = nullptr;   // a batch of one runs the world's own plan
  mc_status st = find_plan(ws, n, s, &plan);
  if (st != MC_OK) return st;
  if (!plan->tuned && n_steps >= kGraphSteps) {
    st = mc::plan_tune(ws, n, *plan, s, true);
    if (st != MC_OK) return st;
  }
  st = run_steps(*plan, n_steps, s);
  if (st == MC_OK)
    for (int k = 0; k < n; ++k) ws[k]->t += n_steps;
  return st;
}

mc_status mc_launch_config_get(mc_world* const* ws, int n, mc_launch_config* out) {
  if (!out) return fail(MC_ERR_INVALID_ARG, "out is NULL");
  Plan* p = nullptr;
  mc_status st = find_plan(ws, n, nullptr, &p);
  if (st != MC_OK) return st;
  out->persistent = p->cfg.persistent;
  out->pbd_warps = p->cfg.pbd_warps;
  out->scan_kernels = p->cfg.scan_kernels;
  out->force_kernel = p->cfg.force_ws;
  return MC_OK;
}

mc_status mc_launch_config_set(mc_world* const* ws, int n, const mc_launch_config* cfg) {
  if (!cfg) return fail(MC_ERR_INVALID_ARG, "cfg is NULL");
  if (cfg->persistent != 0 && cfg->persistent != 3 && cfg->persistent != 4)
    return fail(MC_ERR_INVALID_ARG, "persistent must be 0, 3 or 4");
  if (cfg->pbd_warps != 8 && cfg->pbd_warps != 4 && cfg->pbd_warps != 2)
    return fail(MC_ERR_INVALID_ARG, "pbd_warps must be 8, 4 or 2");
  if (cfg->scan_kernels != 0 && cfg->scan_kernels != 2) return fail(MC_ERR_INVALID_ARG, "scan_kernels must be 0 or 2");
  if (cfg->force_kernel != 0 && cfg->force_kernel != 1) return fail(MC_ERR_INVALID_ARG, "force_kernel must be 0 or 1");
  Plan* p = nullptr;
  mc_status st = find_plan(ws, n, nullptr, &p);
  if (st != MC_OK) return st;
  mc::LaunchCfg c;
  c.persistent = cfg->persistent;
  c.pbd_warps = cfg->pbd_warps;
  c.scan_kernels = cfg->scan_kernels;
  c.force_ws = cfg->force_kernel;
  if (c.persistent && !mc::persistent_supported(*p))
    return fail(MC_ERR_INVALID_ARG, "the persistent step does not support this plan (direct forcing, two layers, "
                                    "filaments over 64 beads or a filter half width other than 4)");
  mc::plan_set_cfg(*p, c);
  p->tuned = true;
  return MC_OK;
}

mc_status mc_autotune(mc_world* const* ws, int n, void* stream, mc_launch_config* chosen) {
  Plan* p = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mc_status st = find_plan(ws, n, s, &p);
  if (st != MC_OK) return st;
  st = mc::plan_tune(ws, n, *p, s, false);
  if (st != MC_OK) return st;
  if (chosen) return mc_launch_config_get(ws, n, chosen);
  return MC_OK;
}

mc_status mc_debug_barrier_test(unsigned extra_arrivals, int64_t timeout_ns) {
  if (extra_arrivals > 1 || timeout_ns < 1000 || timeout_ns > 10000000000LL)
    return fail(MC_ERR_INVALID_ARG, "extra_arrivals must be 0 or 1 and timeout_ns in [1e3, 1e10]");
  mc::persistent_test_settings(extra_arrivals, (unsigned long long)timeout_ns);
  return MC_OK;
}

mc_status mc_step_stage(mc_world* w, int stage, void* stream) {
  if (!w || stage < 0 || stage >= MC_N_STAGES) return fail(MC_ERR_INVALID_ARG, "bad world or stage");
  if (w->h.ib == 1) return fail(MC_ERR_INVALID_ARG, "per-stage steps are defined for the penalty coupling (ib = 0)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Plan& p = w->plan;
  switch (stage) {
    case 0: mc::launch_pbd(p, s); break;
    case 1: mc::launch_bin_scan(p, s); break;
    case 2: mc::launch_bin_scatter(p, s); break;
    case 3: mc::launch_deposit_x(p, s, 0); break;
    case 4: mc::launch_force_spread(p, s, 0); break;
    case 5: mc::launch_lbm(p, s); break;
    case 7: mc::launch_force_lbm(p, s); break;
    default:
      mc::launch_interp_advance(p, s);
      w->t += 1;
      break;
  }
  MC_CUDA(cudaGetLastError());
  return MC_OK;
}

mc_status mc_world_get_state(const mc_world* w, float* x, float* y, float* theta, float* disp, float* fdev,
                             int mem_kind, void* stream) {
  if (!w) return fail(MC_ERR_INVALID_ARG, "world is NULL");
  if (mem_kind != MC_MEM_HOST && mem_kind != MC_MEM_DEVICE) return fail(MC_ERR_INVALID_ARG, "bad mem_kind");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const WorldDev& h = w->h;
  const size_t HW = (size_t)h.H * h.W;
  const bool host = mem_kind == MC_MEM_HOST;
  // device scratch for outputs that need a kernel when the target is host memory
  float *dx = nullptr, *dy = nullptr, *df = nullptr;
  const size_t need = (host && (x || y) ? 2 * (size_t)h.N : 0) + (host && fdev ? 9 * HW : 0);
  void* scratch = nullptr;
  if (need) MC_CUDA(cudaMallocAsync(&scratch, need * sizeof(float), s));
  float* sp = static_cast<float*>(scratch);
  if (x || y) {
    dx = host ? sp : x;
    dy = host ? sp + h.N : y;
    mc::launch_positions_out(h, x ? dx : nullptr, y ? dy : nullptr, s);
    if (host) {
      if (x && h.N) MC_CUDA(cudaMemcpyAsync(x, dx, h.N * sizeof(float), cudaMemcpyDeviceToHost, s));
      if (y && h.N) MC_CUDA(cudaMemcpyAsync(y, dy, h.N * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (host) sp += 2 * (size_t)h.N;
  }
  const cudaMemcpyKind dk = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (theta && h.E) MC_CUDA(cudaMemcpyAsync(theta, h.theta, h.E * sizeof(float), dk, s));
  if (disp && h.N) MC_CUDA(cudaMemcpyAsync(disp, h.disp, h.N * sizeof(float2), dk, s));
  if (fdev) {
    df = host ? sp : fdev;
    mc::launch_stream_out(h.g[w->t & 1], df, h.H, h.W, s);
    if (host) MC_CUDA(cudaMemcpyAsync(fdev, df, 9 * HW * sizeof(float), cudaMemcpyDeviceToHost, s));
  }
  MC_CUDA(cudaGetLastError());
  if (scratch) MC_CUDA(cudaFreeAsync(scratch, s));
  if (host) MC_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

mc_status mc_world_get_field(const mc_world* w, int field, void* out, int mem_kind, void* stream) {
  if (!w || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  if (mem_kind != MC_MEM_HOST && mem_kind != MC_MEM_DEVICE) return fail(MC_ERR_INVALID_ARG, "bad mem_kind");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const WorldDev& h = w->h;
  const size_t HW = (size_t)h.H * h.W;
  const bool host = mem_kind == MC_MEM_HOST;
  const cudaMemcpyKind dk = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (field) {
    case MC_FIELD_FEL: src = h.fel; bytes = h.N * sizeof(float2); break;
    case MC_FIELD_FS: src = h.fs; bytes = h.N * sizeof(float2); break;
    case MC_FIELD_UBEAD: src = h.ubead; bytes = h.N * sizeof(float2); break;
    case MC_FIELD_RHO_S:
    case MC_FIELD_RHO_BAR:
      // the step keeps these in shared memory only: re-run the steric
      // stages on the last step's binned beads with field output on (they
      // are deterministic, so rho_x, F and F_s are rewritten identically)
      mc::launch_deposit_x(w->plan, s, field == MC_FIELD_RHO_S);
      if (field == MC_FIELD_RHO_BAR) mc::launch_force_spread(w->plan, s, 1, 1);
      MC_CUDA(cudaGetLastError());
      src = field == MC_FIELD_RHO_S ? (const void*)h.rho_s : (const void*)h.rho_b;
      bytes = HW * sizeof(float);
      break;
    case MC_FIELD_FORCE:
      // the step hands F from the spread to the collision in shared memory:
      // re-run the spread on the last step's binned beads (deterministic);
      // a direct-forcing step leaves its total F in device memory
      if (h.ib != 1) mc::launch_force_spread(w->plan, s, 0, 1);
      MC_CUDA(cudaGetLastError());
      src = h.F;
      bytes = HW * sizeof(float2);
      break;
    case MC_FIELD_U: src = h.u; bytes = HW * sizeof(float2); break;
    case MC_FIELD_BIN: src = h.bead_bin; bytes = h.N * sizeof(int); break;
    case MC_FIELD_BIN_OFF: src = h.bin_off; bytes = (h.n_bins + 1) * sizeof(int); break;
    case MC_FIELD_BIN_BEADS:   // the id word of each bin-ordered record
      if (h.N)
        MC_CUDA(cudaMemcpy2DAsync(out, sizeof(int), reinterpret_cast<const char*>(h.srec) + 2 * sizeof(float),
                                  sizeof(float4), sizeof(int), h.N, dk, s));
      if (host) MC_CUDA(cudaStreamSynchronize(s));
      return MC_OK;
    case MC_FIELD_EBEAD:
      if (!h.ebead) return fail(MC_ERR_INVALID_ARG, "the world has no energy field");
      src = h.ebead;
      bytes = h.N * sizeof(float);
      break;
    case MC_FIELD_CELL: {
      if (h.N == 0) return MC_OK;
      int* dst = static_cast<int*>(out);
      void* scratch = nullptr;
      if (host) {
        MC_CUDA(cudaMallocAsync(&scratch, h.N * sizeof(int), s));
        dst = static_cast<int*>(scratch);
      }
      mc::launch_cells_out(h, dst, s);
      MC_CUDA(cudaGetLastError());
      if (host) {
        MC_CUDA(cudaMemcpyAsync(out, dst, h.N * sizeof(int), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaFreeAsync(scratch, s));
        MC_CUDA(cudaStreamSynchronize(s));
      }
      return MC_OK;
    }
    default:
      return fail(MC_ERR_INVALID_ARG, "unknown field");
  }
  if (bytes) MC_CUDA(cudaMemcpyAsync(out, src, bytes, dk, s));
  if (host) MC_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

mc_status mc_world_get_observables(const mc_world* w, double* out, void* stream) {
  if (!w || !out) return fail(MC_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long v[3];
  MC_CUDA(cudaMemcpyAsync(v, w->h.obs, sizeof(v), cudaMemcpyDeviceToHost, s));
  MC_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 3; ++k) out[k] = (double)(long long)v[k] / (double)mc::kObsScale;
  return MC_OK;
}

mc_status mc_world_check(const mc_world* w, void* stream) {
  if (!w) return fail(MC_ERR_INVALID_ARG, "world is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned flags = 0;
  MC_CUDA(cudaMemcpyAsync(&flags, w->h.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MC_CUDA(cudaStreamSynchronize(s));
  if (flags & mc::kFlagTimeout)
    return fail(MC_ERR_TIMEOUT,
                "a grid barrier of the persistent step or a wait for bulk copies ran out of time; the world's state is "
                "unspecified");
  if (flags & mc::kFlagUnstable) return fail(MC_ERR_UNSTABLE, "bead velocity watchdog tripped (|U| > 0.5 or not finite)");
  return MC_OK;
}

mc_status mc_world_clear_flags(mc_world* w, void* stream) {
  if (!w) return fail(MC_ERR_INVALID_ARG, "world is NULL");
  MC_CUDA(cudaMemsetAsync(w->h.flags, 0, sizeof(unsigned), static_cast<cudaStream_t>(stream)));
  return MC_OK;
}

}  // extern "C"

namespace mc {
const WorldDev& world_dev(const mc_world* w) { return w->h; }
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace mc
