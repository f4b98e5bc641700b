// C ABI of libgslm (include/gslm.h): contexts, caches and the host-side order
// of the device work of Algorithm 1 and of one LM step (Sec. 3.2, 3.3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace gslm;

namespace gslm {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace gslm


// Per-phase CUDA-event timing of one LM step (options.profile).
struct PhaseTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  std::vector<cudaEvent_t> pool;
  int open_phase = -1;
  cudaEvent_t open_ev = nullptr;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // Opens a phase unless one is already open (nested calls are attributed to
  // the outer phase); returns whether end() must close it.
  bool begin(int phase) {
    if (!on || open_phase >= 0) return false;
    open_phase = phase;
    open_ev = get();
    cudaEventRecord(open_ev, st);
    return true;
  }
  void end(bool opened) {
    if (!opened) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    marks.push_back({open_phase, {open_ev, e}});
    open_phase = -1;
  }
  // Sums elapsed ms per phase (after the stream has been synchronised).
  void collect(double* ms, int n) {
    for (auto& m : marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, m.second.first, m.second.second) == cudaSuccess && m.first < n) ms[m.first] += t;
      pool.push_back(m.second.first);
      pool.push_back(m.second.second);
    }
    marks.clear();
  }
  ~PhaseTimer() {
    for (auto& m : marks) {
      cudaEventDestroy(m.second.first);
      cudaEventDestroy(m.second.second);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

enum { PH_BUILD = 0, PH_DIAG, PH_TANGENT, PH_APPLY_J, PH_APPLY_JT, PH_VJP, PH_VEC, PH_RHO };

struct gslm_ctx {
  gslm_options opt;
  cudaStream_t st = nullptr;
  int device = 0;
  std::string err;
  PhaseTimer timer;
  int var_J[3] = {-1, -1, -1};      // autotuned apply kernel variants per cache format
  int var_JT[3] = {-1, -1, -1};
  float ms_J[3] = {0.f, 0.f, 0.f};
  float ms_JT[3] = {0.f, 0.f, 0.f};
  // scratch reused across calls
  Buf ydot, seg_ybar, seg_q, u, partials, scalars, reduce_out;
  Buf r, z, p, g;
  Buf lm_num, lm_den, lm_delta, lm_trial, lm_x, lm_b, lm_M, lm_tgt, lm_img, lm_D;
  gslm_precond* pc = nullptr;       // learned preconditioner used by lm_step, if set
  // batched solves: stacked per-subset vectors and per-subset scratch
  Buf bt_b, bt_M, bt_D, bt_x, bt_z, bt_p, bt_g, bt_u, bt_ydot, bt_segy, bt_part, bt_sc, bt_queue;
  int bvar_J[3] = {-1, -1, -1};     // autotuned (variant, CTAs per SM) of the persistent tile kernels
  int bvar_JT[3] = {-1, -1, -1};
  int bctas_J[3] = {0, 0, 0};
  int bctas_JT[3] = {0, 0, 0};
  cudaGraphExec_t graph_exec[3] = {nullptr, nullptr, nullptr};   // start + first chunk, full chunk, last chunk
  cudaStream_t cap_st = nullptr;    // private stream the batched solve is captured on
  void* noalloc_scratch = nullptr;  // gslm_apply_JT_noalloc's array on this device (looked up at creation)
  ~gslm_ctx() {
    for (auto ge : graph_exec)
      if (ge != nullptr) cudaGraphExecDestroy(ge);
    if (cap_st != nullptr) cudaStreamDestroy(cap_st);
  }
};

struct gslm_cache {
  gslm_ctx* ctx = nullptr;
  const float* params = nullptr;
  int N = 0;
  long long ld = 0;
  int V = 0;
  int smooth = 0;
  int fmt = 0;
  int n_tiles = 0;
  long long n_pix = 0;
  long long n_vis = 0, n_keys = 0, n_seg = 0, n_entries = 0, n_active = 0;
  double cost = 0.0;
  std::vector<DevCam> hcams;
  Buf cams, rec, slot_active, tile_seg_off, seg_entry_off, seg_slot, seg_rec, payload, seg_scale, pixoff;
  Buf slot_seg_start, slot_seg_end, slot_seg_list, seg_pos, F, own_params, vmask, act_off;
  Buf W;   // residual-to-pixel weights [n_pix][3] (L1 + SSIM objective only)
  // thin caches (GSLM_CACHE_THIN) only
  Buf thin_rec, img, n_live, win_off, win_tile, ckpt;
  long long n_win = 0;

  CacheView view() const {
    CacheView cv;
    cv.cams = cams.as<DevCam>();
    cv.V = V;
    cv.n_tiles = n_tiles;
    cv.n_pix = n_pix;
    cv.N = N;
    cv.n_slots = (long long)N * V;
    cv.rec = rec.as<SplatRec>();
    cv.tile_seg_off = tile_seg_off.as<uint32_t>();
    cv.seg_entry_off = seg_entry_off.as<unsigned long long>();
    cv.seg_slot = seg_slot.as<uint32_t>();
    cv.seg_rec = seg_rec.as<SegRec>();
    cv.payload = payload.p;
    cv.seg_scale = seg_scale.as<float>();
    cv.pixoff = pixoff.as<uint8_t>();
    cv.slot_seg_start = slot_seg_start.as<uint32_t>();
    cv.slot_seg_end = slot_seg_end.as<uint32_t>();
    cv.slot_seg_list = slot_seg_list.as<uint32_t>();
    cv.seg_pos = seg_pos.as<uint32_t>();
    cv.slot_active = slot_active.as<uint8_t>();
    cv.vmask = vmask.as<unsigned long long>();
    cv.act_off = act_off.as<uint32_t>();
    cv.n_seg = n_seg;
    cv.n_entries = n_entries;
    cv.fmt = fmt;
    cv.skip = nullptr;
    cv.wres = W.as<float>();
    cv.thin_rec = thin_rec.as<SplatRec>();
    cv.img = img.as<float>();
    cv.n_live = n_live.as<uint32_t>();
    cv.win_off = win_off.as<uint32_t>();
    cv.win_tile = win_tile.as<uint32_t>();
    cv.ckpt = ckpt.as<float4>();
    cv.n_win = n_win;
    return cv;
  }
  // splat tangents the tangent kernel writes: one per active splat (compact
  // index) when the view masks exist, else one per (view, Gaussian) slot
  long long tangent_rows() const { return act_off.p != nullptr ? std::max<long long>(n_active, 1) : std::max<long long>((long long)N * V, 1); }
  size_t device_bytes() const {
    return cams.bytes + rec.bytes + slot_active.bytes + tile_seg_off.bytes + seg_entry_off.bytes + seg_slot.bytes +
           seg_rec.bytes +
           payload.bytes + seg_scale.bytes + pixoff.bytes + slot_seg_start.bytes + slot_seg_end.bytes +
           slot_seg_list.bytes + seg_pos.bytes + F.bytes + own_params.bytes + vmask.bytes + act_off.bytes + W.bytes +
           thin_rec.bytes + img.bytes + n_live.bytes + win_off.bytes + win_tile.bytes + ckpt.bytes;
  }
  // Algorithmic bytes of one J p + J^T u pair through this cache (N Gaussians):
  // entries (payload and pixel offset), or for a thin cache the segment
  // records, checkpoints and per-pixel counts the kernels read; u written and
  // read, p read and g written, and the per-splat tangent and adjoint records.
  double pair_bytes(int N_) const {
    const double stream = fmt == GSLM_CACHE_THIN
                              ? (double)n_seg * 96.0 + (double)n_win * kTilePix * 16.0 + (double)n_tiles * kTilePix * 8.0
                              : (double)n_entries * (double)((fmt == GSLM_CACHE_FP32 ? 16 : 8) + 1);
    return 2.0 * stream + 24.0 * (double)n_pix + 472.0 * (double)N_ + 192.0 * (double)n_active;
  }
};

namespace {

gslm_status fail(gslm_ctx* c, gslm_status s, const std::string& msg) {
  if (c != nullptr) c->err = msg;
  return s;
}

gslm_status cuda_fail(gslm_ctx* c, cudaError_t e, const char* where) {
  const gslm_status s = (e == cudaErrorMemoryAllocation) ? GSLM_E_OOM : GSLM_E_CUDA;
  cudaGetLastError();
  return fail(c, s, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                                  \
  do {                                                            \
    const cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);      \
  } while (0)

#define CKS(expr)                                                 \
  do {                                                            \
    const gslm_status s_ = (expr);                                \
    if (s_ != GSLM_OK) return s_;                                 \
  } while (0)

int bits_for(unsigned long long n) {
  int b = 0;
  while (b < 64 && (1ull << b) < n) ++b;
  return b;
}

size_t payload_bytes(int fmt) { return fmt == GSLM_CACHE_FP32 ? 16 : fmt == GSLM_CACHE_THIN ? 0 : 8; }

// Cameras of a call with their tile/pixel offsets.
gslm_status make_cams(gslm_ctx* ctx, const gslm_camera* cams, int V, std::vector<DevCam>& out, int& n_tiles,
                      long long& n_pix) {
  out.resize(V);
  long long toff = 0, poff = 0;
  for (int v = 0; v < V; ++v) {
    const gslm_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * kTile || c.height > 65535 * kTile)
      return fail(ctx, GSLM_E_INVALID, "camera size out of range");
    DevCam& d = out[v];
    std::memcpy(d.R, c.R, sizeof(d.R));
    std::memcpy(d.t, c.t, sizeof(d.t));
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    for (int i = 0; i < 3; ++i)
      d.campos[i] = -(c.R[0 * 3 + i] * c.t[0] + c.R[1 * 3 + i] * c.t[1] + c.R[2 * 3 + i] * c.t[2]);
    d.W = c.width;
    d.H = c.height;
    d.tiles_x = (c.width + kTile - 1) / kTile;
    d.tiles_y = (c.height + kTile - 1) / kTile;
    d.tile_off = (int)toff;
    d.pad = 0;
    d.pix_off = poff;
    toff += (long long)d.tiles_x * d.tiles_y;
    poff += (long long)c.width * c.height;
    if (toff >= (1ll << 31)) return fail(ctx, GSLM_E_INVALID, "too many tiles");
  }
  n_tiles = (int)toff;
  n_pix = poff;
  return GSLM_OK;
}

gslm_status check_vec_args(gslm_ctx* ctx, long long N, long long ld) {
  if (ctx == nullptr) return GSLM_E_INVALID;
  if (N <= 0 || N >= (1ll << 31)) return fail(ctx, GSLM_E_INVALID, "N out of range");
  if (ld < N || (ld & 3) != 0) return fail(ctx, GSLM_E_INVALID, "ld must be >= N and a multiple of 4");
  return GSLM_OK;
}

// Projection, depth sort, tile keys and tile ranges of a call (shared by render
// and build_cache). Leaves the per-tile splat lists in (tile_start, tile_end,
// tile_vals) and the splats in rec.
struct Binning {
  Buf cams, rec, ntiles, rect, tmask, depth, flags, pos, vis, keys_a, vals_a, keys_b, vals_b, sort_tmp, key_off;
  Buf tile_start, tile_end, scan_tmp;
  uint32_t* tile_vals = nullptr;
  uint32_t* tile_keys = nullptr;
  long long n_vis = 0, n_keys = 0;
};

gslm_status bin_splats(gslm_ctx* ctx, const float* params, int N, long long ld, const std::vector<DevCam>& hc,
                       int n_tiles, int smooth, Binning& B) {
  cudaStream_t st = ctx->st;
  const int V = (int)hc.size();
  const long long S = (long long)N * V;
  if (S >= (1ll << 32) - 1) return fail(ctx, GSLM_E_INVALID, "views x Gaussians exceeds 2^32 splats");
  CK(B.cams.alloc(sizeof(DevCam) * V, st));
  CK(cudaMemcpyAsync(B.cams.p, hc.data(), sizeof(DevCam) * V, cudaMemcpyHostToDevice, st));
  CK(B.rec.alloc(sizeof(SplatRec) * S, st));
  CK(B.ntiles.alloc(sizeof(uint32_t) * S, st));
  CK(B.rect.alloc(sizeof(uint2) * S, st));
  CK(B.depth.alloc(sizeof(uint32_t) * S, st));
  CK(B.tmask.alloc(sizeof(unsigned long long) * S, st));
  CK(launch_project(params, N, ld, B.cams.as<DevCam>(), V, smooth, B.rec.as<SplatRec>(), B.ntiles.as<uint32_t>(),
                    B.rect.as<uint2>(), B.depth.as<uint32_t>(), B.tmask.as<unsigned long long>(), st));
  // visible splats, compacted in slot order
  CK(B.flags.alloc(sizeof(uint32_t) * S, st));
  CK(B.pos.alloc(sizeof(uint32_t) * (S + 1), st));
  CK(B.scan_tmp.alloc(std::max(scan_temp_bytes(S), scan_temp_bytes(n_tiles + 1)), st));
  CK(launch_flags(B.ntiles.as<uint32_t>(), S, B.flags.as<uint32_t>(), st));
  CK(exclusive_scan_u32(B.flags.as<uint32_t>(), B.pos.as<uint32_t>(), S, B.scan_tmp.p, st));
  uint32_t nvis = 0;
  CK(cudaMemcpyAsync(&nvis, B.pos.as<uint32_t>() + S, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  B.n_vis = nvis;
  const long long nv = std::max<long long>(B.n_vis, 1);
  CK(B.vis.alloc(sizeof(uint32_t) * nv, st));
  CK(launch_compact_flags(B.ntiles.as<uint32_t>(), B.pos.as<uint32_t>(), S, B.vis.as<uint32_t>(), st));
  // depth order (stable: ties keep the Gaussian order)
  CK(B.keys_a.alloc(sizeof(uint32_t) * nv, st));
  CK(B.keys_b.alloc(sizeof(uint32_t) * nv, st));
  CK(B.vals_b.alloc(sizeof(uint32_t) * nv, st));
  CK(launch_gather_u32(B.depth.as<uint32_t>(), B.vis.as<uint32_t>(), B.n_vis, B.keys_a.as<uint32_t>(), st));
  CK(B.sort_tmp.alloc(radix_temp_bytes(nv), st));
  uint32_t *dk = nullptr, *dv = nullptr;
  CK(radix_sort_pairs(B.keys_a.as<uint32_t>(), B.vis.as<uint32_t>(), B.keys_b.as<uint32_t>(),
                      B.vals_b.as<uint32_t>(), B.n_vis, 32, B.sort_tmp.p, &dk, &dv, st));
  // tiles per sorted splat -> key offsets
  CK(launch_gather_u32(B.ntiles.as<uint32_t>(), dv, B.n_vis, dk, st));
  CK(B.key_off.alloc(sizeof(unsigned long long) * (nv + 1), st));
  CK(B.scan_tmp.ensure(scan_temp_bytes(nv + 1), st));
  CK(exclusive_scan_u64(dk, B.key_off.as<unsigned long long>(), B.n_vis, B.scan_tmp.p, st));
  unsigned long long nkeys = 0;
  CK(cudaMemcpyAsync(&nkeys, B.key_off.as<unsigned long long>() + B.n_vis, sizeof(nkeys), cudaMemcpyDeviceToHost,
                     st));
  CK(cudaStreamSynchronize(st));
  if (nkeys >= (1ull << 32) - 1) return fail(ctx, GSLM_E_CACHE_OVERFLOW, "more than 2^32 tile keys");
  B.n_keys = (long long)nkeys;
  const long long nk = std::max<long long>(B.n_keys, 1);
  // the depth-sorted slot list must survive the key emission: keep it in vals_b or vis
  Buf sorted_slots;
  CK(sorted_slots.alloc(sizeof(uint32_t) * nv, st));
  CK(cudaMemcpyAsync(sorted_slots.p, dv, sizeof(uint32_t) * B.n_vis, cudaMemcpyDeviceToDevice, st));
  // Per-slot buffers are dropped as soon as they are dead, so that the peak
  // of a build is the splat records plus the key buffers.
  for (Buf* b : {&B.keys_a, &B.keys_b, &B.vals_b, &B.vis, &B.ntiles, &B.depth, &B.flags, &B.pos}) b->release();
  CK(B.keys_a.alloc(sizeof(uint32_t) * nk, st));
  CK(B.vals_a.alloc(sizeof(uint32_t) * nk, st));
  CK(launch_emit_keys(sorted_slots.as<uint32_t>(), B.n_vis, B.rect.as<uint2>(), B.tmask.as<unsigned long long>(),
                      B.cams.as<DevCam>(), V, N,
                      B.key_off.as<unsigned long long>(), B.keys_a.as<uint32_t>(), B.vals_a.as<uint32_t>(), st));
  for (Buf* b : {&sorted_slots, &B.rect, &B.tmask, &B.key_off}) b->release();
  CK(B.keys_b.alloc(sizeof(uint32_t) * nk, st));
  CK(B.vals_b.alloc(sizeof(uint32_t) * nk, st));
  CK(B.sort_tmp.ensure(radix_temp_bytes(nk), st));
  CK(radix_sort_pairs(B.keys_a.as<uint32_t>(), B.vals_a.as<uint32_t>(), B.keys_b.as<uint32_t>(),
                      B.vals_b.as<uint32_t>(), B.n_keys, bits_for((unsigned long long)n_tiles), B.sort_tmp.p,
                      &B.tile_keys, &B.tile_vals, st));
  CK(B.tile_start.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
  CK(B.tile_end.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
  CK(cudaMemsetAsync(B.tile_start.p, 0, sizeof(uint32_t) * (n_tiles + 1), st));
  CK(cudaMemsetAsync(B.tile_end.p, 0, sizeof(uint32_t) * (n_tiles + 1), st));
  CK(launch_ranges(B.tile_keys, B.n_keys, B.tile_start.as<uint32_t>(), B.tile_end.as<uint32_t>(), st));
  // only the sorted splat list of the keys is read from here on
  const bool vals_in_a = B.tile_vals == B.vals_a.as<uint32_t>();
  for (Buf* b : {&B.keys_a, &B.keys_b, vals_in_a ? &B.vals_b : &B.vals_a, &B.sort_tmp}) b->release();
  B.tile_keys = nullptr;
  return GSLM_OK;
}

gslm_status reduce_to_host(gslm_ctx* ctx, const double* partials, int n, double* host) {
  cudaStream_t st = ctx->st;
  CK(ctx->reduce_out.ensure(sizeof(double), st));
  CK(launch_reduce_partials(partials, n, ctx->reduce_out.as<double>(), st));
  CK(cudaMemcpyAsync(host, ctx->reduce_out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return GSLM_OK;
}

constexpr int kDefaultVariant = 9;   // the fastest on the 1.5M-Gaussian workload, both formats
// Solves of more than kCheckEvery iterations read the done flags back every
// kCheckEvery iterations and stop launching once every solve has ended.
constexpr int kCheckEvery = 16;

// Autotuner: times every kernel variant twice on the caller's real inputs
// (two rounds over all variants; all compute the same result, so the last one
// run leaves valid outputs) and returns the one with the fastest run. Runs
// synchronously, once per context and cache format.
constexpr int kTuneRounds = 2;
template <class F>
gslm_status tune_variant(gslm_ctx* ctx, F&& launch, int* chosen, float* chosen_ms) {
  cudaStream_t st = ctx->st;
  const int n = apply_variants();
  std::vector<cudaEvent_t> ev(kTuneRounds * n + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  struct Ev {
    std::vector<cudaEvent_t>& v;
    ~Ev() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evg{ev};
  CK(cudaEventRecord(ev[0], st));
  for (int i = 0; i < kTuneRounds * n; ++i) {
    CK(launch(i % n));
    CK(cudaEventRecord(ev[i + 1], st));
  }
  CK(cudaEventSynchronize(ev[kTuneRounds * n]));
  int best = kDefaultVariant;
  float best_ms = 1e30f;
  for (int i = 0; i < kTuneRounds * n; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    if (t < best_ms) {
      best_ms = t;
      best = i % n;
    }
  }
  // run the chosen variant last so that its result is the one left behind
  CK(launch(best));
  *chosen = best;
  *chosen_ms = best_ms;
  return GSLM_OK;
}

// J p through the cache: per-Gaussian tangent, then the tile kernel.
gslm_status do_apply_J(gslm_ctx* ctx, const gslm_cache* c, const float* p, float* u, const float* z_beta,
                       float* p_out, const PcgScalars* sc, const float* Fadd, double* sq_partials) {
  cudaStream_t st = ctx->st;
  const long long S = (long long)c->N * c->V;
  (void)S;
  CK(ctx->ydot.ensure(sizeof(float) * 12 * c->tangent_rows(), st));
  bool t = ctx->timer.begin(PH_TANGENT);
  CK(launch_tangent(c->params, c->N, c->ld, c->cams.as<DevCam>(), c->V, c->smooth, c->slot_active.as<uint8_t>(),
                    c->vmask.as<unsigned long long>(), c->act_off.as<uint32_t>(), p,
                    ctx->ydot.as<float>(), z_beta, p_out, sc, st));
  CacheView cv = c->view();
  cv.skip = sc != nullptr ? &sc->done : nullptr;
  ctx->timer.end(t);
  t = ctx->timer.begin(PH_APPLY_J);
  if (c->fmt == GSLM_CACHE_THIN) {   // blends the tile's segments again; no kernel variants
    CK(launch_thin_apply_J(cv, ctx->ydot.as<float>(), Fadd, u, sq_partials, st));
    ctx->timer.end(t);
    return GSLM_OK;
  }
  int& var = ctx->var_J[c->fmt];
  if (ctx->opt.apply_variant > 0) {
    CK(launch_apply_J(cv, ctx->ydot.as<float>(), Fadd, u, sq_partials, ctx->opt.apply_variant - 1, st));
  } else if (var < 0 && ctx->opt.autotune) {
    const float* yd = ctx->ydot.as<float>();
    CKS(tune_variant(ctx, [&](int v) { return launch_apply_J(cv, yd, Fadd, u, sq_partials, v, st); }, &var,
                     &ctx->ms_J[c->fmt]));
  } else {
    CK(launch_apply_J(cv, ctx->ydot.as<float>(), Fadd, u, sq_partials, var < 0 ? kDefaultVariant : var, st));
  }
  ctx->timer.end(t);
  return GSLM_OK;
}

gslm_status do_apply_JT(gslm_ctx* ctx, const gslm_cache* c, const float* u, float* g, float scale, const float* p,
                        const float* M, float lambda, double* partials, const PcgScalars* sc) {
  cudaStream_t st = ctx->st;
  CK(ctx->seg_ybar.ensure(sizeof(float) * 12 * std::max<long long>(c->n_seg, 1), st));
  CacheView cv = c->view();
  cv.skip = sc != nullptr ? &sc->done : nullptr;
  bool t = ctx->timer.begin(PH_APPLY_JT);
  float* sy = ctx->seg_ybar.as<float>();
  int var_dummy = 0;
  int& var = c->fmt == GSLM_CACHE_THIN ? var_dummy : ctx->var_JT[c->fmt];
  if (c->fmt == GSLM_CACHE_THIN) {   // window by window from the checkpoints
    CK(launch_thin_apply_JT(cv, u, sy, st));
  } else if (ctx->opt.apply_variant > 0) {
    CK(launch_apply_JT(cv, u, sy, ctx->opt.apply_variant - 1, st));
  } else if (var < 0 && ctx->opt.autotune) {
    CKS(tune_variant(ctx, [&](int v) { return launch_apply_JT(cv, u, sy, v, st); }, &var, &ctx->ms_JT[c->fmt]));
  } else {
    CK(launch_apply_JT(cv, u, sy, var < 0 ? kDefaultVariant : var, st));
  }
  ctx->timer.end(t);
  t = ctx->timer.begin(PH_VJP);
  // with compact splat keys, the per-splat sums go to the tangent buffer (free
  // once J p has read it) and the adjoint reads one record per splat
  float* splat_ybar = nullptr;
  if (c->act_off.p != nullptr) {
    CK(ctx->ydot.ensure(sizeof(float) * 12 * c->tangent_rows(), st));
    splat_ybar = ctx->ydot.as<float>();
    CK(launch_splat_sum(c->n_active, c->slot_seg_start.as<uint32_t>(), c->slot_seg_end.as<uint32_t>(), sy,
                        splat_ybar, sc, st));
  }
  CK(launch_vjp(c->params, c->N, c->ld, c->cams.as<DevCam>(), c->V, c->smooth, c->slot_seg_start.as<uint32_t>(),
                c->slot_seg_end.as<uint32_t>(), c->vmask.as<unsigned long long>(), c->act_off.as<uint32_t>(), sy,
                splat_ybar, scale, g, p, M, lambda, partials, sc, st));
  ctx->timer.end(t);
  return GSLM_OK;
}

gslm_status pcg_enqueue(gslm_ctx* ctx, const gslm_cache* c, const float* b, const float* diag, const float* D,
                        float lambda, float* x) {
  cudaStream_t st = ctx->st;
  const int N = c->N;
  const long long ld = c->ld;
  const size_t vb = sizeof(float) * kNP * (size_t)ld;
  CK(ctx->r.ensure(vb, st));
  CK(ctx->z.ensure(vb, st));
  CK(ctx->p.ensure(vb, st));
  CK(ctx->g.ensure(vb, st));
  CK(ctx->u.ensure(sizeof(float) * 3 * std::max<long long>(c->n_pix, 1), st));
  const int nvec = pcg_blocks(N), nvjp = vjp_blocks(N);
  CK(ctx->partials.ensure(sizeof(double) * 2 * std::max(nvec, nvjp), st));
  CK(ctx->scalars.ensure(sizeof(PcgScalars), st));
  PcgScalars* sc = ctx->scalars.as<PcgScalars>();
  double* part = ctx->partials.as<double>();
  float *r = ctx->r.as<float>(), *z = ctx->z.as<float>(), *p = ctx->p.as<float>(), *g = ctx->g.as<float>();
  float* u = ctx->u.as<float>();
  // x0 = M^-1 b
  bool t = ctx->timer.begin(PH_VEC);
  CK(launch_pcg_init(N, ld, b, diag, D, x, part, st));
  CK(launch_pcg_scalars(sc, part, nvec, 0, ctx->opt.break_rel2, st));
  ctx->timer.end(t);
  // u0 = J x0; g0 = J^T u0; r0 = b - (g0 + lambda M x0); z0 = M^-1 r0; p0 = z0
  CKS(do_apply_J(ctx, c, x, u, nullptr, nullptr, nullptr, nullptr, nullptr));
  CKS(do_apply_JT(ctx, c, u, g, 1.f, nullptr, nullptr, 0.f, nullptr, nullptr));
  t = ctx->timer.begin(PH_VEC);
  CK(launch_pcg_residual0(N, ld, b, g, diag, D, x, lambda, r, z, p, part, st));
  CK(launch_pcg_scalars(sc, part, nvec, 1, ctx->opt.break_rel2, st));
  ctx->timer.end(t);
  for (int it = 0; it < ctx->opt.n_iters; ++it) {
    if (it > 0 && it % kCheckEvery == 0) {
      // long solves: stop launching once the break test (or a breakdown) has ended the solve
      int done = 0;
      CK(cudaMemcpyAsync(&done, &sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (done) break;
    }
    // p_i = z_i + beta p_{i-1} (fused), u_i = J p_i
    CKS(do_apply_J(ctx, c, p, u, it > 0 ? z : nullptr, it > 0 ? p : nullptr, sc, nullptr, nullptr));
    // g_i = J^T u_i + lambda M p_i, p^T g
    CKS(do_apply_JT(ctx, c, u, g, 1.f, p, diag, lambda, part, sc));
    t = ctx->timer.begin(PH_VEC);
    CK(launch_pcg_scalars(sc, part, nvjp, 2, ctx->opt.break_rel2, st));
    CK(launch_pcg_update(N, ld, sc, p, g, diag, D, x, r, z, part, st));
    CK(launch_pcg_scalars(sc, part, nvec, 3, ctx->opt.break_rel2, st));
    ctx->timer.end(t);
  }
  return GSLM_OK;
}


// Candidates of the persistent tile kernels' autotuner: (variant, CTAs per SM),
// each variant at the residency its registers allow and one CTA fewer.
constexpr int kBatchCand = 20;   // 2 x apply_variants()
inline int cand_variant(int c) { return c / 2; }
inline int cand_ctas(int c, bool jt) {
  const int cap = variant_cta_cap(c / 2, jt);
  return (c & 1) ? cap - 1 : cap;
}

// Times every candidate twice (two rounds; each computes the same result) and
// keeps the one with the fastest run.
template <class F>
gslm_status tune_batch(gslm_ctx* ctx, F&& launch, bool jt, int* var, int* ctas) {
  cudaStream_t st = ctx->st;
  std::vector<cudaEvent_t> ev(kTuneRounds * kBatchCand + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  struct Ev {
    std::vector<cudaEvent_t>& v;
    ~Ev() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evg{ev};
  CK(cudaEventRecord(ev[0], st));
  for (int i = 0; i < kTuneRounds * kBatchCand; ++i) {
    const int c = i % kBatchCand;
    CKS(launch(cand_variant(c), cand_ctas(c, jt)));
    CK(cudaEventRecord(ev[i + 1], st));
  }
  CK(cudaEventSynchronize(ev[kTuneRounds * kBatchCand]));
  int best = 2 * kDefaultVariant;
  float best_ms = 1e30f;
  for (int i = 0; i < kTuneRounds * kBatchCand; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    if (t < best_ms) {
      best_ms = t;
      best = i % kBatchCand;
    }
  }
  *var = cand_variant(best);
  *ctas = cand_ctas(best, jt);
  return GSLM_OK;
}

// Stacked layout of a batch of n subsets of the same Gaussians.
struct BatchLayout {
  int n = 0;
  long long vs = 0;                 // floats per stacked vector
  long long u_off[kMaxBatch + 1];   // floats
  long long y_off[kMaxBatch + 1];   // floats (ydot)
  long long s_off[kMaxBatch + 1];   // floats (segment adjoints)
};

gslm_status batch_layout(gslm_ctx* ctx, const gslm_cache* const* cs, int n, BatchLayout* L) {
  if (n < 1 || n > kMaxBatch) return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: 1 to 16 subsets per batch");
  const gslm_cache* c0 = cs[0];
  L->n = n;
  L->vs = (long long)kNP * c0->ld;
  L->u_off[0] = L->y_off[0] = L->s_off[0] = 0;
  for (int i = 0; i < n; ++i) {
    const gslm_cache* c = cs[i];
    if (c == nullptr) return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: null cache");
    if (c->N != c0->N || c->ld != c0->ld || c->fmt != c0->fmt || c->smooth != c0->smooth || c->params == nullptr)
      return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: caches differ in N, ld, format or mode");
    auto up = [](long long v) { return (v + 3) & ~3ll; };   // 16-byte aligned sub-buffers
    L->u_off[i + 1] = L->u_off[i] + up(3 * std::max<long long>(c->n_pix, 1));
    L->y_off[i + 1] = L->y_off[i] + up(12 * c->tangent_rows());
    L->s_off[i + 1] = L->s_off[i] + up(12 * std::max<long long>(c->n_seg, 1));
  }
  return GSLM_OK;
}

gslm_status batch_alloc(gslm_ctx* ctx, const BatchLayout& L, unsigned d_mask, size_t limit) {
  cudaStream_t st = ctx->st;
  const size_t vb = sizeof(float) * (size_t)L.vs * L.n;
  const size_t need = (d_mask != 0 ? 7 : 6) * vb + sizeof(float) * (L.u_off[L.n] + L.y_off[L.n] + L.s_off[L.n]);
  if (limit != 0 && need > limit) return fail(ctx, GSLM_E_OOM, "batch: stacked vectors above options.batch_mem");
  // r lives in b's place (b is read only by the first residual); M^-1 is not stored
  for (Buf* b : {&ctx->bt_b, &ctx->bt_M, &ctx->bt_x, &ctx->bt_z, &ctx->bt_p, &ctx->bt_g}) CK(b->ensure(vb, st));
  if (d_mask != 0) CK(ctx->bt_D.ensure(vb, st));
  CK(ctx->bt_u.ensure(sizeof(float) * L.u_off[L.n], st));
  CK(ctx->bt_ydot.ensure(sizeof(float) * L.y_off[L.n], st));
  CK(ctx->bt_segy.ensure(sizeof(float) * L.s_off[L.n], st));
  return GSLM_OK;
}

// Enqueues Algorithm 1 for a batch whose stacked b, M (raw diagonal) and
// optional D are in ctx->bt_b, bt_M, bt_D (subset i uses D when bit i of
// d_mask is set); x ends in ctx->bt_x, the scalars in ctx->bt_sc[i]. Nothing
// here synchronises unless `tune` (first use: the tile kernels are autotuned).
gslm_status pcg_batch_enqueue(gslm_ctx* ctx, const gslm_cache* const* cs, const BatchLayout& L, unsigned d_mask,
                              float lambda, bool tune, bool init, int it0, int it1) {
  cudaStream_t st = ctx->st;
  const gslm_cache* c0 = cs[0];
  const int n = L.n, N = c0->N, fmt = c0->fmt;
  const long long ld = c0->ld, vs = L.vs;
  const int nvec = pcg_blocks(N), nvjp = vjp_blocks(N);
  PcgScalars* sc = ctx->bt_sc.as<PcgScalars>();
  double* part = ctx->bt_part.as<double>();
  float *b = ctx->bt_b.as<float>(), *M = ctx->bt_M.as<float>(), *D = ctx->bt_D.as<float>();
  float *x = ctx->bt_x.as<float>(), *r = b, *z = ctx->bt_z.as<float>();   // r overwrites b
  float *p = ctx->bt_p.as<float>(), *g = ctx->bt_g.as<float>();
  GaussBatch gb;
  TileBatch tb;
  gb.n = tb.n = n;
  tb.fmt = fmt;
  tb.queue = ctx->bt_queue.as<unsigned int>();
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    const gslm_cache* c = cs[i];
    SubsetRefs& R = gb.s[i];
    R.cams = c->cams.as<DevCam>();
    R.V = c->V;
    R.slot_active = c->slot_active.as<uint8_t>();
    R.vmask = c->vmask.as<unsigned long long>();
    R.act_off = c->act_off.as<uint32_t>();
    R.s_start = c->slot_seg_start.as<uint32_t>();
    R.s_end = c->slot_seg_end.as<uint32_t>();
    R.s_list = c->slot_seg_list.as<uint32_t>();
    R.ydot = ctx->bt_ydot.as<float>() + L.y_off[i];
    R.seg_ybar = ctx->bt_segy.as<float>() + L.s_off[i];
    R.n_splats = c->act_off.p != nullptr ? c->n_active : 0;
    tiles += c->n_tiles;
    tb.tile_end[i] = tiles;
    tb.v[i] = c->view();
    tb.ydot[i] = R.ydot;
    tb.u[i] = ctx->bt_u.as<float>() + L.u_off[i];
    tb.seg_ybar[i] = R.seg_ybar;
  }
  tb.total_tiles = tiles;
  const float* params = c0->params;
  const int smooth = c0->smooth;
  int& vJ = ctx->bvar_J[fmt];
  int& vJT = ctx->bvar_JT[fmt];
  int& cJ = ctx->bctas_J[fmt];
  int& cJT = ctx->bctas_JT[fmt];
  auto runJ = [&](int var, int ctas) -> gslm_status {
    CK(cudaMemsetAsync(tb.queue, 0, sizeof(unsigned int), st));
    CK(launch_apply_J_batch(tb, var, ctas, st));
    return GSLM_OK;
  };
  auto runJT = [&](int var, int ctas) -> gslm_status {
    CK(cudaMemsetAsync(tb.queue, 0, sizeof(unsigned int), st));
    CK(launch_apply_JT_batch(tb, var, ctas, st));
    return GSLM_OK;
  };
  const int forced = ctx->opt.apply_variant - 1;
  auto apply_pair = [&]() -> gslm_status {
    bool t = ctx->timer.begin(PH_APPLY_J);
    if (forced >= 0) {
      CKS(runJ(forced, ctx->opt.batch_ctas > 0 ? ctx->opt.batch_ctas : 6));
      ctx->timer.end(t);
      t = ctx->timer.begin(PH_APPLY_JT);
      CKS(runJT(forced, ctx->opt.batch_ctas > 0 ? ctx->opt.batch_ctas : 6));
      ctx->timer.end(t);
      return GSLM_OK;
    }
    if (vJ < 0 && tune) {
      CKS(tune_batch(ctx, runJ, false, &vJ, &cJ));
    } else {
      CKS(runJ(vJ < 0 ? kDefaultVariant : vJ, ctx->opt.batch_ctas > 0 ? ctx->opt.batch_ctas : (cJ > 0 ? cJ : 4)));
    }
    ctx->timer.end(t);
    t = ctx->timer.begin(PH_APPLY_JT);
    if (vJT < 0 && tune) {
      CKS(tune_batch(ctx, runJT, true, &vJT, &cJT));
    } else {
      CKS(runJT(vJT < 0 ? kDefaultVariant : vJT,
                ctx->opt.batch_ctas > 0 ? ctx->opt.batch_ctas : (cJT > 0 ? cJT : 4)));
    }
    ctx->timer.end(t);
    return GSLM_OK;
  };
  bool t = false;
  if (init) {
    // x0 = M^-1 b
    t = ctx->timer.begin(PH_VEC);
    CK(launch_pcg_init_batch(n, N, ld, vs, b, M, D, d_mask, x, part, st));
    CK(launch_pcg_scalars_batch(n, sc, part, nvec, nvec, 0, ctx->opt.break_rel2, st));
    ctx->timer.end(t);
    // u0 = J x0; g0 = J^T u0; r0 = b - (g0 + lambda M x0); z0 = M^-1 r0; p0 = z0
    for (int i = 0; i < n; ++i) tb.v[i].skip = nullptr;
    t = ctx->timer.begin(PH_TANGENT);
    CK(launch_tangent_batch(params, N, ld, smooth, gb, x, vs, nullptr, nullptr, nullptr, st));
    ctx->timer.end(t);
    CKS(apply_pair());
    t = ctx->timer.begin(PH_VJP);
    CK(launch_splat_sum_batch(gb, nullptr, st));
    CK(launch_vjp_batch(params, N, ld, smooth, gb, g, vs, nullptr, nullptr, 0.f, nullptr, nullptr, st));
    ctx->timer.end(t);
    t = ctx->timer.begin(PH_VEC);
    CK(launch_pcg_residual0_batch(n, N, ld, vs, b, g, M, D, d_mask, x, lambda, r, z, p, part, st));
    CK(launch_pcg_scalars_batch(n, sc, part, nvec, nvec, 1, ctx->opt.break_rel2, st));
    ctx->timer.end(t);
  }
  for (int i = 0; i < n; ++i) tb.v[i].skip = &sc[i].done;
  for (int it = it0; it < it1; ++it) {
    t = ctx->timer.begin(PH_TANGENT);
    CK(launch_tangent_batch(params, N, ld, smooth, gb, p, vs, it > 0 ? z : nullptr, it > 0 ? p : nullptr, sc, st));
    ctx->timer.end(t);
    CKS(apply_pair());
    t = ctx->timer.begin(PH_VJP);
    CK(launch_splat_sum_batch(gb, sc, st));
    CK(launch_vjp_batch(params, N, ld, smooth, gb, g, vs, p, M, lambda, part, sc, st));
    ctx->timer.end(t);
    t = ctx->timer.begin(PH_VEC);
    CK(launch_pcg_scalars_batch(n, sc, part, nvjp, nvjp, 2, ctx->opt.break_rel2, st));
    CK(launch_pcg_update_batch(n, N, ld, vs, sc, p, g, M, D, d_mask, x, r, z, part, st));
    CK(launch_pcg_scalars_batch(n, sc, part, nvec, 2 * nvec, 3, ctx->opt.break_rel2, st));
    ctx->timer.end(t);
  }
  return GSLM_OK;
}

// Runs a batch whose inputs are already stacked: directly the first time (it
// autotunes), else from captured CUDA graphs when options.graph is set and no
// per-phase profile is wanted: one graph for the start and the first chunk of
// kCheckEvery iterations, one for each later chunk (replayed), one for a
// shorter last chunk. Between chunks the done flags are read back and no more
// work is launched once every solve has ended.
gslm_status pcg_batch_run(gslm_ctx* ctx, const gslm_cache* const* cs, const BatchLayout& L, unsigned d_mask,
                          float lambda) {
  cudaStream_t st = ctx->st;
  const int fmt = cs[0]->fmt;
  const int N = cs[0]->N;
  const int n_iters = ctx->opt.n_iters;
  CK(ctx->bt_part.ensure(sizeof(double) * L.n * std::max(2 * pcg_blocks(N), vjp_blocks(N)), st));
  CK(ctx->bt_sc.ensure(sizeof(PcgScalars) * L.n, st));
  CK(ctx->bt_queue.ensure(sizeof(unsigned int), st));
  const bool tuned = !ctx->opt.autotune || (ctx->bvar_J[fmt] >= 0 && ctx->bvar_JT[fmt] >= 0);
  const bool use_graph = ctx->opt.graph && tuned && !ctx->timer.on;
  auto all_done = [&](bool* out) -> gslm_status {
    std::vector<PcgScalars> h(L.n);
    CK(cudaMemcpyAsync(h.data(), ctx->bt_sc.p, sizeof(PcgScalars) * L.n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool d = true;
    for (const auto& x : h) d = d && x.done != 0;
    *out = d;
    return GSLM_OK;
  };
  if (!use_graph) {
    const int first = std::min(n_iters, kCheckEvery);
    CKS(pcg_batch_enqueue(ctx, cs, L, d_mask, lambda, !tuned, true, 0, first));
    for (int it = first; it < n_iters; it += kCheckEvery) {
      bool done = false;
      CKS(all_done(&done));
      if (done) break;
      CKS(pcg_batch_enqueue(ctx, cs, L, d_mask, lambda, false, false, it, std::min(n_iters, it + kCheckEvery)));
    }
    return GSLM_OK;
  }
  // Capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graphs are launched on the caller's.
  if (ctx->cap_st == nullptr) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
  (void)device_sm_count();
  for (auto& ge : ctx->graph_exec) {
    if (ge != nullptr) CK(cudaGraphExecDestroy(ge));
    ge = nullptr;
  }
  auto capture = [&](bool init, int it0, int it1, cudaGraphExec_t* out) -> gslm_status {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
    ctx->st = ctx->cap_st;
    const gslm_status s = pcg_batch_enqueue(ctx, cs, L, d_mask, lambda, false, init, it0, it1);
    ctx->st = st;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_st, &graph);
    if (s != GSLM_OK) {
      if (graph != nullptr) cudaGraphDestroy(graph);
      return s;
    }
    CK(e);
    const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    return GSLM_OK;
  };
  const int first = std::min(n_iters, kCheckEvery);
  CKS(capture(true, 0, first, &ctx->graph_exec[0]));
  CK(cudaGraphLaunch(ctx->graph_exec[0], st));
  for (int it = first; it < n_iters; it += kCheckEvery) {
    bool done = false;
    CKS(all_done(&done));
    if (done) break;
    const int len = std::min(kCheckEvery, n_iters - it);
    cudaGraphExec_t& ge = ctx->graph_exec[len == kCheckEvery ? 1 : 2];
    if (ge == nullptr) CKS(capture(false, it, it + len, &ge));
    CK(cudaGraphLaunch(ge, st));
  }
  return GSLM_OK;
}

}  // namespace

namespace gslm {

bool cache_parts(const gslm_cache* c, CacheParts* out) {
  if (c == nullptr || out == nullptr) return false;
  out->view = c->view();
  out->params = c->params;
  out->N = c->N;
  out->ld = c->ld;
  out->cams = c->cams.as<DevCam>();
  out->V = c->V;
  out->smooth = c->smooth;
  return true;
}

bool context_parts(const gslm_ctx* c, int cache_fmt, ContextParts* out) {
  if (c == nullptr || out == nullptr || cache_fmt < 0 || cache_fmt > 3) return false;
  out->st = c->st;
  // the variant do_apply_JT would run: forced by the options, else tuned, else
  // the default (thin caches have one kernel)
  if (cache_fmt == GSLM_CACHE_THIN) out->variant_JT = 0;
  else if (c->opt.apply_variant > 0) out->variant_JT = c->opt.apply_variant - 1;
  else out->variant_JT = c->var_JT[cache_fmt] >= 0 ? c->var_JT[cache_fmt] : kDefaultVariant;
  out->device = c->device;
  out->noalloc_scratch = c->noalloc_scratch;
  return true;
}

void set_context_error(gslm_ctx* c, const char* msg) {
  if (c != nullptr) c->err = msg;
}

cudaStream_t context_stream(const gslm_ctx* c) { return c->st; }

gslm_status apply_A(gslm_ctx* ctx, const gslm_cache* c, const float* v, const float* M, float lambda, float* out) {
  CK(ctx->u.ensure(sizeof(float) * 3 * std::max<long long>(c->n_pix, 1), ctx->st));
  CKS(do_apply_J(ctx, c, v, ctx->u.as<float>(), nullptr, nullptr, nullptr, nullptr, nullptr));
  CKS(do_apply_JT(ctx, c, ctx->u.as<float>(), out, 1.f, v, M, lambda, nullptr, nullptr));
  return GSLM_OK;
}

}  // namespace gslm

extern "C" {

const char* gslm_version(void) { return "gslm 0.1 (sm_103a)"; }

int64_t gslm_kernel_launches(void) { return (int64_t)g_launches.load(); }

gslm_status gslm_memory_usage(const gslm_ctx* ctx, int32_t reset_peak, int64_t out[3]) {
  if (ctx == nullptr || out == nullptr) return GSLM_E_INVALID;
  cudaMemPool_t pool = nullptr;
  uint64_t used = 0, reserved = 0, high = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess) {
    cudaGetLastError();
    return GSLM_E_CUDA;
  }
  out[0] = (int64_t)used;
  out[1] = (int64_t)reserved;
  out[2] = (int64_t)high;
  if (reset_peak != 0) {
    uint64_t zero = 0;   // the only value the mark can be set to: it restarts from the bytes in use
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) {
      cudaGetLastError();
      return GSLM_E_CUDA;
    }
  }
  return GSLM_OK;
}

gslm_status gslm_autotune_info(const gslm_ctx* ctx, int32_t out[6], float ms[6]) {
  if (ctx == nullptr || out == nullptr) return GSLM_E_INVALID;
  for (int f = 0; f < 3; ++f) {
    out[f] = ctx->var_J[f];
    out[3 + f] = ctx->var_JT[f];
    if (ms != nullptr) {
      ms[f] = ctx->ms_J[f];
      ms[3 + f] = ctx->ms_JT[f];
    }
  }
  return GSLM_OK;
}

void gslm_default_options(gslm_options* o) {
  if (o == nullptr) return;
  std::memset(o, 0, sizeof(*o));
  o->cache_fmt = GSLM_CACHE_FP32;
  o->n_iters = 8;
  o->break_rel2 = 0.01f;
  o->lambda_min = 1e-4f;
  o->lambda_max = 1e4f;
  o->smooth = 0;
  o->mem_budget = 0;
  o->group = 32;
  o->profile = 0;
  o->autotune = 1;
  o->batch = 1;
  o->graph = 1;
  o->batch_ctas = 0;
  o->line_search = 8;
  o->objective = GSLM_OBJ_L2;
  o->lambda_l1 = 0.8f;
  o->lambda_ssim = 0.2f;
  o->res_eps = 1e-4f;
}

static gslm_status validate_opts(const gslm_options* o) {
  if (o->cache_fmt < 0 || o->cache_fmt > 3) return GSLM_E_INVALID;
  if (o->n_iters < 0 || o->n_iters > 100000) return GSLM_E_INVALID;
  if (!(o->lambda_min > 0.f) || !(o->lambda_max >= o->lambda_min)) return GSLM_E_INVALID;
  if (o->group != 0 && o->group != 8 && o->group != 16 && o->group != 32) return GSLM_E_INVALID;
  if (o->batch_ctas < 0 || o->batch_ctas > 6) return GSLM_E_INVALID;
  if (o->apply_variant < 0 || o->apply_variant > 10) return GSLM_E_INVALID;
  if (o->line_search < 0 || o->line_search > 60) return GSLM_E_INVALID;
  if (o->objective != GSLM_OBJ_L2 && o->objective != GSLM_OBJ_L1_SSIM) return GSLM_E_INVALID;
  if (!(o->lambda_l1 >= 0.f) || !(o->lambda_ssim >= 0.f) || !(o->res_eps > 0.f) || !std::isfinite(o->lambda_l1) ||
      !std::isfinite(o->lambda_ssim) || !std::isfinite(o->res_eps))
    return GSLM_E_INVALID;
  return GSLM_OK;
}

gslm_status gslm_create(const gslm_options* opt, void* stream, gslm_ctx** out) {
  if (out == nullptr) return GSLM_E_INVALID;
  *out = nullptr;
  gslm_options o;
  if (opt != nullptr) o = *opt;
  else gslm_default_options(&o);
  if (o.group == 0) o.group = 32;
  if (validate_opts(&o) != GSLM_OK) return GSLM_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GSLM_E_CUDA;
  }
  gslm_ctx* c = new gslm_ctx();
  c->opt = o;
  c->st = static_cast<cudaStream_t>(stream);
  c->device = dev;
  // The library allocates stream-ordered from the device's default memory pool.
  // Caches of tens of GB are freed and rebuilt every LM step: keep freed memory
  // in the pool instead of returning it to the driver at every synchronisation.
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  // Look up gslm_apply_JT_noalloc's fixed array here, with the context's device
  // current: the lookup loads the array's module (24 MiB of device memory), so
  // that the allocation-free call itself never does. A failure leaves the
  // address null and that call returns GSLM_E_CUDA.
  void* scratch = nullptr;
  if (noalloc_scratch_address(&scratch) == cudaSuccess) c->noalloc_scratch = scratch;
  cudaGetLastError();
  *out = c;
  return GSLM_OK;
}

void gslm_destroy(gslm_ctx* ctx) {
  if (ctx == nullptr) return;
  cudaStreamSynchronize(ctx->st);
  const int dev = ctx->device;
  delete ctx;
  // hand the pool's cached memory back to the driver
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    cudaStreamSynchronize(nullptr);
    cudaMemPoolTrimTo(pool, 0);
  }
  cudaGetLastError();
}

const char* gslm_last_error(const gslm_ctx* ctx) { return ctx == nullptr ? "null context" : ctx->err.c_str(); }

gslm_status gslm_set_options(gslm_ctx* ctx, const gslm_options* opt) {
  if (ctx == nullptr || opt == nullptr) return GSLM_E_INVALID;
  gslm_options o = *opt;
  if (o.group == 0) o.group = 32;
  if (validate_opts(&o) != GSLM_OK) return fail(ctx, GSLM_E_INVALID, "invalid options");
  ctx->opt = o;
  return GSLM_OK;
}

gslm_status gslm_render(gslm_ctx* ctx, const float* params, int64_t N, int64_t ld, const gslm_camera* cams,
                        int32_t V, float* img, const float* targets, double* cost) {
  CKS(check_vec_args(ctx, N, ld));
  if (params == nullptr || cams == nullptr || img == nullptr || V <= 0)
    return fail(ctx, GSLM_E_INVALID, "render: null argument or V <= 0");
  std::vector<DevCam> hc;
  int n_tiles = 0;
  long long n_pix = 0;
  CKS(make_cams(ctx, cams, V, hc, n_tiles, n_pix));
  Binning B;
  CKS(bin_splats(ctx, params, (int)N, ld, hc, n_tiles, ctx->opt.smooth, B));
  Buf partials;
  CK(partials.alloc(sizeof(double) * n_tiles, ctx->st));
  CK(launch_raster_count(B.cams.as<DevCam>(), V, n_tiles, B.tile_start.as<uint32_t>(), B.tile_end.as<uint32_t>(),
                         B.tile_vals, B.rec.as<SplatRec>(), ctx->opt.smooth, targets, img, nullptr,
                         targets != nullptr ? partials.as<double>() : nullptr, nullptr, nullptr, ctx->st));
  if (targets != nullptr && cost != nullptr && ctx->opt.objective == GSLM_OBJ_L1_SSIM)
    CK(launch_l1ssim(B.cams.as<DevCam>(), V, n_tiles, img, targets, ctx->opt.lambda_l1, ctx->opt.lambda_ssim,
                     ctx->opt.res_eps, nullptr, nullptr, partials.as<double>(), ctx->st));
  if (targets != nullptr && cost != nullptr) CKS(reduce_to_host(ctx, partials.as<double>(), n_tiles, cost));
  return GSLM_OK;
}

// Builds a cache; with copy_params the cache keeps its own copy of the
// parameters, else it reads the caller's, which must then stay unchanged for
// the cache's lifetime (the LM step's caches: it writes the parameters only
// after its last use of them).
static gslm_status build_cache_impl(gslm_ctx* ctx, const float* params, int64_t N, int64_t ld,
                                    const gslm_camera* cams, int32_t V, const float* targets, gslm_cache** out,
                                    float* F, float* b, double* cost, bool copy_params) {
  CKS(check_vec_args(ctx, N, ld));
  if (out == nullptr) return fail(ctx, GSLM_E_INVALID, "build_cache: null cache pointer");
  *out = nullptr;
  if (params == nullptr || cams == nullptr || targets == nullptr || V <= 0)
    return fail(ctx, GSLM_E_INVALID, "build_cache: null argument or V <= 0");
  cudaStream_t st = ctx->st;
  gslm_cache* c = new gslm_cache();
  struct Guard {
    gslm_cache*& c;
    ~Guard() { delete c; }
  } guard{c};
  c->ctx = ctx;
  c->N = (int)N;
  c->ld = ld;
  c->V = V;
  c->smooth = ctx->opt.smooth;
  c->fmt = ctx->opt.cache_fmt;
  const bool thin = c->fmt == GSLM_CACHE_THIN;
  if (thin && c->smooth) return fail(ctx, GSLM_E_INVALID, "build_cache: thin caches are built in the default mode only");
  CKS(make_cams(ctx, cams, V, c->hcams, c->n_tiles, c->n_pix));
  if (copy_params) {
    CK(c->own_params.alloc(sizeof(float) * kNP * (size_t)ld, st));
    CK(cudaMemcpyAsync(c->own_params.p, params, sizeof(float) * kNP * (size_t)ld, cudaMemcpyDeviceToDevice, st));
    c->params = c->own_params.as<float>();
  } else {
    c->params = params;
  }
  params = c->params;
  const int n_tiles = c->n_tiles;
  const long long S = (long long)N * V;
  Binning B;
  CKS(bin_splats(ctx, params, (int)N, ld, c->hcams, n_tiles, c->smooth, B));
  c->n_vis = B.n_vis;
  c->n_keys = B.n_keys;
  // blend + count entries and segments per tile
  Buf img, cost_part, tile_entries, tile_segs, tile_entry_off;
  CK(img.alloc(sizeof(float) * 3 * c->n_pix, st));
  CK(c->F.alloc(sizeof(float) * 3 * c->n_pix, st));
  CK(cost_part.alloc(sizeof(double) * n_tiles, st));
  CK(tile_entries.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
  CK(tile_segs.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
  CK(launch_raster_count(B.cams.as<DevCam>(), V, n_tiles, B.tile_start.as<uint32_t>(), B.tile_end.as<uint32_t>(),
                         B.tile_vals, B.rec.as<SplatRec>(), c->smooth, targets, img.as<float>(), c->F.as<float>(),
                         cost_part.as<double>(), tile_entries.as<uint32_t>(), tile_segs.as<uint32_t>(), st));
  CK(tile_entry_off.alloc(sizeof(unsigned long long) * (n_tiles + 1), st));
  CK(c->tile_seg_off.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
  CK(B.scan_tmp.ensure(scan_temp_bytes(n_tiles + 1), st));
  CK(exclusive_scan_u64(tile_entries.as<uint32_t>(), tile_entry_off.as<unsigned long long>(), n_tiles,
                        B.scan_tmp.p, st));
  CK(exclusive_scan_u32(tile_segs.as<uint32_t>(), c->tile_seg_off.as<uint32_t>(), n_tiles, B.scan_tmp.p, st));
  unsigned long long E = 0;
  uint32_t nseg = 0, nwin = 0;
  CK(cudaMemcpyAsync(&E, tile_entry_off.as<unsigned long long>() + n_tiles, sizeof(E), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&nseg, c->tile_seg_off.as<uint32_t>() + n_tiles, sizeof(nseg), cudaMemcpyDeviceToHost, st));
  if (thin) {
    // checkpoint windows: ceil(segments / 32) per tile
    Buf wcount;
    CK(wcount.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
    CK(c->win_off.alloc(sizeof(uint32_t) * (n_tiles + 1), st));
    CK(launch_thin_window_counts(c->tile_seg_off.as<uint32_t>(), n_tiles, wcount.as<uint32_t>(), st));
    CK(exclusive_scan_u32(wcount.as<uint32_t>(), c->win_off.as<uint32_t>(), n_tiles, B.scan_tmp.p, st));
    CK(cudaMemcpyAsync(&nwin, c->win_off.as<uint32_t>() + n_tiles, sizeof(nwin), cudaMemcpyDeviceToHost, st));
  }
  CKS(reduce_to_host(ctx, cost_part.as<double>(), n_tiles, &c->cost));
  if (ctx->opt.objective == GSLM_OBJ_L1_SSIM) {
    // Eq. gn-loss: F becomes e = sum (dr/dc) r, the weights w = sum (dr/dc)^2 are kept
    CK(c->W.alloc(sizeof(float) * 3 * std::max<long long>(c->n_pix, 1), st));
    CK(launch_l1ssim(B.cams.as<DevCam>(), V, n_tiles, img.as<float>(), targets, ctx->opt.lambda_l1,
                     ctx->opt.lambda_ssim, ctx->opt.res_eps, c->F.as<float>(), c->W.as<float>(),
                     cost_part.as<double>(), st));
    CKS(reduce_to_host(ctx, cost_part.as<double>(), n_tiles, &c->cost));
  }
  c->n_entries = (long long)E;
  c->n_seg = nseg;
  c->n_win = nwin;
  const size_t need = (thin ? (size_t)nseg * sizeof(SplatRec) + (size_t)nwin * kTilePix * 16 +
                                  (size_t)n_tiles * kTilePix * 4 + 12 * (size_t)c->n_pix
                            : E * (payload_bytes(c->fmt) + 1)) +
                      (size_t)nseg * (8 + 4 + 4 + 48 + 4 * (c->fmt == 2)) + (size_t)S * (sizeof(SplatRec) + 1 + 8);
  if (ctx->opt.mem_budget != 0 && need > ctx->opt.mem_budget) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "cache needs %zu bytes (%llu entries), budget %zu", need, E,
                  ctx->opt.mem_budget);
    return fail(ctx, GSLM_E_CACHE_OVERFLOW, msg);
  }
  const long long ns = std::max<long long>(nseg, 1);
  ThinOut tout{};
  if (thin) {
    // no entries: the segments' splats, per-pixel live counts and checkpoints
    CK(c->thin_rec.alloc(sizeof(SplatRec) * ns, st));
    CK(c->ckpt.alloc((size_t)std::max<uint32_t>(nwin, 1) * kTilePix * sizeof(float4), st));
    CK(c->n_live.alloc((size_t)std::max(n_tiles, 1) * kTilePix * sizeof(uint32_t), st));
    CK(c->win_tile.alloc(sizeof(uint32_t) * std::max<uint32_t>(nwin, 1), st));
    CK(launch_thin_window_tiles(c->win_off.as<uint32_t>(), n_tiles, c->win_tile.as<uint32_t>(), st));
    tout.rec = c->thin_rec.as<SplatRec>();
    tout.ckpt = c->ckpt.as<float4>();
    tout.win_off = c->win_off.as<uint32_t>();
    tout.n_live = c->n_live.as<uint32_t>();
  }
  // 32 bytes of slack: the tile kernels' L2 prefetches cover whole 16-byte
  // blocks around a segment's entries, up to 15 bytes past the last entry
  CK(c->payload.alloc(thin ? 16 : payload_bytes(c->fmt) * std::max<unsigned long long>(E, 1) + 32, st));
  CK(c->pixoff.alloc(thin ? 16 : std::max<unsigned long long>(E, 1) + 32, st));
  CK(c->seg_entry_off.alloc(sizeof(unsigned long long) * (ns + 1), st));
  CK(c->seg_slot.alloc(sizeof(uint32_t) * ns, st));
  CK(c->seg_rec.alloc(sizeof(SegRec) * ns, st));
  if (c->fmt == GSLM_CACHE_FP16S) CK(c->seg_scale.alloc(sizeof(float) * ns, st));
  CK(c->slot_active.alloc(std::max<long long>(S, 1), st));
  CK(cudaMemsetAsync(c->slot_active.p, 0, std::max<long long>(S, 1), st));
  Buf errflag;
  CK(errflag.alloc(sizeof(int), st));
  CK(cudaMemsetAsync(errflag.p, 0, sizeof(int), st));
  CK(launch_raster_write(B.cams.as<DevCam>(), V, n_tiles, B.tile_start.as<uint32_t>(), B.tile_end.as<uint32_t>(),
                         B.tile_vals, B.rec.as<SplatRec>(), c->smooth, img.as<float>(),
                         tile_entry_off.as<unsigned long long>(), c->tile_seg_off.as<uint32_t>(), c->fmt,
                         c->payload.p, c->seg_scale.as<float>(), c->pixoff.as<uint8_t>(),
                         c->seg_entry_off.as<unsigned long long>(), c->seg_slot.as<uint32_t>(),
                         c->seg_rec.as<SegRec>(), c->slot_active.as<uint8_t>(), errflag.as<int>(), tout, st));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, errflag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr != 0) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "cache write disagreed with the counting pass (flags %d)", herr);
    return fail(ctx, GSLM_E_NUMERIC, msg);
  }
  CK(cudaMemcpyAsync(c->seg_entry_off.as<unsigned long long>() + nseg, &E, sizeof(E), cudaMemcpyHostToDevice, st));
  if (V <= 64) {
    CK(c->vmask.alloc(sizeof(unsigned long long) * (size_t)N, st));
    CK(launch_view_mask(c->slot_active.as<uint8_t>(), (int)N, V, c->vmask.as<unsigned long long>(), st));
  }
  {
    Buf cnt;
    CK(cnt.alloc(sizeof(unsigned long long), st));
    CK(launch_count_nonzero_u8(c->slot_active.as<uint8_t>(), S, cnt.as<unsigned long long>(), st));
    unsigned long long na = 0;
    CK(cudaMemcpyAsync(&na, cnt.p, sizeof(na), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->n_active = (long long)na;
  }
  if (c->vmask.p != nullptr) c->slot_active.release();   // the view masks replace the per-slot flags
  // Segments ordered by splat (the paper's sortCacheByGaussians, on segments).
  // With the view masks the splat key is the compact splat index (act_off from
  // the masks; SegRec.slot rewritten to it): Gaussian-major, so a Gaussian's
  // segments of all its views are one contiguous run. Else the slot v * N + g.
  {
    Buf ka, va, kb, vb, tmp;
    CK(ka.alloc(sizeof(uint32_t) * ns, st));
    CK(va.alloc(sizeof(uint32_t) * ns, st));
    CK(kb.alloc(sizeof(uint32_t) * ns, st));
    CK(vb.alloc(sizeof(uint32_t) * ns, st));
    long long n_keys = S;
    if (c->vmask.p != nullptr) {
      CK(c->act_off.alloc(sizeof(uint32_t) * ((size_t)N + 1), st));
      CK(tmp.alloc(sizeof(uint32_t) * ((size_t)N + 1) + 64 + scan_temp_bytes((long long)N + 1), st));
      CK(launch_compact_splats(c->vmask.as<unsigned long long>(), (int)N, c->act_off.as<uint32_t>(), tmp.p,
                               c->seg_slot.as<uint32_t>(), c->n_seg, c->seg_rec.as<SegRec>(), ka.as<uint32_t>(),
                               st));
      n_keys = c->n_active;
    } else {
      CK(cudaMemcpyAsync(ka.p, c->seg_slot.p, sizeof(uint32_t) * nseg, cudaMemcpyDeviceToDevice, st));
    }
    c->seg_slot.release();   // the segment records hold the splat key
    CK(tmp.ensure(radix_temp_bytes(ns), st));
    CK(launch_iota_u32(va.as<uint32_t>(), nseg, st));
    uint32_t *sk = nullptr, *sv = nullptr;
    CK(radix_sort_pairs(ka.as<uint32_t>(), va.as<uint32_t>(), kb.as<uint32_t>(), vb.as<uint32_t>(), nseg,
                        bits_for((unsigned long long)n_keys), tmp.p, &sk, &sv, st));
    const long long nr = std::max<long long>(n_keys, 1);
    CK(c->slot_seg_start.alloc(sizeof(uint32_t) * nr, st));
    CK(c->slot_seg_end.alloc(sizeof(uint32_t) * nr, st));
    CK(cudaMemsetAsync(c->slot_seg_start.p, 0, sizeof(uint32_t) * nr, st));
    CK(cudaMemsetAsync(c->slot_seg_end.p, 0, sizeof(uint32_t) * nr, st));
    CK(launch_ranges(sk, nseg, c->slot_seg_start.as<uint32_t>(), c->slot_seg_end.as<uint32_t>(), st));
    CK(c->slot_seg_list.alloc(sizeof(uint32_t) * ns, st));
    CK(cudaMemcpyAsync(c->slot_seg_list.p, sv, sizeof(uint32_t) * nseg, cudaMemcpyDeviceToDevice, st));
    CK(c->seg_pos.alloc(sizeof(uint32_t) * ns, st));
    CK(launch_scatter_index_u32(sv, nseg, c->seg_pos.as<uint32_t>(), st));
  }
  // keep the cameras; drop the per-slot splat records (the segment records
  // hold what the kernels need) and the binning buffers
  c->cams.p = B.cams.p;
  c->cams.bytes = B.cams.bytes;
  c->cams.st = st;
  B.cams.p = nullptr;
  if (thin) {   // a thin cache keeps the rendered image (each pixel's final colour)
    c->img.p = img.p;
    c->img.bytes = img.bytes;
    c->img.st = img.st;
    img.p = nullptr;
    img.bytes = 0;
  }
  // b = -J^T F
  if (b != nullptr) CKS(do_apply_JT(ctx, c, c->F.as<float>(), b, -1.f, nullptr, nullptr, 0.f, nullptr, nullptr));
  if (F != nullptr)
    CK(cudaMemcpyAsync(F, c->F.p, sizeof(float) * 3 * c->n_pix, cudaMemcpyDeviceToDevice, st));
  if (cost != nullptr) *cost = c->cost;
  *out = c;
  c = nullptr;   // release from the guard
  return GSLM_OK;
}

gslm_status gslm_build_cache(gslm_ctx* ctx, const float* params, int64_t N, int64_t ld, const gslm_camera* cams,
                             int32_t V, const float* targets, gslm_cache** out, float* F, float* b, double* cost) {
  // the public cache keeps its own copy of the parameters it linearises around
  return build_cache_impl(ctx, params, N, ld, cams, V, targets, out, F, b, cost, true);
}

gslm_status gslm_cache_stats(const gslm_cache* c, gslm_cache_info* info) {
  if (c == nullptr || info == nullptr) return GSLM_E_INVALID;
  info->entries = c->n_entries;
  info->segments = c->n_seg;
  info->splats = c->n_vis;
  info->keys = c->n_keys;
  info->bytes = (int64_t)c->device_bytes();
  info->pixels = c->n_pix;
  info->views = c->V;
  info->cache_fmt = c->fmt;
  info->active_splats = c->n_active;
  return GSLM_OK;
}

gslm_status gslm_cache_weights(const gslm_cache* c, float* w) {
  if (c == nullptr || w == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = c->ctx;
  const long long n = 3 * c->n_pix;
  if (c->W.p != nullptr) CK(cudaMemcpyAsync(w, c->W.p, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->st));
  else CK(launch_fill_f32(n, 1.f, w, ctx->st));
  return GSLM_OK;
}

void gslm_cache_free(gslm_cache* c) { delete c; }

gslm_status gslm_apply_J(gslm_ctx* ctx, const gslm_cache* c, const float* p, float* u) {
  if (ctx == nullptr || c == nullptr || p == nullptr || u == nullptr) return fail(ctx, GSLM_E_INVALID, "apply_J: null");
  return do_apply_J(ctx, c, p, u, nullptr, nullptr, nullptr, nullptr, nullptr);
}

gslm_status gslm_apply_JT(gslm_ctx* ctx, const gslm_cache* c, const float* u, float* g) {
  if (ctx == nullptr || c == nullptr || u == nullptr || g == nullptr) return fail(ctx, GSLM_E_INVALID, "apply_JT: null");
  return do_apply_JT(ctx, c, u, g, 1.f, nullptr, nullptr, 0.f, nullptr, nullptr);
}

gslm_status gslm_jacobi_diag(gslm_ctx* ctx, const gslm_cache* c, float* diag) {
  if (ctx == nullptr || c == nullptr || diag == nullptr) return fail(ctx, GSLM_E_INVALID, "jacobi_diag: null");
  cudaStream_t st = ctx->st;
  CK(ctx->seg_q.ensure(sizeof(float) * kDiagBlock * std::max<long long>(c->n_seg, 1), st));
  if (c->fmt == GSLM_CACHE_THIN) CK(launch_thin_diag(c->view(), ctx->seg_q.as<float>(), st));
  else CK(launch_diag_entries(c->view(), ctx->seg_q.as<float>(), st));
  // with compact splat keys, one block per splat first (segments summed in splat order)
  float* splat_q = nullptr;
  Buf sq;
  if (c->act_off.p != nullptr) {
    CK(sq.alloc(sizeof(float) * kDiagBlock * std::max<long long>(c->n_active, 1), st));
    splat_q = sq.as<float>();
    CK(launch_splat_sum_q(c->n_active, c->slot_seg_start.as<uint32_t>(), c->slot_seg_end.as<uint32_t>(),
                          ctx->seg_q.as<float>(), splat_q, st));
  }
  CK(launch_diag(c->params, c->N, c->ld, c->cams.as<DevCam>(), c->V, c->smooth, c->slot_seg_start.as<uint32_t>(),
                 c->slot_seg_end.as<uint32_t>(), c->vmask.as<unsigned long long>(), c->act_off.as<uint32_t>(),
                 ctx->seg_q.as<float>(), splat_q, diag, st));
  return GSLM_OK;
}

gslm_status gslm_pcg_solve(gslm_ctx* ctx, const gslm_cache* c, const float* b, const float* diag, const float* D,
                           float lambda, float* x, gslm_pcg_stats* stats) {
  if (ctx == nullptr || c == nullptr || b == nullptr || diag == nullptr || x == nullptr)
    return fail(ctx, GSLM_E_INVALID, "pcg_solve: null");
  // the vector kernels move float4s
  for (const void* v : {(const void*)b, (const void*)diag, (const void*)D, (const void*)x})
    if ((reinterpret_cast<uintptr_t>(v) & 15u) != 0) return fail(ctx, GSLM_E_INVALID, "pcg_solve: vector not 16-byte aligned");
  CKS(pcg_enqueue(ctx, c, b, diag, D, lambda, x));
  if (stats != nullptr) {
    PcgScalars h;
    CK(cudaMemcpyAsync(&h, ctx->scalars.p, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    stats->iters = h.iters;
    stats->breakdown = h.breakdown;
    stats->rr = h.rr;
    stats->bb = h.bb;
    if (h.breakdown) return GSLM_W_PCG_BREAKDOWN;
  }
  return GSLM_OK;
}

gslm_status gslm_pcg_solve_batch(gslm_ctx* ctx, const gslm_cache* const* caches, int32_t n_b, const float* const* b,
                                 const float* const* diag, const float* const* D, float lambda, float* const* x,
                                 gslm_pcg_stats* stats) {
  if (ctx == nullptr) return GSLM_E_INVALID;
  if (caches == nullptr || b == nullptr || diag == nullptr || x == nullptr || n_b < 1)
    return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: null argument or no subsets");
  for (int i = 0; i < n_b; ++i)
    if (caches[i] == nullptr || b[i] == nullptr || diag[i] == nullptr || x[i] == nullptr)
      return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: null entry");
  cudaStream_t st = ctx->st;
  bool breakdown = false;
  if (caches[0]->fmt == GSLM_CACHE_THIN) {
    // thin caches: the subsets one after another, with the arithmetic of gslm_pcg_solve
    for (int i = 0; i < n_b; ++i) {
      if (caches[i]->fmt != GSLM_CACHE_THIN) return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: mixed cache formats");
      for (const void* v : {(const void*)b[i], (const void*)diag[i], (const void*)x[i]})
        if ((reinterpret_cast<uintptr_t>(v) & 15u) != 0)
          return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: vector not 16-byte aligned");
      CKS(pcg_enqueue(ctx, caches[i], b[i], diag[i], D != nullptr ? D[i] : nullptr, lambda, x[i]));
      PcgScalars h;
      CK(cudaMemcpyAsync(&h, ctx->scalars.p, sizeof(h), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      breakdown |= h.breakdown != 0;
      if (stats != nullptr) {
        stats[i].iters = h.iters;
        stats[i].breakdown = h.breakdown;
        stats[i].rr = h.rr;
        stats[i].bb = h.bb;
      }
    }
    return breakdown ? GSLM_W_PCG_BREAKDOWN : GSLM_OK;
  }
  for (int g0 = 0; g0 < n_b; g0 += kMaxBatch) {
    const int gn = std::min(kMaxBatch, n_b - g0);
    BatchLayout L;
    CKS(batch_layout(ctx, caches + g0, gn, &L));
    if (caches[g0]->N != caches[0]->N || caches[g0]->ld != caches[0]->ld)
      return fail(ctx, GSLM_E_INVALID, "pcg_solve_batch: caches differ in N or ld");
    unsigned mask = 0;
    for (int k = 0; k < gn; ++k)
      if (D != nullptr && D[g0 + k] != nullptr) mask |= 1u << k;
    CKS(batch_alloc(ctx, L, mask, 0));
    const size_t vb = sizeof(float) * (size_t)L.vs;
    for (int k = 0; k < gn; ++k) {
      const int i = g0 + k;
      CK(cudaMemcpyAsync(ctx->bt_b.as<float>() + k * L.vs, b[i], vb, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ctx->bt_M.as<float>() + k * L.vs, diag[i], vb, cudaMemcpyDeviceToDevice, st));
      if ((mask >> k) & 1u)
        CK(cudaMemcpyAsync(ctx->bt_D.as<float>() + k * L.vs, D[i], vb, cudaMemcpyDeviceToDevice, st));
    }
    CKS(pcg_batch_run(ctx, caches + g0, L, mask, lambda));
    for (int k = 0; k < gn; ++k)
      CK(cudaMemcpyAsync(x[g0 + k], ctx->bt_x.as<float>() + k * L.vs, vb, cudaMemcpyDeviceToDevice, st));
    std::vector<PcgScalars> h(gn);
    CK(cudaMemcpyAsync(h.data(), ctx->bt_sc.p, sizeof(PcgScalars) * gn, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < gn; ++k) {
      breakdown |= h[k].breakdown != 0;
      if (stats != nullptr) {
        stats[g0 + k].iters = h[k].iters;
        stats[g0 + k].breakdown = h[k].breakdown;
        stats[g0 + k].rr = h[k].rr;
        stats[g0 + k].bb = h[k].bb;
      }
    }
  }
  return breakdown ? GSLM_W_PCG_BREAKDOWN : GSLM_OK;
}

gslm_status gslm_combine_accumulate(gslm_ctx* ctx, int64_t N, int64_t ld, const float* d, const float* m, float* num,
                                    float* den) {
  CKS(check_vec_args(ctx, N, ld));
  if (d == nullptr || m == nullptr || num == nullptr || den == nullptr) return fail(ctx, GSLM_E_INVALID, "combine: null");
  CK(launch_combine_acc((int)N, ld, d, m, num, den, ctx->st));
  return GSLM_OK;
}

gslm_status gslm_combine_finish(gslm_ctx* ctx, int64_t N, int64_t ld, const float* num, const float* den,
                                float* delta) {
  CKS(check_vec_args(ctx, N, ld));
  if (num == nullptr || den == nullptr || delta == nullptr) return fail(ctx, GSLM_E_INVALID, "combine: null");
  CK(launch_combine_finish((int)N, ld, num, den, delta, ctx->st));
  return GSLM_OK;
}

gslm_status gslm_set_precond(gslm_ctx* ctx, gslm_precond* pc) {
  if (ctx == nullptr) return GSLM_E_INVALID;
  ctx->pc = pc;
  return GSLM_OK;
}

gslm_status gslm_lm_step(gslm_ctx* ctx, float* params, int64_t N, int64_t ld, const gslm_camera* cams,
                         int32_t n_cams, const float* targets, const int32_t* subset_views,
                         const int32_t* subset_off, int32_t n_b, const float* const* precond, gslm_lm_state* state,
                         gslm_lm_stats* stats) {
  CKS(check_vec_args(ctx, N, ld));
  if (params == nullptr || cams == nullptr || targets == nullptr || subset_views == nullptr ||
      subset_off == nullptr || n_b <= 0 || state == nullptr)
    return fail(ctx, GSLM_E_INVALID, "lm_step: null argument");
  if (precond != nullptr)
    for (int i = 0; i < n_b; ++i)
      if ((reinterpret_cast<uintptr_t>(precond[i]) & 15u) != 0)
        return fail(ctx, GSLM_E_INVALID, "lm_step: preconditioner not 16-byte aligned");
  cudaStream_t st = ctx->st;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  CK(cudaEventRecord(ev0, st));
  // camera pixel offsets inside `targets`
  std::vector<long long> cam_pix(n_cams + 1, 0);
  for (int i = 0; i < n_cams; ++i) cam_pix[i + 1] = cam_pix[i] + (long long)cams[i].width * cams[i].height;
  const size_t vb = sizeof(float) * kNP * (size_t)ld;
  CK(ctx->lm_num.ensure(vb, st));
  CK(ctx->lm_den.ensure(vb, st));
  CK(ctx->lm_delta.ensure(vb, st));
  CK(ctx->lm_trial.ensure(vb, st));
  // thin caches have no persistent batched tile kernels: their subsets are solved one after another
  const bool batched = ctx->opt.batch != 0 && ctx->opt.cache_fmt != GSLM_CACHE_THIN;
  if (!batched) {
    CK(ctx->lm_x.ensure(vb, st));
    CK(ctx->lm_b.ensure(vb, st));
    CK(ctx->lm_M.ensure(vb, st));
  }
  CK(cudaMemsetAsync(ctx->lm_num.p, 0, vb, st));
  CK(cudaMemsetAsync(ctx->lm_den.p, 0, vb, st));
  std::vector<gslm_cache*> caches(n_b, nullptr);
  struct CacheGuard {
    std::vector<gslm_cache*>& v;
    ~CacheGuard() {
      for (auto* c : v) delete c;
    }
  } cg{caches};
  std::vector<std::vector<gslm_camera>> scams(n_b);
  std::vector<std::vector<int>> sviews(n_b);
  // the targets of the first nv views of subset i, made contiguous in lm_tgt
  auto stage_targets = [&](int i, int nv) -> gslm_status {
    long long pix = 0;
    for (int q = 0; q < nv; ++q) pix += cam_pix[sviews[i][q] + 1] - cam_pix[sviews[i][q]];
    CK(ctx->lm_tgt.ensure(sizeof(float) * 3 * std::max<long long>(pix, 1), st));
    long long o = 0;
    for (int q = 0; q < nv; ++q) {
      const int v = sviews[i][q];
      const long long np = cam_pix[v + 1] - cam_pix[v];
      CK(cudaMemcpyAsync(ctx->lm_tgt.as<float>() + 3 * o, targets + 3 * cam_pix[v], sizeof(float) * 3 * np,
                         cudaMemcpyDeviceToDevice, st));
      o += np;
    }
    return GSLM_OK;
  };
  double cost0 = 0.0, pair_bytes = 0.0;
  int pcg_iters = 0, n_pairs = 0, seq_groups = 0;
  long long segs = 0, actives = 0;
  ctx->timer.on = ctx->opt.profile != 0;
  ctx->timer.st = st;
  struct TimerOff {
    PhaseTimer& t;
    ~TimerOff() { t.on = false; t.open_phase = -1; }
  } toff{ctx->timer};
  long long entries = 0, bytes = 0;
  const float lambda = state->lambda;
  const long long vsn = (long long)kNP * ld;
  std::vector<long long> spix(n_b, 0);
  for (int i = 0; i < n_b; ++i) {
    const int a = subset_off[i], e = subset_off[i + 1];
    if (e <= a) return fail(ctx, GSLM_E_INVALID, "lm_step: empty subset");
    for (int q = a; q < e; ++q) {
      const int v = subset_views[q];
      if (v < 0 || v >= n_cams) return fail(ctx, GSLM_E_INVALID, "lm_step: bad camera index");
      scams[i].push_back(cams[v]);
      sviews[i].push_back(v);
      spix[i] += cam_pix[v + 1] - cam_pix[v];
    }
  }
  for (int g0 = 0; g0 < n_b; g0 += batched ? kMaxBatch : 1) {
    const int gn = batched ? std::min(kMaxBatch, n_b - g0) : 1;
    if (batched) {
      CK(ctx->bt_b.ensure(vb * gn, st));
      CK(ctx->bt_M.ensure(vb * gn, st));
      if (precond != nullptr || ctx->pc != nullptr) CK(ctx->bt_D.ensure(vb * gn, st));
    }
    // A group's caches are built largest first: each build's transient buffers
    // then come when the fewest caches are resident, and the memory pool reuses
    // the large blocks they leave for the smaller caches that follow.
    std::vector<int> order(gn);
    for (int k = 0; k < gn; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return spix[g0 + x] > spix[g0 + y]; });
    unsigned dmask = 0;
    for (int kk = 0; kk < gn; ++kk) {
      const int k = order[kk];
      const int i = g0 + k;
      CKS(stage_targets(i, (int)sviews[i].size()));
      float* bi = batched ? ctx->bt_b.as<float>() + k * vsn : ctx->lm_b.as<float>();
      float* Mi = batched ? ctx->bt_M.as<float>() + k * vsn : ctx->lm_M.as<float>();
      double ci = 0.0;
      bool t = ctx->timer.begin(PH_BUILD);
      CKS(build_cache_impl(ctx, params, N, ld, scams[i].data(), (int)scams[i].size(), ctx->lm_tgt.as<float>(),
                           &caches[i], nullptr, bi, &ci, false));
      ctx->timer.end(t);
      cost0 += ci;
      entries += caches[i]->n_entries;
      segs += caches[i]->n_seg;
      actives += caches[i]->n_active;
      bytes += (long long)caches[i]->device_bytes();
      t = ctx->timer.begin(PH_DIAG);
      CKS(gslm_jacobi_diag(ctx, caches[i], Mi));
      ctx->timer.end(t);
      const float* D = precond != nullptr ? precond[i] : nullptr;
      float* Dslot = batched ? ctx->bt_D.as<float>() + k * vsn : nullptr;
      if (D == nullptr && ctx->pc != nullptr) {
        if (!batched) CK(ctx->lm_D.ensure(vb, st));
        float* Dout = batched ? Dslot : ctx->lm_D.as<float>();
        CKS(precond_for_cache(ctx->pc, ctx, caches[i], Mi, Dout));
        D = Dout;
      } else if (D != nullptr && batched) {
        CK(cudaMemcpyAsync(Dslot, D, vb, cudaMemcpyDeviceToDevice, st));
      }
      if (D != nullptr) dmask |= 1u << k;
      if (batched) continue;
      CKS(pcg_enqueue(ctx, caches[i], bi, Mi, D, lambda, ctx->lm_x.as<float>()));
      PcgScalars h;
      CK(cudaMemcpyAsync(&h, ctx->scalars.p, sizeof(h), cudaMemcpyDeviceToHost, st));
      CK(launch_combine_acc((int)N, ld, ctx->lm_x.as<float>(), Mi, ctx->lm_num.as<float>(), ctx->lm_den.as<float>(),
                            st));
      CK(cudaStreamSynchronize(st));
      pcg_iters += h.iters;
      const gslm_cache* c = caches[i];
      n_pairs += 1 + h.iters;
      pair_bytes += (1.0 + h.iters) * c->pair_bytes((int)N);
    }
    if (!batched) continue;
    BatchLayout L;
    CKS(batch_layout(ctx, caches.data() + g0, gn, &L));
    const gslm_status sa = batch_alloc(ctx, L, dmask, ctx->opt.batch_mem);
    std::vector<PcgScalars> h(gn);
    if (sa == GSLM_E_OOM) {
      // The stacked vectors of the group do not fit beside its caches: solve
      // the subsets one after another with one set of scratch vectors.
      for (Buf* bf : {&ctx->bt_x, &ctx->bt_z, &ctx->bt_p, &ctx->bt_g, &ctx->bt_u, &ctx->bt_ydot, &ctx->bt_segy})
        bf->release();
      ctx->err.clear();
      ++seq_groups;
      CK(ctx->lm_x.ensure(vb, st));
      for (int k = 0; k < gn; ++k) {
        float* Mk = ctx->bt_M.as<float>() + k * vsn;
        const float* Dk = ((dmask >> k) & 1u) ? ctx->bt_D.as<float>() + k * vsn : nullptr;
        CKS(pcg_enqueue(ctx, caches[g0 + k], ctx->bt_b.as<float>() + k * vsn, Mk, Dk, lambda,
                        ctx->lm_x.as<float>()));
        CK(cudaMemcpyAsync(&h[k], ctx->scalars.p, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CK(launch_combine_acc((int)N, ld, ctx->lm_x.as<float>(), Mk, ctx->lm_num.as<float>(),
                              ctx->lm_den.as<float>(), st));
      }
    } else {
      CKS(sa);
      CKS(pcg_batch_run(ctx, caches.data() + g0, L, dmask, lambda));
      CK(cudaMemcpyAsync(h.data(), ctx->bt_sc.p, sizeof(PcgScalars) * gn, cudaMemcpyDeviceToHost, st));
      for (int k = 0; k < gn; ++k)
        CK(launch_combine_acc((int)N, ld, ctx->bt_x.as<float>() + k * vsn, ctx->bt_M.as<float>() + k * vsn,
                              ctx->lm_num.as<float>(), ctx->lm_den.as<float>(), st));
    }
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < gn; ++k) {
      const gslm_cache* c = caches[g0 + k];
      pcg_iters += h[k].iters;
      n_pairs += 1 + h[k].iters;
      pair_bytes += (1.0 + h[k].iters) * c->pair_bytes((int)N);
    }
    // back to the pool (which keeps them for the next step): the trial renders
    // below need room beside the caches
    for (Buf* bf : {&ctx->bt_b, &ctx->bt_M, &ctx->bt_D, &ctx->bt_x, &ctx->bt_z, &ctx->bt_p, &ctx->bt_g, &ctx->bt_u,
                    &ctx->bt_ydot, &ctx->bt_segy})
      bf->release();
  }
  CK(launch_combine_finish((int)N, ld, ctx->lm_num.as<float>(), ctx->lm_den.as<float>(), ctx->lm_delta.as<float>(),
                           st));
  // predicted cost at any step scale gamma, the Gauss-Newton model
  // cost0 + gamma B + gamma^2 A with u_i = (dc/dx)_i Delta, B = 2 sum_i e_i.u_i and
  // A = sum_i w_i.u_i^2 (for L2, e = F and w = 1: sum_i ||gamma u_i + F_i||^2)
  bool trho = ctx->timer.begin(PH_RHO);
  double pA = 0.0, pB = 0.0;
  for (int i = 0; i < n_b; ++i) {
    gslm_cache* c = caches[i];
    CK(ctx->partials.ensure(sizeof(double) * 2 * std::max(c->n_tiles, 1), st));
    CKS(do_apply_J(ctx, c, ctx->lm_delta.as<float>(), nullptr, nullptr, nullptr, nullptr, c->F.as<float>(),
                   ctx->partials.as<double>()));
    double a = 0.0, eu = 0.0;
    CKS(reduce_to_host(ctx, ctx->partials.as<double>(), c->n_tiles, &eu));
    CKS(reduce_to_host(ctx, ctx->partials.as<double>() + c->n_tiles, c->n_tiles, &a));
    pB += 2.0 * eu;
    pA += a;
  }
  // the trial render of params + g Delta over the first nv[i] views of every
  // subset i; +inf when the trial splats exceed the renderer's tile-key capacity
  // (counted in trial_overflows)
  int trial_overflows = 0;
  auto trial_cost = [&](double g, const std::vector<int>& nv, double* out) -> gslm_status {
    CK(launch_axpy_params((int)N, ld, params, (float)g, ctx->lm_delta.as<float>(), ctx->lm_trial.as<float>(), st));
    double e = 0.0;
    for (int i = 0; i < n_b; ++i) {
      if (nv[i] == 0) continue;
      long long pix = 0;
      for (int k = 0; k < nv[i]; ++k) pix += (long long)scams[i][k].width * scams[i][k].height;
      CK(ctx->lm_img.ensure(sizeof(float) * 3 * std::max<long long>(pix, 1), st));
      CKS(stage_targets(i, nv[i]));
      double ci = 0.0;
      const gslm_status rs = gslm_render(ctx, ctx->lm_trial.as<float>(), N, ld, scams[i].data(), nv[i],
                                         ctx->lm_img.as<float>(), ctx->lm_tgt.as<float>(), &ci);
      if (rs == GSLM_E_CACHE_OVERFLOW) {
        ++trial_overflows;
        ctx->err.clear();
        *out = INFINITY;
        return GSLM_OK;
      }
      CKS(rs);
      e += ci;
    }
    *out = e;
    return GSLM_OK;
  };
  // Eq. line-search: gamma = 1, 1/2, ... on the first 30% of the step's views
  // (in subset order), stopping at the first cost above the previous finite one
  double gamma = 1.0;
  int ls_evals = 0;
  if (ctx->opt.line_search > 0) {
    long long total = 0;
    for (int i = 0; i < n_b; ++i) total += (long long)scams[i].size();
    long long left = (long long)std::ceil(0.3 * (double)total);
    std::vector<int> nv(n_b, 0);
    for (int i = 0; i < n_b; ++i) {
      nv[i] = (int)std::min<long long>((long long)scams[i].size(), std::max<long long>(left, 0));
      left -= nv[i];
    }
    double best = INFINITY, prev = INFINITY;
    for (int k = 0; k < ctx->opt.line_search; ++k) {
      const double g = std::ldexp(1.0, -k);
      double e = 0.0;
      CKS(trial_cost(g, nv, &e));
      ++ls_evals;
      if (e < best) {
        best = e;
        gamma = g;
      }
      if (std::isfinite(prev) && e > prev) break;
      prev = e;
    }
  }
  const double pred = cost0 + gamma * pB + gamma * gamma * pA;
  // actual: ||F(x + gamma Delta)||^2 over all views of the step
  double cost1 = 0.0;
  {
    std::vector<int> all(n_b);
    for (int i = 0; i < n_b; ++i) all[i] = (int)scams[i].size();
    CKS(trial_cost(gamma, all, &cost1));
  }
  ctx->timer.end(trho);
  const double den = cost0 - pred;
  const double rho = den > 0.0 ? (cost0 - cost1) / den : -INFINITY;
  const bool accept = den > 0.0 && rho > 1e-5;
  double lam = state->lambda;
  if (accept) {   // lm_trial holds params + gamma Delta
    CK(cudaMemcpyAsync(params, ctx->lm_trial.p, vb, cudaMemcpyDeviceToDevice, st));
    lam *= 1.0 - std::pow(2.0 * rho - 1.0, 3.0);
  } else {
    lam *= 2.0;
  }
  lam = std::min<double>(std::max<double>(lam, ctx->opt.lambda_min), ctx->opt.lambda_max);
  state->lambda = (float)lam;
  state->step += 1;
  CK(cudaEventRecord(ev1, st));
  CK(cudaEventSynchronize(ev1));
  if (stats != nullptr) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    stats->cost = cost0;
    stats->cost_new = cost1;
    stats->predicted = pred;
    stats->rho = rho;
    stats->accepted = accept ? 1 : 0;
    stats->pcg_iters = pcg_iters;
    stats->cache_entries = entries;
    stats->cache_bytes = bytes;
    stats->ms_total = ms;
    for (int k = 0; k < 8; ++k) stats->ms_phase[k] = 0.0;
    ctx->timer.collect(stats->ms_phase, 8);
    stats->n_pairs = n_pairs;
    stats->trial_overflows = trial_overflows;
    stats->pair_bytes = pair_bytes;
    stats->cache_segments = segs;
    stats->active_splats = actives;
    stats->gamma = gamma;
    stats->ls_evals = ls_evals;
    stats->seq_groups = seq_groups;
  } else {
    double dummy[8] = {0};
    ctx->timer.collect(dummy, 8);
  }
  return GSLM_OK;
}

}  // extern "C"
