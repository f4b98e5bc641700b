// Internal declarations shared by the CUDA translation units of libgslm.
// Everything here is private to the library; the public ABI is include/gslm.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "gslm.h"

namespace gslm {

// Rasterizer constants. The paper (Sec. 3.1) uses the 3DGS rasterizer without
// stating its constants; these are the values this library adopts.
constexpr int kTile = 16;                   // 16 x 16 pixel tiles
constexpr int kTilePix = kTile * kTile;     // one thread per pixel in the tile kernels
constexpr float kDilation = 0.3f;           // added to the 2D covariance diagonal
constexpr float kNear = 0.2f;               // visible only if camera-space z > kNear
constexpr float kRadiusSigmas = 3.0f;       // splat radius in standard deviations
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kShOffset = 0.5f;
constexpr int kNP = 59;                     // parameters per Gaussian
constexpr int kDiagBlock = 44;              // floats per segment block of diag(J^T J) (42 used)
// Bounds applied to diag(J^T J) where it serves as the Jacobi preconditioner and
// as the LM damping term (the Levenberg-Marquardt diagonal bounds of Ceres, whose
// LM implementation the paper follows, Sec. 3.2). Subset weights use the raw diagonal.
constexpr float kDiagMin = 1e-6f;
constexpr float kDiagMax = 1e32f;
__host__ __device__ __forceinline__ float clamp_diag(float m) { return fminf(fmaxf(m, kDiagMin), kDiagMax); }

// Tile culling. A splat's tile rectangle (radius 3 sigma) holds tiles where its
// alpha stays below 1/255 at every pixel, which blending skips pixel by pixel.
// For rectangles of at most kCullMaxTiles tiles the projection tests each tile
// and keeps a mask of the tiles the splat can reach; only those get a tile key.
// The test is conservative (it keeps a tile unless the splat provably misses
// every pixel centre in it), so blending sees the same contributions.
constexpr int kCullMaxTiles = 64;
// Whether alpha = o exp(-q/2), q = A dx^2 + 2 B dx dy + C dy^2 with (dx, dy) =
// pixel centre - (mx, my), can reach 1/255 at a pixel centre of tile (tx, ty):
// the least q over the box of the tile's pixel centres (0 if the mean is in the
// box, else its least value on the four edges, each a 1-D quadratic) against
// 2 ln(255 o), with margins far above float32 rounding.
__device__ __forceinline__ bool tile_reachable(float mx, float my, float A, float B, float C, float o, int tx,
                                               int ty) {
  if (!(A > 0.f) || !(C > 0.f) || !(o > 0.f)) return true;
  const float t = 2.f * logf(255.f * o);
  const float x0 = (float)(tx * kTile) + 0.5f - mx, x1 = x0 + (float)(kTile - 1);
  const float y0 = (float)(ty * kTile) + 0.5f - my, y1 = y0 + (float)(kTile - 1);
  if (x0 <= 0.f && 0.f <= x1 && y0 <= 0.f && 0.f <= y1) return true;
  float qmin = INFINITY, scale = 0.f;
  auto at = [&](float x, float y) {
    const float q = A * x * x + 2.f * B * x * y + C * y * y;
    if (q < qmin) {
      qmin = q;
      scale = A * x * x + 2.f * fabsf(B * x * y) + C * y * y;
    }
  };
  at(x0, fminf(fmaxf(-B * x0 / C, y0), y1));
  at(x1, fminf(fmaxf(-B * x1 / C, y0), y1));
  at(fminf(fmaxf(-B * y0 / A, x0), x1), y0);
  at(fminf(fmaxf(-B * y1 / A, x0), x1), y1);
  return !(qmin > t + 0.05f * (1.f + fabsf(t)) + 1e-3f * scale);
}

// Stream-ordered device buffer.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  void release() {
    if (p != nullptr) cudaFreeAsync(p, st);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t alloc(size_t n, cudaStream_t s) {
    release();
    st = s;
    if (n == 0) n = 16;
    cudaError_t e = cudaMallocAsync(&p, n, s);
    if (e == cudaErrorMemoryAllocation) {
      // The pool keeps freed blocks reserved; hand them back to the device
      // and try once more (not while a graph is being captured).
      cudaGetLastError();
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        cudaMemPool_t pool;
        int dev = 0;
        if (cudaStreamSynchronize(s) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
          e = cudaMallocAsync(&p, n, s);
        if (e != cudaSuccess) cudaGetLastError();
      }
    }
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = n;
    return cudaSuccess;
  }
  cudaError_t ensure(size_t n, cudaStream_t s) {
    if (p != nullptr && bytes >= n) return cudaSuccess;
    return alloc(n, s);
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};


// Camera of one view of a call, with the view's place in the call's tile and
// pixel index spaces.
struct DevCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];          // camera centre in world coordinates, -R^T t
  int W, H;
  int tiles_x, tiles_y;
  int tile_off;             // first tile of this view in the call's tile numbering
  int pad;
  long long pix_off;        // first pixel of this view in the call's residual vector
};

// Projected splat as read by the blending and apply kernels.
//   a = (mu_x, mu_y, conic A, conic B), b = (conic C, opacity, depth, 0),
//   c = (r, g, b, 0)
struct SplatRec {
  float4 a, b, c;
};

// One non-empty (tile, splat) segment of the cache, as the apply kernels read
// it: a single 48-byte broadcast load gives everything a warp needs to walk the
// segment's entries.
struct SegRec {
  unsigned long long e0, e1;  // entry range [e0, e1)
  uint32_t slot;              // splat (view * N + Gaussian)
  float mx, my;               // 2D mean relative to the centre of the tile's first pixel
  float A, B, C;              // conic
  float io;                   // 1 / opacity
  float scale;                // FP16S payload scale (1 for the other formats)
};
static_assert(sizeof(SegRec) == 48, "SegRec is three 16-byte words");

// Device-side scalars of one PCG solve (Algorithm 1).
struct PcgScalars {
  double bb;        // ||b||^2
  double rz;        // r^T z of the current iterate
  double rz_new;
  double pg;        // p^T g
  double rr;        // ||r||^2
  double alpha, beta;
  int done;         // set when the break test fires or on breakdown
  int iters;
  int breakdown;
  int pad;
};

// Everything the apply kernels need about one cache (device pointers).
struct CacheView {
  const DevCam* cams;
  int V;
  int n_tiles;
  long long n_pix;                 // pixels over all views
  int N;                           // Gaussians
  long long n_slots;               // V * N
  const SplatRec* rec;             // [n_slots]
  const uint32_t* tile_seg_off;    // [n_tiles + 1]
  const unsigned long long* seg_entry_off;  // [n_seg + 1]
  const uint32_t* seg_slot;        // [n_seg]
  const SegRec* seg_rec;           // [n_seg]
  const void* payload;             // [E] float4 (FP32) or 4 x 16-bit
  const float* seg_scale;          // [n_seg] (FP16S only)
  const uint8_t* pixoff;           // [E] pixel index inside the tile (row-major 16 x 16)
  const uint32_t* slot_seg_start;  // segments of a splat, as a range of slot_seg_list; indexed by the
  const uint32_t* slot_seg_end;    // compact splat index [n_active] with vmask, else by slot [n_slots]
  const uint32_t* slot_seg_list;   // [n_seg] segment ids in splat order (compact index or slot; stable)
  const uint32_t* seg_pos;         // [n_seg] position of a segment in slot_seg_list: per-segment
                                   // adjoints and diagonal blocks are stored in this (splat) order
  const uint8_t* slot_active;      // [n_slots] (null when vmask is set)
  const unsigned long long* vmask; // [N] active views per Gaussian (null when V > 64)
  const uint32_t* act_off;         // [N + 1] with vmask: first compact splat index of each Gaussian; the
                                   // splat tangents are stored by compact index (act_off[g] + rank of the
                                   // view among g's active views) and SegRec.slot holds that index
  long long n_seg;
  long long n_entries;
  int fmt;
  const int* skip;                 // if non-null and *skip != 0 the kernels do nothing (PCG finished)
  const float* wres;               // [n_pix][3] residual-to-pixel weights (dr/dc)^2, or null (L2: 1)
  // GSLM_CACHE_THIN only (null otherwise): no entries; the kernels blend again
  const SplatRec* thin_rec;        // [n_seg] the projected splat of each segment, as the blending read it
  const float* img;                // [n_pix][3] final colour of each pixel
  const uint32_t* n_live;          // [n_tiles * 256] segments of its tile a pixel takes before it stops
  const uint32_t* win_off;         // [n_tiles + 1] first window of each tile (32 segments per window)
  const uint32_t* win_tile;        // [n_win] tile of each window
  const float4* ckpt;              // [n_win * 256] (T, colour prefix) of each pixel before the window
  long long n_win;
};

// Thin-cache outputs of the cache-writing pass (GSLM_CACHE_THIN).
constexpr int kThinWindow = 32;    // segments per checkpoint window
struct ThinOut {
  SplatRec* rec;                   // [n_seg]
  float4* ckpt;                    // [n_win * 256]
  const uint32_t* win_off;         // [n_tiles + 1]
  uint32_t* n_live;                // [n_tiles * 256]
};

// Counts kernel launches of this library (reported by gslm_kernel_launches).
void note_launch();

// Views of a cache and of a context for entry points defined outside api.cu.
// ----------------------------------------------------------------------------
// Batched solves: the PCG solves of up to kMaxBatch image subsets advance in
// lock step, each phase one launch over every subset. Parameter-space vectors
// of the subsets are stacked with a fixed stride (vs floats); float64 partials
// with a fixed stride per subset; one PcgScalars per subset.
constexpr int kMaxBatch = 16;

// Per-subset geometry and per-subset buffers of the per-Gaussian kernels.
struct SubsetRefs {
  const DevCam* cams;
  int V;
  const uint8_t* slot_active;           // [N * V] (null when vmask is set)
  const unsigned long long* vmask;      // [N] or null
  const uint32_t* act_off;              // [N + 1] compact splat offsets (with vmask) or null
  const uint32_t* s_start;              // segments of a splat (vjp), keyed as CacheView.slot_seg_start
  const uint32_t* s_end;
  const uint32_t* s_list;
  float* ydot;                          // [splats][12] splat tangents; after J p, the per-splat sums
                                        // of the J^T u partials (compact splat keys only)
  float* seg_ybar;                      // [n_seg][12] per-segment adjoints, in splat order
  long long n_splats;                   // compact splats (n_active) with act_off, else 0
};
struct GaussBatch {
  int n;
  SubsetRefs s[kMaxBatch];
};

// The tile kernels' view of a batch: subset b owns the global tiles
// [tile_end[b - 1], tile_end[b]).
struct TileBatch {
  int n;
  int fmt;
  long long total_tiles;
  long long tile_end[kMaxBatch];
  CacheView v[kMaxBatch];
  const float* ydot[kMaxBatch];
  float* u[kMaxBatch];
  float* seg_ybar[kMaxBatch];
  unsigned int* queue;      // persistent mode: global tile counter (zero at launch)
};

struct CacheParts {
  CacheView view;
  const float* params;
  int N;
  long long ld;
  const DevCam* cams;
  int V;
  int smooth;
};
struct ContextParts {
  cudaStream_t st;
  int variant_JT;   // apply_JT kernel variant for the cache format asked about (forced, tuned or default)
  int device;
  void* noalloc_scratch;   // device address of the allocation-free J^T u's array on the context's device, or null
};
bool cache_parts(const gslm_cache* c, CacheParts* out);
// out = (J^T J + lambda clamp(M)) v through the cache (api.cu).
gslm_status apply_A(gslm_ctx* ctx, const gslm_cache* c, const float* v, const float* M, float lambda, float* out);
cudaStream_t context_stream(const gslm_ctx* c);
// D = the learned preconditioner of a cache's system with diagonal M (precond.cu).
gslm_status precond_for_cache(gslm_precond* pc, gslm_ctx* ctx, const gslm_cache* c, const float* M, float* D);
bool context_parts(const gslm_ctx* c, int cache_fmt, ContextParts* out);
void set_context_error(gslm_ctx* c, const char* msg);
// Device address, on the current device, of the fixed array gslm_apply_JT_noalloc
// uses (noalloc.cu); looking it up loads the array's module on that device.
cudaError_t noalloc_scratch_address(void** out);

// ----------------------------------------------------------------------------
// Launchers (each defined in the .cu file that holds the kernel).
// All return cudaGetLastError() of the launch.

// project.cu
// tmask (may be null: no tile culling): per slot, the tiles of its rectangle
// (row-major, bit (ty - y0) * width + (tx - x0)) the splat can reach, for
// rectangles of at most kCullMaxTiles tiles; ntiles counts those tiles.
cudaError_t launch_project(const float* params, int N, long long ld, const DevCam* cams, int V,
                           int smooth, SplatRec* rec, uint32_t* ntiles, uint2* rect,
                           uint32_t* depth_key, unsigned long long* tmask, cudaStream_t st);
cudaError_t launch_view_mask(const uint8_t* slot_active, int N, int V, unsigned long long* vmask,
                             cudaStream_t st);
// vmask (per Gaussian, bit v = view v has cache entries) may be null, and must
// be null when V > 64; the kernels then visit every view.
// act_off (with vmask; may be null): ydot stored by compact splat index (CacheView.act_off).
cudaError_t launch_tangent(const float* params, int N, long long ld, const DevCam* cams, int V,
                           int smooth, const uint8_t* slot_active, const unsigned long long* vmask,
                           const uint32_t* act_off, const float* p, float* ydot, const float* z_beta,
                           float* p_out, const PcgScalars* sc, cudaStream_t st);
// act_off[0..N] from the view masks, SegRec.slot rewritten to the compact
// splat index, and that index per segment in key[n_seg] (the sort key of the
// splat order).
cudaError_t launch_compact_splats(const unsigned long long* vmask, int N, uint32_t* act_off, void* scan_temp,
                                  const uint32_t* seg_slot, long long n_seg, SegRec* seg_rec, uint32_t* key,
                                  cudaStream_t st);
// s_start/s_end: segment positions of a splat, keyed by compact splat index
// when vmask (and act_off) are given, else by slot v * N + g.
// splat_ybar (with vmask and act_off; may be null): the per-splat sums of
// launch_splat_sum, read instead of the segment ranges.
cudaError_t launch_vjp(const float* params, int N, long long ld, const DevCam* cams, int V,
                       int smooth, const uint32_t* s_start, const uint32_t* s_end,
                       const unsigned long long* vmask, const uint32_t* act_off,
                       const float* seg_ybar, const float* splat_ybar, float scale, float* g, const float* p,
                       const float* M, float lambda, double* dot_partials, const PcgScalars* sc, cudaStream_t st);
// splat_q (with compact keys; may be null): the per-splat sums of the
// segment blocks (launch_splat_sum_q), read instead of the segment ranges.
cudaError_t launch_diag(const float* params, int N, long long ld, const DevCam* cams, int V,
                        int smooth, const uint32_t* s_start, const uint32_t* s_end,
                        const unsigned long long* vmask, const uint32_t* act_off,
                        const float* seg_q, const float* splat_q, float* diag, cudaStream_t st);
cudaError_t launch_splat_sum_q(long long n_splats, const uint32_t* s_start, const uint32_t* s_end, const float* seg_q,
                               float* splat_q, cudaStream_t st);
int vjp_blocks(int N);
// Batched forms: blockIdx.y = subset; p, z, pout, g, M stacked with stride vs;
// scalars sc[b]; vjp partials at partials + b * vjp_blocks(N).
cudaError_t launch_tangent_batch(const float* params, int N, long long ld, int smooth, const GaussBatch& gb,
                                 const float* p, long long vs, const float* z_beta, float* p_out,
                                 const PcgScalars* sc, cudaStream_t st);
// Per compact splat c < n_splats: splat_ybar[c] = sum of seg_ybar over the
// splat's segment range [s_start[c], s_end[c]) (12 floats). Skipped when
// sc->done. The batched form does every subset whose act_off is set, into its
// ydot buffer.
cudaError_t launch_splat_sum(long long n_splats, const uint32_t* s_start, const uint32_t* s_end,
                             const float* seg_ybar, float* splat_ybar, const PcgScalars* sc, cudaStream_t st);
cudaError_t launch_splat_sum_batch(const GaussBatch& gb, const PcgScalars* sc, cudaStream_t st);
cudaError_t launch_vjp_batch(const float* params, int N, long long ld, int smooth, const GaussBatch& gb,
                             float* g, long long vs, const float* p, const float* M, float lambda,
                             double* partials, const PcgScalars* sc, cudaStream_t st);

// sort.cu
size_t scan_temp_bytes(long long n);
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* temp,
                               cudaStream_t st);   // out[n] = total
cudaError_t exclusive_scan_u64(const uint32_t* in, unsigned long long* out, long long n,
                               void* temp, cudaStream_t st);   // out[n] = total
size_t radix_temp_bytes(long long n);
// Stable LSD sort of (key, value) pairs on the low `bits` bits of the key. The
// sorted result ends in (keys_out, vals_out); the *_tmp buffers are scratch.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                             uint32_t* vals_tmp, long long n, int bits, void* temp,
                             uint32_t** keys_out, uint32_t** vals_out, cudaStream_t st);
cudaError_t launch_flags(const uint32_t* counts, long long n, uint32_t* flags, cudaStream_t st);
cudaError_t launch_compact_flags(const uint32_t* counts, const uint32_t* pos, long long n,
                                 uint32_t* list, cudaStream_t st);
cudaError_t launch_gather_u32(const uint32_t* src, const uint32_t* idx, long long n,
                              uint32_t* dst, cudaStream_t st);
cudaError_t launch_iota_u32(uint32_t* dst, long long n, cudaStream_t st);
// dst[idx[i]] = i for i < n (inverse of a permutation)
cudaError_t launch_scatter_index_u32(const uint32_t* idx, long long n, uint32_t* dst, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t* sorted_keys, long long n, uint32_t* start,
                          uint32_t* end, cudaStream_t st);

// raster.cu
// tmask as written by launch_project (may be null: every tile of the rectangle).
cudaError_t launch_emit_keys(const uint32_t* sorted_slots, long long n_vis, const uint2* rect,
                             const unsigned long long* tmask, const DevCam* cams, int V, int N,
                             const unsigned long long* key_off, uint32_t* tile_keys, uint32_t* tile_vals,
                             cudaStream_t st);
// Blend every tile. mode 0: render only; mode 1: also count entries/segments.
cudaError_t launch_raster_count(const DevCam* cams, int V, int n_tiles, const uint32_t* tile_start,
                                const uint32_t* tile_end, const uint32_t* tile_vals,
                                const SplatRec* rec, int smooth, const float* targets,
                                float* img, float* F, double* cost_partials, uint32_t* tile_entries,
                                uint32_t* tile_segs, cudaStream_t st);
// fmt GSLM_CACHE_THIN: no payload or pixel offsets; writes thin instead.
cudaError_t launch_raster_write(const DevCam* cams, int V, int n_tiles, const uint32_t* tile_start,
                                const uint32_t* tile_end, const uint32_t* tile_vals,
                                const SplatRec* rec, int smooth, const float* img,
                                const unsigned long long* tile_entry_off,
                                const uint32_t* tile_seg_off, int fmt, void* payload,
                                float* seg_scale, uint8_t* pixoff,
                                unsigned long long* seg_entry_off, uint32_t* seg_slot, SegRec* seg_rec,
                                uint8_t* slot_active, int* err, const ThinOut& thin, cudaStream_t st);

// thin.cu: the thin cache's windows and its J p, J^T u and diag(J^T J) blocks
// (same outputs as launch_apply_J / launch_apply_JT / launch_diag_entries).
// win_count: [n_tiles] windows per tile (ceil(segments / 32)).
cudaError_t launch_thin_window_counts(const uint32_t* tile_seg_off, int n_tiles, uint32_t* win_count,
                                      cudaStream_t st);
cudaError_t launch_thin_window_tiles(const uint32_t* win_off, int n_tiles, uint32_t* win_tile, cudaStream_t st);
cudaError_t launch_thin_apply_J(const CacheView& cv, const float* ydot, const float* F_add, float* u,
                                double* sq_partials, cudaStream_t st);
cudaError_t launch_thin_apply_JT(const CacheView& cv, const float* u, float* seg_ybar, cudaStream_t st);
cudaError_t launch_thin_diag(const CacheView& cv, float* seg_q, cudaStream_t st);

// apply.cu. `variant` selects one of apply_variants() kernel configurations
// (entries in flight per lane and register budget); all compute the same result.
int apply_variants();
// Most 256-thread CTAs of a variant's J p (jt false) or J^T u kernel that fit
// one SM (registers, shared memory).
inline int variant_cta_cap(int v, bool jt) {
  if (jt) return (v == 1 || v == 7 || v == 9) ? 5 : (v == 3 || v == 5 || v == 6) ? 4 : 6;
  return v == 1 ? 5 : (v == 3 || v == 5 || v == 6 || v == 8 || v == 9) ? 4 : 6;
}
// sq_partials (may be null): [2][n_tiles] per-tile sums of ||u + F_add||^2 and ||u||^2.
cudaError_t launch_apply_J(const CacheView& cv, const float* ydot, const float* F_add,
                           float* u, double* sq_partials, int variant, cudaStream_t st);
cudaError_t launch_apply_JT(const CacheView& cv, const float* u, float* seg_ybar, int variant,
                            cudaStream_t st);
cudaError_t launch_diag_entries(const CacheView& cv, float* seg_q, cudaStream_t st);
int apply_J_partials(const CacheView& cv);
// Batched persistent forms: `ctas_per_sm` resident CTAs per SM take the tiles
// of every subset from tb.queue (which must be zero at launch).
cudaError_t launch_apply_J_batch(const TileBatch& tb, int variant, int ctas_per_sm, cudaStream_t st);
cudaError_t launch_apply_JT_batch(const TileBatch& tb, int variant, int ctas_per_sm, cudaStream_t st);
int device_sm_count();

// residual.cu: e (may be null), w (may be null) [n_pix][3] and per-tile float64
// energies of the L1 + SSIM objective for rendered img against tgt.
cudaError_t launch_l1ssim(const DevCam* cams, int V, int n_tiles, const float* img, const float* tgt, float lam1,
                          float lam2, float eps, float* e, float* w, double* cost_partials, cudaStream_t st);
cudaError_t launch_fill_f32(long long n, float v, float* out, cudaStream_t st);

// pcg.cu
cudaError_t launch_reduce_partials(const double* partials, int n, double* out, cudaStream_t st);
// M^-1 of Algorithm 1 is D where given, else 1 / clamp(M) (not stored).
// residual0: r may be b itself.
cudaError_t launch_pcg_init(int N, long long ld, const float* b, const float* M, const float* D, float* x,
                            double* partials, cudaStream_t st);
cudaError_t launch_pcg_residual0(int N, long long ld, const float* b, const float* g, const float* M, const float* D,
                                 const float* x, float lambda, float* r, float* z, float* p, double* partials,
                                 cudaStream_t st);
cudaError_t launch_pcg_scalars(PcgScalars* sc, const double* partials, int n_partials, int stage,
                               float break_rel2, cudaStream_t st);
cudaError_t launch_pcg_update(int N, long long ld, const PcgScalars* sc, const float* p, const float* g,
                              const float* M, const float* D, float* x, float* r, float* z, double* partials,
                              cudaStream_t st);
int pcg_blocks(int N);
// Batched forms: n subsets, grid (pcg_blocks(N), n); vectors at stride vs,
// partials at stride pcg_blocks(N) (update: 2 * pcg_blocks(N)), scalars sc[b].
// Subset b uses D + b * vs when bit b of d_mask is set, else 1 / clamp(M).
cudaError_t launch_pcg_init_batch(int n, int N, long long ld, long long vs, const float* b, const float* M,
                                  const float* D, unsigned d_mask, float* x, double* partials, cudaStream_t st);
cudaError_t launch_pcg_residual0_batch(int n, int N, long long ld, long long vs, const float* b, const float* g,
                                       const float* M, const float* D, unsigned d_mask, const float* x, float lambda,
                                       float* r, float* z, float* p, double* partials, cudaStream_t st);
cudaError_t launch_pcg_update_batch(int n, int N, long long ld, long long vs, const PcgScalars* sc, const float* p,
                                    const float* g, const float* M, const float* D, unsigned d_mask, float* x,
                                    float* r, float* z, double* partials, cudaStream_t st);
// scalars of n subsets; subset b reduces partials + b * pstride (n_partials of them).
cudaError_t launch_pcg_scalars_batch(int n, PcgScalars* sc, const double* partials, int n_partials, int pstride,
                                     int stage, float break_rel2, cudaStream_t st);
cudaError_t launch_combine_acc(int N, long long ld, const float* delta, const float* diag,
                               float* num, float* den, cudaStream_t st);
cudaError_t launch_combine_finish(int N, long long ld, const float* num, const float* den,
                                  float* delta, cudaStream_t st);
// out = x + a d over [59][ld]
cudaError_t launch_axpy_params(int N, long long ld, const float* x, float a, const float* d, float* out,
                               cudaStream_t st);
cudaError_t launch_neg_copy(long long n, const float* src, float* dst, cudaStream_t st);
cudaError_t launch_count_nonzero_u8(const uint8_t* v, long long n, unsigned long long* out, cudaStream_t st);

}  // namespace gslm
