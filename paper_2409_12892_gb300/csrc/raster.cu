// Tile rasterizer and gradient-cache construction (Sec. 3.1 Eq. alpha-blending;
// Sec. 3.3 "buildCache").
//
//   k_emit_keys     one (tile, splat) key per tile overlapped by a splat, in the
//                   depth order of the splats (ties: Gaussian index)
//   k_raster_count  one CTA per 16x16 tile, one thread per pixel: front-to-back
//                   blending; writes the image, F = c - C and its squared norm,
//                   and (counting mode) the number of cache entries and of
//                   non-empty (tile, splat) segments of the tile
//   k_raster_write  the same walk again, writing one cache entry per
//                   contributing (pixel, splat) pair
//
// Cache layout (the paper stores the cache by pixel and re-sorts it by
// Gaussian, Sec. 3.3; here it is written directly grouped by (tile, splat)):
//   segments of a tile in depth order; within a segment, the entries of the
//   contributing pixels in row-major pixel order. Entry payload (w, h0, h1, h2):
//     w    = alpha_s T_s                    (= dc/dc_s)
//     h_ch = alpha_s * dc_ch/dalpha_s       (0 where alpha is clamped)
//   with dc/dalpha_s = T_s c_s - (colour behind s) / (1 - alpha_s) and the
//   colour behind s = final colour - colour accumulated up to and including s.
//   A 1-byte pixel offset inside the tile accompanies every entry.
#include "internal.cuh"

namespace gslm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int find_view(const DevCam* __restrict__ cams, int V, int tile) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cams[mid].tile_off <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_emit_keys(const uint32_t* __restrict__ sorted_slots, long long n_vis,
                            const uint2* __restrict__ rect, const unsigned long long* __restrict__ tmask,
                            const DevCam* __restrict__ cams, int N, const unsigned long long* __restrict__ key_off,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_vis) return;
  const uint32_t slot = sorted_slots[i];
  const int v = (int)(slot / (uint32_t)N);
  const DevCam& cam = cams[v];
  const uint2 r = rect[slot];
  const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
  // the tiles the projection kept (key_off counts exactly those)
  const bool masked = tmask != nullptr && (x1 - x0) * (y1 - y0) <= kCullMaxTiles;
  const unsigned long long m = masked ? tmask[slot] : ~0ull;
  unsigned long long o = key_off[i];
  int bit = 0;
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx, ++bit) {
      if (masked && !((m >> bit) & 1ull)) continue;
      keys[o] = (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx);
      vals[o] = slot;
      ++o;
    }
}

// Blending weight of a splat at a pixel. Written with explicit round-to-nearest
// intrinsics so that the counting and the writing walks, compiled as separate
// kernels, take bit-identical decisions (no differing FMA contraction).
struct Blend {
  float araw;    // opacity * G
  float alpha;   // blending alpha (clamped unless smooth)
  bool valid;    // alpha >= 1/255 (always in smooth mode)
};

__device__ __forceinline__ Blend blend_weight(float px, float py, float4 a, float2 bb, int smooth) {
  const float dx = __fsub_rn(px, a.x), dy = __fsub_rn(py, a.y);
  const float q = __fadd_rn(__fmul_rn(a.z, __fmul_rn(dx, dx)), __fmul_rn(bb.x, __fmul_rn(dy, dy)));
  const float power = __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(a.w, __fmul_rn(dx, dy)));
  Blend r;
  r.araw = __fmul_rn(bb.y, expf(power));
  r.alpha = smooth ? r.araw : fminf(kAlphaMax, r.araw);
  r.valid = smooth || r.alpha >= kAlphaMin;
  return r;
}

__device__ __forceinline__ float transmit(float T, float alpha) { return __fmul_rn(T, __fsub_rn(1.f, alpha)); }

// Row reach of a splat: the largest |py - mean y| at which some pixel of the
// row can take alpha >= 1/255 (blend_weight's test). With the conic
// Q = [[A, B], [B, C]] (A = a.z, B = a.w, C = b.x) the blend is valid where
// Q(d) <= L = 2 ln(255 o), and the least Q over a row at offset dy is
// dy^2 det(Q) / A, so rows with |dy| > sqrt(L A / det(Q)) hold no valid pixel.
// Widened by 0.1% and 0.01 pixel, far beyond float32 rounding of the blend's
// own arithmetic; -1 where the splat is never valid (o <= 1/255), +inf where
// nothing is skipped (smooth mode, a degenerate conic, NaN). A warp (two rows
// of the tile) skips a splat whose reach misses both rows: every decision the
// blend would take there is "not valid", so nothing changes but the work.
__device__ __forceinline__ float row_reach(const SplatRec& r, int smooth) {
  if (smooth) return INFINITY;
  const float A = r.a.z, B = r.a.w, C = r.b.x, o = r.b.y;
  const float L = 2.f * logf(255.f * o);
  if (!(L > 0.f)) return -1.f;
  const float det = A * C - B * B;
  if (!(A > 0.f) || !(det > 0.f)) return INFINITY;
  const float y = sqrtf(L * A / det);
  return y == y ? y * 1.001f + 0.01f : INFINITY;
}

// True when a splat with mean y `my` and row reach `reach` misses both rows of
// a warp whose first row's pixel centres lie at yc0 (NaN: false).
__device__ __forceinline__ bool misses_rows(float my, float reach, float yc0) {
  return yc0 - my > reach || my - (yc0 + 1.f) > reach;
}

struct TileSetup {
  int x, y;
  bool inside;
  float px, py;
  long long pix;
  int x0, y0;
};

__device__ __forceinline__ TileSetup tile_setup(const DevCam& cam, int tile) {
  TileSetup s;
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  s.x0 = tx * kTile;
  s.y0 = ty * kTile;
  s.x = s.x0 + (threadIdx.x & (kTile - 1));
  s.y = s.y0 + (threadIdx.x / kTile);
  s.inside = s.x < cam.W && s.y < cam.H;
  s.px = s.x + 0.5f;
  s.py = s.y + 0.5f;
  s.pix = cam.pix_off + (long long)s.y * cam.W + s.x;
  return s;
}

template <bool kCount>
__global__ void __launch_bounds__(kTilePix) k_raster_count(
    const DevCam* __restrict__ cams, int V, const uint32_t* __restrict__ tstart,
    const uint32_t* __restrict__ tend, const uint32_t* __restrict__ tvals, const SplatRec* __restrict__ rec,
    int smooth, const float* __restrict__ targets, float* __restrict__ img, float* __restrict__ F,
    double* __restrict__ cost_partials, uint32_t* __restrict__ tile_entries, uint32_t* __restrict__ tile_segs) {
  __shared__ float4 sA[kTilePix];
  __shared__ float2 sB[kTilePix];
  __shared__ float4 sC[kTilePix];
  __shared__ float sY[kTilePix];             // row reach of each splat
  __shared__ unsigned flag[kTilePix / 32];   // bit j of word b: splat 32 b + j of the batch contributes
  __shared__ double dred[kTilePix / 32];
  __shared__ uint32_t ured[kTilePix / 32];
  const int tile = blockIdx.x;
  const int v = find_view(cams, V, tile);
  const DevCam& cam = cams[v];
  const TileSetup ts = tile_setup(cam, tile);
  const int lane = threadIdx.x & 31;
  const float yc0 = (float)(ts.y0 + 2 * (int)(threadIdx.x >> 5)) + 0.5f;   // the warp's first row
  const uint32_t s0 = tstart[tile], s1 = tend[tile];
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  uint32_t n = 0, nseg = 0;
  bool done = !ts.inside;
  for (uint32_t b = s0; b < s1; b += kTilePix) {
    if (__syncthreads_count(done) == kTilePix) break;
    const uint32_t i = b + threadIdx.x;
    if (i < s1) {
      const SplatRec& r = rec[tvals[i]];
      sA[threadIdx.x] = r.a;
      sB[threadIdx.x] = make_float2(r.b.x, r.b.y);
      sC[threadIdx.x] = r.c;
      sY[threadIdx.x] = row_reach(r, smooth);
    }
    if (kCount && threadIdx.x < kTilePix / 32) flag[threadIdx.x] = 0u;
    __syncthreads();
    const int cnt = (int)min((uint32_t)kTilePix, s1 - b);
    // 32 splats at a time; a warp whose pixels are all done leaves the batch
    for (int jb = 0; jb < cnt; jb += 32) {
      if (__all_sync(kFull, done)) break;
      const int jn = min(32, cnt - jb);
      const unsigned wskip = __ballot_sync(kFull, lane < jn && misses_rows(sA[jb + lane].y, sY[jb + lane], yc0));
      unsigned mine = 0u;   // this pixel's contributions among the 32
      for (int jj = 0; jj < jn; ++jj) {
        if (done) break;
        if ((wskip >> jj) & 1u) continue;
        const int j = jb + jj;
        const Blend bl = blend_weight(ts.px, ts.py, sA[j], sB[j], smooth);
        const float alpha = bl.alpha;
        if (bl.valid) {
          const float test = transmit(T, alpha);
          if (!smooth && test < kTMin) {
            done = true;
          } else {
            const float w = __fmul_rn(alpha, T);
            const float4 c = sC[j];
            c0 = __fmaf_rn(c.x, w, c0);
            c1 = __fmaf_rn(c.y, w, c1);
            c2 = __fmaf_rn(c.z, w, c2);
            T = test;
            ++n;
            mine |= 1u << jj;
          }
        }
      }
      if (kCount) {
        const unsigned any = __reduce_or_sync(kFull, mine);
        if (lane == 0 && any != 0u) atomicOr(&flag[jb >> 5], any);
      }
    }
    if (kCount) {
      __syncthreads();
      nseg += (uint32_t)__syncthreads_count(threadIdx.x < (unsigned)cnt &&
                                            ((flag[threadIdx.x >> 5] >> (threadIdx.x & 31)) & 1u));
    }
  }
  double local = 0.0;
  if (ts.inside) {
    float* o = img + ts.pix * 3;
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
    if (targets != nullptr) {
      const float* t = targets + ts.pix * 3;
      const float f0 = c0 - t[0], f1 = c1 - t[1], f2 = c2 - t[2];
      if (F != nullptr) {
        float* f = F + ts.pix * 3;
        f[0] = f0;
        f[1] = f1;
        f[2] = f2;
      }
      local = (double)f0 * f0 + (double)f1 * f1 + (double)f2 * f2;
    }
  }
  if (cost_partials != nullptr || kCount) {
    for (int o = 16; o > 0; o >>= 1) {
      local += __shfl_xor_sync(kFull, local, o);
      n += __shfl_xor_sync(kFull, n, o);
    }
    if (lane == 0) {
      dred[threadIdx.x >> 5] = local;
      ured[threadIdx.x >> 5] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      uint32_t e = 0;
      for (int w = 0; w < kTilePix / 32; ++w) {
        s += dred[w];
        e += ured[w];
      }
      if (cost_partials != nullptr) cost_partials[tile] = s;
      if (kCount) {
        tile_entries[tile] = e;
        tile_segs[tile] = nseg;
      }
    }
  }
}

template <int kFmt>
__device__ __forceinline__ void store_entry(void* payload, unsigned long long pos, float w, float h0, float h1,
                                            float h2, float inv_scale) {
  if (kFmt == GSLM_CACHE_FP32) {
    reinterpret_cast<float4*>(payload)[pos] = make_float4(w, h0, h1, h2);
  } else if (kFmt == GSLM_CACHE_BF16) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(w, h0);
    const __nv_bfloat162 b = __floats2bfloat162_rn(h1, h2);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&a);
    u.y = *reinterpret_cast<const uint32_t*>(&b);
    reinterpret_cast<uint2*>(payload)[pos] = u;
  } else {
    const __half2 a = __floats2half2_rn(w * inv_scale, h0 * inv_scale);
    const __half2 b = __floats2half2_rn(h1 * inv_scale, h2 * inv_scale);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&a);
    u.y = *reinterpret_cast<const uint32_t*>(&b);
    reinterpret_cast<uint2*>(payload)[pos] = u;
  }
}

// kFmt GSLM_CACHE_THIN writes no entries: per segment the projected splat
// (thin.rec), per pixel the number of its tile's segments it takes before it
// stops (thin.n_live) and, before every kThinWindow-th segment of the tile, the
// pixel's transmittance and colour prefix (thin.ckpt). Segment records and
// entry offsets are written as for the other formats (the entry offsets count
// the entries a full cache would hold).
template <int kFmt>
__global__ void __launch_bounds__(kTilePix) k_raster_write(
    const DevCam* __restrict__ cams, int V, const uint32_t* __restrict__ tstart,
    const uint32_t* __restrict__ tend, const uint32_t* __restrict__ tvals, const SplatRec* __restrict__ rec,
    int smooth, const float* __restrict__ img, const unsigned long long* __restrict__ tile_entry_off,
    const uint32_t* __restrict__ tile_seg_off, void* __restrict__ payload, float* __restrict__ seg_scale,
    uint8_t* __restrict__ pixoff, unsigned long long* __restrict__ seg_entry_off,
    uint32_t* __restrict__ seg_slot, SegRec* __restrict__ seg_rec, uint8_t* __restrict__ slot_active,
    int* __restrict__ err, const ThinOut thin) {
  constexpr bool kThin = kFmt == GSLM_CACHE_THIN;
  __shared__ float4 sA[kTilePix];
  __shared__ float2 sB[kTilePix];
  __shared__ float4 sC[kTilePix];
  __shared__ float sY[kTilePix];   // row reach of each splat
  __shared__ uint32_t sSlot[kTilePix];
  // Per sub-batch of 32 splats every warp works out the splats' entry and
  // segment offsets itself (lane = splat) from all warps' ballots, so one
  // barrier per sub-batch suffices; the ballots alternate between two buffers
  // so that a warp already in the next sub-batch cannot overwrite ballots
  // another warp still reads.
  __shared__ uint32_t bal[2][kTilePix / 32][32];
  __shared__ uint32_t wpos[kTilePix / 32][32];   // a warp's first entry position of each splat (own row)
  __shared__ int wseg[kTilePix / 32][32];        // segment index of each splat or -1 (own row)
  __shared__ uint32_t segmax[32];
  __shared__ float sAraw[32][kTilePix];   // o G of the sub-batch's splats at each pixel (phase A -> D)
  const int tile = blockIdx.x;
  const int v = find_view(cams, V, tile);
  const DevCam& cam = cams[v];
  const TileSetup ts = tile_setup(cam, tile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const float yc0 = (float)(ts.y0 + 2 * warp) + 0.5f;   // the warp's first row
  const uint32_t s0 = tstart[tile], s1 = tend[tile];
  float Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f;
  if (ts.inside) {
    Cf0 = img[ts.pix * 3 + 0];
    Cf1 = img[ts.pix * 3 + 1];
    Cf2 = img[ts.pix * 3 + 2];
  }
  const unsigned long long ebase = tile_entry_off[tile], eend = tile_entry_off[tile + 1];
  const uint32_t sbase = tile_seg_off[tile], send = tile_seg_off[tile + 1];
  uint32_t erun = 0, srun = 0;
  float T = 1.f, p0 = 0.f, p1 = 0.f, p2 = 0.f;
  bool done = !ts.inside;
  uint32_t nlive = done ? 0u : 0xffffffffu;   // thin: set where the pixel stops
  for (uint32_t b = s0; b < s1; b += kTilePix) {
    if (__syncthreads_count(done) == kTilePix) break;
    const uint32_t i = b + threadIdx.x;
    if (i < s1) {
      const uint32_t slot = tvals[i];
      const SplatRec& r = rec[slot];
      sA[threadIdx.x] = r.a;
      sB[threadIdx.x] = make_float2(r.b.x, r.b.y);
      sC[threadIdx.x] = r.c;
      sY[threadIdx.x] = row_reach(r, smooth);
      sSlot[threadIdx.x] = slot;
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kTilePix, s1 - b);
    for (int sub = 0; sub < cnt; sub += 32) {
      const int m = min(32, cnt - sub);
      // A: which of the next m splats contribute to this pixel
      uint32_t mask = 0;
      float Tl = T;
      bool dl = done;
      int jstop = -1;
      const unsigned wskip = __ballot_sync(kFull, lane < m && misses_rows(sA[sub + lane].y, sY[sub + lane], yc0));
      for (int j = 0; j < m; ++j) {
        if (dl) break;
        if ((wskip >> j) & 1u) continue;
        const Blend bl = blend_weight(ts.px, ts.py, sA[sub + j], sB[sub + j], smooth);
        if (bl.valid) {
          const float test = transmit(Tl, bl.alpha);
          if (!smooth && test < kTMin) {
            dl = true;
            jstop = j;
          } else {
            mask |= 1u << j;
            Tl = test;
            sAraw[j][threadIdx.x] = bl.araw;
          }
        }
      }
      // B: per-warp ballots, one per splat
      const int par = (sub >> 5) & 1;
#pragma unroll 4
      for (int j = 0; j < 32; ++j) {
        const unsigned bj = __ballot_sync(kFull, (mask >> j) & 1u);
        if (lane == j) bal[par][warp][j] = bj;
      }
      __syncthreads();
      // C: segment and entry offsets of the m splats, in every warp (lane =
      // splat); warp 0 also writes the segment records
      uint32_t add_e, add_s;
      unsigned nzs;
      {
        const int j = lane;
        uint32_t cj = 0, own = 0;
#pragma unroll
        for (int w = 0; w < kTilePix / 32; ++w) {
          const uint32_t c = __popc(bal[par][w][j]);
          own += w < warp ? c : 0u;
          cj += c;
        }
        uint32_t inc = cj;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, inc, o);
          if (lane >= o) inc += t;
        }
        const uint32_t excl = inc - cj;
        const unsigned nz = __ballot_sync(kFull, cj > 0);
        const uint32_t sidx = sbase + srun + __popc(nz & lt);
        wpos[warp][j] = erun + excl + own;
        wseg[warp][j] = cj > 0 && sidx < send ? (int)sidx : -1;
        add_e = __shfl_sync(kFull, inc, 31);
        add_s = (uint32_t)__popc(nz);
        nzs = nz;
        if (warp == 0 && cj > 0) {
          const uint32_t slot = sSlot[sub + j];
          if (sidx < send) {
            seg_slot[sidx] = slot;
            seg_entry_off[sidx] = ebase + erun + excl;
            slot_active[slot] = 1;
            const float4 a = sA[sub + j];
            const float2 bb = sB[sub + j];
            SegRec r;
            r.e0 = ebase + erun + excl;
            r.e1 = r.e0 + cj;
            r.slot = slot;
            r.mx = a.x - (ts.x0 + 0.5f);
            r.my = a.y - (ts.y0 + 0.5f);
            r.A = a.z;
            r.B = a.w;
            r.C = bb.x;
            r.io = 1.f / bb.y;
            r.scale = 1.f;
            seg_rec[sidx] = r;
            if (kThin) {
              SplatRec t;
              t.a = a;
              t.b = make_float4(bb.x, bb.y, 0.f, 0.f);
              t.c = sC[sub + j];
              thin.rec[sidx] = t;
            }
          } else {
            atomicOr(err, 2);
          }
        }
        if (kFmt == GSLM_CACHE_FP16S && warp == 0) segmax[j] = 0u;
      }
      __syncwarp();
      if (kThin) {
        // checkpoints before the window-opening segments, the pixel's state
        // advanced over its own contributions; where the pixel stopped
        const uint32_t wbase = thin.win_off[tile];
        for (int j = 0; j < m; ++j) {
          const int sj = wseg[warp][j];
          if (sj >= 0 && ((uint32_t)(sj - (int)sbase) % kThinWindow) == 0u)
            thin.ckpt[(size_t)(wbase + (uint32_t)(sj - (int)sbase) / kThinWindow) * kTilePix + threadIdx.x] =
                make_float4(T, p0, p1, p2);
          if (!((mask >> j) & 1u)) continue;
          const float araw = sAraw[j][threadIdx.x];
          const float alpha = smooth ? araw : fminf(kAlphaMax, araw);
          const float4 c = sC[sub + j];
          const float w = __fmul_rn(alpha, T);
          p0 = __fmaf_rn(c.x, w, p0);
          p1 = __fmaf_rn(c.y, w, p1);
          p2 = __fmaf_rn(c.z, w, p2);
          T = transmit(T, alpha);
        }
        if (jstop >= 0) nlive = srun + (uint32_t)__popc(nzs & ((1u << jstop) - 1u));
        done = dl;
        erun += add_e;
        srun += add_s;
        continue;
      }
      // D: entries. FP16S first needs every segment's largest magnitude.
      if (kFmt == GSLM_CACHE_FP16S) {
        __syncthreads();   // segmax cleared by warp 0
        float Tq = T, q0 = p0, q1 = p1, q2 = p2;
        for (unsigned mm = mask; mm != 0u; mm &= mm - 1u) {
          const int j = __ffs(mm) - 1;
          const float araw = sAraw[j][threadIdx.x];
          const float alpha = smooth ? araw : fminf(kAlphaMax, araw);
          const float4 c = sC[sub + j];
          const float w = __fmul_rn(alpha, Tq);
          q0 = __fmaf_rn(c.x, w, q0);
          q1 = __fmaf_rn(c.y, w, q1);
          q2 = __fmaf_rn(c.z, w, q2);
          const float inv1m = __fdividef(1.f, 1.f - alpha);
          const bool clamped = !smooth && araw > kAlphaMax;
          const float h0 = clamped ? 0.f : alpha * (Tq * c.x - (Cf0 - q0) * inv1m);
          const float h1 = clamped ? 0.f : alpha * (Tq * c.y - (Cf1 - q1) * inv1m);
          const float h2 = clamped ? 0.f : alpha * (Tq * c.z - (Cf2 - q2) * inv1m);
          const float mx = fmaxf(fmaxf(fabsf(w), fabsf(h0)), fmaxf(fabsf(h1), fabsf(h2)));
          atomicMax(&segmax[j], __float_as_uint(mx));
          Tq = transmit(Tq, alpha);
        }
        __syncthreads();
        if (threadIdx.x < 32 && wseg[0][threadIdx.x] >= 0) {
          seg_scale[wseg[0][threadIdx.x]] = __uint_as_float(segmax[threadIdx.x]);
          seg_rec[wseg[0][threadIdx.x]].scale = __uint_as_float(segmax[threadIdx.x]);
        }
      }
      // the pixel's own contributions in splat order (set bits of its mask)
      for (unsigned mm = mask; mm != 0u; mm &= mm - 1u) {
        const int j = __ffs(mm) - 1;
        const float araw = sAraw[j][threadIdx.x];   // as blend_weight computed it in phase A
        const float alpha = smooth ? araw : fminf(kAlphaMax, araw);
        const float4 c = sC[sub + j];
        const float w = __fmul_rn(alpha, T);
        p0 = __fmaf_rn(c.x, w, p0);
        p1 = __fmaf_rn(c.y, w, p1);
        p2 = __fmaf_rn(c.z, w, p2);
        const float inv1m = __fdividef(1.f, 1.f - alpha);   // 0 < 1 - alpha <= 1
        const bool clamped = !smooth && araw > kAlphaMax;
        const float h0 = clamped ? 0.f : alpha * (T * c.x - (Cf0 - p0) * inv1m);
        const float h1 = clamped ? 0.f : alpha * (T * c.y - (Cf1 - p1) * inv1m);
        const float h2 = clamped ? 0.f : alpha * (T * c.z - (Cf2 - p2) * inv1m);
        const unsigned long long pos = ebase + wpos[warp][j] + (uint32_t)__popc(bal[par][warp][j] & lt);
        float inv_scale = 1.f;
        if (kFmt == GSLM_CACHE_FP16S) {
          const float s = __uint_as_float(segmax[j]);
          inv_scale = s > 0.f ? 1.f / s : 0.f;
        }
        if (pos < eend) {
          store_entry<kFmt>(payload, pos, w, h0, h1, h2, inv_scale);
          pixoff[pos] = (uint8_t)threadIdx.x;
        } else {
          atomicOr(err, 1);
        }
        T = transmit(T, alpha);
      }
      done = dl;
      erun += add_e;
      srun += add_s;
    }
  }
  if (kThin) thin.n_live[(size_t)tile * kTilePix + threadIdx.x] = nlive == 0xffffffffu ? srun : nlive;
  if (threadIdx.x == 0 && (ebase + erun != eend || sbase + srun != send)) atomicOr(err, 4);
}

}  // namespace

cudaError_t launch_emit_keys(const uint32_t* sorted_slots, long long n_vis, const uint2* rect,
                             const unsigned long long* tmask, const DevCam* cams, int V, int N,
                             const unsigned long long* key_off, uint32_t* tile_keys, uint32_t* tile_vals,
                             cudaStream_t st) {
  (void)V;
  if (n_vis <= 0) return cudaSuccess;
  { k_emit_keys<<<(unsigned)((n_vis + 255) / 256), 256, 0, st>>>(sorted_slots, n_vis, rect, tmask, cams, N, key_off,
                                                               tile_keys, tile_vals); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_raster_count(const DevCam* cams, int V, int n_tiles, const uint32_t* tile_start,
                                const uint32_t* tile_end, const uint32_t* tile_vals, const SplatRec* rec,
                                int smooth, const float* targets, float* img, float* F, double* cost_partials,
                                uint32_t* tile_entries, uint32_t* tile_segs, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (tile_entries != nullptr)
    { k_raster_count<true><<<n_tiles, kTilePix, 0, st>>>(cams, V, tile_start, tile_end, tile_vals, rec, smooth,
                                                       targets, img, F, cost_partials, tile_entries, tile_segs); note_launch(); }
  else
    { k_raster_count<false><<<n_tiles, kTilePix, 0, st>>>(cams, V, tile_start, tile_end, tile_vals, rec, smooth,
                                                        targets, img, F, cost_partials, nullptr, nullptr); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_raster_write(const DevCam* cams, int V, int n_tiles, const uint32_t* tile_start,
                                const uint32_t* tile_end, const uint32_t* tile_vals, const SplatRec* rec,
                                int smooth, const float* img, const unsigned long long* tile_entry_off,
                                const uint32_t* tile_seg_off, int fmt, void* payload, float* seg_scale,
                                uint8_t* pixoff, unsigned long long* seg_entry_off, uint32_t* seg_slot,
                                SegRec* seg_rec, uint8_t* slot_active, int* err, const ThinOut& thin,
                                cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
#define GSLM_WRITE(F)                                                                                         \
  do {                                                                                                        \
    k_raster_write<F><<<n_tiles, kTilePix, 0, st>>>(cams, V, tile_start, tile_end, tile_vals, rec, smooth, img, \
                                                    tile_entry_off, tile_seg_off, payload, seg_scale, pixoff,   \
                                                    seg_entry_off, seg_slot, seg_rec, slot_active, err, thin);  \
    note_launch();                                                                                            \
  } while (0)
  if (fmt == GSLM_CACHE_FP32) GSLM_WRITE(GSLM_CACHE_FP32);
  else if (fmt == GSLM_CACHE_BF16) GSLM_WRITE(GSLM_CACHE_BF16);
  else if (fmt == GSLM_CACHE_THIN) GSLM_WRITE(GSLM_CACHE_THIN);
  else GSLM_WRITE(GSLM_CACHE_FP16S);
#undef GSLM_WRITE
  return cudaGetLastError();
}

}  // namespace gslm
