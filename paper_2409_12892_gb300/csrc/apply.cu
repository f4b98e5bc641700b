// J p, J^T u and the per-splat blocks of diag(J^T J) from the gradient cache
// (Sec. 3.3 "per-pixel-per-splat" parallelisation; Sec. A, Eq. apply-j,
// Eq. apply-jt, Eq. diag-jtj).
//
// One CTA per 16x16 tile; a group of G lanes walks one (tile, splat) segment at
// a time, reading consecutive cache entries with coalesced loads.
//
// For an entry (pixel, splat s) with payload (w, h0, h1, h2) and
// d = pixel centre - splat mean, the splat-attribute gradient of channel ch is
//   dc_ch/dy = [h_ch * gamma, w * e_ch],
//   gamma = (A dx + B dy, B dx + C dy, -dx^2/2, -dx dy, -dy^2/2, 1/o)
// (y = mean (2), conic (3), opacity, colour (3)). Hence
//   J p:    u_ch += w * rgbdot_ch + h_ch * (gamma . ydot_geo)
//   J^T u:  ybar_geo += (sum_ch h_ch u_ch) * gamma,  ybar_rgb_ch += w * u_ch
// apply_J accumulates u of the tile in shared memory and writes it once (no
// global atomics). apply_JT reads u of the tile from shared memory, reduces each
// segment inside its lane group and stores one 9-float partial per segment;
// the per-Gaussian adjoint kernel sums a splat's segments.
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

template <int kFmt>
__device__ __forceinline__ float4 load_entry(const void* __restrict__ payload, unsigned long long e, float scale) {
  if (kFmt == GSLM_CACHE_FP32) {
    return __ldcs(reinterpret_cast<const float4*>(payload) + e);
  } else {
    const uint2 u = __ldcs(reinterpret_cast<const uint2*>(payload) + e);
    if (kFmt == GSLM_CACHE_BF16) {
      const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
      const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
      const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      return make_float4(fa.x, fa.y, fb.x, fb.y);
    } else {
      const __half2 a = *reinterpret_cast<const __half2*>(&u.x);
      const __half2 b = *reinterpret_cast<const __half2*>(&u.y);
      const float2 fa = __half22float2(a), fb = __half22float2(b);
      return make_float4(fa.x * scale, fa.y * scale, fb.x * scale, fb.y * scale);
    }
  }
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if (G == 32) return kFull;
  const int lane = threadIdx.x & 31;
  return ((1u << G) - 1u) << (lane & ~(G - 1));
}

// ---------------------------------------------------------------------------
// Work distribution of both tile kernels: the tile's segment records are staged
// in shared memory first (below), then the warps of the tile's CTA take the
// staged segments from a shared counter (long and short segments balance) and
// stream each segment's entries with every lane keeping U loads in flight.
constexpr int kWarps = kTilePix / 32;

// Shared-memory index of pixel p of colour plane ch, padded by one word every
// 32 pixels (two tile rows) to spread a segment's pixels over more banks.
__device__ __forceinline__ int upad(int ch, int p) { return ch * (kTilePix + kTilePix / 32) + p + (p >> 5); }
constexpr int kPlane3 = 3 * (kTilePix + kTilePix / 32);   // floats of one padded 3-plane tile of u



// Raw payload as loaded (float4 for FP32, two 32-bit words for the 16-bit
// formats), decoded only when used so that U loads stay cheap in registers.
template <int kFmt>
struct Raw {
  using T = uint2;
};
template <>
struct Raw<GSLM_CACHE_FP32> {
  using T = float4;
};

template <int kFmt>
__device__ __forceinline__ typename Raw<kFmt>::T load_raw(const void* __restrict__ payload, unsigned long long e) {
  return __ldcs(reinterpret_cast<const typename Raw<kFmt>::T*>(payload) + e);
}

template <int kFmt>
__device__ __forceinline__ float4 decode(const typename Raw<kFmt>::T& r, float scale) {
  if constexpr (kFmt == GSLM_CACHE_FP32) {
    return r;
  } else if constexpr (kFmt == GSLM_CACHE_BF16) {
    const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  } else {
    const float2 fa = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 fb = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(fa.x * scale, fa.y * scale, fb.x * scale, fb.y * scale);
  }
}

// ---------------------------------------------------------------------------
// Tile kernels. A CTA (256 threads) works on one 16 x 16 tile at a time. The
// tile's segment records (and for J p the splat tangents the records point
// to) are first staged in shared memory, kStage segments at a time, by one
// coalesced cooperative load, so no warp waits on a chain of dependent
// global loads. Warps then take the staged segments in order; a warp works
// on 32 / G segments at once, one per group of G lanes, in lock step, with
// each lane keeping U entries in flight.
constexpr int kStage = 256;

__device__ __forceinline__ SegRec rec_from(const uint4& a, const uint4& b, const uint4& c) {
  SegRec s;
  s.e0 = ((unsigned long long)a.y << 32) | a.x;
  s.e1 = ((unsigned long long)a.w << 32) | a.z;
  s.slot = b.x;
  s.mx = __uint_as_float(b.y);
  s.my = __uint_as_float(b.z);
  s.A = __uint_as_float(b.w);
  s.B = __uint_as_float(c.x);
  s.C = __uint_as_float(c.y);
  s.io = __uint_as_float(c.z);
  s.scale = __uint_as_float(c.w);
  return s;
}

// Both tile kernels take a pixel's position as its offset (x', y') from the
// tile centre (7.5, 7.5) and fold the splat mean into per-segment constants,
// so no entry spends instructions on the offset from the mean: with e = mean -
// centre, the exponent tangent of J p is re-expanded in (x', y') and the
// J^T u moments about the centre are shifted to the mean after the sums.
constexpr float kTileCentre = 0.5f * (kTile - 1);

// Shared staging of one chunk of segments for J p: what a lane reads, prepared
// once per segment. The tangent of log alpha (alpha = o exp(-d^T Sigma'^-1 d / 2),
// the splat's blending weight at the pixel) is the quadratic
// q = K0 + x' (K1 + K3 x' + K4 y') + y' (K2 + K5 y').
struct StageJ {
  uint4 w0[kStage];     // e0 (low, high word), entry count, FP16S scale
  float4 w1[kStage];    // K0, K1, K2, K3
  float4 w2[kStage];    // K4, K5, colour tangents dr, dg
  float w3[kStage];     // colour tangent db
};
// For J^T u: the entry range read while streaming, and what the moments need
// after the sums (read then, so it holds no registers during the stream).
struct StageJT {
  uint4 w0[kStage];     // e0 (low, high word), entry count, FP16S scale
  float4 w1[kStage];    // e = mean - centre (x, y), conic A, B
  float2 w2[kStage];    // conic C, 1 / opacity
  uint32_t pos[kStage]; // splat-order position of the segment (output row)
  uint16_t order[kStage];   // processing order (groups of G < 32 lanes): by passes, most first
  uint32_t bcount[16];      // pass-count buckets (zero between stages)
};

// Groups of G < 32 lanes work on 32 / G segments per warp in lock step, each
// pass as long as the longest: the staged segments are taken in the order of
// their pass counts (ceil(entries / P), P = G U; most passes first, a counting
// sort in shared memory), so the segments a warp takes together need the same
// number of passes. Which group takes which segment does not change any
// result. Thread t holds staged segment t (cnt <= kStage = the CTA's threads).
template <int P>
__device__ __forceinline__ void order_by_passes(StageJT& S, int cnt) {
  constexpr int kB = kTilePix / P;
  static_assert(kB >= 1 && kB <= 16, "buckets");
  const int t = threadIdx.x;
  int bk = 0;
  if (t < cnt) {
    bk = kB - 1 - (int)min((S.w0[t].z - 1u) / (uint32_t)P, (uint32_t)(kB - 1));
    atomicAdd(&S.bcount[bk], 1u);
  }
  __syncthreads();
  if (t < 32) {   // bucket starts: exclusive scan of the counts
    const uint32_t c = t < kB ? S.bcount[t] : 0u;
    uint32_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(kFull, inc, o);
      if (t >= o) inc += x;
    }
    if (t < kB) S.bcount[t] = inc - c;
  }
  __syncthreads();
  if (t < cnt) S.order[atomicAdd(&S.bcount[bk], 1u)] = (uint16_t)t;
  __syncthreads();
  if (t < kB) S.bcount[t] = 0u;
}

__device__ __forceinline__ uint4 entry_word(const uint4& a, const uint4& c) {
  return make_uint4(a.x, a.y, a.z - a.x, c.w);   // segments hold < 2^32 entries
}

// The tile kernels' variants 8 and 9 ask L2 to fetch a segment's entries
// (payload and pixel offsets: two bulk prefetches, no completion to wait for,
// no registers held) kPf segments before a lane group takes it, so that its
// loads hit L2 instead of waiting on DRAM; the diagonal kernel asks for a
// group's next segment while it works on the current one. The prefetched ranges are widened to 16-byte
// boundaries; the cache's payload and pixel-offset arrays are allocated 32
// bytes long for this.
template <int kFmt>
__device__ __forceinline__ void prefetch_range_l2(const CacheView& cv, unsigned long long e0, unsigned long long e1) {
  constexpr unsigned long long B = kFmt == GSLM_CACHE_FP32 ? 16 : 8;
  const unsigned long long p0 = (e0 * B) & ~15ull, p1 = (e1 * B + 15ull) & ~15ull;
  const unsigned long long x0 = e0 & ~15ull, x1 = (e1 + 15ull) & ~15ull;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const unsigned char*>(cv.payload) + p0),
               "r"((uint32_t)(p1 - p0))
               : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(cv.pixoff + x0), "r"((uint32_t)(x1 - x0))
               : "memory");
}

template <int kFmt>
__device__ __forceinline__ void prefetch_segment_l2(const CacheView& cv, const uint4& w0) {
  const unsigned long long e0 = ((unsigned long long)w0.y << 32) | w0.x;
  prefetch_range_l2<kFmt>(cv, e0, e0 + w0.z);
}

// Stages segments [first, first + cnt) of the cache for J p; ydot holds the
// splat tangents (12 floats per splat: dmx, dmy, dA, dB, dC, do, dr, dg, db).
// With kPf > 0 the first kPf segments' entries are prefetched to L2.
template <int kFmt, int kPf>
__device__ __forceinline__ void stage_chunk_J(const CacheView& cv, uint32_t first, int cnt, StageJ& S,
                                              const float* __restrict__ ydot) {
  for (int t = threadIdx.x; t < cnt; t += kTilePix) {
    const uint4* q = reinterpret_cast<const uint4*>(cv.seg_rec + first + t);
    const uint4 a = q[0], b = q[1], c = q[2];
    if (kPf > 0 && t < kPf) prefetch_segment_l2<kFmt>(cv, entry_word(a, c));
    const SegRec r = rec_from(a, b, c);
    const float4* yd = reinterpret_cast<const float4*>(ydot + (size_t)r.slot * 12);
    const float4 y0 = yd[0], y1 = yd[1];
    const float db = ydot[(size_t)r.slot * 12 + 8];
    // q about the mean: k0 + dx (k1 + k3 dx + k4 dy) + dy (k2 + k5 dy)
    const float k1 = r.A * y0.x + r.B * y0.y, k2 = r.B * y0.x + r.C * y0.y;
    const float k3 = -0.5f * y0.z, k4 = -y0.w, k5 = -0.5f * y1.x, k0 = y1.y * r.io;
    // with dx = x' - ex, dy = y' - ey
    const float ex = r.mx - kTileCentre, ey = r.my - kTileCentre;
    const float K1 = k1 - 2.f * k3 * ex - k4 * ey, K2 = k2 - 2.f * k5 * ey - k4 * ex;
    const float K0 = k0 - ex * (k1 - k3 * ex - k4 * ey) - ey * (k2 - k5 * ey);
    S.w0[t] = entry_word(a, c);
    S.w1[t] = make_float4(K0, K1, K2, k3);
    S.w2[t] = make_float4(k4, k5, y1.z, y1.w);
    S.w3[t] = db;
  }
}

// Stages segments [first, first + cnt) of the cache for J^T u (kPf as for J p).
template <int kFmt, int kPf>
__device__ __forceinline__ void stage_chunk_JT(const CacheView& cv, uint32_t first, int cnt, StageJT& S) {
  for (int t = threadIdx.x; t < cnt; t += kTilePix) {
    const uint4* q = reinterpret_cast<const uint4*>(cv.seg_rec + first + t);
    const uint4 a = q[0], b = q[1], c = q[2];
    if (kPf > 0 && t < kPf) prefetch_segment_l2<kFmt>(cv, entry_word(a, c));
    const SegRec r = rec_from(a, b, c);
    S.w0[t] = entry_word(a, c);
    S.w1[t] = make_float4(r.mx - kTileCentre, r.my - kTileCentre, r.A, r.B);
    S.w2[t] = make_float2(r.C, r.io);
    S.pos[t] = cv.seg_pos[first + t];
  }
}

// Pixel p's offset from the tile centre.
__device__ __forceinline__ float2 centred_xy(int p) {
  return make_float2((float)(p & (kTile - 1)) - kTileCentre, (float)(p / kTile) - kTileCentre);
}

// Largest value of v over the groups of G lanes of the warp (all lanes converged).
template <int G>
__device__ __forceinline__ uint32_t warp_max_groups(uint32_t v) {
#pragma unroll
  for (int o = G; o < 32; o <<= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// J p over one tile. su (u of the tile, padded planes) must be zero on entry;
// sxy holds the pixels' offsets from the tile centre; the caller synchronises
// before.
// Epilogue of a J p tile: u = w (dc/dx) p with the residual-to-pixel weights
// (1 without them); for the predicted decrease, per-tile sums of e.u (Fadd
// holds e, or F for L2) and w.u^2, where u is the unweighted (dc/dx) p. The
// caller has synchronised after the last accumulation.
template <int kMode>
__device__ __forceinline__ void apply_J_epilogue(const CacheView& cv, int tile, const DevCam& cam, int tx, int ty,
                                                 const float* su, const float* __restrict__ Fadd,
                                                 float* __restrict__ u, double* __restrict__ sq_partials,
                                                 double* dred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx * kTile + (threadIdx.x & (kTile - 1)), y = ty * kTile + threadIdx.x / kTile;
  double local = 0.0, local2 = 0.0;
  if (x < cam.W && y < cam.H) {
    const long long pix = cam.pix_off + (long long)y * cam.W + x;
    const int p = threadIdx.x;
    float u0, u1, u2;
    if constexpr (kMode == 2) {
      u0 = u1 = u2 = 0.f;
      const float4* s4 = reinterpret_cast<const float4*>(su);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const float4 t = s4[w * kTilePix + p];
        u0 += t.x;
        u1 += t.y;
        u2 += t.z;
      }
    } else if constexpr (kMode == 1) {
      u0 = u1 = u2 = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        u0 += su[w * (3 * kTilePix) + p];
        u1 += su[w * (3 * kTilePix) + kTilePix + p];
        u2 += su[w * (3 * kTilePix) + 2 * kTilePix + p];
      }
    } else {
      u0 = su[upad(0, p)];
      u1 = su[upad(1, p)];
      u2 = su[upad(2, p)];
    }
    float w0 = 1.f, w1 = 1.f, w2 = 1.f;
    if (cv.wres != nullptr) {
      w0 = cv.wres[pix * 3 + 0];
      w1 = cv.wres[pix * 3 + 1];
      w2 = cv.wres[pix * 3 + 2];
    }
    if (u != nullptr) {
      u[pix * 3 + 0] = w0 * u0;
      u[pix * 3 + 1] = w1 * u1;
      u[pix * 3 + 2] = w2 * u2;
    }
    if (sq_partials != nullptr) {
      const float* f = Fadd + pix * 3;
      local = (double)(f[0] * u0 + f[1] * u1 + f[2] * u2);
      local2 = (double)(w0 * u0 * u0 + w1 * u1 * u1 + w2 * u2 * u2);
    }
  }
  if (sq_partials != nullptr) {
    for (int o = 16; o > 0; o >>= 1) {
      local += __shfl_xor_sync(kFull, local, o);
      local2 += __shfl_xor_sync(kFull, local2, o);
    }
    if (lane == 0) {
      dred[warp] = local;
      dred[kWarps + warp] = local2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0, s2 = 0.0;
      for (int w = 0; w < kWarps; ++w) {
        s += dred[w];
        s2 += dred[kWarps + w];
      }
      sq_partials[tile] = s;
      sq_partials[cv.n_tiles + tile] = s2;
    }
  }
}

// kMode 0: one tile of u accumulated with shared-memory atomics. kMode 1 (G =
// 32 only): a warp works on one segment at a time, whose entries are distinct
// pixels, so each warp adds into its own copy of the tile with plain
// read-modify-writes and the copies are summed in the epilogue. kMode 2: as 1
// with the copy's three channels of a pixel in one float4 (one 16-byte load
// and one store per entry instead of three of each).
template <int kFmt, int G, int U, int kMode, int kPf>
__device__ __forceinline__ void apply_J_tile(const CacheView& cv, int tile, const float* __restrict__ ydot,
                                             const float* __restrict__ Fadd, float* __restrict__ u,
                                             double* __restrict__ sq_partials, float* su, const float2* sxy,
                                             double* dred, unsigned int* next_seg, StageJ& S) {
  static_assert(G == 8 || G == 16 || G == 32, "group size");
  static_assert(kMode == 0 || G == 32, "private tiles need one segment per warp");
  constexpr int kGPW = 32 / G;
  const int v = find_view(cv.cams, cv.V, tile);
  const DevCam& cam = cv.cams[v];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (G - 1), grp = lane / G;
  const uint32_t g0 = cv.tile_seg_off[tile];
  const uint32_t n = cv.tile_seg_off[tile + 1] - g0;
  for (uint32_t c0 = 0; c0 < n; c0 += kStage) {
    const int cnt = (int)min((uint32_t)kStage, n - c0);
    stage_chunk_J<kFmt, kPf>(cv, g0 + c0, cnt, S, ydot);
    if (threadIdx.x == 0) *next_seg = 0;
    __syncthreads();
    for (;;) {
      uint32_t kb = 0;
      if (lane == 0) kb = atomicAdd(next_seg, (unsigned)kGPW);
      kb = __shfl_sync(kFull, kb, 0);
      if (kb >= (uint32_t)cnt) break;
      const uint32_t k = kb + grp;
      const bool has = k < (uint32_t)cnt;
      if constexpr (kPf > 0) {
        if (gl == 0 && k + kPf < (uint32_t)cnt) prefetch_segment_l2<kFmt>(cv, S.w0[k + kPf]);
      }
      uint4 w0 = make_uint4(0u, 0u, 0u, 0u);
      float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f), w2 = w1;
      float db = 0.f;
      if (has) {
        w0 = S.w0[k];
        w1 = S.w1[k];
        w2 = S.w2[k];
        db = S.w3[k];
      }
      const uint32_t len = w0.z;
      const float scale = __uint_as_float(w0.w);
      const unsigned long long e0 = ((unsigned long long)w0.y << 32) | w0.x;
      const float K0 = w1.x, K1 = w1.y, K2 = w1.z, K3 = w1.w, K4 = w2.x, K5 = w2.y, dr = w2.z, dg = w2.w;
      const uint32_t mlen = warp_max_groups<G>(len);
      const typename Raw<kFmt>::T* pl = reinterpret_cast<const typename Raw<kFmt>::T*>(cv.payload) + e0;
      const uint8_t* po = cv.pixoff + e0;
      for (uint32_t base = 0; base < mlen; base += G * U) {
        typename Raw<kFmt>::T raw[U];
        int pp[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const uint32_t i = base + gl + G * j;
          if (i < len) {
            raw[j] = __ldcs(pl + i);
            pp[j] = po[i];
          }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const uint32_t i = base + gl + G * j;
          if (i < len) {
            const int p = pp[j];
            const float4 pe = decode<kFmt>(raw[j], scale);
            const float2 c = sxy[p];
            const float q = fmaf(c.x, fmaf(K3, c.x, fmaf(K4, c.y, K1)), fmaf(c.y, fmaf(K5, c.y, K2), K0));
            const float v0 = fmaf(pe.x, dr, pe.y * q), v1 = fmaf(pe.x, dg, pe.z * q);
            const float v2 = fmaf(pe.x, db, pe.w * q);
            if constexpr (kMode == 2) {   // the warp's own tile of float4 [p]
              float4* sp = reinterpret_cast<float4*>(su) + warp * kTilePix + p;
              float4 t = *sp;
              t.x += v0;
              t.y += v1;
              t.z += v2;
              *sp = t;
            } else if constexpr (kMode == 1) {   // the warp's own unpadded planes [ch][p]
              float* sp = su + warp * (3 * kTilePix) + p;
              sp[0] += v0;
              sp[kTilePix] += v1;
              sp[2 * kTilePix] += v2;
            } else {   // upad(ch, p) = sp + ch * (kTilePix + kTilePix / 32)
              float* sp = su + p + (p >> 5);
              atomicAdd(sp, v0);
              atomicAdd(sp + (kTilePix + kTilePix / 32), v1);
              atomicAdd(sp + 2 * (kTilePix + kTilePix / 32), v2);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  apply_J_epilogue<kMode>(cv, tile, cam, tx, ty, su, Fadd, u, sq_partials, dred);
}

// Floats of the J p accumulation tile(s) of each mode.
constexpr int su_floats(int mode) { return mode == 2 ? kWarps * 4 * kTilePix : mode == 1 ? kWarps * 3 * kTilePix : kPlane3; }

#define APPLY_J_SHARED                                   \
  __shared__ __align__(16) float su[su_floats(kMode)];   \
  __shared__ float2 sxy[kTilePix];                       \
  __shared__ double dred[2 * kWarps];                    \
  __shared__ unsigned int next_seg;                      \
  __shared__ StageJ S;                                   \
  sxy[threadIdx.x] = centred_xy(threadIdx.x);

template <int kFmt, int G, int U, int kMinBlocks, int kMode, int kPf>
__global__ void __launch_bounds__(kTilePix, kMinBlocks) k_apply_J(CacheView cv, const float* __restrict__ ydot,
                                                                  const float* __restrict__ Fadd,
                                                                  float* __restrict__ u,
                                                                  double* __restrict__ sq_partials) {
  if (cv.skip != nullptr && *cv.skip) return;
  APPLY_J_SHARED
  for (int i = threadIdx.x; i < su_floats(kMode); i += kTilePix) su[i] = 0.f;
  __syncthreads();
  apply_J_tile<kFmt, G, U, kMode, kPf>(cv, blockIdx.x, ydot, Fadd, u, sq_partials, su, sxy, dred, &next_seg, S);
}

// Subset of a global tile index of a batch.
__device__ __forceinline__ int batch_subset(const TileBatch& tb, long long gt) {
  int b = 0;
  while (b + 1 < tb.n && gt >= tb.tile_end[b]) ++b;
  return b;
}

// Persistent J p over every subset of a batch: each CTA takes tiles from the
// batch's queue until all are done (tiles of finished solves are skipped).
template <int kFmt, int G, int U, int kMinBlocks, int kMode, int kPf>
__global__ void __launch_bounds__(kTilePix, kMinBlocks) k_apply_J_batch(const __grid_constant__ TileBatch tb) {
  APPLY_J_SHARED
  __shared__ long long s_tile;
  for (;;) {
    for (int i = threadIdx.x; i < su_floats(kMode); i += kTilePix) su[i] = 0.f;
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(tb.queue, 1u);
    __syncthreads();
    const long long gt = s_tile;
    if (gt >= tb.total_tiles) break;
    const int b = batch_subset(tb, gt);
    const CacheView& cv = tb.v[b];
    if (cv.skip == nullptr || *cv.skip == 0)
      apply_J_tile<kFmt, G, U, kMode, kPf>(cv, (int)(gt - (b > 0 ? tb.tile_end[b - 1] : 0)), tb.ydot[b], nullptr, tb.u[b],
                               nullptr, su, sxy, dred, &next_seg, S);
    __syncthreads();
  }
}

// One step of a recursive-halving reduction: lanes whose `upper` bit is set keep
// the upper half of their N values, the others the lower half; each kept value
// gains the partner lane's matching value.
template <int N>
__device__ __forceinline__ void halve(float (&v)[16], bool upper, int o) {
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    const float send = upper ? v[k] : v[k + N / 2];
    const float keep = upper ? v[k + N / 2] : v[k];
    v[k] = keep + __shfl_xor_sync(kFull, send, o);
  }
}

// Sums 16 values over each group of G lanes (all 32 lanes converged). G = 32:
// lanes 0, 2, ..., 30 then hold the sum of value index lane / 2 in v[0]; G = 16:
// lane l of a group holds the sum of value index l in v[0]; G = 8: lane l of
// a group holds the sums of value indices 2l and 2l + 1 in v[0] and v[1].
template <int G>
__device__ __forceinline__ void group_sum16(float (&v)[16], int lane) {
  if constexpr (G == 32) {
    halve<16>(v, lane & 16, 16);
    halve<8>(v, lane & 8, 8);
    halve<4>(v, lane & 4, 4);
    halve<2>(v, lane & 2, 2);
    v[0] += __shfl_xor_sync(kFull, v[0], 1);
  } else if constexpr (G == 16) {
    halve<16>(v, lane & 8, 8);
    halve<8>(v, lane & 4, 4);
    halve<4>(v, lane & 2, 2);
    halve<2>(v, lane & 1, 1);
  } else {
    halve<16>(v, lane & 4, 4);
    halve<8>(v, lane & 2, 2);
    halve<4>(v, lane & 1, 1);
  }
}

// Moment i of the group after group_sum16<G>, on every lane of the group.
template <int G>
__device__ __forceinline__ float group_moment(const float (&v)[16], int i) {
  if constexpr (G == 32) return __shfl_sync(kFull, v[0], 2 * i, 32);
  else if constexpr (G == 16) return __shfl_sync(kFull, v[0], i, 16);
  else return __shfl_sync(kFull, (i & 1) ? v[1] : v[0], i >> 1, 8);
}

// Shared-memory transpose of a 16-lane group's 9 partial sums: rows of 20
// floats (16 lanes + 4 of padding, so that the 16-byte row reads of lanes
// 0..7 hit distinct banks) and a group stride of 208 floats (16 banks apart,
// so that the two groups of a warp store without conflicts).
constexpr int kRedRow = 20;
constexpr int kRedGroup = 208;
static_assert(9 * kRedRow <= kRedGroup && kRedGroup % 32 == 16 && kRedRow % 4 == 0, "transpose layout");

// J^T u over one tile into per-segment partials, stored at each segment's
// splat-order position (so the adjoint kernel reads a splat's partials as one
// contiguous range). The caller synchronises before. su4 / sxy are filled here.
template <int kFmt, int G, int U, int kPf>
__device__ __forceinline__ void apply_JT_tile(const CacheView& cv, int tile, const float* __restrict__ u,
                                              float* __restrict__ seg_ybar, float4* su4, float2* sxy,
                                              unsigned int* next_seg, StageJT& S, float* sred) {
  static_assert(G == 8 || G == 16 || G == 32, "group size");
  constexpr int kGPW = 32 / G;
  const uint32_t g0 = cv.tile_seg_off[tile];
  const uint32_t n = cv.tile_seg_off[tile + 1] - g0;
  if (n == 0) return;
  const int v = find_view(cv.cams, cv.V, tile);
  const DevCam& cam = cv.cams[v];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  {
    const int x = tx * kTile + (threadIdx.x & (kTile - 1)), y = ty * kTile + threadIdx.x / kTile;
    float4 uv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x < cam.W && y < cam.H) {
      const long long pix = cam.pix_off + (long long)y * cam.W + x;
      uv = make_float4(u[pix * 3 + 0], u[pix * 3 + 1], u[pix * 3 + 2], 0.f);
    }
    su4[threadIdx.x] = uv;
    sxy[threadIdx.x] = centred_xy(threadIdx.x);
  }
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1), grp = lane / G;
  for (uint32_t c0 = 0; c0 < n; c0 += kStage) {
    const int cnt = (int)min((uint32_t)kStage, n - c0);
    stage_chunk_JT<kFmt, kPf>(cv, g0 + c0, cnt, S);
    if (threadIdx.x == 0) *next_seg = 0;
    if constexpr (G < 32) order_by_passes<G * U>(S, cnt);
    else __syncthreads();
    for (;;) {
      uint32_t kb = 0;
      if (lane == 0) kb = atomicAdd(next_seg, (unsigned)kGPW);
      kb = __shfl_sync(kFull, kb, 0);
      if (kb >= (uint32_t)cnt) break;
      const bool has = kb + grp < (uint32_t)cnt;
      const uint32_t k = !has ? 0u : G < 32 ? (uint32_t)S.order[kb + grp] : kb + grp;   // staged index
      if constexpr (kPf > 0) {
        const uint32_t kp = kb + grp + kPf;
        if (gl == 0 && kp < (uint32_t)cnt) prefetch_segment_l2<kFmt>(cv, S.w0[G < 32 ? (uint32_t)S.order[kp] : kp]);
      }
      const uint4 w0 = has ? S.w0[k] : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t len = w0.z;
      const float scale = __uint_as_float(w0.w);
      const unsigned long long e0 = ((unsigned long long)w0.y << 32) | w0.x;
      const uint32_t mlen = warp_max_groups<G>(len);
      // moments of s = h . u over the segment's pixels, taken about the tile
      // centre, and sums of w u; the shift to the mean and the conic are
      // applied once per segment
      float a[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] = 0.f;
      const typename Raw<kFmt>::T* pl = reinterpret_cast<const typename Raw<kFmt>::T*>(cv.payload) + e0;
      const uint8_t* po = cv.pixoff + e0;
      for (uint32_t base = 0; base < mlen; base += G * U) {
        typename Raw<kFmt>::T raw[U];
        int pp[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const uint32_t i = base + gl + G * j;
          if (i < len) {
            raw[j] = __ldcs(pl + i);
            pp[j] = po[i];
          }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const uint32_t i = base + gl + G * j;
          if (i < len) {
            const int p = pp[j];
            const float4 pej = decode<kFmt>(raw[j], scale);
            const float4 uv = su4[p];
            const float2 c = sxy[p];
            const float sv = pej.y * uv.x + pej.z * uv.y + pej.w * uv.z;
            const float t1 = sv * c.x, t2 = sv * c.y;
            a[0] += sv;
            a[1] += t1;
            a[2] += t2;
            a[3] += t1 * c.x;
            a[4] += t1 * c.y;
            a[5] += t2 * c.y;
            a[6] += pej.x * uv.x;
            a[7] += pej.x * uv.y;
            a[8] += pej.x * uv.z;
          }
        }
      }
      // sums about the centre: S0 = sum s, Sx = sum s x', Sy = sum s y', Sxx,
      // Sxy, Syy, then the three sums of w u. With e = mean - centre the moments
      // about the mean are m1 = Sx - ex S0, m2 = Sy - ey S0, m3 = sum s dx^2 =
      // Sxx - ex (Sx + m1), m4 = sum s dx dy = Sxy - ey Sx - ex m2 and
      // m5 = sum s dy^2 = Syy - ey (Sy + m2)
      if constexpr (G == 16) {
        // the group's 16 x 9 partials transposed through shared memory: lane o
        // (o < 9) reads row o (the 16 lanes' partials of sum o) with four
        // 16-byte loads, in place of a 16-value shuffle reduction
        float* rb = sred + ((threadIdx.x >> 5) * 2 + grp) * kRedGroup;
#pragma unroll
        for (int i = 0; i < 9; ++i) rb[i * kRedRow + gl] = a[i];
        __syncwarp();
        float so = 0.f;
        if (gl < 9) {
          const float4* row = reinterpret_cast<const float4*>(rb + gl * kRedRow);
          const float4 q0 = row[0], q1 = row[1], q2 = row[2], q3 = row[3];
          so = ((q0.x + q0.y) + (q0.z + q0.w) + ((q1.x + q1.y) + (q1.z + q1.w))) +
               ((q2.x + q2.y) + (q2.z + q2.w) + ((q3.x + q3.y) + (q3.z + q3.w)));
        }
        __syncwarp();   // the next segment's partials overwrite rb
        // lane o of the group holds sum o: output o needs sum o (6..8), its
        // neighbour's (2..4) and S0, Sx, Sy (four shuffles in all)
        const float sn = __shfl_down_sync(kFull, so, 1, 16);
        const float s0 = __shfl_sync(kFull, so, 0, 16);
        const float s1 = __shfl_sync(kFull, so, 1, 16);
        const float s2 = __shfl_sync(kFull, so, 2, 16);
        if (has && gl < 9) {
          const float4 w1 = S.w1[k];
          const float2 w2 = S.w2[k];
          const float ex = w1.x, ey = w1.y;
          const float m1 = fmaf(-ex, s0, s1), m2 = fmaf(-ey, s0, s2);
          float val = so;
          if (gl == 0) val = w1.z * m1 + w1.w * m2;
          else if (gl == 1) val = w1.w * m1 + w2.x * m2;
          else if (gl == 2) val = -0.5f * fmaf(-ex, s1 + m1, sn);
          else if (gl == 3) val = -fmaf(-ey, s1, fmaf(-ex, m2, sn));
          else if (gl == 4) val = -0.5f * fmaf(-ey, s2 + m2, sn);
          else if (gl == 5) val = s0 * w2.y;
          seg_ybar[(size_t)S.pos[k] * 12 + gl] = val;
        }
        continue;
      }
      group_sum16<G>(a, lane);
      float m[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) m[i] = group_moment<G>(a, i);
      if (has) {
        const float4 w1 = S.w1[k];
        const float2 w2 = S.w2[k];
        const float ex = w1.x, ey = w1.y;
        const float m1 = fmaf(-ex, m[0], m[1]), m2 = fmaf(-ey, m[0], m[2]);
        // output o of the segment's 9 (G = 8: lane 0 also writes output 8)
        for (int o = gl; o < 9; o += G) {
          float val = m[o];
          if (o == 0) val = w1.z * m1 + w1.w * m2;
          else if (o == 1) val = w1.w * m1 + w2.x * m2;
          else if (o == 2) val = -0.5f * fmaf(-ex, m[1] + m1, m[3]);
          else if (o == 3) val = -fmaf(-ey, m[1], fmaf(-ex, m2, m[4]));
          else if (o == 4) val = -0.5f * fmaf(-ey, m[2] + m2, m[5]);
          else if (o == 5) val = m[0] * w2.y;
          seg_ybar[(size_t)S.pos[k] * 12 + o] = val;
        }
      }
    }
    __syncthreads();
  }
}

#define APPLY_JT_SHARED                                      \
  __shared__ float4 su4[kTilePix];                           \
  __shared__ float2 sxy[kTilePix];                           \
  __shared__ unsigned int next_seg;                          \
  __shared__ StageJT S;                                      \
  __shared__ __align__(16) float sred[G == 16 ? kWarps * 2 * kRedGroup : 4];

template <int kFmt, int G, int U, int kMinBlocks, int kPf>
__global__ void __launch_bounds__(kTilePix, kMinBlocks) k_apply_JT(CacheView cv, const float* __restrict__ u,
                                                                   float* __restrict__ seg_ybar) {
  APPLY_JT_SHARED
  if (cv.skip != nullptr && *cv.skip) return;
  if (threadIdx.x < 16) S.bcount[threadIdx.x] = 0u;
  __syncthreads();
  apply_JT_tile<kFmt, G, U, kPf>(cv, blockIdx.x, u, seg_ybar, su4, sxy, &next_seg, S, sred);
}

// Persistent J^T u over every subset of a batch (see k_apply_J_batch).
template <int kFmt, int G, int U, int kMinBlocks, int kPf>
__global__ void __launch_bounds__(kTilePix, kMinBlocks) k_apply_JT_batch(const __grid_constant__ TileBatch tb) {
  APPLY_JT_SHARED
  __shared__ long long s_tile;
  if (threadIdx.x < 16) S.bcount[threadIdx.x] = 0u;   // the loop's first barrier orders it
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(tb.queue, 1u);
    __syncthreads();
    const long long gt = s_tile;
    if (gt >= tb.total_tiles) break;
    const int b = batch_subset(tb, gt);
    const CacheView& cv = tb.v[b];
    if (cv.skip == nullptr || *cv.skip == 0)
      apply_JT_tile<kFmt, G, U, kPf>(cv, (int)(gt - (b > 0 ? tb.tile_end[b - 1] : 0)), tb.u[b], tb.seg_ybar[b], su4, sxy,
                                &next_seg, S, sred);
    __syncthreads();
  }
}

// Per segment: Q = sum over entries and channels of rho_ch a_ch a_ch^T with
// a_ch = [h_ch gamma, w e_ch] and rho_ch the residual-to-pixel weight of the
// entry's pixel channel (1 for L2); stored as kDiagBlock floats: Qgg (21,
// upper triangle of the 6x6 block, row-major), X (18, 6x3: sum rho_c w h_c
// gamma_i), D_ch (3: sum rho_ch w^2) and two zeros of padding. A group of
// kDiagG lanes takes one segment (two segments per warp in lock step), so
// short segments leave fewer lanes idle and the three 16-value reductions
// serve two segments at once.
constexpr int kDiagG = 16;

template <int kFmt, bool kWeighted>
__global__ void __launch_bounds__(kTilePix) k_diag_entries(CacheView cv, float* __restrict__ seg_q) {
  constexpr int kGPW = 32 / kDiagG;
  constexpr int kPass = 2 * kDiagG;   // entries per pass of a group (two per lane)
  constexpr int kBk = kTilePix / kPass;
  __shared__ float sw[3][kWeighted ? kTilePix : 1];   // residual-to-pixel weights of the tile's pixels
  __shared__ uint16_t sorder[kTilePix];               // a chunk's segments by pass count, most first
  __shared__ uint32_t sbc[kBk];
  const int tile = blockIdx.x;
  const uint32_t g0 = cv.tile_seg_off[tile], g1 = cv.tile_seg_off[tile + 1];
  if (g0 == g1) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (kDiagG - 1), grp = lane / kDiagG;
  if constexpr (kWeighted) {
    const DevCam& cam = cv.cams[find_view(cv.cams, cv.V, tile)];
    const int lt = tile - cam.tile_off;
    const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
    const int x = tx * kTile + (threadIdx.x & (kTile - 1)), y = ty * kTile + threadIdx.x / kTile;
    float w0 = 1.f, w1 = 1.f, w2 = 1.f;
    if (x < cam.W && y < cam.H) {
      const long long pix = cam.pix_off + (long long)y * cam.W + x;
      w0 = cv.wres[pix * 3 + 0];
      w1 = cv.wres[pix * 3 + 1];
      w2 = cv.wres[pix * 3 + 2];
    }
    sw[0][threadIdx.x] = w0;
    sw[1][threadIdx.x] = w1;
    sw[2][threadIdx.x] = w2;
  }
  if (threadIdx.x < kBk) sbc[threadIdx.x] = 0u;
  __syncthreads();
  // The tile's segments in chunks of 256, each taken in the order of its
  // segments' pass counts (as the J^T u kernel does), so that the two
  // segments a warp works on together need the same number of passes.
  for (uint32_t c0 = g0; c0 < g1; c0 += kTilePix) {
    const int cnt = (int)min((uint32_t)kTilePix, g1 - c0);
    int bk = 0;
    if ((int)threadIdx.x < cnt) {
      const uint32_t len = (uint32_t)(cv.seg_entry_off[c0 + threadIdx.x + 1] - cv.seg_entry_off[c0 + threadIdx.x]);
      bk = kBk - 1 - (int)min((len - 1u) / (uint32_t)kPass, (uint32_t)(kBk - 1));
      atomicAdd(&sbc[bk], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t c = threadIdx.x < kBk ? sbc[threadIdx.x] : 0u;
      uint32_t inc = c;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, inc, o);
        if ((int)threadIdx.x >= o) inc += x;
      }
      if (threadIdx.x < kBk) sbc[threadIdx.x] = inc - c;
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) sorder[atomicAdd(&sbc[bk], 1u)] = (uint16_t)threadIdx.x;
    __syncthreads();
    if (threadIdx.x < kBk) sbc[threadIdx.x] = 0u;
    // every lane of a warp runs the same number of rounds (the reductions shuffle over the warp)
    for (int qb = warp * kGPW; qb < cnt; qb += kWarps * kGPW) {
      const bool has = qb + grp < cnt;
      const uint32_t seg = c0 + (has ? (uint32_t)sorder[qb + grp] : 0u);
      float q[42];
  #pragma unroll
      for (int i = 0; i < 42; ++i) q[i] = 0.f;
      if (has) {
        const uint4* rq = reinterpret_cast<const uint4*>(cv.seg_rec + seg);
        const SegRec r = rec_from(rq[0], rq[1], rq[2]);   // tile-local mean, conic, 1/o, FP16 scale
        const float mx = r.mx, my = r.my, A = r.A, B = r.B, C = r.C, io = r.io;
        const float scale = kFmt == GSLM_CACHE_FP16S ? r.scale : 1.f;
        // the entry range of the group's next segment, asked of L2 after this one's entries
        const int nq = qb + grp + kWarps * kGPW;
        const bool pf = gl == 0 && nq < cnt;
        unsigned long long ne0 = 0, ne1 = 0;
        if (pf) {
          const uint32_t nseg = c0 + sorder[nq];
          ne0 = cv.seg_entry_off[nseg];
          ne1 = cv.seg_entry_off[nseg + 1];
        }
        auto add_entry = [&](const float4& pe, int p) {
          float wr = 1.f, wg = 1.f, wb = 1.f;
          if constexpr (kWeighted) {
            wr = sw[0][p];
            wg = sw[1][p];
            wb = sw[2][p];
          }
          const float dx = (float)(p & (kTile - 1)) - mx, dy = (float)(p / kTile) - my;
          float gam[6] = {A * dx + B * dy, B * dx + C * dy, -0.5f * dx * dx, -dx * dy, -0.5f * dy * dy, io};
          const float H2 = wr * pe.y * pe.y + wg * pe.z * pe.z + wb * pe.w * pe.w;
          int k = 0;
  #pragma unroll
          for (int i = 0; i < 6; ++i)
  #pragma unroll
            for (int j = i; j < 6; ++j) q[k++] += H2 * gam[i] * gam[j];
          const float xr = wr * pe.x * pe.y, xg = wg * pe.x * pe.z, xb = wb * pe.x * pe.w;
  #pragma unroll
          for (int i = 0; i < 6; ++i) {
            q[21 + 3 * i + 0] += xr * gam[i];
            q[21 + 3 * i + 1] += xg * gam[i];
            q[21 + 3 * i + 2] += xb * gam[i];
          }
          const float aa = pe.x * pe.x;
          q[39] += wr * aa;
          q[40] += wg * aa;
          q[41] += wb * aa;
        };
        // two entries per lane in flight
        unsigned long long e = r.e0 + gl;
        for (; e + kDiagG < r.e1; e += 2 * kDiagG) {
          const float4 pa = load_entry<kFmt>(cv.payload, e, scale);
          const float4 pb = load_entry<kFmt>(cv.payload, e + kDiagG, scale);
          const int xa = cv.pixoff[e], xb = cv.pixoff[e + kDiagG];
          add_entry(pa, xa);
          add_entry(pb, xb);
        }
        if (e < r.e1) add_entry(load_entry<kFmt>(cv.payload, e, scale), cv.pixoff[e]);
        if (pf) prefetch_range_l2<kFmt>(cv, ne0, ne1);
      }
      // three recursive-halving reductions of 16 values over the group: lane gl
      // then holds sum gl of each block
      float b0[16], b1[16], b2[16];
  #pragma unroll
      for (int i = 0; i < 16; ++i) {
        b0[i] = q[i];
        b1[i] = q[16 + i];
        b2[i] = i < 10 ? q[32 + i] : 0.f;
      }
      group_sum16<kDiagG>(b0, lane);
      group_sum16<kDiagG>(b1, lane);
      group_sum16<kDiagG>(b2, lane);
      if (has) {
        float* out = seg_q + (size_t)cv.seg_pos[seg] * kDiagBlock;
        out[gl] = b0[0];
        out[16 + gl] = b1[0];
        if (gl < kDiagBlock - 32) out[32 + gl] = b2[0];   // the last two are zero padding
      }
    }
    __syncthreads();   // sorder is rewritten by the next chunk
  }
}

// Variants: lanes per segment (G), entries each lane keeps in flight (U) and
// the minimum number of resident 256-thread blocks per SM the registers must
// allow: 0 = (16, 2, 6), 1 = (16, 4, 5), 2 = (32, 2, 6), 3 = (32, 4, 4),
// 4 = (8, 2, 6); 5 = J p with per-warp private tiles (32, 2, 4) and J^T u
// (16, 4, 4); 6 = J p private tiles (32, 3, 4) and J^T u (32, 3, 4); 7 = J p
// (32, 3, 6) and J^T u (16, 3, 5). U = 3 fills a 94-entry segment (the paper
// workload's mean) with 96 lane slots at G = 32 or 2 x 48 at G = 16.
// With L2 prefetch of the segment 16 ahead: 8 = J p private tiles (32, 3, 4)
// and J^T u (8, 2, 6); 9 = J p float4 private tiles (32, 4, 4) and J^T u
// (8, 4, 5).
template <int kFmt, int G, int U, int B, int kMode = 0, int kPf = 0>
cudaError_t run_J(const CacheView& cv, const float* ydot, const float* F_add, float* u, double* sq, cudaStream_t st) {
  k_apply_J<kFmt, G, U, B, kMode, kPf><<<cv.n_tiles, kTilePix, 0, st>>>(cv, ydot, F_add, u, sq);
  note_launch();
  return cudaGetLastError();
}

template <int kFmt, int G, int U, int B, int kPf = 0>
cudaError_t run_JT(const CacheView& cv, const float* u, float* seg_ybar, cudaStream_t st) {
  k_apply_JT<kFmt, G, U, B, kPf><<<cv.n_tiles, kTilePix, 0, st>>>(cv, u, seg_ybar);
  note_launch();
  return cudaGetLastError();
}

template <int kFmt, int G, int U, int B, int kMode = 0, int kPf = 0>
cudaError_t run_J_batch(const TileBatch& tb, int ctas, cudaStream_t st) {
  k_apply_J_batch<kFmt, G, U, B, kMode, kPf><<<ctas, kTilePix, 0, st>>>(tb);
  note_launch();
  return cudaGetLastError();
}

template <int kFmt, int G, int U, int B, int kPf = 0>
cudaError_t run_JT_batch(const TileBatch& tb, int ctas, cudaStream_t st) {
  k_apply_JT_batch<kFmt, G, U, B, kPf><<<ctas, kTilePix, 0, st>>>(tb);
  note_launch();
  return cudaGetLastError();
}

template <int kFmt>
cudaError_t apply_J_batch_variant(int variant, const TileBatch& tb, int ctas, cudaStream_t st) {
  switch (variant) {
    case 0: return run_J_batch<kFmt, 16, 2, 6>(tb, ctas, st);
    case 1: return run_J_batch<kFmt, 16, 4, 5>(tb, ctas, st);
    case 2: return run_J_batch<kFmt, 32, 2, 6>(tb, ctas, st);
    case 3: return run_J_batch<kFmt, 32, 4, 4>(tb, ctas, st);
    case 5: return run_J_batch<kFmt, 32, 2, 4, 1>(tb, ctas, st);
    case 6: return run_J_batch<kFmt, 32, 3, 4, 1>(tb, ctas, st);
    case 7: return run_J_batch<kFmt, 32, 3, 6>(tb, ctas, st);
    case 8: return run_J_batch<kFmt, 32, 3, 4, 1, 16>(tb, ctas, st);
    case 9: return run_J_batch<kFmt, 32, 4, 4, 2, 16>(tb, ctas, st);
    default: return run_J_batch<kFmt, 8, 2, 6>(tb, ctas, st);
  }
}

template <int kFmt>
cudaError_t apply_JT_batch_variant(int variant, const TileBatch& tb, int ctas, cudaStream_t st) {
  switch (variant) {
    case 0: return run_JT_batch<kFmt, 16, 2, 6>(tb, ctas, st);
    case 1: return run_JT_batch<kFmt, 16, 4, 5>(tb, ctas, st);
    case 2: return run_JT_batch<kFmt, 32, 2, 6>(tb, ctas, st);
    case 3: return run_JT_batch<kFmt, 32, 4, 4>(tb, ctas, st);
    case 5: return run_JT_batch<kFmt, 16, 4, 4>(tb, ctas, st);
    case 6: return run_JT_batch<kFmt, 32, 3, 4>(tb, ctas, st);
    case 7: return run_JT_batch<kFmt, 16, 3, 5>(tb, ctas, st);
    case 8: return run_JT_batch<kFmt, 8, 2, 6, 16>(tb, ctas, st);
    case 9: return run_JT_batch<kFmt, 8, 4, 5, 16>(tb, ctas, st);
    default: return run_JT_batch<kFmt, 8, 2, 6>(tb, ctas, st);
  }
}

template <int kFmt>
cudaError_t apply_J_variant(int variant, const CacheView& cv, const float* ydot, const float* F_add, float* u,
                            double* sq, cudaStream_t st) {
  switch (variant) {
    case 0: return run_J<kFmt, 16, 2, 6>(cv, ydot, F_add, u, sq, st);
    case 1: return run_J<kFmt, 16, 4, 5>(cv, ydot, F_add, u, sq, st);
    case 2: return run_J<kFmt, 32, 2, 6>(cv, ydot, F_add, u, sq, st);
    case 3: return run_J<kFmt, 32, 4, 4>(cv, ydot, F_add, u, sq, st);
    case 5: return run_J<kFmt, 32, 2, 4, 1>(cv, ydot, F_add, u, sq, st);
    case 6: return run_J<kFmt, 32, 3, 4, 1>(cv, ydot, F_add, u, sq, st);
    case 7: return run_J<kFmt, 32, 3, 6>(cv, ydot, F_add, u, sq, st);
    case 8: return run_J<kFmt, 32, 3, 4, 1, 16>(cv, ydot, F_add, u, sq, st);
    case 9: return run_J<kFmt, 32, 4, 4, 2, 16>(cv, ydot, F_add, u, sq, st);
    default: return run_J<kFmt, 8, 2, 6>(cv, ydot, F_add, u, sq, st);
  }
}

template <int kFmt>
cudaError_t apply_JT_variant(int variant, const CacheView& cv, const float* u, float* seg_ybar, cudaStream_t st) {
  switch (variant) {
    case 0: return run_JT<kFmt, 16, 2, 6>(cv, u, seg_ybar, st);
    case 1: return run_JT<kFmt, 16, 4, 5>(cv, u, seg_ybar, st);
    case 2: return run_JT<kFmt, 32, 2, 6>(cv, u, seg_ybar, st);
    case 3: return run_JT<kFmt, 32, 4, 4>(cv, u, seg_ybar, st);
    case 5: return run_JT<kFmt, 16, 4, 4>(cv, u, seg_ybar, st);
    case 6: return run_JT<kFmt, 32, 3, 4>(cv, u, seg_ybar, st);
    case 7: return run_JT<kFmt, 16, 3, 5>(cv, u, seg_ybar, st);
    case 8: return run_JT<kFmt, 8, 2, 6, 16>(cv, u, seg_ybar, st);
    case 9: return run_JT<kFmt, 8, 4, 5, 16>(cv, u, seg_ybar, st);
    default: return run_JT<kFmt, 8, 2, 6>(cv, u, seg_ybar, st);
  }
}

}  // namespace

int apply_J_partials(const CacheView& cv) { return cv.n_tiles; }

int apply_variants() { return 10; }

cudaError_t launch_apply_J(const CacheView& cv, const float* ydot, const float* F_add, float* u,
                           double* sq_partials, int variant, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  if (cv.fmt == GSLM_CACHE_FP32) return apply_J_variant<GSLM_CACHE_FP32>(variant, cv, ydot, F_add, u, sq_partials, st);
  if (cv.fmt == GSLM_CACHE_BF16) return apply_J_variant<GSLM_CACHE_BF16>(variant, cv, ydot, F_add, u, sq_partials, st);
  return apply_J_variant<GSLM_CACHE_FP16S>(variant, cv, ydot, F_add, u, sq_partials, st);
}

cudaError_t launch_apply_JT(const CacheView& cv, const float* u, float* seg_ybar, int variant, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  if (cv.fmt == GSLM_CACHE_FP32) return apply_JT_variant<GSLM_CACHE_FP32>(variant, cv, u, seg_ybar, st);
  if (cv.fmt == GSLM_CACHE_BF16) return apply_JT_variant<GSLM_CACHE_BF16>(variant, cv, u, seg_ybar, st);
  return apply_JT_variant<GSLM_CACHE_FP16S>(variant, cv, u, seg_ybar, st);
}

int device_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// Resident CTAs of a persistent grid: never more than the kernel variant's
// register and shared-memory budget lets share an SM (variant_cta_cap), never
// more CTAs than tiles.
static int batch_ctas(const TileBatch& tb, int variant, bool jt, int ctas_per_sm) {
  const int cap = variant_cta_cap(variant, jt);
  const int per = ctas_per_sm < 1 ? 1 : (ctas_per_sm > cap ? cap : ctas_per_sm);
  const long long c = (long long)device_sm_count() * per;
  return (int)(c < tb.total_tiles ? c : tb.total_tiles);
}

cudaError_t launch_apply_J_batch(const TileBatch& tb, int variant, int ctas_per_sm, cudaStream_t st) {
  if (tb.n <= 0 || tb.total_tiles <= 0) return cudaSuccess;
  const int ctas = batch_ctas(tb, variant, false, ctas_per_sm);
  if (tb.fmt == GSLM_CACHE_FP32) return apply_J_batch_variant<GSLM_CACHE_FP32>(variant, tb, ctas, st);
  if (tb.fmt == GSLM_CACHE_BF16) return apply_J_batch_variant<GSLM_CACHE_BF16>(variant, tb, ctas, st);
  return apply_J_batch_variant<GSLM_CACHE_FP16S>(variant, tb, ctas, st);
}

cudaError_t launch_apply_JT_batch(const TileBatch& tb, int variant, int ctas_per_sm, cudaStream_t st) {
  if (tb.n <= 0 || tb.total_tiles <= 0) return cudaSuccess;
  const int ctas = batch_ctas(tb, variant, true, ctas_per_sm);
  if (tb.fmt == GSLM_CACHE_FP32) return apply_JT_batch_variant<GSLM_CACHE_FP32>(variant, tb, ctas, st);
  if (tb.fmt == GSLM_CACHE_BF16) return apply_JT_batch_variant<GSLM_CACHE_BF16>(variant, tb, ctas, st);
  return apply_JT_batch_variant<GSLM_CACHE_FP16S>(variant, tb, ctas, st);
}

cudaError_t launch_diag_entries(const CacheView& cv, float* seg_q, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
#define DIAG_LAUNCH(F, W) { k_diag_entries<F, W><<<cv.n_tiles, kTilePix, 0, st>>>(cv, seg_q); note_launch(); }
  const bool w = cv.wres != nullptr;
  if (cv.fmt == GSLM_CACHE_FP32) { if (w) DIAG_LAUNCH(GSLM_CACHE_FP32, true) else DIAG_LAUNCH(GSLM_CACHE_FP32, false) }
  else if (cv.fmt == GSLM_CACHE_BF16) { if (w) DIAG_LAUNCH(GSLM_CACHE_BF16, true) else DIAG_LAUNCH(GSLM_CACHE_BF16, false) }
  else { if (w) DIAG_LAUNCH(GSLM_CACHE_FP16S, true) else DIAG_LAUNCH(GSLM_CACHE_FP16S, false) }
#undef DIAG_LAUNCH
  return cudaGetLastError();
}

}  // namespace gslm
