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

template <int G, int kFmt>
__global__ void __launch_bounds__(kTilePix) k_apply_J(CacheView cv, const float* __restrict__ ydot,
                                                      const float* __restrict__ Fadd, float* __restrict__ u,
                                                      double* __restrict__ sq_partials) {
  __shared__ float su[3 * kTilePix];
  __shared__ double dred[kTilePix / 32];
  if (cv.skip != nullptr && *cv.skip) return;
  const int tile = blockIdx.x;
  const int v = find_view(cv.cams, cv.V, tile);
  const DevCam& cam = cv.cams[v];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  const float ox = tx * kTile + 0.5f, oy = ty * kTile + 0.5f;
  for (int i = threadIdx.x; i < 3 * kTilePix; i += kTilePix) su[i] = 0.f;
  __syncthreads();
  const uint32_t g0 = cv.tile_seg_off[tile], g1 = cv.tile_seg_off[tile + 1];
  const int gid = threadIdx.x / G, gl = threadIdx.x % G;
  constexpr int kGroups = kTilePix / G;
  for (uint32_t seg = g0 + gid; seg < g1; seg += kGroups) {
    const uint32_t slot = cv.seg_slot[seg];
    const unsigned long long e0 = cv.seg_entry_off[seg], e1 = cv.seg_entry_off[seg + 1];
    const float4 ra = cv.rec[slot].a;
    const float2 rb = *reinterpret_cast<const float2*>(&cv.rec[slot].b);
    const float4* yd = reinterpret_cast<const float4*>(ydot + (size_t)slot * 12);
    const float4 y0 = yd[0], y1 = yd[1], y2 = yd[2];
    const float mx = ra.x - ox, my = ra.y - oy, A = ra.z, B = ra.w, C = rb.x;
    const float od = y1.y / rb.y;
    const float scale = kFmt == GSLM_CACHE_FP16S ? cv.seg_scale[seg] : 1.f;
    for (unsigned long long e = e0 + gl; e < e1; e += G) {
      const float4 pe = load_entry<kFmt>(cv.payload, e, scale);
      const int p = cv.pixoff[e];
      const float dx = (float)(p & (kTile - 1)) - mx, dy = (float)(p / kTile) - my;
      const float q = (A * dx + B * dy) * y0.x + (B * dx + C * dy) * y0.y -
                      0.5f * dx * dx * y0.z - dx * dy * y0.w - 0.5f * dy * dy * y1.x + od;
      atomicAdd(&su[p], pe.x * y1.z + pe.y * q);
      atomicAdd(&su[kTilePix + p], pe.x * y1.w + pe.z * q);
      atomicAdd(&su[2 * kTilePix + p], pe.x * y2.x + pe.w * q);
    }
  }
  __syncthreads();
  const int x = tx * kTile + (threadIdx.x & (kTile - 1)), y = ty * kTile + threadIdx.x / kTile;
  double local = 0.0;
  if (x < cam.W && y < cam.H) {
    const long long pix = cam.pix_off + (long long)y * cam.W + x;
    const float u0 = su[threadIdx.x], u1 = su[kTilePix + threadIdx.x], u2 = su[2 * kTilePix + threadIdx.x];
    if (u != nullptr) {
      u[pix * 3 + 0] = u0;
      u[pix * 3 + 1] = u1;
      u[pix * 3 + 2] = u2;
    }
    if (sq_partials != nullptr) {
      const float* f = Fadd + pix * 3;
      const double a0 = (double)u0 + f[0], a1 = (double)u1 + f[1], a2 = (double)u2 + f[2];
      local = a0 * a0 + a1 * a1 + a2 * a2;
    }
  }
  if (sq_partials != nullptr) {
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kTilePix / 32; ++w) s += dred[w];
      sq_partials[tile] = s;
    }
  }
}

template <int G, int kFmt>
__global__ void __launch_bounds__(kTilePix) k_apply_JT(CacheView cv, const float* __restrict__ u,
                                                       float* __restrict__ seg_ybar) {
  __shared__ float su[3 * kTilePix];
  if (cv.skip != nullptr && *cv.skip) return;
  const int tile = blockIdx.x;
  const uint32_t g0 = cv.tile_seg_off[tile], g1 = cv.tile_seg_off[tile + 1];
  if (g0 == g1) return;
  const int v = find_view(cv.cams, cv.V, tile);
  const DevCam& cam = cv.cams[v];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  const float ox = tx * kTile + 0.5f, oy = ty * kTile + 0.5f;
  {
    const int x = tx * kTile + (threadIdx.x & (kTile - 1)), y = ty * kTile + threadIdx.x / kTile;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f;
    if (x < cam.W && y < cam.H) {
      const long long pix = cam.pix_off + (long long)y * cam.W + x;
      u0 = u[pix * 3 + 0];
      u1 = u[pix * 3 + 1];
      u2 = u[pix * 3 + 2];
    }
    su[threadIdx.x] = u0;
    su[kTilePix + threadIdx.x] = u1;
    su[2 * kTilePix + threadIdx.x] = u2;
  }
  __syncthreads();
  const int gid = threadIdx.x / G, gl = threadIdx.x % G;
  constexpr int kGroups = kTilePix / G;
  const unsigned gm = group_mask<G>();
  for (uint32_t seg = g0 + gid; seg < g1; seg += kGroups) {
    const uint32_t slot = cv.seg_slot[seg];
    const unsigned long long e0 = cv.seg_entry_off[seg], e1 = cv.seg_entry_off[seg + 1];
    const float4 ra = cv.rec[slot].a;
    const float2 rb = *reinterpret_cast<const float2*>(&cv.rec[slot].b);
    const float mx = ra.x - ox, my = ra.y - oy, A = ra.z, B = ra.w, C = rb.x;
    const float scale = kFmt == GSLM_CACHE_FP16S ? cv.seg_scale[seg] : 1.f;
    // sums of s, s*dx, s*dy, s*dx^2, s*dx*dy, s*dy^2 and w*u_ch
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
    for (unsigned long long e = e0 + gl; e < e1; e += G) {
      const float4 pe = load_entry<kFmt>(cv.payload, e, scale);
      const int p = cv.pixoff[e];
      const float dx = (float)(p & (kTile - 1)) - mx, dy = (float)(p / kTile) - my;
      const float u0 = su[p], u1 = su[kTilePix + p], u2 = su[2 * kTilePix + p];
      const float s = pe.y * u0 + pe.z * u1 + pe.w * u2;
      a0 += s;
      a1 += s * dx;
      a2 += s * dy;
      a3 += s * dx * dx;
      a4 += s * dx * dy;
      a5 += s * dy * dy;
      r0 += pe.x * u0;
      r1 += pe.x * u1;
      r2 += pe.x * u2;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(gm, a0, o);
      a1 += __shfl_xor_sync(gm, a1, o);
      a2 += __shfl_xor_sync(gm, a2, o);
      a3 += __shfl_xor_sync(gm, a3, o);
      a4 += __shfl_xor_sync(gm, a4, o);
      a5 += __shfl_xor_sync(gm, a5, o);
      r0 += __shfl_xor_sync(gm, r0, o);
      r1 += __shfl_xor_sync(gm, r1, o);
      r2 += __shfl_xor_sync(gm, r2, o);
    }
    if (gl == 0) {
      float4* out = reinterpret_cast<float4*>(seg_ybar + (size_t)seg * 12);
      out[0] = make_float4(A * a1 + B * a2, B * a1 + C * a2, -0.5f * a3, -a4);
      out[1] = make_float4(-0.5f * a5, a0 / rb.y, r0, r1);
      out[2] = make_float4(r2, 0.f, 0.f, 0.f);
    }
  }
}

// Per segment: Q = sum over entries and channels of a_ch a_ch^T with
// a_ch = [h_ch gamma, w e_ch]; stored as Qgg (21, upper triangle of the 6x6
// block, row-major), X (18, 6x3: sum w h_c gamma_i), D (sum w^2).
template <int kFmt>
__global__ void __launch_bounds__(kTilePix) k_diag_entries(CacheView cv, float* __restrict__ seg_q) {
  const int tile = blockIdx.x;
  const uint32_t g0 = cv.tile_seg_off[tile], g1 = cv.tile_seg_off[tile + 1];
  if (g0 == g1) return;
  const int v = find_view(cv.cams, cv.V, tile);
  const DevCam& cam = cv.cams[v];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  const float ox = tx * kTile + 0.5f, oy = ty * kTile + 0.5f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t seg = g0 + warp; seg < g1; seg += kTilePix / 32) {
    const uint32_t slot = cv.seg_slot[seg];
    const unsigned long long e0 = cv.seg_entry_off[seg], e1 = cv.seg_entry_off[seg + 1];
    const float4 ra = cv.rec[slot].a;
    const float2 rb = *reinterpret_cast<const float2*>(&cv.rec[slot].b);
    const float mx = ra.x - ox, my = ra.y - oy, A = ra.z, B = ra.w, C = rb.x;
    const float io = 1.f / rb.y;
    const float scale = kFmt == GSLM_CACHE_FP16S ? cv.seg_scale[seg] : 1.f;
    float q[40];
#pragma unroll
    for (int i = 0; i < 40; ++i) q[i] = 0.f;
    for (unsigned long long e = e0 + lane; e < e1; e += 32) {
      const float4 pe = load_entry<kFmt>(cv.payload, e, scale);
      const int p = cv.pixoff[e];
      const float dx = (float)(p & (kTile - 1)) - mx, dy = (float)(p / kTile) - my;
      float gam[6] = {A * dx + B * dy, B * dx + C * dy, -0.5f * dx * dx, -dx * dy, -0.5f * dy * dy, io};
      const float H2 = pe.y * pe.y + pe.z * pe.z + pe.w * pe.w;
      int k = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) q[k++] += H2 * gam[i] * gam[j];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        q[21 + 3 * i + 0] += pe.x * pe.y * gam[i];
        q[21 + 3 * i + 1] += pe.x * pe.z * gam[i];
        q[21 + 3 * i + 2] += pe.x * pe.w * gam[i];
      }
      q[39] += pe.x * pe.x;
    }
#pragma unroll
    for (int i = 0; i < 40; ++i)
      for (int o = 16; o > 0; o >>= 1) q[i] += __shfl_xor_sync(kFull, q[i], o);
    if (lane < 10) {
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 10; ++i)
        if (lane == i) val = make_float4(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]);
      reinterpret_cast<float4*>(seg_q + (size_t)seg * 40)[lane] = val;
    }
  }
}

template <int G>
cudaError_t apply_J_g(const CacheView& cv, const float* ydot, const float* F_add, float* u, double* sq,
                      cudaStream_t st) {
  if (cv.fmt == GSLM_CACHE_FP32) { k_apply_J<G, GSLM_CACHE_FP32><<<cv.n_tiles, kTilePix, 0, st>>>(cv, ydot, F_add, u, sq); note_launch(); }
  else if (cv.fmt == GSLM_CACHE_BF16) { k_apply_J<G, GSLM_CACHE_BF16><<<cv.n_tiles, kTilePix, 0, st>>>(cv, ydot, F_add, u, sq); note_launch(); }
  else { k_apply_J<G, GSLM_CACHE_FP16S><<<cv.n_tiles, kTilePix, 0, st>>>(cv, ydot, F_add, u, sq); note_launch(); }
  return cudaGetLastError();
}

template <int G>
cudaError_t apply_JT_g(const CacheView& cv, const float* u, float* seg_ybar, cudaStream_t st) {
  if (cv.fmt == GSLM_CACHE_FP32) { k_apply_JT<G, GSLM_CACHE_FP32><<<cv.n_tiles, kTilePix, 0, st>>>(cv, u, seg_ybar); note_launch(); }
  else if (cv.fmt == GSLM_CACHE_BF16) { k_apply_JT<G, GSLM_CACHE_BF16><<<cv.n_tiles, kTilePix, 0, st>>>(cv, u, seg_ybar); note_launch(); }
  else { k_apply_JT<G, GSLM_CACHE_FP16S><<<cv.n_tiles, kTilePix, 0, st>>>(cv, u, seg_ybar); note_launch(); }
  return cudaGetLastError();
}

}  // namespace

int apply_J_partials(const CacheView& cv) { return cv.n_tiles; }

cudaError_t launch_apply_J(const CacheView& cv, const float* ydot, const float* F_add, float* u,
                           double* sq_partials, int group, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  switch (group) {
    case 8: return apply_J_g<8>(cv, ydot, F_add, u, sq_partials, st);
    case 16: return apply_J_g<16>(cv, ydot, F_add, u, sq_partials, st);
    default: return apply_J_g<32>(cv, ydot, F_add, u, sq_partials, st);
  }
}

cudaError_t launch_apply_JT(const CacheView& cv, const float* u, float* seg_ybar, int group, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  switch (group) {
    case 8: return apply_JT_g<8>(cv, u, seg_ybar, st);
    case 16: return apply_JT_g<16>(cv, u, seg_ybar, st);
    default: return apply_JT_g<32>(cv, u, seg_ybar, st);
  }
}

cudaError_t launch_diag_entries(const CacheView& cv, float* seg_q, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  if (cv.fmt == GSLM_CACHE_FP32) { k_diag_entries<GSLM_CACHE_FP32><<<cv.n_tiles, kTilePix, 0, st>>>(cv, seg_q); note_launch(); }
  else if (cv.fmt == GSLM_CACHE_BF16) { k_diag_entries<GSLM_CACHE_BF16><<<cv.n_tiles, kTilePix, 0, st>>>(cv, seg_q); note_launch(); }
  else { k_diag_entries<GSLM_CACHE_FP16S><<<cv.n_tiles, kTilePix, 0, st>>>(cv, seg_q); note_launch(); }
  return cudaGetLastError();
}

}  // namespace gslm
