// J p, J^T u and the per-segment blocks of diag(J^T J) from a thin cache
// (GSLM_CACHE_THIN): the cache thinning the paper names among its limitations,
// which keeps gradient state only every 32nd splat along a ray and blends the
// splats in between again when the products need them.
//
// A thin cache holds no per-(pixel, splat) entries. It keeps, per (tile,
// splat) segment in depth order, the projected splat (mean, conic, opacity,
// colour) exactly as the blending pass read it; per pixel its final colour C
// and n_live, the number of its tile's segments it takes before blending stops;
// and before every 32nd segment of a tile (a window) each pixel's
// transmittance T and colour prefix P (the checkpoints). Blending the
// segments again with the same float32 operations as the blending pass
// reproduces that pass's decisions and T, and for a contributing (pixel,
// splat s) pair gives the entry a full cache would hold:
//   w    = alpha_s T_s
//   h_ch = alpha_s (T_s c_ch - (C_ch - P_ch) / (1 - alpha_s))   (0 where alpha is clamped)
// with P the prefix including s (Sec. 3.3; Sec. A, Eq. apply-j, Eq. apply-jt,
// Eq. diag-jtj use these as the cache's T_s and dc/dalpha_s).
//
//   k_thin_apply_J   one CTA per tile, thread per pixel, walks the tile's
//                    segments front to back and sums u = sum_s w rgbdot + h q
//                    in registers (no atomics, no checkpoints needed)
//   k_thin_apply_JT  one CTA per window (32 segments): every pixel starts from
//                    its checkpoint; each segment's 9 adjoint sums are reduced
//                    over the pixels (warp halving, then shared atomics) and
//                    stored at the segment's splat-order position, as the
//                    entry-cache kernel stores them
//   k_thin_diag      the same per window for the 42 values of a segment's
//                    diagonal block
#include "internal.cuh"

namespace gslm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kTilePix / 32;

__device__ __forceinline__ int find_view(const DevCam* __restrict__ cams, int V, int tile) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cams[mid].tile_off <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The blending pass's weight of a splat at a pixel, with the same explicit
// round-to-nearest operations, so that every decision and every T is
// reproduced bit for bit. a = (mean x, mean y, conic A, conic B), bb = (conic
// C, opacity).
struct Weight {
  float araw, alpha, dx, dy;
  bool valid;
};
__device__ __forceinline__ Weight weight(float px, float py, const float4& a, float2 bb, int smooth) {
  Weight r;
  r.dx = __fsub_rn(px, a.x);
  r.dy = __fsub_rn(py, a.y);
  const float q = __fadd_rn(__fmul_rn(a.z, __fmul_rn(r.dx, r.dx)), __fmul_rn(bb.x, __fmul_rn(r.dy, r.dy)));
  const float power = __fsub_rn(__fmul_rn(-0.5f, q), __fmul_rn(a.w, __fmul_rn(r.dx, r.dy)));
  r.araw = __fmul_rn(bb.y, expf(power));
  r.alpha = smooth ? r.araw : fminf(kAlphaMax, r.araw);
  r.valid = smooth || r.alpha >= kAlphaMin;
  return r;
}

__device__ __forceinline__ float transmit(float T, float alpha) { return __fmul_rn(T, __fsub_rn(1.f, alpha)); }

struct Pixel {
  int x, y;
  bool inside;
  float px, py;
  long long pix;
};
__device__ __forceinline__ Pixel pixel_of(const DevCam& cam, int tile) {
  Pixel s;
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  s.x = tx * kTile + (threadIdx.x & (kTile - 1));
  s.y = ty * kTile + (threadIdx.x / kTile);
  s.inside = s.x < cam.W && s.y < cam.H;
  s.px = s.x + 0.5f;
  s.py = s.y + 0.5f;
  s.pix = cam.pix_off + (long long)s.y * cam.W + s.x;
  return s;
}

// One contributing (pixel, splat) pair: w = alpha T and h (alpha dc/dalpha),
// the prefix P advanced over the splat, T left for the caller to advance.
struct Entry {
  float w, h0, h1, h2;
};
__device__ __forceinline__ Entry entry_of(const Weight& bl, float T, const float4& c, const float3& Cf, float& p0,
                                          float& p1, float& p2, int smooth) {
  Entry e;
  e.w = __fmul_rn(bl.alpha, T);
  p0 = __fmaf_rn(c.x, e.w, p0);
  p1 = __fmaf_rn(c.y, e.w, p1);
  p2 = __fmaf_rn(c.z, e.w, p2);
  const float inv1m = __fdividef(1.f, 1.f - bl.alpha);   // as the cache-writing pass
  const bool clamped = !smooth && bl.araw > kAlphaMax;
  e.h0 = clamped ? 0.f : bl.alpha * (T * c.x - (Cf.x - p0) * inv1m);
  e.h1 = clamped ? 0.f : bl.alpha * (T * c.y - (Cf.y - p1) * inv1m);
  e.h2 = clamped ? 0.f : bl.alpha * (T * c.z - (Cf.z - p2) * inv1m);
  return e;
}

// gamma = d(log alpha)/d(mean x, mean y, A, B, C) and d/d(opacity), with
// d = pixel centre - mean: (A dx + B dy, B dx + C dy, -dx^2/2, -dx dy, -dy^2/2, 1/o).
__device__ __forceinline__ void gamma_of(const Weight& bl, const float4& a, float2 bb, float (&g)[6]) {
  g[0] = a.z * bl.dx + a.w * bl.dy;
  g[1] = a.w * bl.dx + bb.x * bl.dy;
  g[2] = -0.5f * bl.dx * bl.dx;
  g[3] = -bl.dx * bl.dy;
  g[4] = -0.5f * bl.dy * bl.dy;
  g[5] = 1.f / bb.y;
}

// ---------------------------------------------------------------------------
// Windows: win_count[t] = ceil(segments of tile t / 32); win_tile[w] = tile of window w.
__global__ void k_window_counts(const uint32_t* __restrict__ tile_seg_off, int n_tiles, uint32_t* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint32_t n = tile_seg_off[t + 1] - tile_seg_off[t];
  cnt[t] = (n + kThinWindow - 1) / kThinWindow;
}

__global__ void k_window_tiles(const uint32_t* __restrict__ win_off, int n_tiles, uint32_t* __restrict__ win_tile) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  for (uint32_t w = win_off[t]; w < win_off[t + 1]; ++w) win_tile[w] = (uint32_t)t;
}

// ---------------------------------------------------------------------------
// J p. Shared staging per chunk of 256 segments: the splat (a, (C, o), colour)
// and its tangent ydot (dmx, dmy, dA, dB, dC, do, dr, dg, db).
struct StageJ {
  float4 a[kTilePix];
  float4 bc[kTilePix];     // C, o, r, g
  float4 y0[kTilePix];     // dmx, dmy, dA, dB
  float4 y1[kTilePix];     // dC, do, dr, dg
  float2 y2[kTilePix];     // db, colour b
};

__global__ void __launch_bounds__(kTilePix) k_thin_apply_J(CacheView cv, const float* __restrict__ ydot,
                                                           const float* __restrict__ Fadd, float* __restrict__ u,
                                                           double* __restrict__ sq_partials) {
  if (cv.skip != nullptr && *cv.skip) return;
  __shared__ StageJ S;
  __shared__ double dred[2 * kWarps];
  __shared__ uint32_t smax;
  const int tile = blockIdx.x;
  const DevCam& cam = cv.cams[find_view(cv.cams, cv.V, tile)];
  const Pixel px = pixel_of(cam, tile);
  const uint32_t g0 = cv.tile_seg_off[tile], n = cv.tile_seg_off[tile + 1] - g0;
  const uint32_t nl = cv.n_live[(size_t)tile * kTilePix + threadIdx.x];
  float3 Cf = make_float3(0.f, 0.f, 0.f);
  if (px.inside) Cf = make_float3(cv.img[px.pix * 3 + 0], cv.img[px.pix * 3 + 1], cv.img[px.pix * 3 + 2]);
  if (threadIdx.x == 0) smax = 0u;
  __syncthreads();
  atomicMax(&smax, nl);
  __syncthreads();
  const uint32_t nmax = min(smax, n);
  const int smooth = 0;   // thin caches are built in the default mode only
  float T = 1.f, p0 = 0.f, p1 = 0.f, p2 = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f;
  for (uint32_t c0 = 0; c0 < nmax; c0 += kTilePix) {
    const uint32_t cnt = min((uint32_t)kTilePix, nmax - c0);
    if (threadIdx.x < cnt) {
      const uint32_t sg = g0 + c0 + threadIdx.x;
      const SplatRec r = cv.thin_rec[sg];
      const float4* yd = reinterpret_cast<const float4*>(ydot + (size_t)cv.seg_rec[sg].slot * 12);
      const float4 y0 = yd[0], y1 = yd[1], y2 = yd[2];
      S.a[threadIdx.x] = r.a;
      S.bc[threadIdx.x] = make_float4(r.b.x, r.b.y, r.c.x, r.c.y);
      S.y0[threadIdx.x] = y0;
      S.y1[threadIdx.x] = y1;
      S.y2[threadIdx.x] = make_float2(y2.x, r.c.z);
    }
    __syncthreads();
    const uint32_t mine = nl > c0 ? min(cnt, nl - c0) : 0u;
    for (uint32_t j = 0; j < mine; ++j) {
      const float4 a = S.a[j], bc = S.bc[j];
      const Weight bl = weight(px.px, px.py, a, make_float2(bc.x, bc.y), smooth);
      if (!bl.valid) continue;
      const float2 y2 = S.y2[j];
      const float4 c = make_float4(bc.z, bc.w, y2.y, 0.f);
      const Entry e = entry_of(bl, T, c, Cf, p0, p1, p2, smooth);
      const float4 y0 = S.y0[j], y1 = S.y1[j];
      float g[6];
      gamma_of(bl, a, make_float2(bc.x, bc.y), g);
      const float q = g[0] * y0.x + g[1] * y0.y + g[2] * y0.z + g[3] * y0.w + g[4] * y1.x + g[5] * y1.y;
      u0 = fmaf(e.w, y1.z, fmaf(e.h0, q, u0));
      u1 = fmaf(e.w, y1.w, fmaf(e.h1, q, u1));
      u2 = fmaf(e.w, y2.x, fmaf(e.h2, q, u2));
      T = transmit(T, bl.alpha);
    }
    __syncthreads();
  }
  // epilogue as the entry-cache kernel's: u = w (dc/dx) p; per-tile sums of
  // e.u and w.u^2 with the unweighted u (predicted decrease)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double local = 0.0, local2 = 0.0;
  if (px.inside) {
    float w0 = 1.f, w1 = 1.f, w2 = 1.f;
    if (cv.wres != nullptr) {
      w0 = cv.wres[px.pix * 3 + 0];
      w1 = cv.wres[px.pix * 3 + 1];
      w2 = cv.wres[px.pix * 3 + 2];
    }
    if (u != nullptr) {
      u[px.pix * 3 + 0] = w0 * u0;
      u[px.pix * 3 + 1] = w1 * u1;
      u[px.pix * 3 + 2] = w2 * u2;
    }
    if (sq_partials != nullptr) {
      const float* f = Fadd + px.pix * 3;
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

// ---------------------------------------------------------------------------
// Warp sums of 16 values by recursive halving: afterwards lane 2i holds the
// sum of value i (i < 16) in v[0].
template <int N>
__device__ __forceinline__ void halve(float (&v)[16], bool upper, int o) {
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    const float send = upper ? v[k] : v[k + N / 2];
    const float keep = upper ? v[k + N / 2] : v[k];
    v[k] = keep + __shfl_xor_sync(kFull, send, o);
  }
}
__device__ __forceinline__ void warp_sum16(float (&v)[16], int lane) {
  halve<16>(v, lane & 16, 16);
  halve<8>(v, lane & 8, 8);
  halve<4>(v, lane & 4, 4);
  halve<2>(v, lane & 2, 2);
  v[0] += __shfl_xor_sync(kFull, v[0], 1);
}

// Shared staging of one window: the splats and their output positions.
struct StageWin {
  float4 a[kThinWindow];
  float4 bc[kThinWindow];   // C, o, r, g
  float b2[kThinWindow];    // colour b
  uint32_t pos[kThinWindow];
};

// Per window: pixel state from its checkpoint; the window's segments staged.
struct WinSetup {
  int tile;
  uint32_t k0, cnt, nl;
  Pixel px;
  float3 Cf;
  float4 st;   // T, prefix
};
__device__ __forceinline__ WinSetup window_setup(const CacheView& cv, uint32_t win, StageWin& S) {
  WinSetup w;
  w.tile = (int)cv.win_tile[win];
  const uint32_t g0 = cv.tile_seg_off[w.tile], n = cv.tile_seg_off[w.tile + 1] - g0;
  w.k0 = (win - cv.win_off[w.tile]) * kThinWindow;
  w.cnt = min((uint32_t)kThinWindow, n - w.k0);
  const DevCam& cam = cv.cams[find_view(cv.cams, cv.V, w.tile)];
  w.px = pixel_of(cam, w.tile);
  w.nl = cv.n_live[(size_t)w.tile * kTilePix + threadIdx.x];
  w.Cf = make_float3(0.f, 0.f, 0.f);
  if (w.px.inside) w.Cf = make_float3(cv.img[w.px.pix * 3 + 0], cv.img[w.px.pix * 3 + 1], cv.img[w.px.pix * 3 + 2]);
  w.st = cv.ckpt[(size_t)win * kTilePix + threadIdx.x];
  if (threadIdx.x < w.cnt) {
    const uint32_t sg = g0 + w.k0 + threadIdx.x;
    const SplatRec r = cv.thin_rec[sg];
    S.a[threadIdx.x] = r.a;
    S.bc[threadIdx.x] = make_float4(r.b.x, r.b.y, r.c.x, r.c.y);
    S.b2[threadIdx.x] = r.c.z;
    S.pos[threadIdx.x] = cv.seg_pos[sg];
  }
  return w;
}

// J^T u: per segment, ybar = sum over its pixels of
// (s gamma, w u_r, w u_g, w u_b) with s = h . u, stored as 12 floats at the
// segment's splat-order position (9 used), the layout of the entry-cache kernel.
__global__ void __launch_bounds__(kTilePix) k_thin_apply_JT(CacheView cv, const float* __restrict__ u,
                                                            float* __restrict__ seg_ybar) {
  if (cv.skip != nullptr && *cv.skip) return;
  __shared__ StageWin S;
  __shared__ float acc[kThinWindow][9];
  for (int i = threadIdx.x; i < kThinWindow * 9; i += kTilePix) (&acc[0][0])[i] = 0.f;
  const WinSetup W = window_setup(cv, blockIdx.x, S);
  float3 uv = make_float3(0.f, 0.f, 0.f);
  if (W.px.inside) uv = make_float3(u[W.px.pix * 3 + 0], u[W.px.pix * 3 + 1], u[W.px.pix * 3 + 2]);
  __syncthreads();
  const int smooth = 0;
  const int lane = threadIdx.x & 31;
  float T = W.st.x, p0 = W.st.y, p1 = W.st.z, p2 = W.st.w;
  for (uint32_t j = 0; j < W.cnt; ++j) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0.f;
    bool contrib = false;
    if (W.k0 + j < W.nl) {
      const float4 a = S.a[j], bc = S.bc[j];
      const Weight bl = weight(W.px.px, W.px.py, a, make_float2(bc.x, bc.y), smooth);
      if (bl.valid) {
        contrib = true;
        const float4 c = make_float4(bc.z, bc.w, S.b2[j], 0.f);
        const Entry e = entry_of(bl, T, c, W.Cf, p0, p1, p2, smooth);
        float g[6];
        gamma_of(bl, a, make_float2(bc.x, bc.y), g);
        const float s = e.h0 * uv.x + e.h1 * uv.y + e.h2 * uv.z;
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = s * g[i];
        v[6] = e.w * uv.x;
        v[7] = e.w * uv.y;
        v[8] = e.w * uv.z;
        T = transmit(T, bl.alpha);
      }
    }
    if (__any_sync(kFull, contrib)) {
      warp_sum16(v, lane);
      if ((lane & 1) == 0 && lane < 18) atomicAdd(&acc[j][lane >> 1], v[0]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)W.cnt * 9; i += kTilePix) {
    const int j = i / 9, o = i - 9 * j;
    seg_ybar[(size_t)S.pos[j] * 12 + o] = acc[j][o];
  }
}

// diag(J^T J) blocks: per segment, Q = sum over pixels and channels of
// rho_ch a_ch a_ch^T with a_ch = [h_ch gamma, w e_ch] (rho: residual-to-pixel
// weights, 1 for L2), as kDiagBlock floats: Qgg (21, upper triangle of the 6x6
// block, row-major), X (18: sum rho_c w h_c gamma_i, index 3 i + c), D_ch (3:
// sum rho_ch w^2), two zeros.
__global__ void __launch_bounds__(kTilePix) k_thin_diag(CacheView cv, float* __restrict__ seg_q) {
  __shared__ StageWin S;
  __shared__ float acc[kThinWindow][42];
  for (int i = threadIdx.x; i < kThinWindow * 42; i += kTilePix) (&acc[0][0])[i] = 0.f;
  const WinSetup W = window_setup(cv, blockIdx.x, S);
  float r0 = 1.f, r1 = 1.f, r2 = 1.f;
  if (cv.wres != nullptr && W.px.inside) {
    r0 = cv.wres[W.px.pix * 3 + 0];
    r1 = cv.wres[W.px.pix * 3 + 1];
    r2 = cv.wres[W.px.pix * 3 + 2];
  }
  __syncthreads();
  const int smooth = 0;
  const int lane = threadIdx.x & 31;
  float T = W.st.x, p0 = W.st.y, p1 = W.st.z, p2 = W.st.w;
  for (uint32_t j = 0; j < W.cnt; ++j) {
    float q[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) q[i] = 0.f;
    bool contrib = false;
    if (W.k0 + j < W.nl) {
      const float4 a = S.a[j], bc = S.bc[j];
      const Weight bl = weight(W.px.px, W.px.py, a, make_float2(bc.x, bc.y), smooth);
      if (bl.valid) {
        contrib = true;
        const float4 c = make_float4(bc.z, bc.w, S.b2[j], 0.f);
        const Entry e = entry_of(bl, T, c, W.Cf, p0, p1, p2, smooth);
        float g[6];
        gamma_of(bl, a, make_float2(bc.x, bc.y), g);
        const float H2 = r0 * e.h0 * e.h0 + r1 * e.h1 * e.h1 + r2 * e.h2 * e.h2;
        int k = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int jj = i; jj < 6; ++jj) q[k++] = H2 * g[i] * g[jj];
        const float xr = r0 * e.w * e.h0, xg = r1 * e.w * e.h1, xb = r2 * e.w * e.h2;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          q[21 + 3 * i + 0] = xr * g[i];
          q[21 + 3 * i + 1] = xg * g[i];
          q[21 + 3 * i + 2] = xb * g[i];
        }
        const float ww = e.w * e.w;
        q[39] = r0 * ww;
        q[40] = r1 * ww;
        q[41] = r2 * ww;
        T = transmit(T, bl.alpha);
      }
    }
    if (__any_sync(kFull, contrib)) {
#pragma unroll
      for (int part = 0; part < 3; ++part) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = q[16 * part + i];
        warp_sum16(v, lane);
        const int o = 16 * part + (lane >> 1);
        if ((lane & 1) == 0 && o < 42) atomicAdd(&acc[j][o], v[0]);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)W.cnt * kDiagBlock; i += kTilePix) {
    const int j = i / kDiagBlock, o = i - kDiagBlock * j;
    seg_q[(size_t)S.pos[j] * kDiagBlock + o] = o < 42 ? acc[j][o] : 0.f;
  }
}

}  // namespace

cudaError_t launch_thin_window_counts(const uint32_t* tile_seg_off, int n_tiles, uint32_t* win_count,
                                      cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  k_window_counts<<<(n_tiles + 255) / 256, 256, 0, st>>>(tile_seg_off, n_tiles, win_count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_thin_window_tiles(const uint32_t* win_off, int n_tiles, uint32_t* win_tile, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  k_window_tiles<<<(n_tiles + 255) / 256, 256, 0, st>>>(win_off, n_tiles, win_tile);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_thin_apply_J(const CacheView& cv, const float* ydot, const float* F_add, float* u,
                                double* sq_partials, cudaStream_t st) {
  if (cv.n_tiles <= 0) return cudaSuccess;
  k_thin_apply_J<<<cv.n_tiles, kTilePix, 0, st>>>(cv, ydot, F_add, u, sq_partials);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_thin_apply_JT(const CacheView& cv, const float* u, float* seg_ybar, cudaStream_t st) {
  if (cv.n_win <= 0) return cudaSuccess;
  k_thin_apply_JT<<<(unsigned)cv.n_win, kTilePix, 0, st>>>(cv, u, seg_ybar);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_thin_diag(const CacheView& cv, float* seg_q, cudaStream_t st) {
  if (cv.n_win <= 0) return cudaSuccess;
  k_thin_diag<<<(unsigned)cv.n_win, kTilePix, 0, st>>>(cv, seg_q);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gslm
