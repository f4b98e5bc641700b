// Residuals of the L1 + SSIM objective (Eq. gn-loss) and their residual-to-
// pixel weights (Sec. C, "Precomputation Of Residual-To-Pixel Weights").
//
// Per pixel i and colour channel the objective has two residuals,
// r1 = sqrt(l1 |c - C|) and r2 = sqrt(l2 (1 - SSIM_i)). The cache keeps, per
// pixel channel, e = (dr1/dc) r1 + (dr2/dc) r2 (so that J^T F = (dc/dx)^T e) in
// place of F, and w = (dr1/dc)^2 + (dr2/dc)^2, which the J p tile kernel
// multiplies into its output and the diagonal kernel into every entry.
//
// SSIM per channel: local means, variances and covariance from an 11 x 11
// Gaussian window (sd 1.5, normalised), zero outside the view, C1 = 0.01^2,
// C2 = 0.03^2. dSSIM_i/dc_i keeps only the centre pixel's own term (the paper
// propagates each pixel's score to its centre pixel only): the centre pixel
// enters its own window's statistics with weight w0 = g_mid^2. The derivatives
// floor |c - C| and 1 - SSIM at eps under their square roots.
//
// One 256-thread block per 16 x 16 tile of a view: the tile and a 5-pixel halo
// of the rendered image and the target are staged in shared memory, the window
// is applied as a horizontal then a vertical pass, and every thread finishes
// one pixel's three channels. Statistics are float32 (as the 3DGS loss
// computes them); the energy is summed in float64.
#include "internal.cuh"

namespace gslm {
namespace {

constexpr int kHalo = 5;                    // 11-tap window
constexpr int kReg = kTile + 2 * kHalo;     // staged region: 26 x 26 pixels
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;
constexpr int kWarps = kTilePix / 32;

__device__ __forceinline__ int view_of_tile(const DevCam* __restrict__ cams, int V, int tile) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cams[mid].tile_off <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kTilePix) k_l1ssim(const DevCam* __restrict__ cams, int V,
                                                     const float* __restrict__ img, const float* __restrict__ tgt,
                                                     float lam1, float lam2, float eps, float* __restrict__ e_out,
                                                     float* __restrict__ w_out, double* __restrict__ cost_part) {
  __shared__ float sx[kReg * kReg * 3];          // [row][col][channel] of the region, 0 outside the view
  __shared__ float sy[kReg * kReg * 3];
  __shared__ float sh[5][kReg][kTile * 3];       // horizontal window sums of x, y, x^2, y^2, x y
  __shared__ float g[2 * kHalo + 1];
  __shared__ double red[kWarps];
  const int tile = blockIdx.x;
  const DevCam& cam = cams[view_of_tile(cams, V, tile)];
  const int lt = tile - cam.tile_off;
  const int ty = lt / cam.tiles_x, tx = lt - ty * cam.tiles_x;
  const int x0 = tx * kTile - kHalo, y0 = ty * kTile - kHalo;
  if (threadIdx.x <= 2 * kHalo) {
    float sum = 0.f;
    for (int t = -kHalo; t <= kHalo; ++t) sum += expf(-(float)(t * t) / 4.5f);
    const int t = (int)threadIdx.x - kHalo;
    g[threadIdx.x] = expf(-(float)(t * t) / 4.5f) / sum;
  }
  for (int i = threadIdx.x; i < kReg * kReg * 3; i += kTilePix) {
    const int c = i % 3, q = i / 3, r = q / kReg, col = q - r * kReg;
    const int gx = x0 + col, gy = y0 + r;
    float a = 0.f, b = 0.f;
    if (gx >= 0 && gx < cam.W && gy >= 0 && gy < cam.H) {
      const long long o = (cam.pix_off + (long long)gy * cam.W + gx) * 3 + c;
      a = img[o];
      b = tgt[o];
    }
    sx[i] = a;
    sy[i] = b;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kReg * kTile * 3; i += kTilePix) {
    const int r = i / (kTile * 3), k = i - r * (kTile * 3), col = k / 3, c = k - col * 3;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
    for (int t = 0; t <= 2 * kHalo; ++t) {
      const int o = (r * kReg + col + t) * 3 + c;
      const float a = sx[o], b = sy[o], gt = g[t];
      m0 = fmaf(gt, a, m0);
      m1 = fmaf(gt, b, m1);
      m2 = fmaf(gt * a, a, m2);
      m3 = fmaf(gt * b, b, m3);
      m4 = fmaf(gt * a, b, m4);
    }
    sh[0][r][k] = m0;
    sh[1][r][k] = m1;
    sh[2][r][k] = m2;
    sh[3][r][k] = m3;
    sh[4][r][k] = m4;
  }
  __syncthreads();
  const int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
  const int px = tx * kTile + lx, py = ty * kTile + ly;
  double local = 0.0;
  if (px < cam.W && py < cam.H) {
    const long long pix = cam.pix_off + (long long)py * cam.W + px;
    const float w0 = g[kHalo] * g[kHalo];
    const float sl1 = sqrtf(lam1), sl2 = sqrtf(lam2);
    float lc = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kHalo; ++t) {
        const int k = lx * 3 + c, r = ly + t;
        const float gt = g[t];
        mx = fmaf(gt, sh[0][r][k], mx);
        my = fmaf(gt, sh[1][r][k], my);
        exx = fmaf(gt, sh[2][r][k], exx);
        eyy = fmaf(gt, sh[3][r][k], eyy);
        exy = fmaf(gt, sh[4][r][k], exy);
      }
      const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
      const float den = B1 * B2;
      const float S = A1 * A2 / den;
      const int o = ((ly + kHalo) * kReg + lx + kHalo) * 3 + c;
      const float xc = sx[o], yc = sy[o];
      // quotient rule with d mu_x = w0, d var_x = 2 w0 (x - mu_x), d cov = w0 (y - mu_y)
      const float dS = (2.f * w0 * my * A2 + A1 * 2.f * w0 * (yc - my)) / den -
                       S * (2.f * w0 * mx / B1 + 2.f * w0 * (xc - mx) / B2);
      const float d = xc - yc, ad = fabsf(d);
      const float r1 = sqrtf(lam1 * ad);
      const float dr1 = d == 0.f ? 0.f : copysignf(sl1 / (2.f * sqrtf(fmaxf(ad, eps))), d);
      const float om = 1.f - S;
      const float r2 = sqrtf(lam2 * fmaxf(om, 0.f));
      const float dr2 = -sl2 * dS / (2.f * sqrtf(fmaxf(om, eps)));
      if (e_out != nullptr) e_out[pix * 3 + c] = dr1 * r1 + dr2 * r2;
      if (w_out != nullptr) w_out[pix * 3 + c] = dr1 * dr1 + dr2 * dr2;
      lc += lam1 * ad + lam2 * fmaxf(om, 0.f);
    }
    local = (double)lc;
  }
  if (cost_part != nullptr) {
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kWarps; ++w) s += red[w];
      cost_part[tile] = s;
    }
  }
}

__global__ void k_fill(long long n, float v, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}

}  // namespace

cudaError_t launch_l1ssim(const DevCam* cams, int V, int n_tiles, const float* img, const float* tgt, float lam1,
                          float lam2, float eps, float* e, float* w, double* cost_partials, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  { k_l1ssim<<<n_tiles, kTilePix, 0, st>>>(cams, V, img, tgt, lam1, lam2, eps, e, w, cost_partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_fill_f32(long long n, float v, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, v, out); note_launch(); }
  return cudaGetLastError();
}

}  // namespace gslm
