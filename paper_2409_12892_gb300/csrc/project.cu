// Gaussian -> splat projection and the per-Gaussian factor dy/dx of the chain
// rule in Eq. backward-pass (Sec. 3.3): forward (k_project), its tangent
// (k_tangent: ydot = (dy/dx) p, used by J p) and its adjoint (k_vjp:
// (dy/dx)^T ybar, used by J^T u), plus the diag(J^T J) finalisation (k_diag).
//
// The per-Gaussian kernels keep one lane per Gaussian for everything read or
// written per Gaussian, so each Gaussian's 59 parameters and 59 vector entries
// are read once per call (coalesced, structure-of-arrays), and sum its views'
// results per Gaussian: this is the paper's applyJT_p2/p3 and the "sortX" it
// needs before applyJ (Sec. A), replaced by one pass in the [59][ld] layout.
// The per-view work itself is dealt out: a warp spreads the (Gaussian, view)
// pairs of its 32 Gaussians over its 32 lanes (WarpDeal), since most Gaussians
// have no view in a given image subset and the others 1 to 64.
//
// Splat attributes y (9): mean (mx, my), conic (A, B, C) = inverse of the 2D
// covariance [[a, b], [b, c]], opacity o, colour (r, g, b).
#include <algorithm>

#include "internal.cuh"

namespace gslm {
namespace {

// Real spherical harmonics, degree <= 3, with the Condon-Shortley phase
// (sign (-1)^m); normalisation constants are the closed forms
// 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4,
// sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.09254843059207907f;
constexpr float kY2b = 0.31539156525252001f;
constexpr float kY2c = 0.54627421529603953f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.89061144264055405f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011540f;
constexpr float kY3e = 1.44530572132027702f;

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kY0;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// g = sum_k w_k grad Y_k(x, y, z), the polynomial gradient (no re-normalisation).
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float w[16], float g[3]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  gy += -kY1 * w[1];
  gz += kY1 * w[2];
  gx += -kY1 * w[3];
  gx += kY2a * y * w[4];            gy += kY2a * x * w[4];
  gy += -kY2a * z * w[5];           gz += -kY2a * y * w[5];
  gx += -2.f * kY2b * x * w[6];     gy += -2.f * kY2b * y * w[6];     gz += 4.f * kY2b * z * w[6];
  gx += -kY2a * z * w[7];           gz += -kY2a * x * w[7];
  gx += 2.f * kY2c * x * w[8];      gy += -2.f * kY2c * y * w[8];
  gx += -kY3a * 6.f * x * y * w[9]; gy += -kY3a * (3.f * xx - 3.f * yy) * w[9];
  gx += kY3b * y * z * w[10];       gy += kY3b * x * z * w[10];       gz += kY3b * x * y * w[10];
  gx += kY3c * 2.f * x * y * w[11];
  gy += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz += -kY3c * 8.f * y * z * w[11];
  gx += -kY3d * 6.f * x * z * w[12];
  gy += -kY3d * 6.f * y * z * w[12];
  gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
  gy += kY3c * 2.f * x * y * w[13];
  gz += -kY3c * 8.f * x * z * w[13];
  gx += kY3e * 2.f * x * z * w[14]; gy += -kY3e * 2.f * y * z * w[14]; gz += kY3e * (xx - yy) * w[14];
  gx += -kY3a * (3.f * xx - 3.f * yy) * w[15];
  gy += kY3a * 6.f * x * y * w[15];
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
}

// View-independent state of one Gaussian.
struct GaussGeo {
  float mu[3];
  float qn[4];
  float qinv;      // 1 / |q|
  float R[9];      // rotation of the normalised quaternion, row-major
  float S[3];      // exp(log-scale)
  float M[9];      // R diag(S)
  float Sig[6];    // 3D covariance M M^T: xx, xy, xz, yy, yz, zz
  float o;         // opacity
};

__device__ __forceinline__ float sym(const float s[6], int i, int j) {
  // index of (i, j) in xx, xy, xz, yy, yz, zz
  const int a = i < j ? i : j, b = i < j ? j : i;
  const int idx = a == 0 ? b : (a == 1 ? 2 + b : 5);
  return s[idx];
}

__device__ __forceinline__ void gauss_geo(const float* __restrict__ P, long long ld, int g, GaussGeo& G) {
  G.mu[0] = P[0 * ld + g];
  G.mu[1] = P[1 * ld + g];
  G.mu[2] = P[2 * ld + g];
  const float q0 = P[6 * ld + g], q1 = P[7 * ld + g], q2 = P[8 * ld + g], q3 = P[9 * ld + g];
  const float len = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  G.qinv = 1.f / len;
  const float w = q0 * G.qinv, x = q1 * G.qinv, y = q2 * G.qinv, z = q3 * G.qinv;
  G.qn[0] = w; G.qn[1] = x; G.qn[2] = y; G.qn[3] = z;
  G.R[0] = 1.f - 2.f * (y * y + z * z); G.R[1] = 2.f * (x * y - w * z); G.R[2] = 2.f * (x * z + w * y);
  G.R[3] = 2.f * (x * y + w * z); G.R[4] = 1.f - 2.f * (x * x + z * z); G.R[5] = 2.f * (y * z - w * x);
  G.R[6] = 2.f * (x * z - w * y); G.R[7] = 2.f * (y * z + w * x); G.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int j = 0; j < 3; ++j) G.S[j] = expf(P[(3 + j) * ld + g]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) G.M[i * 3 + j] = G.R[i * 3 + j] * G.S[j];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      G.Sig[k++] = G.M[i * 3 + 0] * G.M[j * 3 + 0] + G.M[i * 3 + 1] * G.M[j * 3 + 1] +
                   G.M[i * 3 + 2] * G.M[j * 3 + 2];
    }
  G.o = 1.f / (1.f + expf(-P[10 * ld + g]));
}

// Per-view state of one splat.
struct ViewGeo {
  float tc[3];
  float iz;
  float T0[3], T1[3];      // T = Jp W (2 x 3)
  float ST0[3], ST1[3];    // Sigma T0^T, Sigma T1^T
  float a, b, c;           // 2D covariance incl. dilation
  float A, B, C;           // conic
  float det;
  float mx, my;
  float dir[3];
  float inv_dlen;
};

__device__ __forceinline__ void view_geo(const GaussGeo& G, const DevCam& cam, ViewGeo& V) {
  const float* W = cam.R;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    V.tc[i] = W[i * 3 + 0] * G.mu[0] + W[i * 3 + 1] * G.mu[1] + W[i * 3 + 2] * G.mu[2] + cam.t[i];
  V.iz = 1.f / V.tc[2];
  const float iz2 = V.iz * V.iz;
  const float J00 = cam.fx * V.iz, J02 = -cam.fx * V.tc[0] * iz2;
  const float J11 = cam.fy * V.iz, J12 = -cam.fy * V.tc[1] * iz2;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    V.T0[k] = J00 * W[0 * 3 + k] + J02 * W[2 * 3 + k];
    V.T1[k] = J11 * W[1 * 3 + k] + J12 * W[2 * 3 + k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    V.ST0[i] = sym(G.Sig, i, 0) * V.T0[0] + sym(G.Sig, i, 1) * V.T0[1] + sym(G.Sig, i, 2) * V.T0[2];
    V.ST1[i] = sym(G.Sig, i, 0) * V.T1[0] + sym(G.Sig, i, 1) * V.T1[1] + sym(G.Sig, i, 2) * V.T1[2];
  }
  V.a = V.T0[0] * V.ST0[0] + V.T0[1] * V.ST0[1] + V.T0[2] * V.ST0[2] + kDilation;
  V.b = V.T0[0] * V.ST1[0] + V.T0[1] * V.ST1[1] + V.T0[2] * V.ST1[2];
  V.c = V.T1[0] * V.ST1[0] + V.T1[1] * V.ST1[1] + V.T1[2] * V.ST1[2] + kDilation;
  V.det = V.a * V.c - V.b * V.b;
  const float inv = 1.f / V.det;
  V.A = V.c * inv;
  V.B = -V.b * inv;
  V.C = V.a * inv;
  V.mx = cam.fx * V.tc[0] * V.iz + cam.cx;
  V.my = cam.fy * V.tc[1] * V.iz + cam.cy;
  const float d0 = G.mu[0] - cam.campos[0], d1 = G.mu[1] - cam.campos[1], d2 = G.mu[2] - cam.campos[2];
  const float dl = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  V.inv_dlen = 1.f / dl;
  V.dir[0] = d0 * V.inv_dlen;
  V.dir[1] = d1 * V.inv_dlen;
  V.dir[2] = d2 * V.inv_dlen;
}

// d(R(qn)) for a tangent qdn of the normalised quaternion.
__device__ __forceinline__ void rot_tangent(const float qn[4], const float qd[4], float Rd[9]) {
  const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  const float dw = qd[0], dx = qd[1], dy = qd[2], dz = qd[3];
  Rd[0] = -4.f * (y * dy + z * dz);
  Rd[1] = 2.f * (dx * y + x * dy - dw * z - w * dz);
  Rd[2] = 2.f * (dx * z + x * dz + dw * y + w * dy);
  Rd[3] = 2.f * (dx * y + x * dy + dw * z + w * dz);
  Rd[4] = -4.f * (x * dx + z * dz);
  Rd[5] = 2.f * (dy * z + y * dz - dw * x - w * dx);
  Rd[6] = 2.f * (dx * z + x * dz - dw * y - w * dy);
  Rd[7] = 2.f * (dy * z + y * dz + dw * x + w * dx);
  Rd[8] = -4.f * (x * dx + y * dy);
}

// Tangent of the 3D covariance for parameter tangents (ds, dq).
__device__ __forceinline__ void sigma_tangent(const GaussGeo& G, const float ds[3], const float dq[4],
                                              float Sd[6]) {
  const float qdot = G.qn[0] * dq[0] + G.qn[1] * dq[1] + G.qn[2] * dq[2] + G.qn[3] * dq[3];
  float qnd[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) qnd[i] = (dq[i] - G.qn[i] * qdot) * G.qinv;
  float Rd[9];
  rot_tangent(G.qn, qnd, Rd);
  float Md[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Md[i * 3 + j] = Rd[i * 3 + j] * G.S[j] + G.R[i * 3 + j] * G.S[j] * ds[j];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      Sd[k++] = Md[i * 3 + 0] * G.M[j * 3 + 0] + Md[i * 3 + 1] * G.M[j * 3 + 1] + Md[i * 3 + 2] * G.M[j * 3 + 2] +
                G.M[i * 3 + 0] * Md[j * 3 + 0] + G.M[i * 3 + 1] * Md[j * 3 + 1] + G.M[i * 3 + 2] * Md[j * 3 + 2];
    }
}

// Geometric part of ydot: (mx, my, A, B, C) tangents for mean tangent mud and
// covariance tangent Sd.
__device__ __forceinline__ void geo_tangent(const ViewGeo& V, const DevCam& cam, const float mud[3],
                                            const float Sd[6], float yd[5]) {
  const float* W = cam.R;
  float td[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) td[i] = W[i * 3 + 0] * mud[0] + W[i * 3 + 1] * mud[1] + W[i * 3 + 2] * mud[2];
  const float iz = V.iz, iz2 = iz * iz, iz3 = iz2 * iz;
  yd[0] = cam.fx * (td[0] * iz - V.tc[0] * iz2 * td[2]);
  yd[1] = cam.fy * (td[1] * iz - V.tc[1] * iz2 * td[2]);
  const float J00d = -cam.fx * iz2 * td[2];
  const float J02d = -cam.fx * (td[0] * iz2 - 2.f * V.tc[0] * iz3 * td[2]);
  const float J11d = -cam.fy * iz2 * td[2];
  const float J12d = -cam.fy * (td[1] * iz2 - 2.f * V.tc[1] * iz3 * td[2]);
  float T0d[3], T1d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T0d[k] = J00d * W[0 * 3 + k] + J02d * W[2 * 3 + k];
    T1d[k] = J11d * W[1 * 3 + k] + J12d * W[2 * 3 + k];
  }
  // T0 Sd T0^T etc.
  float SdT0[3], SdT1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    SdT0[i] = sym(Sd, i, 0) * V.T0[0] + sym(Sd, i, 1) * V.T0[1] + sym(Sd, i, 2) * V.T0[2];
    SdT1[i] = sym(Sd, i, 0) * V.T1[0] + sym(Sd, i, 1) * V.T1[1] + sym(Sd, i, 2) * V.T1[2];
  }
  const float ad = 2.f * (T0d[0] * V.ST0[0] + T0d[1] * V.ST0[1] + T0d[2] * V.ST0[2]) +
                   (V.T0[0] * SdT0[0] + V.T0[1] * SdT0[1] + V.T0[2] * SdT0[2]);
  const float bd = (T0d[0] * V.ST1[0] + T0d[1] * V.ST1[1] + T0d[2] * V.ST1[2]) +
                   (T1d[0] * V.ST0[0] + T1d[1] * V.ST0[1] + T1d[2] * V.ST0[2]) +
                   (V.T0[0] * SdT1[0] + V.T0[1] * SdT1[1] + V.T0[2] * SdT1[2]);
  const float cd = 2.f * (T1d[0] * V.ST1[0] + T1d[1] * V.ST1[1] + T1d[2] * V.ST1[2]) +
                   (V.T1[0] * SdT1[0] + V.T1[1] * SdT1[1] + V.T1[2] * SdT1[2]);
  const float A = V.A, B = V.B, C = V.C;
  yd[2] = -(A * A * ad + 2.f * A * B * bd + B * B * cd);
  yd[3] = -(A * B * ad + (A * C + B * B) * bd + B * C * cd);
  yd[4] = -(B * B * ad + 2.f * B * C * bd + C * C * cd);
}

__device__ __forceinline__ long long n_slots(int N, int V) { return (long long)N * V; }

// Iteration over the views of one Gaussian: with a view mask (bit v set when the
// splat of view v has cache entries; only for V <= 64) the set bits in
// ascending order, otherwise every view. `mm` holds the bits not yet visited.
__device__ __forceinline__ int next_view(bool use_mask, unsigned long long& mm, int v, int V) {
  if (!use_mask) return v + 1;
  if (mm == 0) return V;
  const int b = __ffsll((long long)mm) - 1;
  mm &= mm - 1;
  return b;
}

__global__ void k_view_mask(const uint8_t* __restrict__ slot_active, int N, int V,
                            unsigned long long* __restrict__ vmask) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  unsigned long long m = 0;
  for (int v = 0; v < V && v < 64; ++v)
    if (slot_active[(long long)v * N + g]) m |= 1ull << v;
  vmask[g] = m;
}

__global__ void k_project(const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams,
                          int V, int smooth, SplatRec* __restrict__ rec, uint32_t* __restrict__ ntiles,
                          uint2* __restrict__ rect, uint32_t* __restrict__ depth_key,
                          unsigned long long* __restrict__ tmask) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots(N, V)) return;
  const int v = (int)(s / N);
  const int g = (int)(s - (long long)v * N);
  const DevCam& cam = cams[v];
  const float tz = cam.R[6] * P[0 * ld + g] + cam.R[7] * P[1 * ld + g] + cam.R[8] * P[2 * ld + g] + cam.t[2];
  ntiles[s] = 0;
  depth_key[s] = 0xffffffffu;
  if (!(tz > kNear)) return;
  GaussGeo G;
  gauss_geo(P, ld, g, G);
  ViewGeo VG;
  view_geo(G, cam, VG);
  if (!(VG.det > 0.f) || !isfinite(VG.A) || !isfinite(VG.mx) || !isfinite(VG.my)) return;
  const float mid = 0.5f * (VG.a + VG.c);
  const float disc = fmaxf(0.25f * (VG.a - VG.c) * (VG.a - VG.c) + VG.b * VG.b, 0.f);
  const float lam = mid + sqrtf(disc);
  const float r = ceilf(kRadiusSigmas * sqrtf(lam));
  int x0, y0, x1, y1;
  if (smooth) {
    x0 = 0; y0 = 0; x1 = cam.tiles_x; y1 = cam.tiles_y;
  } else {
    const float inv = 1.f / kTile;
    x0 = (int)fminf(fmaxf(floorf((VG.mx - r) * inv), 0.f), (float)cam.tiles_x);
    y0 = (int)fminf(fmaxf(floorf((VG.my - r) * inv), 0.f), (float)cam.tiles_y);
    x1 = (int)fminf(fmaxf(floorf((VG.mx + r) * inv) + 1.f, 0.f), (float)cam.tiles_x);
    y1 = (int)fminf(fmaxf(floorf((VG.my + r) * inv) + 1.f, 0.f), (float)cam.tiles_y);
  }
  if (x1 <= x0 || y1 <= y0) return;
  // tiles of a small rectangle the splat can reach (all for a large one)
  // (the key emission reads the mask of every rectangle of at most
  // kCullMaxTiles tiles, so it is written for each of them: all bits in smooth mode)
  uint32_t nt = (uint32_t)((x1 - x0) * (y1 - y0));
  if (tmask != nullptr && nt <= (uint32_t)kCullMaxTiles) {
    unsigned long long m = nt == 64u ? ~0ull : (1ull << nt) - 1ull;
    if (!smooth) {
      m = 0ull;
      int bit = 0;
      for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx, ++bit)
          if (tile_reachable(VG.mx, VG.my, VG.A, VG.B, VG.C, G.o, tx, ty)) m |= 1ull << bit;
    }
    nt = (uint32_t)__popcll(m);
    tmask[s] = m;
    if (nt == 0) return;   // the splat reaches no pixel
  }
  float Y[16];
  sh_basis(VG.dir[0], VG.dir[1], VG.dir[2], Y);
  float rgb[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += Y[k] * P[(11 + 3 * k + ch) * ld + g];
    acc += kShOffset;
    rgb[ch] = smooth ? acc : fmaxf(acc, 0.f);
  }
  SplatRec R;
  R.a = make_float4(VG.mx, VG.my, VG.A, VG.B);
  R.b = make_float4(VG.C, G.o, VG.tc[2], 0.f);
  R.c = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
  rec[s] = R;
  ntiles[s] = nt;
  rect[s] = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
  depth_key[s] = __float_as_uint(VG.tc[2]);
}

// The per-Gaussian kernels split each Gaussian's work over the four warps of a
// 128-thread block (32 Gaussians per block, lane = Gaussian): warp 0 takes the
// geometry (mean, scale, rotation, opacity), warp 1 + c the SH coefficients of
// colour channel c and that channel's view-direction term of the mean. Warps
// never diverge on the role, and no thread holds all 59 parameters at once.
constexpr int kGPB = 32;   // Gaussians per block

// Parameter rows owned by a role: 0 -> rows 0..10; 1 + c -> rows 11 + 3k + c.
__device__ __forceinline__ int role_rows(int role) { return role == 0 ? 11 : 16; }
__device__ __forceinline__ int role_row(int role, int i) { return role == 0 ? i : 11 + 3 * i + (role - 1); }

// (Gaussian, view) pairs of a warp's 32 Gaussians, dealt to its lanes. Lane l
// owns Gaussian g0 + l with view mask m_l (ascending set bits = its active
// views) and compact splat index base b_l; pair t of the warp (t < total) is
// view number r of owner o, where o is the last lane whose exclusive prefix of
// the mask popcounts is <= t and r = t - prefix_o. Whatever the owners' view
// counts, every lane of the warp takes ceil(total / 32) pairs, where a loop
// over each lane's own views would run as long as the busiest lane's.
struct WarpDeal {
  unsigned long long mask[kGPB];
  uint32_t base[kGPB];
  uint32_t off[kGPB];   // exclusive prefix of the popcounts
};

// Position of the r-th (from 0) set bit of m; r < popc(m).
__device__ __forceinline__ int nth_set_bit(unsigned long long m, uint32_t r) {
  int pos = 0;
#pragma unroll
  for (int w = 32; w >= 1; w >>= 1) {
    const unsigned long long low = m & ((1ull << w) - 1ull);
    const uint32_t c = (uint32_t)__popcll(low);
    if (r >= c) {
      r -= c;
      m >>= w;
      pos += w;
    } else {
      m = low;
    }
  }
  return pos;
}

// Fills the warp's deal table (all 32 lanes call it) and returns the number of
// pairs.
__device__ __forceinline__ uint32_t deal_setup(WarpDeal& D, unsigned long long m, uint32_t base, int lane) {
  const uint32_t c = (uint32_t)__popcll(m);
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  D.mask[lane] = m;
  D.base[lane] = base;
  D.off[lane] = inc - c;
  __syncwarp();
  return __shfl_sync(0xffffffffu, inc, 31);
}

// Owner lane, view and compact splat index of pair t.
__device__ __forceinline__ void deal_pair(const WarpDeal& D, uint32_t t, int& o, int& v, long long& key) {
  o = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1)
    if (D.off[o + step] <= t) o += step;
  const uint32_t r = t - D.off[o];
  v = nth_set_bit(D.mask[o], r);
  key = (long long)D.base[o] + r;
}

// Per-warp staging of the tangent's per-Gaussian inputs, [field][lane]: the
// geometry warp keeps mu (3), Sigma (6), the mean tangent (3), the covariance
// tangent (6) and the opacity tangent; a colour warp the channel's 16 SH
// coefficients, their 16 tangents, mu (3) and the mean tangent (3).
constexpr int kTanFields = 38;
struct TangentShared {
  float f[4][kTanFields][kGPB];
  WarpDeal deal[4];
};

// ydot[slot] = (dy/dx) p for every active slot of Gaussian g. With z_beta
// given, first p = z + beta p (Algorithm 1's last vector update, fused), and
// the new p is written back to p_out. Roles: see above; the geometry warp
// writes floats 0..5 of the slot's 12, warp 1 + c float 6 + c. With view masks
// each warp deals its Gaussians' (Gaussian, view) pairs to all its lanes
// (WarpDeal); without them (more than 64 views) each lane walks its own views.
// All 32 lanes of a warp call this (g >= N on the lanes past the last Gaussian).
__device__ __forceinline__ void tangent_body(
    int g, int role, const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V,
    int smooth, const uint8_t* __restrict__ slot_active, const unsigned long long* __restrict__ vmask,
    const uint32_t* __restrict__ act_off, const float* __restrict__ pin, float* __restrict__ ydot,
    const float* __restrict__ zb, float* __restrict__ pout, const PcgScalars* __restrict__ sc, TangentShared& S) {
  if (sc != nullptr && sc->done) return;   // the same for the whole block
  const bool valid = g < N;
  const int lane = threadIdx.x & 31;
  const float beta = zb != nullptr ? (float)sc->beta : 0.f;
  auto pval = [&](int row) -> float {
    const long long o = (long long)row * ld + g;
    return zb != nullptr ? zb[o] + beta * pin[o] : pin[o];
  };
  // own rows (updated and written back when fused), and the mean rows
  float pm[3] = {0.f, 0.f, 0.f};
  if (valid) {
#pragma unroll
    for (int i = 0; i < 3; ++i) pm[i] = pval(i);
  }
  const bool use_mask = vmask != nullptr;
  const unsigned long long m0 = (use_mask && valid) ? vmask[g] : 0ull;
  float (*F)[kGPB] = S.f[role];
  if (role == 0) {
    float pg[11];
    if (valid) {
#pragma unroll
      for (int i = 0; i < 11; ++i) {
        pg[i] = i < 3 ? pm[i] : pval(i);
        if (pout != nullptr) pout[(long long)i * ld + g] = pg[i];
      }
    }
    if (!use_mask) {
      if (!valid) return;
      GaussGeo G;
      gauss_geo(P, ld, g, G);
      float Sd[6];
      sigma_tangent(G, pg + 3, pg + 6, Sd);
      const float od = G.o * (1.f - G.o) * pg[10];
      for (int v = 0; v < V; ++v) {
        const long long slot = (long long)v * N + g;
        if (!slot_active[slot]) continue;
        const DevCam& cam = cams[v];
        ViewGeo VG;
        view_geo(G, cam, VG);
        float yd[5];
        geo_tangent(VG, cam, pm, Sd, yd);
        float* out = ydot + slot * 12;
        reinterpret_cast<float4*>(out)[0] = make_float4(yd[0], yd[1], yd[2], yd[3]);
        reinterpret_cast<float2*>(out)[2] = make_float2(yd[4], od);
      }
      return;
    }
    if (m0 != 0ull) {
      GaussGeo G;
      gauss_geo(P, ld, g, G);
      float Sd[6];
      sigma_tangent(G, pg + 3, pg + 6, Sd);
#pragma unroll
      for (int i = 0; i < 3; ++i) F[i][lane] = G.mu[i];
#pragma unroll
      for (int i = 0; i < 6; ++i) F[3 + i][lane] = G.Sig[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) F[9 + i][lane] = pm[i];
#pragma unroll
      for (int i = 0; i < 6; ++i) F[12 + i][lane] = Sd[i];
      F[18][lane] = G.o * (1.f - G.o) * pg[10];
    }
    const uint32_t total = deal_setup(S.deal[0], m0, m0 != 0ull ? act_off[g] : 0u, lane);
    for (uint32_t t = lane; t < total; t += 32) {
      int o, v;
      long long ti;
      deal_pair(S.deal[0], t, o, v, ti);
      GaussGeo G;   // view_geo reads mu and Sigma only
#pragma unroll
      for (int i = 0; i < 3; ++i) G.mu[i] = F[i][o];
#pragma unroll
      for (int i = 0; i < 6; ++i) G.Sig[i] = F[3 + i][o];
      float pmo[3], Sd[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) pmo[i] = F[9 + i][o];
#pragma unroll
      for (int i = 0; i < 6; ++i) Sd[i] = F[12 + i][o];
      const DevCam& cam = cams[v];
      ViewGeo VG;
      view_geo(G, cam, VG);
      float yd[5];
      geo_tangent(VG, cam, pmo, Sd, yd);
      float* out = ydot + ti * 12;
      reinterpret_cast<float4*>(out)[0] = make_float4(yd[0], yd[1], yd[2], yd[3]);
      reinterpret_cast<float2*>(out)[2] = make_float2(yd[4], F[18][o]);
    }
  } else {
    const int ch = role - 1;
    float ps[16], w[16];
    if (valid) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int row = 11 + 3 * k + ch;
        ps[k] = pval(row);
        if (pout != nullptr) pout[(long long)row * ld + g] = ps[k];
      }
    }
    // view v of Gaussian gg: the colour tangent of channel ch
    auto colour = [&](const float (&wv)[16], const float (&psv)[16], const float (&mu)[3], const float (&pmv)[3],
                      const DevCam& cam) -> float {
      const float d0 = mu[0] - cam.campos[0], d1 = mu[1] - cam.campos[1], d2 = mu[2] - cam.campos[2];
      const float inv_dlen = 1.f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      const float dir[3] = {d0 * inv_dlen, d1 * inv_dlen, d2 * inv_dlen};
      float Y[16];
      sh_basis(dir[0], dir[1], dir[2], Y);
      const float mdot = dir[0] * pmv[0] + dir[1] * pmv[1] + dir[2] * pmv[2];
      float raw = kShOffset, acc = 0.f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        raw += Y[k] * wv[k];
        acc += Y[k] * psv[k];
      }
      float gr[3];
      sh_grad(dir[0], dir[1], dir[2], wv, gr);
#pragma unroll
      for (int i = 0; i < 3; ++i) acc += gr[i] * (pmv[i] - dir[i] * mdot) * inv_dlen;
      return (!smooth && raw < 0.f) ? 0.f : acc;
    };
    if (!use_mask) {
      if (!valid) return;
#pragma unroll
      for (int k = 0; k < 16; ++k) w[k] = P[(11 + 3 * k + ch) * ld + g];
      const float mu[3] = {P[g], P[ld + g], P[2 * ld + g]};
      for (int v = 0; v < V; ++v) {
        const long long slot = (long long)v * N + g;
        if (!slot_active[slot]) continue;
        ydot[slot * 12 + 6 + ch] = colour(w, ps, mu, pm, cams[v]);
      }
      return;
    }
    if (m0 != 0ull) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        F[k][lane] = P[(11 + 3 * k + ch) * ld + g];
        F[16 + k][lane] = ps[k];
      }
      F[32][lane] = P[g];
      F[33][lane] = P[ld + g];
      F[34][lane] = P[2 * ld + g];
#pragma unroll
      for (int i = 0; i < 3; ++i) F[35 + i][lane] = pm[i];
    }
    const uint32_t total = deal_setup(S.deal[role], m0, m0 != 0ull ? act_off[g] : 0u, lane);
    for (uint32_t t = lane; t < total; t += 32) {
      int o, v;
      long long ti;
      deal_pair(S.deal[role], t, o, v, ti);
      float wo[16], pso[16], mu[3], pmo[3];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        wo[k] = F[k][o];
        pso[k] = F[16 + k][o];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        mu[i] = F[32 + i][o];
        pmo[i] = F[35 + i][o];
      }
      ydot[ti * 12 + 6 + ch] = colour(wo, pso, mu, pmo, cams[v]);
    }
  }
}

// Per-view terms of the adjoint. Geometry: for the splat's ybar (mean 2,
// conic 3, opacity) the view's terms of the 3D covariance gradient GS (6,
// symmetric), of the opacity sum and of the mean gradient (3).
__device__ __forceinline__ void vjp_geo_terms(const GaussGeo& G, const DevCam& cam, const float yb[6], float GS[6],
                                              float& ob, float mub[3]) {
  ViewGeo VG;
  view_geo(G, cam, VG);
  ob += yb[5];
  // conic -> 2D covariance
  const float A = VG.A, B = VG.B, C = VG.C;
  const float ab = -(A * A * yb[2] + A * B * yb[3] + B * B * yb[4]);
  const float bb = -(2.f * A * B * yb[2] + (A * C + B * B) * yb[3] + 2.f * B * C * yb[4]);
  const float cb = -(B * B * yb[2] + B * C * yb[3] + C * C * yb[4]);
  // 2D covariance -> 3D covariance (symmetric full-matrix gradient) and T
  {
    int k = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        GS[k++] += ab * VG.T0[i] * VG.T0[j] + 0.5f * bb * (VG.T0[i] * VG.T1[j] + VG.T1[i] * VG.T0[j]) +
                   cb * VG.T1[i] * VG.T1[j];
      }
  }
  float T0b[3], T1b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T0b[i] = 2.f * ab * VG.ST0[i] + bb * VG.ST1[i];
    T1b[i] = bb * VG.ST0[i] + 2.f * cb * VG.ST1[i];
  }
  const float* W = cam.R;
  const float J00b = T0b[0] * W[0] + T0b[1] * W[1] + T0b[2] * W[2];
  const float J02b = T0b[0] * W[6] + T0b[1] * W[7] + T0b[2] * W[8];
  const float J11b = T1b[0] * W[3] + T1b[1] * W[4] + T1b[2] * W[5];
  const float J12b = T1b[0] * W[6] + T1b[1] * W[7] + T1b[2] * W[8];
  const float iz = VG.iz, iz2 = iz * iz, iz3 = iz2 * iz;
  const float tx = VG.tc[0], ty = VG.tc[1];
  float tb[3];
  tb[0] = -cam.fx * iz2 * J02b + cam.fx * iz * yb[0];
  tb[1] = -cam.fy * iz2 * J12b + cam.fy * iz * yb[1];
  tb[2] = -cam.fx * iz2 * J00b + 2.f * cam.fx * tx * iz3 * J02b - cam.fy * iz2 * J11b +
          2.f * cam.fy * ty * iz3 * J12b - cam.fx * tx * iz2 * yb[0] - cam.fy * ty * iz2 * yb[1];
#pragma unroll
  for (int i = 0; i < 3; ++i) mub[i] += W[0 * 3 + i] * tb[0] + W[1 * 3 + i] * tb[1] + W[2 * 3 + i] * tb[2];
}

// Colour channel: for the splat's colour ybar yc, the view's terms of the
// channel's 16 SH coefficient gradients and of the mean gradient (3).
__device__ __forceinline__ void vjp_colour_terms(const float w[16], const float mu[3], const DevCam& cam, float yc,
                                                 int smooth, float out[16], float mub[3]) {
  const float d0 = mu[0] - cam.campos[0], d1 = mu[1] - cam.campos[1], d2 = mu[2] - cam.campos[2];
  const float inv_dlen = 1.f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  const float dir[3] = {d0 * inv_dlen, d1 * inv_dlen, d2 * inv_dlen};
  float Y[16];
  sh_basis(dir[0], dir[1], dir[2], Y);
  float raw = kShOffset;
#pragma unroll
  for (int k = 0; k < 16; ++k) raw += Y[k] * w[k];
  const float rb = (!smooth && raw < 0.f) ? 0.f : yc;
  float wsum[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    out[k] += Y[k] * rb;
    wsum[k] = rb * w[k];
  }
  float db[3];
  sh_grad(dir[0], dir[1], dir[2], wsum, db);
  const float dd = dir[0] * db[0] + dir[1] * db[1] + dir[2] * db[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) mub[i] += (db[i] - dir[i] * dd) * inv_dlen;
}

// The splat's ybar: its record (one per Gaussian and view), or the sum of its
// segments' partials. Returns false for a splat without segments.
__device__ __forceinline__ bool splat_ybar6(const float* __restrict__ splat_ybar, const float* __restrict__ seg_ybar,
                                            const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
                                            long long sk, float yb[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) yb[i] = 0.f;
  if (splat_ybar != nullptr) {
    const float* sy = splat_ybar + (size_t)sk * 12;
    const float4 u0 = *reinterpret_cast<const float4*>(sy);
    const float2 u1 = *reinterpret_cast<const float2*>(sy + 4);
    yb[0] = u0.x; yb[1] = u0.y; yb[2] = u0.z; yb[3] = u0.w; yb[4] = u1.x; yb[5] = u1.y;
    return true;
  }
  const uint32_t a = s_start[sk], b = s_end[sk];
  for (uint32_t j = a; j < b; ++j) {
    const float* sy = seg_ybar + (size_t)j * 12;
    const float4 u0 = *reinterpret_cast<const float4*>(sy);
    const float2 u1 = *reinterpret_cast<const float2*>(sy + 4);
    yb[0] += u0.x; yb[1] += u0.y; yb[2] += u0.z; yb[3] += u0.w; yb[4] += u1.x; yb[5] += u1.y;
  }
  return a != b;
}

__device__ __forceinline__ bool splat_ybar_colour(const float* __restrict__ splat_ybar,
                                                  const float* __restrict__ seg_ybar,
                                                  const uint32_t* __restrict__ s_start,
                                                  const uint32_t* __restrict__ s_end, long long sk, int ch,
                                                  float& yc) {
  yc = 0.f;
  if (splat_ybar != nullptr) {
    yc = splat_ybar[(size_t)sk * 12 + 6 + ch];
    return true;
  }
  const uint32_t a = s_start[sk], b = s_end[sk];
  for (uint32_t j = a; j < b; ++j) yc += seg_ybar[(size_t)j * 12 + 6 + ch];
  return a != b;
}

// Shared staging of the adjoint with view masks: each warp deals its
// Gaussians' (Gaussian, view) pairs to its lanes in chunks of kVjpChunk; a
// pair's terms go to the chunk's rows, and each owner lane then adds its own
// rows in view order (the order a lane walking its own views adds them in).
constexpr int kVjpChunk = 32;
constexpr int kGeoTerms = 10, kGeoRow = 11;     // GS (6), ob, mub (3); odd row stride
constexpr int kColTerms = 19, kColRow = 19;     // out (16), mub (3)
struct VjpShared {
  float gin[9][kGPB];                           // geometry warp: mu (3), Sigma (6)
  float gt[kVjpChunk * kGeoRow];
  float cin[3][19][kGPB];                       // colour warp c: w (16), mu (3)
  float ct[3][kVjpChunk * kColRow];
  WarpDeal deal[4];
  float mub[4][kGPB][3];                        // the warps' mean-gradient sums
  float ep[4][16][kGPB], em[4][16][kGPB];       // the epilogue's p and M rows, copied ahead (cp.async)
};

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// g = scale * (dy/dx)^T ybar summed over the views; ybar of a slot is the sum
// of its segments' partial sums, which the tile kernel stores in splat order:
// the splat's range [s_start, s_end) of positions. A splat is keyed by its
// compact index act_off[g] + (rank of the view among g's active views) when
// the view masks exist, so that a Gaussian's segments of all its views form
// one contiguous run; else by its slot v * N + g.
// Epilogue (M != null): g += lambda M p and a per-block float64 partial of
// p^T g. Roles as for the tangent; the colour warps hand their view-direction
// terms of the mean gradient to the geometry warp through shared memory. With
// view masks each warp deals its Gaussians' (Gaussian, view) pairs to all its
// lanes (as the tangent does) and every owner adds its pairs' terms in view
// order; without them each lane walks its own views.
// All 128 threads of the block call this with the same g0.
__device__ __forceinline__ void vjp_body(
    int g0, const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V, int smooth,
    const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
    const unsigned long long* __restrict__ vmask, const uint32_t* __restrict__ act_off,
    const float* __restrict__ seg_ybar, const float* __restrict__ splat_ybar, float scale,
    float* __restrict__ gout, const float* __restrict__ p, const float* __restrict__ Mdiag, float lambda,
    VjpShared& S, double& local) {
  const int lane = threadIdx.x & 31, role = threadIdx.x >> 5;
  const int g = g0 + lane;
  const bool valid = g < N;
  const bool use_mask = vmask != nullptr;
  const unsigned long long m0 = (use_mask && valid) ? vmask[g] : 0ull;
  const uint32_t base = m0 != 0ull ? act_off[g] : 0u;   // compact splat index of the first active view
  // the epilogue's rows of p and M start moving now and land while the views
  // are worked on (each lane later reads only its own copies)
  const bool epi = valid && Mdiag != nullptr;
  if (epi) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (i < role_rows(role)) {
        const long long o = (long long)role_row(role, i) * ld + g;
        cp_async4(&S.ep[role][i][lane], p + o);
        cp_async4(&S.em[role][i][lane], Mdiag + o);
      }
    }
    cp_async_commit();
  }
  float mub[3] = {0.f, 0.f, 0.f};
  float out[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) out[k] = 0.f;
  if (role == 0) {
    float GS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float ob = 0.f;
    bool any = false;
    GaussGeo G;
    if (!use_mask) {
      for (int v = 0; valid && v < V; ++v) {
        float yb[6];
        if (!splat_ybar6(nullptr, seg_ybar, s_start, s_end, (long long)v * N + g, yb)) continue;
        if (!any) {
          gauss_geo(P, ld, g, G);
          any = true;
        }
        vjp_geo_terms(G, cams[v], yb, GS, ob, mub);
      }
    } else {
      if (m0 != 0ull) {
        gauss_geo(P, ld, g, G);
        any = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) S.gin[i][lane] = G.mu[i];
#pragma unroll
        for (int i = 0; i < 6; ++i) S.gin[3 + i][lane] = G.Sig[i];
      }
      WarpDeal& D = S.deal[0];
      const uint32_t total = deal_setup(D, m0, base, lane);
      const uint32_t my0 = D.off[lane], my1 = my0 + (uint32_t)__popcll(m0);
      for (uint32_t cb = 0; cb < total; cb += kVjpChunk) {
        const uint32_t ce = min(total, cb + (uint32_t)kVjpChunk);
        for (uint32_t t = cb + lane; t < ce; t += 32) {
          int o, v;
          long long sk;
          deal_pair(D, t, o, v, sk);
          float tGS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, tob = 0.f, tmub[3] = {0.f, 0.f, 0.f};
          float yb[6];
          if (splat_ybar6(splat_ybar, seg_ybar, s_start, s_end, sk, yb)) {
            GaussGeo Go;   // view_geo reads mu and Sigma only
#pragma unroll
            for (int i = 0; i < 3; ++i) Go.mu[i] = S.gin[i][o];
#pragma unroll
            for (int i = 0; i < 6; ++i) Go.Sig[i] = S.gin[3 + i][o];
            vjp_geo_terms(Go, cams[v], yb, tGS, tob, tmub);
          }
          float* row = S.gt + (t - cb) * kGeoRow;
#pragma unroll
          for (int i = 0; i < 6; ++i) row[i] = tGS[i];
          row[6] = tob;
#pragma unroll
          for (int i = 0; i < 3; ++i) row[7 + i] = tmub[i];
        }
        __syncwarp();
        for (uint32_t t = max(my0, cb); t < min(my1, ce); ++t) {
          const float* row = S.gt + (t - cb) * kGeoRow;
#pragma unroll
          for (int i = 0; i < 6; ++i) GS[i] += row[i];
          ob += row[6];
#pragma unroll
          for (int i = 0; i < 3; ++i) mub[i] += row[7 + i];
        }
        __syncwarp();   // the next chunk rewrites the rows
      }
    }
    if (any) {
      // 3D covariance -> M = R diag(S): Mb = 2 GS M
      float Mb[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          Mb[i * 3 + j] = 2.f * (sym(GS, i, 0) * G.M[0 * 3 + j] + sym(GS, i, 1) * G.M[1 * 3 + j] +
                                 sym(GS, i, 2) * G.M[2 * 3 + j]);
      float Rb[9];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float sbar = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          Rb[i * 3 + j] = Mb[i * 3 + j] * G.S[j];
          sbar += Mb[i * 3 + j] * G.R[i * 3 + j];
        }
        out[3 + j] = sbar * G.S[j];
      }
      const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
      float qb[4];
      qb[0] = 2.f * (-Rb[1] * z + Rb[2] * y + Rb[3] * z - Rb[5] * x - Rb[6] * y + Rb[7] * x);
      qb[1] = -4.f * x * (Rb[4] + Rb[8]) + 2.f * (Rb[1] * y + Rb[2] * z + Rb[3] * y - Rb[5] * w + Rb[6] * z + Rb[7] * w);
      qb[2] = -4.f * y * (Rb[0] + Rb[8]) + 2.f * (Rb[1] * x + Rb[2] * w + Rb[3] * x + Rb[5] * z - Rb[6] * w + Rb[7] * z);
      qb[3] = -4.f * z * (Rb[0] + Rb[4]) + 2.f * (-Rb[1] * w + Rb[2] * x + Rb[3] * w + Rb[5] * y + Rb[6] * x + Rb[7] * y);
      const float qd = G.qn[0] * qb[0] + G.qn[1] * qb[1] + G.qn[2] * qb[2] + G.qn[3] * qb[3];
#pragma unroll
      for (int i = 0; i < 4; ++i) out[6 + i] = (qb[i] - G.qn[i] * qd) * G.qinv;
      out[10] = ob * G.o * (1.f - G.o);
    }
  } else {
    // colour channel ch: SH coefficient gradients and the view-direction term of the mean
    const int ch = role - 1;
    if (!use_mask) {
      if (valid) {
        float w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = P[(11 + 3 * k + ch) * ld + g];
        const float mu[3] = {P[g], P[ld + g], P[2 * ld + g]};
        for (int v = 0; v < V; ++v) {
          float yc;
          if (!splat_ybar_colour(nullptr, seg_ybar, s_start, s_end, (long long)v * N + g, ch, yc)) continue;
          vjp_colour_terms(w, mu, cams[v], yc, smooth, out, mub);
        }
      }
    } else {
      float (*cin)[kGPB] = S.cin[ch];
      float* ct = S.ct[ch];
      if (m0 != 0ull) {
#pragma unroll
        for (int k = 0; k < 16; ++k) cin[k][lane] = P[(11 + 3 * k + ch) * ld + g];
        cin[16][lane] = P[g];
        cin[17][lane] = P[ld + g];
        cin[18][lane] = P[2 * ld + g];
      }
      WarpDeal& D = S.deal[role];
      const uint32_t total = deal_setup(D, m0, base, lane);
      const uint32_t my0 = D.off[lane], my1 = my0 + (uint32_t)__popcll(m0);
      for (uint32_t cb = 0; cb < total; cb += kVjpChunk) {
        const uint32_t ce = min(total, cb + (uint32_t)kVjpChunk);
        for (uint32_t t = cb + lane; t < ce; t += 32) {
          int o, v;
          long long sk;
          deal_pair(D, t, o, v, sk);
          float tout[16], tmub[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 0; k < 16; ++k) tout[k] = 0.f;
          float yc;
          if (splat_ybar_colour(splat_ybar, seg_ybar, s_start, s_end, sk, ch, yc)) {
            float w[16], mu[3];
#pragma unroll
            for (int k = 0; k < 16; ++k) w[k] = cin[k][o];
#pragma unroll
            for (int i = 0; i < 3; ++i) mu[i] = cin[16 + i][o];
            vjp_colour_terms(w, mu, cams[v], yc, smooth, tout, tmub);
          }
          float* row = ct + (t - cb) * kColRow;
#pragma unroll
          for (int k = 0; k < 16; ++k) row[k] = tout[k];
#pragma unroll
          for (int i = 0; i < 3; ++i) row[16 + i] = tmub[i];
        }
        __syncwarp();
        for (uint32_t t = max(my0, cb); t < min(my1, ce); ++t) {
          const float* row = ct + (t - cb) * kColRow;
#pragma unroll
          for (int k = 0; k < 16; ++k) out[k] += row[k];
#pragma unroll
          for (int i = 0; i < 3; ++i) mub[i] += row[16 + i];
        }
        __syncwarp();   // the next chunk rewrites the rows
      }
    }
  }
  S.mub[role][lane][0] = mub[0];
  S.mub[role][lane][1] = mub[1];
  S.mub[role][lane][2] = mub[2];
  __syncthreads();
  if (role == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = S.mub[0][lane][i] + S.mub[1][lane][i] + S.mub[2][lane][i] + S.mub[3][lane][i];
  }
  if (valid) {
    if (epi) cp_async_wait_all();
    const int nr = role_rows(role);
    float lf = 0.f;   // this role's rows of p^T g in float32; the sum over Gaussians in float64
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (i < nr) {
        const long long o = (long long)role_row(role, i) * ld + g;
        if (Mdiag != nullptr) {
          const float pk = S.ep[role][i][lane];
          const float gk = scale * out[i] + lambda * clamp_diag(S.em[role][i][lane]) * pk;
          gout[o] = gk;
          lf = fmaf(pk, gk, lf);
        } else {
          gout[o] = scale * out[i];
        }
      }
    }
    local += (double)lf;
  }
  __syncthreads();   // S is reused by the next group of Gaussians
}

// Block reduction of the float64 partial dot into partials[blockIdx.x].
__device__ __forceinline__ void write_dot_partial(double local, double* __restrict__ partials) {
  __shared__ double red[4];
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

__global__ void __launch_bounds__(128) k_tangent(
    const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V, int smooth,
    const uint8_t* __restrict__ slot_active, const unsigned long long* __restrict__ vmask,
    const uint32_t* __restrict__ act_off, const float* __restrict__ pin, float* __restrict__ ydot,
    const float* __restrict__ zb, float* __restrict__ pout, const PcgScalars* __restrict__ sc) {
  __shared__ TangentShared S;
  tangent_body(blockIdx.x * kGPB + (threadIdx.x & 31), threadIdx.x >> 5, P, N, ld, cams, V, smooth, slot_active,
               vmask, act_off, pin, ydot, zb, pout, sc, S);
}

// Batched: blockIdx.y is the subset; its p, z and pout sit at offset
// blockIdx.y * vs, its scalars at sc[blockIdx.y]. 7 blocks per SM (72
// registers, no spills): the paper workload's tangent phase took 12.6 ms per LM
// step against 15.7 at the 6 blocks its natural 80 registers allow.
__global__ void __launch_bounds__(128, 7) k_tangent_batch(const float* __restrict__ P, int N, long long ld, int smooth,
                                                       const __grid_constant__ GaussBatch gb,
                                                       const float* __restrict__ pin, long long vs,
                                                       const float* __restrict__ zb, float* __restrict__ pout,
                                                       const PcgScalars* __restrict__ sc) {
  const int b = blockIdx.y;
  const SubsetRefs& s = gb.s[b];
  const long long off = (long long)b * vs;
  __shared__ TangentShared S;
  tangent_body(blockIdx.x * kGPB + (threadIdx.x & 31), threadIdx.x >> 5, P, N, ld, s.cams, s.V, smooth,
               s.slot_active, s.vmask, s.act_off, pin + off, s.ydot, zb != nullptr ? zb + off : nullptr,
               pout != nullptr ? pout + off : nullptr, sc != nullptr ? sc + b : nullptr, S);
}

// Each block loops over groups of 32 Gaussians (bounded grid: at most
// kVjpBlocks float64 partials per call).
constexpr int kVjpBlocks = 2432;

__device__ __forceinline__ void vjp_blocks_loop(
    const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V, int smooth,
    const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
    const unsigned long long* __restrict__ vmask, const uint32_t* __restrict__ act_off,
    const float* __restrict__ seg_ybar, const float* __restrict__ splat_ybar, float scale,
    float* __restrict__ gout, const float* __restrict__ p, const float* __restrict__ Mdiag, float lambda,
    double* __restrict__ partials, const PcgScalars* __restrict__ sc) {
  __shared__ VjpShared S;
  double local = 0.0;
  if (sc == nullptr || !sc->done) {
    for (int g0 = blockIdx.x * kGPB; g0 < N; g0 += gridDim.x * kGPB)
      vjp_body(g0, P, N, ld, cams, V, smooth, s_start, s_end, vmask, act_off, seg_ybar, splat_ybar, scale, gout, p,
               Mdiag, lambda, S, local);
  }
  if (partials != nullptr) write_dot_partial(local, partials);
}

__global__ void __launch_bounds__(128, 4) k_vjp(
    const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V, int smooth,
    const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
    const unsigned long long* __restrict__ vmask, const uint32_t* __restrict__ act_off,
    const float* __restrict__ seg_ybar, const float* __restrict__ splat_ybar, float scale,
    float* __restrict__ gout, const float* __restrict__ p, const float* __restrict__ Mdiag, float lambda,
    double* __restrict__ partials, const PcgScalars* __restrict__ sc) {
  vjp_blocks_loop(P, N, ld, cams, V, smooth, s_start, s_end, vmask, act_off, seg_ybar, splat_ybar, scale, gout, p,
                  Mdiag, lambda, partials, sc);
}

// Batched: blockIdx.y is the subset; g, p and M at offset blockIdx.y * vs, the
// float64 partials at blockIdx.y * gridDim.x.
__global__ void __launch_bounds__(128, 4) k_vjp_batch(const float* __restrict__ P, int N, long long ld, int smooth,
                                                   const __grid_constant__ GaussBatch gb, float* __restrict__ gout,
                                                   long long vs, const float* __restrict__ p,
                                                   const float* __restrict__ Mdiag, float lambda,
                                                   double* __restrict__ partials, const PcgScalars* __restrict__ sc) {
  const int b = blockIdx.y;
  const SubsetRefs& s = gb.s[b];
  const long long off = (long long)b * vs;
  vjp_blocks_loop(P, N, ld, s.cams, s.V, smooth, s.s_start, s.s_end, s.vmask, s.act_off, s.seg_ybar,
                  s.act_off != nullptr ? s.ydot : nullptr, 1.f, gout + off,
                  p != nullptr ? p + off : nullptr, Mdiag != nullptr ? Mdiag + off : nullptr, lambda,
                  partials != nullptr ? partials + (size_t)b * gridDim.x : nullptr, sc != nullptr ? sc + b : nullptr);
}

// diag(J^T J) for every Gaussian: sum over views of v_k^T Q v_k, where v_k is
// column k of dy/dx and Q (per splat) is the sum over its cache entries and
// channels of (dc/dy)^T (dc/dy), weighted by the residual-to-pixel weights,
// stored as 21 geo-geo + 18 geo-rgb + 3 rgb values (and 2 of padding).

// One view's 59 terms of Gaussian g (geometry G, splat block Q), added to
// acc[k * stride].
__device__ __forceinline__ void diag_view_terms(const GaussGeo& G, const float (&Q)[kDiagBlock], const DevCam& cam,
                                                const float* __restrict__ P, long long ld, int g, int smooth,
                                                float* acc, int stride) {
  ViewGeo VG;
  view_geo(G, cam, VG);
  float Y[16];
  sh_basis(VG.dir[0], VG.dir[1], VG.dir[2], Y);
  bool live[3];
  float grad[3][3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float w[16];
    float raw = kShOffset;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      w[k] = P[(11 + 3 * k + ch) * ld + g];
      raw += Y[k] * w[k];
    }
    live[ch] = smooth || raw >= 0.f;
    sh_grad(VG.dir[0], VG.dir[1], VG.dir[2], w, grad[ch]);
  }
  const float D[3] = {Q[39], Q[40], Q[41]};   // per channel: the weights differ between channels
#pragma unroll
  for (int k = 0; k < 16; ++k)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
      if (live[ch]) acc[(11 + 3 * k + ch) * stride] += D[ch] * Y[k] * Y[k];
  // the 11 geometric parameters: unit tangents
#pragma unroll 1
  for (int k = 0; k < 11; ++k) {
    // unit tangent of parameter k, built with selects (k is not a
    // compile-time index here, and arrays indexed by it would go to local memory)
    float mud[3], ds[3], dq[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mud[i] = k == i ? 1.f : 0.f;
      ds[i] = k == 3 + i ? 1.f : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dq[i] = k == 6 + i ? 1.f : 0.f;
    const float od = k == 10 ? G.o * (1.f - G.o) : 0.f;
    float Sd[6];
    sigma_tangent(G, ds, dq, Sd);
    float yv[9];
    geo_tangent(VG, cam, mud, Sd, yv);
    yv[5] = od;
    if (k < 3) {
      const float md = k == 0 ? VG.dir[0] : k == 1 ? VG.dir[1] : VG.dir[2];
      float dd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) dd[i] = ((i == k ? 1.f : 0.f) - VG.dir[i] * md) * VG.inv_dlen;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch)
        yv[6 + ch] = live[ch] ? grad[ch][0] * dd[0] + grad[ch][1] * dd[1] + grad[ch][2] * dd[2] : 0.f;
    } else {
      yv[6] = yv[7] = yv[8] = 0.f;
    }
    // v^T Q v with Q = [[Qgg, X], [X^T, diag(D)]]
    float a = 0.f;
    int idx = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) {
        const float q = Q[idx++];
        a += (i == j ? 1.f : 2.f) * q * yv[i] * yv[j];
      }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) a += 2.f * Q[21 + i * 3 + c] * yv[i] * yv[6 + c];
    a += D[0] * yv[6] * yv[6] + D[1] * yv[7] * yv[7] + D[2] * yv[8] * yv[8];
    acc[k * stride] += a;
  }
}

// The splat's block Q: its precomputed sum (splat_q), or the sum of its
// segments' blocks. Returns false for a splat without segments.
__device__ __forceinline__ bool splat_block(const float* __restrict__ splat_q, const float* __restrict__ seg_q,
                                            const uint32_t* __restrict__ s_start,
                                            const uint32_t* __restrict__ s_end, long long sk,
                                            float (&Q)[kDiagBlock]) {
#pragma unroll
  for (int i = 0; i < kDiagBlock; ++i) Q[i] = 0.f;
  if (splat_q != nullptr) {
    const float4* q4 = reinterpret_cast<const float4*>(splat_q + (size_t)sk * kDiagBlock);
#pragma unroll
    for (int i = 0; i < kDiagBlock / 4; ++i) {
      const float4 t = q4[i];
      Q[4 * i + 0] = t.x; Q[4 * i + 1] = t.y; Q[4 * i + 2] = t.z; Q[4 * i + 3] = t.w;
    }
    return true;
  }
  const uint32_t a = s_start[sk], b = s_end[sk];
  for (uint32_t j = a; j < b; ++j) {
    const float4* q4 = reinterpret_cast<const float4*>(seg_q + (size_t)j * kDiagBlock);   // splat order
#pragma unroll
    for (int i = 0; i < kDiagBlock / 4; ++i) {
      const float4 t = q4[i];
      Q[4 * i + 0] += t.x; Q[4 * i + 1] += t.y; Q[4 * i + 2] += t.z; Q[4 * i + 3] += t.w;
    }
  }
  return a != b;
}

// Two warps of 32 Gaussians (lane = Gaussian). Each thread's 59 sums sit in
// its own column of shared memory (as a register array indexed by the rolled
// column loop they would live in local memory). With view masks a warp deals
// its Gaussians' (Gaussian, view) pairs to its lanes, 32 at a time: a pair's
// 59 terms go to its row of the warp's chunk, and each owner adds its rows in
// view order (the order of a lane walking its own views). Without masks (more
// than 64 views) each lane walks its own views.
constexpr int kDiagThreads = 64;
struct DiagShared {
  float sd[kNP][kDiagThreads];
  float rows[kDiagThreads / 32][32 * kNP];   // row stride 59 (odd): no bank conflicts
  WarpDeal deal[kDiagThreads / 32];
};
__global__ void __launch_bounds__(kDiagThreads, 6) k_diag(
    const float* __restrict__ P, int N, long long ld, const DevCam* __restrict__ cams, int V, int smooth,
    const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
    const unsigned long long* __restrict__ vmask, const uint32_t* __restrict__ act_off,
    const float* __restrict__ seg_q, const float* __restrict__ splat_q, float* __restrict__ dout) {
  __shared__ DiagShared S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = blockIdx.x * kDiagThreads + threadIdx.x;
  const bool valid = g < N;
  float* d = &S.sd[0][threadIdx.x];   // d[k * kDiagThreads] is sum k
#pragma unroll
  for (int k = 0; k < kNP; ++k) d[k * kDiagThreads] = 0.f;
  if (vmask == nullptr) {
    if (!valid) return;
    GaussGeo G;
    bool any = false;
    for (int v = 0; v < V; ++v) {
      float Q[kDiagBlock];
      if (!splat_block(splat_q, seg_q, s_start, s_end, (long long)v * N + g, Q)) continue;
      if (!any) {
        gauss_geo(P, ld, g, G);
        any = true;
      }
      diag_view_terms(G, Q, cams[v], P, ld, g, smooth, d, kDiagThreads);
    }
  } else {
    const unsigned long long m0 = valid ? vmask[g] : 0ull;
    WarpDeal& D = S.deal[warp];
    const uint32_t total = deal_setup(D, m0, m0 != 0ull ? act_off[g] : 0u, lane);
    const uint32_t my0 = D.off[lane], my1 = my0 + (uint32_t)__popcll(m0);
    const int gw = blockIdx.x * kDiagThreads + warp * 32;   // the warp's first Gaussian
    float* rows = S.rows[warp];
    for (uint32_t cb = 0; cb < total; cb += 32) {
      const uint32_t t = cb + lane;
      if (t < total) {
        float* row = rows + lane * kNP;
#pragma unroll
        for (int k = 0; k < kNP; ++k) row[k] = 0.f;
        int o, v;
        long long sk;
        deal_pair(D, t, o, v, sk);
        float Q[kDiagBlock];
        if (splat_block(splat_q, seg_q, s_start, s_end, sk, Q)) {
          GaussGeo G;
          gauss_geo(P, ld, gw + o, G);
          diag_view_terms(G, Q, cams[v], P, ld, gw + o, smooth, row, 1);
        }
      }
      __syncwarp();
      for (uint32_t tt = max(my0, cb); tt < min(my1, cb + 32u); ++tt) {
        const float* row = rows + (tt - cb) * kNP;
#pragma unroll
        for (int k = 0; k < kNP; ++k) d[k * kDiagThreads] += row[k];
      }
      __syncwarp();   // the next chunk rewrites the rows
    }
    if (!valid) return;
  }
#pragma unroll
  for (int k = 0; k < kNP; ++k) dout[k * ld + g] = d[k * kDiagThreads];
}

// Per compact splat: the sum of its segments' J^T u partials. The segments of
// a splat are one contiguous run in splat order, so consecutive threads read
// consecutive records; the adjoint then reads one record per (Gaussian, view)
// instead of walking a range per view behind a dependent load.
template <int kW4>   // float4s per record
__device__ __forceinline__ void splat_sum_body(long long c, const uint32_t* __restrict__ s_start,
                                               const uint32_t* __restrict__ s_end,
                                               const float* __restrict__ seg_rec, float* __restrict__ out) {
  float4 acc[kW4];
#pragma unroll
  for (int i = 0; i < kW4; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t j = s_start[c], e = s_end[c]; j < e; ++j) {
    const float4* q = reinterpret_cast<const float4*>(seg_rec + (size_t)j * (4 * kW4));
#pragma unroll
    for (int i = 0; i < kW4; ++i) {
      const float4 t = q[i];
      acc[i].x += t.x; acc[i].y += t.y; acc[i].z += t.z; acc[i].w += t.w;
    }
  }
  float4* o = reinterpret_cast<float4*>(out + (size_t)c * (4 * kW4));
#pragma unroll
  for (int i = 0; i < kW4; ++i) o[i] = acc[i];
}

template <int kW4>
__global__ void k_splat_sum(long long n, const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
                            const float* __restrict__ seg_rec, float* __restrict__ out,
                            const PcgScalars* __restrict__ sc) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (sc != nullptr && sc->done)) return;
  splat_sum_body<kW4>(c, s_start, s_end, seg_rec, out);
}

__global__ void k_splat_sum_batch(const __grid_constant__ GaussBatch gb, const PcgScalars* __restrict__ sc) {
  const SubsetRefs& s = gb.s[blockIdx.y];
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s.act_off == nullptr || c >= s.n_splats || (sc != nullptr && sc[blockIdx.y].done)) return;
  splat_sum_body<3>(c, s.s_start, s.s_end, s.seg_ybar, s.ydot);
}

}  // namespace

cudaError_t launch_project(const float* params, int N, long long ld, const DevCam* cams, int V, int smooth,
                           SplatRec* rec, uint32_t* ntiles, uint2* rect, uint32_t* depth_key,
                           unsigned long long* tmask, cudaStream_t st) {
  const long long n = (long long)N * V;
  if (n == 0) return cudaSuccess;
  const int bs = 256;
  { k_project<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(params, N, ld, cams, V, smooth, rec, ntiles, rect,
                                                          depth_key, tmask); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_view_mask(const uint8_t* slot_active, int N, int V, unsigned long long* vmask,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  { k_view_mask<<<(N + 255) / 256, 256, 0, st>>>(slot_active, N, V, vmask); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_tangent(const float* params, int N, long long ld, const DevCam* cams, int V, int smooth,
                           const uint8_t* slot_active, const unsigned long long* vmask, const uint32_t* act_off,
                           const float* p, float* ydot, const float* z_beta, float* p_out, const PcgScalars* sc,
                           cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  { k_tangent<<<(N + kGPB - 1) / kGPB, 128, 0, st>>>(params, N, ld, cams, V, smooth, slot_active, vmask, act_off, p,
                                                     ydot, z_beta, p_out, sc); note_launch(); }
  return cudaGetLastError();
}

__global__ void k_active_count(const unsigned long long* __restrict__ vmask, int N, uint32_t* __restrict__ cnt) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < N) cnt[g] = (uint32_t)__popcll(vmask[g]);
}

__global__ void k_seg_compact_slot(const unsigned long long* __restrict__ vmask, int N,
                                   const uint32_t* __restrict__ act_off, const uint32_t* __restrict__ seg_slot,
                                   long long n_seg, SegRec* __restrict__ seg_rec, uint32_t* __restrict__ key) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_seg) return;
  const uint32_t slot = seg_slot[s];
  const int v = (int)(slot / (uint32_t)N);
  const int g = (int)(slot - (uint32_t)v * (uint32_t)N);
  const unsigned long long below = v > 0 ? (vmask[g] & ((1ull << v) - 1ull)) : 0ull;
  const uint32_t c = act_off[g] + (uint32_t)__popcll(below);
  seg_rec[s].slot = c;
  key[s] = c;
}

cudaError_t launch_compact_splats(const unsigned long long* vmask, int N, uint32_t* act_off, void* scan_temp,
                                  const uint32_t* seg_slot, long long n_seg, SegRec* seg_rec, uint32_t* key,
                                  cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  // counts in act_off[0..N), then an in-place-safe scan into act_off via a second buffer
  uint32_t* cnt = reinterpret_cast<uint32_t*>(scan_temp);
  { k_active_count<<<(N + 255) / 256, 256, 0, st>>>(vmask, N, cnt); note_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* tmp = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(cnt + N + 1) + 63) & ~uintptr_t(63));
  e = exclusive_scan_u32(cnt, act_off, N, tmp, st);   // act_off[N] = the total
  if (e != cudaSuccess || n_seg <= 0) return e;
  { k_seg_compact_slot<<<(unsigned)((n_seg + 255) / 256), 256, 0, st>>>(vmask, N, act_off, seg_slot, n_seg, seg_rec,
                                                                       key);
    note_launch(); }
  return cudaGetLastError();
}

int vjp_blocks(int N) { return std::max(1, std::min((N + kGPB - 1) / kGPB, kVjpBlocks)); }

cudaError_t launch_tangent_batch(const float* params, int N, long long ld, int smooth, const GaussBatch& gb,
                                 const float* p, long long vs, const float* z_beta, float* p_out,
                                 const PcgScalars* sc, cudaStream_t st) {
  if (N == 0 || gb.n <= 0) return cudaSuccess;
  { k_tangent_batch<<<dim3((N + kGPB - 1) / kGPB, gb.n), 128, 0, st>>>(params, N, ld, smooth, gb, p, vs, z_beta,
                                                                       p_out, sc); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_vjp_batch(const float* params, int N, long long ld, int smooth, const GaussBatch& gb,
                             float* g, long long vs, const float* p, const float* M, float lambda,
                             double* partials, const PcgScalars* sc, cudaStream_t st) {
  if (N == 0 || gb.n <= 0) return cudaSuccess;
  { k_vjp_batch<<<dim3(vjp_blocks(N), gb.n), 128, 0, st>>>(params, N, ld, smooth, gb, g, vs, p, M, lambda, partials,
                                                           sc); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_vjp(const float* params, int N, long long ld, const DevCam* cams, int V, int smooth,
                       const uint32_t* s_start, const uint32_t* s_end, const unsigned long long* vmask,
                       const uint32_t* act_off, const float* seg_ybar, const float* splat_ybar, float scale,
                       float* g, const float* p, const float* M, float lambda, double* partials,
                       const PcgScalars* sc, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  { k_vjp<<<vjp_blocks(N), 128, 0, st>>>(params, N, ld, cams, V, smooth, s_start, s_end, vmask, act_off, seg_ybar,
                                       splat_ybar, scale, g, p, M, lambda, partials, sc); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_diag(const float* params, int N, long long ld, const DevCam* cams, int V, int smooth,
                        const uint32_t* s_start, const uint32_t* s_end, const unsigned long long* vmask,
                        const uint32_t* act_off, const float* seg_q, const float* splat_q, float* diag,
                        cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  { k_diag<<<(N + kDiagThreads - 1) / kDiagThreads, kDiagThreads, 0, st>>>(params, N, ld, cams, V, smooth, s_start,
                                                                          s_end, vmask, act_off, seg_q, splat_q,
                                                                          diag); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_splat_sum(long long n_splats, const uint32_t* s_start, const uint32_t* s_end,
                             const float* seg_ybar, float* splat_ybar, const PcgScalars* sc, cudaStream_t st) {
  if (n_splats <= 0) return cudaSuccess;
  { k_splat_sum<3><<<(unsigned)((n_splats + 255) / 256), 256, 0, st>>>(n_splats, s_start, s_end, seg_ybar,
                                                                      splat_ybar, sc); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_splat_sum_q(long long n_splats, const uint32_t* s_start, const uint32_t* s_end, const float* seg_q,
                               float* splat_q, cudaStream_t st) {
  if (n_splats <= 0) return cudaSuccess;
  { k_splat_sum<kDiagBlock / 4><<<(unsigned)((n_splats + 127) / 128), 128, 0, st>>>(n_splats, s_start, s_end, seg_q,
                                                                                   splat_q, nullptr); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_splat_sum_batch(const GaussBatch& gb, const PcgScalars* sc, cudaStream_t st) {
  long long n = 0;
  for (int i = 0; i < gb.n; ++i) n = std::max(n, gb.s[i].act_off != nullptr ? gb.s[i].n_splats : 0ll);
  if (n <= 0 || gb.n <= 0) return cudaSuccess;
  { k_splat_sum_batch<<<dim3((unsigned)((n + 255) / 256), gb.n), 256, 0, st>>>(gb, sc); note_launch(); }
  return cudaGetLastError();
}

}  // namespace gslm
