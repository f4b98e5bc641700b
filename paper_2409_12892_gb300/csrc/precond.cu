// Learned diagonal preconditioner (include/gslm.h, gslm_precond_*). The paper
// uses the Jacobi preconditioner M^-1 of Algorithm 1; this per-Gaussian network
// scales it entry by entry, D_k = softplus(o_k) / clamp(M_k), and is trained on
// the relative PCG residual after K iterations of Algorithm 1 run with D.
//
// Network weights are one float32 vector: W1 (64 x 64, row = output), b1, W2,
// b2, W3 (59 x 64), b3. Parameter-space vectors use the [59][ld] layout of the
// rest of the library; feature arrays are [N][64] row-major.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace gslm;

namespace {

constexpr int kIn = 64, kHid = 64, kOut = 59;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid, kNW = kOffB3 + kOut;
static_assert(kNW == 12155, "weight count");
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kInvSqrt2Pi = 0.39894228040143268f;
constexpr int kVB = 256;   // vector kernels: block size

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * kInvSqrt2)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * kInvSqrt2)) + x * kInvSqrt2Pi * expf(-0.5f * x * x);
}
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid(float x) { return 1.f / (1.f + expf(-x)); }

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------------------- features
__global__ void k_features(const float* __restrict__ P, int N, long long ld, const float* __restrict__ M, int V,
                           const uint32_t* __restrict__ s_start, const uint32_t* __restrict__ s_end,
                           const uint32_t* __restrict__ s_list, const unsigned long long* __restrict__ seg_off,
                           const uint32_t* __restrict__ act_off, float* __restrict__ phi) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  float* f = phi + (size_t)g * kIn;
  for (int k = 0; k < kNP; ++k) f[k] = logf(M[k * ld + g] + 1e-12f);
  f[59] = P[3 * ld + g];
  f[60] = P[4 * ld + g];
  f[61] = P[5 * ld + g];
  f[62] = sigmoid(P[10 * ld + g]);
  unsigned long long entries = 0;
  if (act_off != nullptr) {
    // splats keyed by compact index: the Gaussian's segments are one run
    const uint32_t c0 = act_off[g], c1 = act_off[g + 1];
    if (c1 > c0)
      for (uint32_t j = s_start[c0]; j < s_end[c1 - 1]; ++j) {
        const uint32_t s = s_list[j];
        entries += seg_off[s + 1] - seg_off[s];
      }
  } else {
    for (int v = 0; v < V; ++v) {
      const long long slot = (long long)v * N + g;
      for (uint32_t j = s_start[slot]; j < s_end[slot]; ++j) {
        const uint32_t s = s_list[j];
        entries += seg_off[s + 1] - seg_off[s];
      }
    }
  }
  f[63] = log1pf((float)entries);
}

// Per-feature sums of x and x^2 (float64); 4 rows per 256-thread block.
__global__ void k_feature_sums(const float* __restrict__ phi, int N, double* __restrict__ sums) {
  const int f = threadIdx.x & 63, row0 = threadIdx.x >> 6;
  double s = 0.0, s2 = 0.0;
  for (long long g = (long long)blockIdx.x * 4 + row0; g < N; g += (long long)gridDim.x * 4) {
    const double x = phi[g * kIn + f];
    s += x;
    s2 += x * x;
  }
  atomicAdd(&sums[f], s);
  atomicAdd(&sums[64 + f], s2);
}

__global__ void k_feature_stats(const double* __restrict__ sums, int N, float* __restrict__ mu,
                                float* __restrict__ sd) {
  const int f = threadIdx.x;
  if (f >= kIn) return;
  const double m = sums[f] / N;
  const double var = fmax(sums[64 + f] / N - m * m, 0.0);
  mu[f] = (float)m;
  sd[f] = (float)fmax(sqrt(var), 1e-6);
}

// ---------------------------------------------------------------------------- network
// The network computes with bfloat16 weight matrices and float32 biases,
// activations and sums: W1, W2 and W3 (the float32 master copy that Adam
// updates) are rounded to bfloat16 (round to nearest even) as they are staged
// into shared memory, and the weight gradient is that of the rounded weights.
// The biases stay float32, so the initial network (W3 = 0, b3 = log(e - 1)) is
// exactly the Jacobi preconditioner.
__device__ __forceinline__ float bf16_weight(int i, float w) {
  const bool bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i >= kOffB3;
  return bias ? w : __bfloat162float(__float2bfloat16_rn(w));
}

// D = softplus(o) / clamp(M): one thread per Gaussian, weights in shared memory
// (every lane of a warp reads the same weight: a broadcast).
__global__ void __launch_bounds__(128) k_mlp_infer(const float* __restrict__ W, const float* __restrict__ mu,
                                                   const float* __restrict__ sd, const float* __restrict__ phi,
                                                   int N, long long ld, const float* __restrict__ M,
                                                   float* __restrict__ D) {
  extern __shared__ float sw[];
  float* smu = sw + kNW;
  float* srs = smu + kIn;
  for (int i = threadIdx.x; i < kNW; i += blockDim.x) sw[i] = bf16_weight(i, W[i]);
  if (threadIdx.x < kIn) {
    smu[threadIdx.x] = mu[threadIdx.x];
    srs[threadIdx.x] = 1.f / sd[threadIdx.x];
  }
  __syncthreads();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  float x[kIn], h[kHid];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = (phi[(size_t)g * kIn + i] - smu[i]) * srs[i];
#pragma unroll 2
  for (int o = 0; o < kHid; ++o) {
    float a = sw[kOffB1 + o];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = fmaf(sw[kOffW1 + o * kIn + i], x[i], a);
    h[o] = gelu(a);
  }
#pragma unroll 2
  for (int o = 0; o < kHid; ++o) {
    float a = sw[kOffB2 + o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) a = fmaf(sw[kOffW2 + o * kHid + i], h[i], a);
    x[o] = gelu(a);
  }
  for (int o = 0; o < kOut; ++o) {
    float a = sw[kOffB3 + o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) a = fmaf(sw[kOffW3 + o * kHid + i], x[i], a);
    D[o * ld + g] = softplus(a) / clamp_diag(M[o * ld + g]);
  }
}

// Weight gradient for an upstream dL/dD. Each block walks chunks of kChunk
// Gaussians: one thread per Gaussian reruns the forward pass and the backward
// pass and leaves its activations and pre-activation gradients in shared
// memory; then every thread adds the chunk's outer products to the weight
// gradients it owns (registers), flushed with one atomic each at the end.
constexpr int kChunk = 64;
constexpr int kRowPhi = 0, kRowH1 = kRowPhi + kIn, kRowH2 = kRowH1 + kHid, kRowDo = kRowH2 + kHid;
constexpr int kRowDa2 = kRowDo + kOut, kRowDa1 = kRowDa2 + kHid, kRow = kRowDa1 + kHid;   // 379, odd: no bank conflicts
constexpr int kGradThreads = 256;
constexpr int kOwn = (kNW + kGradThreads - 1) / kGradThreads;

__device__ __forceinline__ void grad_operands(int w, int& ga, int& gb) {
  // gradient of weight w = sum over the chunk of row[ga] * (gb < 0 ? 1 : row[gb])
  if (w < kOffB1) { ga = kRowDa1 + w / kIn; gb = kRowPhi + w % kIn; }
  else if (w < kOffW2) { ga = kRowDa1 + (w - kOffB1); gb = -1; }
  else if (w < kOffB2) { ga = kRowDa2 + (w - kOffW2) / kHid; gb = kRowH1 + (w - kOffW2) % kHid; }
  else if (w < kOffW3) { ga = kRowDa2 + (w - kOffB2); gb = -1; }
  else if (w < kOffB3) { ga = kRowDo + (w - kOffW3) / kHid; gb = kRowH2 + (w - kOffW3) % kHid; }
  else { ga = kRowDo + (w - kOffB3); gb = -1; }
}

__global__ void __launch_bounds__(kGradThreads) k_mlp_backward(
    const float* __restrict__ W, const float* __restrict__ mu, const float* __restrict__ sd,
    const float* __restrict__ phi, int N, long long ld, const float* __restrict__ M, const float* __restrict__ dD,
    float scale, float* __restrict__ grad) {
  extern __shared__ float smem[];
  float* sw = smem;
  float* act = sw + kNW;
  float* smu = act + kChunk * kRow;
  float* srs = smu + kIn;
  for (int i = threadIdx.x; i < kNW; i += blockDim.x) sw[i] = bf16_weight(i, W[i]);
  if (threadIdx.x < kIn) {
    smu[threadIdx.x] = mu[threadIdx.x];
    srs[threadIdx.x] = 1.f / sd[threadIdx.x];
  }
  __syncthreads();
  float acc[kOwn];
#pragma unroll
  for (int j = 0; j < kOwn; ++j) acc[j] = 0.f;
  const long long n_chunks = ((long long)N + kChunk - 1) / kChunk;
  for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const int t = threadIdx.x;
    if (t < kChunk) {
      float* r = act + t * kRow;
      const long long g = c * kChunk + t;
      if (g < N) {
        for (int i = 0; i < kIn; ++i) r[kRowPhi + i] = (phi[g * kIn + i] - smu[i]) * srs[i];
        for (int o = 0; o < kHid; ++o) {
          float a = sw[kOffB1 + o];
          for (int i = 0; i < kIn; ++i) a = fmaf(sw[kOffW1 + o * kIn + i], r[kRowPhi + i], a);
          r[kRowH1 + o] = gelu(a);
          r[kRowDa1 + o] = gelu_grad(a);        // times dL/dh1 below
        }
        for (int o = 0; o < kHid; ++o) {
          float a = sw[kOffB2 + o];
          for (int i = 0; i < kHid; ++i) a = fmaf(sw[kOffW2 + o * kHid + i], r[kRowH1 + i], a);
          r[kRowH2 + o] = gelu(a);
          r[kRowDa2 + o] = gelu_grad(a);        // times dL/dh2 below
        }
        for (int o = 0; o < kOut; ++o) {
          float a = sw[kOffB3 + o];
          for (int i = 0; i < kHid; ++i) a = fmaf(sw[kOffW3 + o * kHid + i], r[kRowH2 + i], a);
          // D = softplus(a) / clamp(M)  =>  dL/da = dL/dD sigmoid(a) / clamp(M)
          r[kRowDo + o] = scale * dD[o * ld + g] * sigmoid(a) / clamp_diag(M[o * ld + g]);
        }
        for (int i = 0; i < kHid; ++i) {
          float s = 0.f;
          for (int o = 0; o < kOut; ++o) s = fmaf(r[kRowDo + o], sw[kOffW3 + o * kHid + i], s);
          r[kRowDa2 + i] *= s;
        }
        for (int i = 0; i < kHid; ++i) {
          float s = 0.f;
          for (int o = 0; o < kHid; ++o) s = fmaf(r[kRowDa2 + o], sw[kOffW2 + o * kHid + i], s);
          r[kRowDa1 + i] *= s;
        }
      } else {
        for (int i = 0; i < kRow; ++i) r[i] = 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kOwn; ++j) {
      const int w = threadIdx.x + j * kGradThreads;
      if (w < kNW) {
        int ga, gb;
        grad_operands(w, ga, gb);
        float s = 0.f;
        if (gb >= 0) {
          for (int n = 0; n < kChunk; ++n) s = fmaf(act[n * kRow + ga], act[n * kRow + gb], s);
        } else {
          for (int n = 0; n < kChunk; ++n) s += act[n * kRow + ga];
        }
        acc[j] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kOwn; ++j) {
    const int w = threadIdx.x + j * kGradThreads;
    if (w < kNW) atomicAdd(&grad[w], acc[j]);
  }
}

__global__ void k_adam(float* __restrict__ W, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float bc1, float bc2, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNW) return;
  const float g = grad[i];
  const float mi = 0.9f * m[i] + 0.1f * g;
  const float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  W[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// ---------------------------------------------------------------------------- unrolled PCG
// Scalars of one unrolled run (float64, device): rho[0..K], pg[0..K-1],
// rhobar[0..K], then single working slots.
struct Unrolled {
  int K;
  double* s;
  __host__ __device__ double* rho() const { return s; }
  __host__ __device__ double* pg() const { return s + (K + 1); }
  __host__ __device__ double* rhobar() const { return s + (2 * K + 1); }
  __host__ __device__ double* betabar() const { return s + (3 * K + 2); }
  __host__ __device__ double* dotv() const { return s + (3 * K + 3); }
  __host__ __device__ double* pgbar() const { return s + (3 * K + 4); }
  __host__ __device__ double* rr() const { return s + (3 * K + 5); }
  __host__ __device__ double* bb() const { return s + (3 * K + 6); }
  static int count(int K) { return 3 * K + 7; }
};

// Grid-stride loop over the Gaussians of a [59][ld] vector; `o` is the element offset.
#define VEC_LOOP(N, ld, ...)                                                   \
  for (int g = blockIdx.x * kVB + threadIdx.x; g < (N); g += gridDim.x * kVB) { \
    for (int k = 0; k < kNP; ++k) {                                            \
      const long long o = (long long)k * (ld) + g;                            \
      __VA_ARGS__                                                              \
    }                                                                          \
  }

#define WRITE_PARTIAL(acc)                             \
  {                                                    \
    __shared__ double red[kVB / 32];                   \
    const double s_ = block_sum((acc), red);           \
    if (threadIdx.x == 0) partials[blockIdx.x] = s_;   \
  }

__global__ void k_dot(int N, long long ld, const float* __restrict__ a, const float* __restrict__ b,
                      double* __restrict__ partials) {
  double acc = 0.0;
  VEC_LOOP(N, ld, acc += (double)a[o] * (double)b[o];)
  WRITE_PARTIAL(acc)
}

__global__ void k_mul(int N, long long ld, const float* __restrict__ a, const float* __restrict__ b,
                      float* __restrict__ out) {
  VEC_LOOP(N, ld, out[o] = a[o] * b[o];)
}

// r0 = b - A x0; z0 = D r0; p0 = z0; partial r0.z0
__global__ void k_u_r0(int N, long long ld, const float* __restrict__ b, const float* __restrict__ Ax,
                       const float* __restrict__ D, float* __restrict__ r, float* __restrict__ p,
                       double* __restrict__ partials) {
  double acc = 0.0;
  VEC_LOOP(N, ld, {
    const float rv = b[o] - Ax[o];
    const float z = D[o] * rv;
    r[o] = rv;
    p[o] = z;
    acc += (double)rv * (double)z;
  })
  WRITE_PARTIAL(acc)
}

// r_{i+1} = r_i - alpha_i g_i, alpha_i = rho_i / pg_i; partial r_{i+1}.(D r_{i+1})
__global__ void k_u_r(int N, long long ld, Unrolled u, int i, const float* __restrict__ r0,
                      const float* __restrict__ gi, const float* __restrict__ D, float* __restrict__ r1,
                      double* __restrict__ partials) {
  const float alpha = (float)(u.rho()[i] / u.pg()[i]);
  double acc = 0.0;
  VEC_LOOP(N, ld, {
    const float rv = r0[o] - alpha * gi[o];
    r1[o] = rv;
    acc += (double)rv * (double)(D[o] * rv);
  })
  WRITE_PARTIAL(acc)
}

// p_{i+1} = D r_{i+1} + beta_i p_i, beta_i = rho_{i+1} / rho_i
__global__ void k_u_p(int N, long long ld, Unrolled u, int i, const float* __restrict__ r1,
                      const float* __restrict__ D, const float* __restrict__ p0, float* __restrict__ p1) {
  const float beta = (float)(u.rho()[i + 1] / u.rho()[i]);
  VEC_LOOP(N, ld, p1[o] = D[o] * r1[o] + beta * p0[o];)
}

// rbar = dL/dr_K = r_K / ||r_K||^2, pbar = 0, dbar = 0
__global__ void k_u_rev_init(int N, long long ld, Unrolled u, const float* __restrict__ rK, float* __restrict__ rbar,
                             float* __restrict__ pbar, float* __restrict__ dbar) {
  const float inv = (float)(1.0 / *u.rr());
  VEC_LOOP(N, ld, {
    rbar[o] = rK[o] * inv;
    pbar[o] = 0.f;
    dbar[o] = 0.f;
  })
}

// beta_i = rho_{i+1} / rho_i: rhobar_{i+1} += betabar / rho_i, rhobar_i -= betabar rho_{i+1} / rho_i^2
__global__ void k_u_scal_beta(Unrolled u, int i) {
  const double bb = *u.betabar(), ri = u.rho()[i], r1 = u.rho()[i + 1];
  u.rhobar()[i + 1] += bb / ri;
  u.rhobar()[i] -= bb * r1 / (ri * ri);
}

// Reverse of z_{i+1} = D r_{i+1}, rho_{i+1} = r_{i+1}.z_{i+1} and of the z part
// of p_{i+1} = z_{i+1} + beta_i p_i; then pbar <- beta_i pbar (its p_i part).
// Partial rbar.g_i for alphabar.
__global__ void k_u_rev_a(int N, long long ld, Unrolled u, int i, const float* __restrict__ r1,
                          const float* __restrict__ gi, const float* __restrict__ D, float* __restrict__ rbar,
                          float* __restrict__ pbar, float* __restrict__ dbar, double* __restrict__ partials) {
  const float rb1 = (float)u.rhobar()[i + 1];
  const float beta = (float)(u.rho()[i + 1] / u.rho()[i]);
  double acc = 0.0;
  VEC_LOOP(N, ld, {
    const float rv = r1[o], d = D[o], pb = pbar[o];
    const float zb = pb + rb1 * rv;
    const float rbv = rbar[o] + rb1 * (d * rv) + d * zb;
    rbar[o] = rbv;
    dbar[o] += rv * zb;
    pbar[o] = beta * pb;
    acc += (double)rbv * (double)gi[o];
  })
  WRITE_PARTIAL(acc)
}

// alpha_i = rho_i / pg_i with alphabar = -rbar.g_i
__global__ void k_u_scal_alpha(Unrolled u, int i) {
  const double ab = -*u.dotv(), ri = u.rho()[i], pg = u.pg()[i];
  u.rhobar()[i] += ab / pg;
  *u.pgbar() = -ab * ri / (pg * pg);
}

// gbar = -alpha_i rbar + pgbar p_i; pbar += pgbar g_i
__global__ void k_u_rev_b(int N, long long ld, Unrolled u, int i, const float* __restrict__ rbar,
                          const float* __restrict__ pi, const float* __restrict__ gi, float* __restrict__ gbar,
                          float* __restrict__ pbar) {
  const float alpha = (float)(u.rho()[i] / u.pg()[i]);
  const float pgb = (float)*u.pgbar();
  VEC_LOOP(N, ld, {
    gbar[o] = -alpha * rbar[o] + pgb * pi[o];
    pbar[o] += pgb * gi[o];
  })
}

__global__ void k_add(int N, long long ld, const float* __restrict__ a, float* __restrict__ out) {
  VEC_LOOP(N, ld, out[o] += a[o];)
}

// Reverse of p0 = z0, rho0 = r0.z0, z0 = D r0 (rbar becomes dL/dr0)
__global__ void k_u_rev_c(int N, long long ld, Unrolled u, const float* __restrict__ r0, const float* __restrict__ D,
                          const float* __restrict__ pbar, float* __restrict__ rbar, float* __restrict__ dbar) {
  const float rb0 = (float)u.rhobar()[0];
  VEC_LOOP(N, ld, {
    const float rv = r0[o], d = D[o];
    const float zb = pbar[o] + rb0 * rv;
    rbar[o] = rbar[o] + rb0 * (d * rv) + d * zb;
    dbar[o] += rv * zb;
  })
}

// Reverse of r0 = b - A x0 and x0 = D b: dbar -= b (A rbar)
__global__ void k_u_rev_d(int N, long long ld, const float* __restrict__ b, const float* __restrict__ Arbar,
                          float* __restrict__ dbar) {
  VEC_LOOP(N, ld, dbar[o] -= b[o] * Arbar[o];)
}

int vec_blocks(int N) { return std::max(1, std::min((N + kVB - 1) / kVB, 2432)); }

// SplitMix64 (Steele, Lea and Flood, 2014) and the Box-Muller transform, for
// the default initial weights.
struct SplitMix64 {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)((next() >> 11) + 1) * (1.0 / 9007199254740992.0); }   // (0, 1]
  double normal() {
    const double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

}  // namespace

struct gslm_precond {
  gslm_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  Buf W, mu, sd, m, v, grad, sums, phi, D, dD;
  int t = 0;
};

namespace {

gslm_status pfail(gslm_ctx* ctx, gslm_status s, const std::string& msg) {
  set_context_error(ctx, msg.c_str());
  return s;
}

#define PCK(expr)                                                                              \
  do {                                                                                         \
    const cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                                   \
      cudaGetLastError();                                                                      \
      return pfail(ctx, e_ == cudaErrorMemoryAllocation ? GSLM_E_OOM : GSLM_E_CUDA,            \
                   std::string(#expr) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                          \
  } while (0)

#define PCKS(expr)                        \
  do {                                    \
    const gslm_status s_ = (expr);        \
    if (s_ != GSLM_OK) return s_;         \
  } while (0)

#define LAUNCH(...)      \
  do {                   \
    __VA_ARGS__;         \
    note_launch();       \
  } while (0)

gslm_status features(gslm_ctx* ctx, const gslm_cache* cache, const float* diag, float* phi) {
  CacheParts cp;
  if (!cache_parts(cache, &cp) || diag == nullptr || phi == nullptr)
    return pfail(ctx, GSLM_E_INVALID, "precond_features: null argument");
  const cudaStream_t st = context_stream(ctx);
  if (cp.N <= 0) return GSLM_OK;
  LAUNCH((k_features<<<(cp.N + 255) / 256, 256, 0, st>>>(cp.params, cp.N, cp.ld, diag, cp.V, cp.view.slot_seg_start,
                                                          cp.view.slot_seg_end, cp.view.slot_seg_list,
                                                          cp.view.seg_entry_off,
                                                          cp.view.vmask != nullptr ? cp.view.act_off : nullptr,
                                                          phi)));
  PCK(cudaGetLastError());
  return GSLM_OK;
}

gslm_status infer(gslm_precond* pc, const float* phi, int N, long long ld, const float* diag, float* D) {
  gslm_ctx* ctx = pc->ctx;
  if (N <= 0) return GSLM_OK;
  const size_t smem = sizeof(float) * (kNW + 2 * kIn);
  PCK(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LAUNCH((k_mlp_infer<<<(N + 127) / 128, 128, smem, pc->st>>>(pc->W.as<float>(), pc->mu.as<float>(),
                                                               pc->sd.as<float>(), phi, N, ld, diag, D)));
  PCK(cudaGetLastError());
  return GSLM_OK;
}

gslm_status backward(gslm_precond* pc, const float* phi, int N, long long ld, const float* diag, const float* dD,
                     float scale, float* grad) {
  gslm_ctx* ctx = pc->ctx;
  if (N <= 0) return GSLM_OK;
  const size_t smem = sizeof(float) * (kNW + kChunk * kRow + 2 * kIn);
  PCK(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int n_chunks = (N + kChunk - 1) / kChunk;
  const int grid = std::max(1, std::min(n_chunks, 152 * 4));
  LAUNCH((k_mlp_backward<<<grid, kGradThreads, smem, pc->st>>>(pc->W.as<float>(), pc->mu.as<float>(),
                                                                pc->sd.as<float>(), phi, N, ld, diag, dD, scale,
                                                                grad)));
  PCK(cudaGetLastError());
  return GSLM_OK;
}

gslm_status reduce_dot(gslm_ctx* ctx, int N, long long ld, const float* a, const float* b, double* partials,
                       double* out, cudaStream_t st) {
  const int nb = vec_blocks(N);
  LAUNCH((k_dot<<<nb, kVB, 0, st>>>(N, ld, a, b, partials)));
  PCK(launch_reduce_partials(partials, nb, out, st));
  return GSLM_OK;
}

// The unrolled loss and dL/dD (include/gslm.h); dD may be null.
gslm_status unrolled(gslm_ctx* ctx, const gslm_cache* cache, const float* b, const float* diag, float lambda,
                     const float* D, int K, double* loss, float* dD) {
  CacheParts cp;
  if (!cache_parts(cache, &cp) || b == nullptr || diag == nullptr || D == nullptr || K < 1 || K > 4096)
    return pfail(ctx, GSLM_E_INVALID, "precond_unrolled_grad: null argument or K outside [1, 4096]");
  const int N = cp.N;
  const long long ld = cp.ld;
  const cudaStream_t st = context_stream(ctx);
  const size_t vb = sizeof(float) * kNP * (size_t)ld;
  std::vector<Buf> r(K + 1), p(K), g(K);
  for (auto& x : r) PCK(x.alloc(vb, st));
  for (auto& x : p) PCK(x.alloc(vb, st));
  for (auto& x : g) PCK(x.alloc(vb, st));
  Buf tmp, rbar, pbar, gbar, dbar, scal, partials;
  PCK(tmp.alloc(vb, st));
  PCK(rbar.alloc(vb, st));
  PCK(pbar.alloc(vb, st));
  PCK(gbar.alloc(vb, st));
  PCK(dbar.alloc(vb, st));
  PCK(scal.alloc(sizeof(double) * Unrolled::count(K), st));
  PCK(partials.alloc(sizeof(double) * vec_blocks(N), st));
  PCK(cudaMemsetAsync(scal.p, 0, sizeof(double) * Unrolled::count(K), st));
  // pad entries (ld > N) are never read by the vector kernels but apply_A reads whole rows
  PCK(cudaMemsetAsync(tmp.p, 0, vb, st));
  PCK(cudaMemsetAsync(gbar.p, 0, vb, st));
  PCK(cudaMemsetAsync(rbar.p, 0, vb, st));
  for (auto& x : p) PCK(cudaMemsetAsync(x.p, 0, vb, st));
  const Unrolled u{K, scal.as<double>()};
  double* part = partials.as<double>();
  const int nb = vec_blocks(N);
  auto F = [](Buf& x) { return x.as<float>(); };
  // forward: x0 = D b, r0 = b - A x0, z0 = D r0, p0 = z0
  LAUNCH((k_mul<<<nb, kVB, 0, st>>>(N, ld, D, b, F(tmp))));
  PCKS(apply_A(ctx, cache, F(tmp), diag, lambda, F(gbar)));
  LAUNCH((k_u_r0<<<nb, kVB, 0, st>>>(N, ld, b, F(gbar), D, F(r[0]), F(p[0]), part)));
  PCK(launch_reduce_partials(part, nb, &u.rho()[0], st));
  PCKS(reduce_dot(ctx, N, ld, b, b, part, u.bb(), st));
  for (int i = 0; i < K; ++i) {
    PCKS(apply_A(ctx, cache, F(p[i]), diag, lambda, F(g[i])));
    PCKS(reduce_dot(ctx, N, ld, F(p[i]), F(g[i]), part, &u.pg()[i], st));
    LAUNCH((k_u_r<<<nb, kVB, 0, st>>>(N, ld, u, i, F(r[i]), F(g[i]), D, F(r[i + 1]), part)));
    PCK(launch_reduce_partials(part, nb, &u.rho()[i + 1], st));
    if (i + 1 < K) LAUNCH((k_u_p<<<nb, kVB, 0, st>>>(N, ld, u, i, F(r[i + 1]), D, F(p[i]), F(p[i + 1]))));
  }
  PCKS(reduce_dot(ctx, N, ld, F(r[K]), F(r[K]), part, u.rr(), st));
  std::vector<double> h(Unrolled::count(K));
  PCK(cudaMemcpyAsync(h.data(), scal.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  PCK(cudaStreamSynchronize(st));
  const Unrolled hu{K, h.data()};
  for (int i = 0; i <= K; ++i) {
    const bool rho_ok = std::isfinite(hu.rho()[i]) && hu.rho()[i] > 0.0;
    const bool pg_ok = i == K || (std::isfinite(hu.pg()[i]) && hu.pg()[i] > 0.0);
    if (!rho_ok || !pg_ok)
      return pfail(ctx, GSLM_E_NUMERIC, "precond_unrolled_grad: r.z or p.Ap not positive and finite");
  }
  if (!(*hu.rr() > 0.0) || !(*hu.bb() > 0.0))
    return pfail(ctx, GSLM_E_NUMERIC, "precond_unrolled_grad: zero residual or right-hand side");
  if (loss != nullptr) *loss = 0.5 * std::log(*hu.rr() / *hu.bb());
  if (dD == nullptr) return GSLM_OK;
  // reverse
  LAUNCH((k_u_rev_init<<<nb, kVB, 0, st>>>(N, ld, u, F(r[K]), F(rbar), F(pbar), F(dbar))));
  for (int i = K - 1; i >= 0; --i) {
    PCKS(reduce_dot(ctx, N, ld, F(pbar), F(p[i]), part, u.betabar(), st));
    LAUNCH((k_u_scal_beta<<<1, 1, 0, st>>>(u, i)));
    LAUNCH((k_u_rev_a<<<nb, kVB, 0, st>>>(N, ld, u, i, F(r[i + 1]), F(g[i]), D, F(rbar), F(pbar), F(dbar), part)));
    PCK(launch_reduce_partials(part, nb, u.dotv(), st));
    LAUNCH((k_u_scal_alpha<<<1, 1, 0, st>>>(u, i)));
    LAUNCH((k_u_rev_b<<<nb, kVB, 0, st>>>(N, ld, u, i, F(rbar), F(p[i]), F(g[i]), F(gbar), F(pbar))));
    PCKS(apply_A(ctx, cache, F(gbar), diag, lambda, F(tmp)));
    LAUNCH((k_add<<<nb, kVB, 0, st>>>(N, ld, F(tmp), F(pbar))));
  }
  LAUNCH((k_u_rev_c<<<nb, kVB, 0, st>>>(N, ld, u, F(r[0]), D, F(pbar), F(rbar), F(dbar))));
  PCKS(apply_A(ctx, cache, F(rbar), diag, lambda, F(tmp)));
  LAUNCH((k_u_rev_d<<<nb, kVB, 0, st>>>(N, ld, b, F(tmp), F(dbar))));
  PCK(cudaGetLastError());
  PCK(cudaMemcpyAsync(dD, dbar.p, vb, cudaMemcpyDeviceToDevice, st));
  PCK(cudaStreamSynchronize(st));
  return GSLM_OK;
}

}  // namespace

namespace gslm {

gslm_status precond_for_cache(gslm_precond* pc, gslm_ctx* ctx, const gslm_cache* c, const float* M, float* D) {
  CacheParts cp;
  if (pc == nullptr || !cache_parts(c, &cp)) return pfail(ctx, GSLM_E_INVALID, "precond: null argument");
  PCK(pc->phi.ensure(sizeof(float) * kIn * (size_t)std::max(cp.N, 1), context_stream(ctx)));
  PCKS(features(ctx, c, M, pc->phi.as<float>()));
  return infer(pc, pc->phi.as<float>(), cp.N, cp.ld, M, D);
}

}  // namespace gslm

extern "C" {

int32_t gslm_precond_weight_count(void) { return kNW; }

gslm_status gslm_precond_create(gslm_ctx* ctx, const float* weights, const float* mean, const float* std_,
                                uint64_t seed, gslm_precond** out) {
  if (ctx == nullptr || out == nullptr) return GSLM_E_INVALID;
  *out = nullptr;
  auto* pc = new gslm_precond();
  pc->ctx = ctx;
  pc->st = context_stream(ctx);
  const cudaStream_t st = pc->st;
  auto bad = [&](cudaError_t e) {
    delete pc;
    cudaGetLastError();
    return pfail(ctx, e == cudaErrorMemoryAllocation ? GSLM_E_OOM : GSLM_E_CUDA,
                 std::string("precond_create: ") + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = pc->W.alloc(sizeof(float) * kNW, st)) != cudaSuccess) return bad(e);
  if ((e = pc->m.alloc(sizeof(float) * kNW, st)) != cudaSuccess) return bad(e);
  if ((e = pc->v.alloc(sizeof(float) * kNW, st)) != cudaSuccess) return bad(e);
  if ((e = pc->grad.alloc(sizeof(float) * kNW, st)) != cudaSuccess) return bad(e);
  if ((e = pc->mu.alloc(sizeof(float) * kIn, st)) != cudaSuccess) return bad(e);
  if ((e = pc->sd.alloc(sizeof(float) * kIn, st)) != cudaSuccess) return bad(e);
  if ((e = pc->sums.alloc(sizeof(double) * 2 * kIn, st)) != cudaSuccess) return bad(e);
  std::vector<float> w(kNW, 0.f), mu(kIn, 0.f), sd(kIn, 1.f);
  if (weights != nullptr) {
    std::memcpy(w.data(), weights, sizeof(float) * kNW);
  } else {
    SplitMix64 rng{seed};
    for (int i = 0; i < kHid * kIn; ++i) w[kOffW1 + i] = (float)(rng.normal() * 0.0625);   // 0.5 / sqrt(64)
    for (int i = 0; i < kHid * kHid; ++i) w[kOffW2 + i] = (float)(rng.normal() * 0.0625);
    for (int i = 0; i < kOut; ++i) w[kOffB3 + i] = (float)std::log(std::exp(1.0) - 1.0);   // softplus = 1
  }
  if (mean != nullptr) std::memcpy(mu.data(), mean, sizeof(float) * kIn);
  if (std_ != nullptr) std::memcpy(sd.data(), std_, sizeof(float) * kIn);
  if ((e = cudaMemcpyAsync(pc->W.p, w.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(pc->mu.p, mu.data(), sizeof(float) * kIn, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(pc->sd.p, sd.data(), sizeof(float) * kIn, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(pc->m.p, 0, sizeof(float) * kNW, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(pc->v.p, 0, sizeof(float) * kNW, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(pc->grad.p, 0, sizeof(float) * kNW, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return bad(e);
  *out = pc;
  return GSLM_OK;
}

void gslm_precond_free(gslm_precond* pc) { delete pc; }

gslm_status gslm_precond_get(const gslm_precond* pc, float* weights, float* mean, float* std_) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  if (weights != nullptr)
    PCK(cudaMemcpyAsync(weights, pc->W.p, sizeof(float) * kNW, cudaMemcpyDeviceToHost, pc->st));
  if (mean != nullptr) PCK(cudaMemcpyAsync(mean, pc->mu.p, sizeof(float) * kIn, cudaMemcpyDeviceToHost, pc->st));
  if (std_ != nullptr) PCK(cudaMemcpyAsync(std_, pc->sd.p, sizeof(float) * kIn, cudaMemcpyDeviceToHost, pc->st));
  PCK(cudaStreamSynchronize(pc->st));
  return GSLM_OK;
}

gslm_status gslm_precond_set(gslm_precond* pc, const float* weights, const float* mean, const float* std_) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  if (weights != nullptr)
    PCK(cudaMemcpyAsync(pc->W.p, weights, sizeof(float) * kNW, cudaMemcpyHostToDevice, pc->st));
  if (mean != nullptr) PCK(cudaMemcpyAsync(pc->mu.p, mean, sizeof(float) * kIn, cudaMemcpyHostToDevice, pc->st));
  if (std_ != nullptr) PCK(cudaMemcpyAsync(pc->sd.p, std_, sizeof(float) * kIn, cudaMemcpyHostToDevice, pc->st));
  PCK(cudaStreamSynchronize(pc->st));   // the host arrays may go away after return
  return GSLM_OK;
}

gslm_status gslm_precond_features(gslm_ctx* ctx, const gslm_cache* cache, const float* diag, float* phi) {
  if (ctx == nullptr) return GSLM_E_INVALID;
  return features(ctx, cache, diag, phi);
}

gslm_status gslm_precond_fit_standardizer(gslm_precond* pc, const float* phi, int64_t N) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  if (phi == nullptr || N <= 0 || N > 0x7fffffff)
    return pfail(ctx, GSLM_E_INVALID, "precond_fit_standardizer: bad argument");
  PCK(cudaMemsetAsync(pc->sums.p, 0, sizeof(double) * 2 * kIn, pc->st));
  LAUNCH((k_feature_sums<<<1024, 256, 0, pc->st>>>(phi, (int)N, pc->sums.as<double>())));
  LAUNCH((k_feature_stats<<<1, kIn, 0, pc->st>>>(pc->sums.as<double>(), (int)N, pc->mu.as<float>(),
                                                  pc->sd.as<float>())));
  PCK(cudaGetLastError());
  PCK(cudaStreamSynchronize(pc->st));
  return GSLM_OK;
}

gslm_status gslm_precond_apply(gslm_precond* pc, const float* phi, int64_t N, int64_t ld, const float* diag,
                               float* D) {
  if (pc == nullptr) return GSLM_E_INVALID;
  if (phi == nullptr || diag == nullptr || D == nullptr || N < 0 || N > 0x7fffffff || ld < N)
    return pfail(pc->ctx, GSLM_E_INVALID, "precond_apply: bad argument");
  return infer(pc, phi, (int)N, ld, diag, D);
}

gslm_status gslm_precond_backward(gslm_precond* pc, const float* phi, int64_t N, int64_t ld, const float* diag,
                                  const float* dD, float* grad, int32_t accumulate) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  if (phi == nullptr || diag == nullptr || dD == nullptr || grad == nullptr || N < 0 || N > 0x7fffffff || ld < N)
    return pfail(ctx, GSLM_E_INVALID, "precond_backward: bad argument");
  if (!accumulate) PCK(cudaMemsetAsync(grad, 0, sizeof(float) * kNW, pc->st));
  return backward(pc, phi, (int)N, ld, diag, dD, 1.f, grad);
}

gslm_status gslm_precond_unrolled_grad(gslm_ctx* ctx, const gslm_cache* cache, const float* b, const float* diag,
                                       float lambda, const float* D, int32_t K, double* loss, float* dD) {
  if (ctx == nullptr) return GSLM_E_INVALID;
  return unrolled(ctx, cache, b, diag, lambda, D, K, loss, dD);
}

gslm_status gslm_precond_accumulate(gslm_precond* pc, const gslm_cache* cache, const float* phi, const float* b,
                                    const float* diag, float lambda, int32_t K, float weight, double* loss) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  CacheParts cp;
  if (!cache_parts(cache, &cp) || phi == nullptr)
    return pfail(ctx, GSLM_E_INVALID, "precond_accumulate: null argument");
  const size_t vb = sizeof(float) * kNP * (size_t)cp.ld;
  PCK(pc->D.ensure(vb, pc->st));
  PCK(pc->dD.ensure(vb, pc->st));
  PCK(cudaMemsetAsync(pc->D.p, 0, vb, pc->st));
  PCKS(infer(pc, phi, cp.N, cp.ld, diag, pc->D.as<float>()));
  PCKS(unrolled(ctx, cache, b, diag, lambda, pc->D.as<float>(), K, loss, pc->dD.as<float>()));
  return backward(pc, phi, cp.N, cp.ld, diag, pc->dD.as<float>(), weight, pc->grad.as<float>());
}

gslm_status gslm_precond_adam(gslm_precond* pc, float lr) {
  if (pc == nullptr) return GSLM_E_INVALID;
  gslm_ctx* ctx = pc->ctx;
  pc->t += 1;
  const float bc1 = (float)(1.0 - std::pow(0.9, pc->t)), bc2 = (float)(1.0 - std::pow(0.999, pc->t));
  LAUNCH((k_adam<<<(kNW + 255) / 256, 256, 0, pc->st>>>(pc->W.as<float>(), pc->grad.as<float>(), pc->m.as<float>(),
                                                         pc->v.as<float>(), bc1, bc2, lr)));
  PCK(cudaGetLastError());
  PCK(cudaMemsetAsync(pc->grad.p, 0, sizeof(float) * kNW, pc->st));
  return GSLM_OK;
}

}  // extern "C"
