// Vector operations of Algorithm 1 (Sec. 3.3; the paper runs these in
// PyTorch), the subset weighted mean (Eq. combine-pcg) and small helpers.
//
// Vectors are [59][ld] float32 (ld a multiple of 4, rows 16-byte aligned).
// Dot products sum a thread's terms of up to eight rows in float32 and those
// sums in float64 (float64 arithmetic runs at a small fraction of the float32
// rate on this GPU, so it is not spent per element): each block writes one
// partial, and a one-block kernel reduces the partials in a
// fixed order and updates the device-side scalars (alpha, beta, the break
// test), so a whole solve runs without host synchronisation.
#include <algorithm>

#include "internal.cuh"

namespace gslm {
namespace {

constexpr int kBS = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// The vector kernels run a bounded grid (at most kVecBlocks blocks), so each
// block writes one float64 partial and the scalar kernel reduces at most
// kVecBlocks of them.
constexpr int kVecBlocks = 2432;   // 16 blocks of 256 threads per SM on 152 SMs

// Batched launches: blockIdx.y is the subset; its vectors sit at offset
// blockIdx.y * vs and its partials at blockIdx.y * gridDim.x (times 2 for the
// update kernel). The preconditioner M^-1 of Algorithm 1 is not stored: it is
// the given diagonal D where subset y has one (bit y of d_mask), else the
// inverse of the bounded Jacobi diagonal, computed where it is used.
__device__ __forceinline__ const float* subset_D(const float* D, unsigned d_mask, long long off) {
  return (D != nullptr && ((d_mask >> blockIdx.y) & 1u)) ? D + off : nullptr;
}

// The vector kernels walk the 59 rows in the outer loop and, inside a row,
// one float4 (four Gaussians) per thread, so the resident warps stream through
// one or two rows at a time with 16-byte accesses. ld is a multiple of 4: a
// row starts on a 16-byte boundary and its last float4 may hold padding
// columns (i >= N), which are read but neither written nor summed. f(o, nv)
// gets the element offset o of the float4 and its nv valid lanes; after every
// eighth row and the last, flush() moves the float32 partial sums to float64.
template <class F, class Flush>
__device__ __forceinline__ void for_each4(int N, long long ld, F&& f, Flush&& flush) {
  const int nq = (N + 3) >> 2;
  const int stride = gridDim.x * kBS;
#pragma unroll 2
  for (int k = 0; k < kNP; ++k) {
    const long long row = (long long)k * ld;
    for (int c = blockIdx.x * kBS + threadIdx.x; c < nq; c += stride) f(row + 4ll * c, min(4, N - 4 * c));
    if ((k & 7) == 7 || k == kNP - 1) flush();
  }
}

__device__ __forceinline__ float4 ld4(const float* __restrict__ a, long long o) {
  return *reinterpret_cast<const float4*>(a + o);
}
__device__ __forceinline__ void st4(float* __restrict__ a, long long o, float4 v, int nv) {
  if (nv == 4) {
    *reinterpret_cast<float4*>(a + o) = v;
  } else {
    a[o] = v.x;
    if (nv > 1) a[o + 1] = v.y;
    if (nv > 2) a[o + 2] = v.z;
  }
}
// sum of the first nv lanes of a * b
__device__ __forceinline__ float dot4(float4 a, float4 b, int nv) {
  float s = a.x * b.x;
  if (nv > 1) s = fmaf(a.y, b.y, s);
  if (nv > 2) s = fmaf(a.z, b.z, s);
  if (nv > 3) s = fmaf(a.w, b.w, s);
  return s;
}
__device__ __forceinline__ float4 minv4(const float* __restrict__ D, const float* __restrict__ M, long long o) {
  if (D != nullptr) return ld4(D, o);
  const float4 m = ld4(M, o);
  return make_float4(1.f / clamp_diag(m.x), 1.f / clamp_diag(m.y), 1.f / clamp_diag(m.z), 1.f / clamp_diag(m.w));
}

__global__ void k_pcg_init(int N, long long ld, long long vs, const float* __restrict__ b,
                           const float* __restrict__ M, const float* __restrict__ D, unsigned d_mask,
                           float* __restrict__ x, double* __restrict__ partials) {
  __shared__ double red[kBS / 32];
  {
    const long long off = (long long)blockIdx.y * vs;
    b += off;
    M += off;
    D = subset_D(D, d_mask, off);
    x += off;
    partials += (size_t)blockIdx.y * gridDim.x;
  }
  double bb = 0.0;
  float bf = 0.f;
  for_each4(
      N, ld,
      [&](long long o, int nv) {
        const float4 bv = ld4(b, o), mi = minv4(D, M, o);
        st4(x, o, make_float4(mi.x * bv.x, mi.y * bv.y, mi.z * bv.z, mi.w * bv.w), nv);
        bf += dot4(bv, bv, nv);
      },
      [&]() {
        bb += (double)bf;
        bf = 0.f;
      });
  const double s = block_sum(bb, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r may be b itself (each element is read before it is written).
__global__ void k_pcg_residual0(int N, long long ld, long long vs, const float* b, const float* __restrict__ g,
                                const float* __restrict__ M, const float* __restrict__ D, unsigned d_mask,
                                const float* __restrict__ x, float lambda, float* r, float* __restrict__ z,
                                float* __restrict__ p, double* __restrict__ partials) {
  __shared__ double red[kBS / 32];
  {
    const long long off = (long long)blockIdx.y * vs;
    b += off;
    g += off;
    M += off;
    D = subset_D(D, d_mask, off);
    x += off;
    r += off;
    z += off;
    p += off;
    partials += (size_t)blockIdx.y * gridDim.x;
  }
  double rz = 0.0;
  float rzf = 0.f;
  for_each4(
      N, ld,
      [&](long long o, int nv) {
        const float4 bv = *reinterpret_cast<const float4*>(b + o), gv = ld4(g, o), mv = ld4(M, o), xv = ld4(x, o);
        float4 rv, mi;
        rv.x = bv.x - (gv.x + lambda * clamp_diag(mv.x) * xv.x);
        rv.y = bv.y - (gv.y + lambda * clamp_diag(mv.y) * xv.y);
        rv.z = bv.z - (gv.z + lambda * clamp_diag(mv.z) * xv.z);
        rv.w = bv.w - (gv.w + lambda * clamp_diag(mv.w) * xv.w);
        if (D != nullptr) {
          mi = ld4(D, o);
        } else {
          mi = make_float4(1.f / clamp_diag(mv.x), 1.f / clamp_diag(mv.y), 1.f / clamp_diag(mv.z),
                           1.f / clamp_diag(mv.w));
        }
        const float4 zv = make_float4(mi.x * rv.x, mi.y * rv.y, mi.z * rv.z, mi.w * rv.w);
        if (nv == 4) {
          *reinterpret_cast<float4*>(r + o) = rv;
        } else {
          r[o] = rv.x;
          if (nv > 1) r[o + 1] = rv.y;
          if (nv > 2) r[o + 2] = rv.z;
        }
        st4(z, o, zv, nv);
        st4(p, o, zv, nv);
        rzf += dot4(rv, zv, nv);
      },
      [&]() {
        rz += (double)rzf;
        rzf = 0.f;
      });
  const double s = block_sum(rz, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_pcg_update(int N, long long ld, long long vs, const PcgScalars* __restrict__ sc,
                             const float* __restrict__ p, const float* __restrict__ g, const float* __restrict__ M,
                             const float* __restrict__ D, unsigned d_mask, float* __restrict__ x,
                             float* __restrict__ r, float* __restrict__ z, double* __restrict__ partials) {
  __shared__ double red[kBS / 32];
  {
    const long long off = (long long)blockIdx.y * vs;
    sc += blockIdx.y;
    p += off;
    g += off;
    M += off;
    D = subset_D(D, d_mask, off);
    x += off;
    r += off;
    z += off;
    partials += (size_t)blockIdx.y * 2 * gridDim.x;
  }
  if (sc->done) return;
  const float alpha = (float)sc->alpha;
  double rz = 0.0, rr = 0.0;
  float rzf = 0.f, rrf = 0.f;
  for_each4(
      N, ld,
      [&](long long o, int nv) {
        const float4 xv = ld4(x, o), pv = ld4(p, o), rv0 = ld4(r, o), gv = ld4(g, o), mi = minv4(D, M, o);
        const float4 xn = make_float4(xv.x + alpha * pv.x, xv.y + alpha * pv.y, xv.z + alpha * pv.z,
                                      xv.w + alpha * pv.w);
        const float4 rv = make_float4(rv0.x - alpha * gv.x, rv0.y - alpha * gv.y, rv0.z - alpha * gv.z,
                                      rv0.w - alpha * gv.w);
        const float4 zv = make_float4(mi.x * rv.x, mi.y * rv.y, mi.z * rv.z, mi.w * rv.w);
        st4(x, o, xn, nv);
        st4(r, o, rv, nv);
        st4(z, o, zv, nv);
        rzf += dot4(rv, zv, nv);
        rrf += dot4(rv, rv, nv);
      },
      [&]() {
        rz += (double)rzf;
        rr += (double)rrf;
        rzf = rrf = 0.f;
      });
  const double s0 = block_sum(rz, red);
  __syncthreads();
  const double s1 = block_sum(rr, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
}

// stage 0: ||b||^2 (resets the solve state); 1: r^T z; 2: p^T g -> alpha;
// 3: (r^T z, ||r||^2) -> beta and the break test.
__global__ void k_pcg_scalars(PcgScalars* __restrict__ sc, const double* __restrict__ partials, int n, int pstride,
                              int stage, float break_rel2) {
  __shared__ double red[kBS / 32];
  sc += blockIdx.y;
  partials += (size_t)blockIdx.y * pstride;
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < n; i += kBS) {
    if (stage == 3) {
      s0 += partials[2 * i];
      s1 += partials[2 * i + 1];
    } else {
      s0 += partials[i];
    }
  }
  const double t0 = block_sum(s0, red);
  __syncthreads();
  const double t1 = block_sum(s1, red);
  if (threadIdx.x != 0) return;
  switch (stage) {
    case 0:
      sc->bb = t0;
      sc->done = 0;
      sc->iters = 0;
      sc->breakdown = 0;
      sc->alpha = 0.0;
      sc->beta = 0.0;
      sc->rr = t0;
      break;
    case 1:
      sc->rz = t0;
      break;
    case 2:
      if (sc->done) break;
      sc->pg = t0;
      if (!(t0 > 0.0) || !isfinite(t0)) {
        sc->done = 1;
        sc->breakdown = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / t0;
      }
      break;
    default:
      if (sc->done) break;
      sc->beta = sc->rz != 0.0 ? t0 / sc->rz : 0.0;
      sc->rz = t0;
      sc->rr = t1;
      sc->iters += 1;
      if (break_rel2 > 0.f && t1 < (double)break_rel2 * sc->bb) sc->done = 1;
      break;
  }
}

__global__ void k_reduce(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double red[kBS / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kBS) s += partials[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) *out = t;
}

__global__ void k_combine_acc(int N, long long ld, const float* __restrict__ d, const float* __restrict__ m,
                              float* __restrict__ num, float* __restrict__ den) {
  const int i = blockIdx.x * kBS + threadIdx.x;
  if (i >= N) return;
  const long long o = (long long)blockIdx.y * ld + i;
  const float mv = m[o];
  num[o] += mv * d[o];
  den[o] += mv;
}

__global__ void k_combine_finish(int N, long long ld, const float* __restrict__ num, const float* __restrict__ den,
                                 float* __restrict__ d) {
  const int i = blockIdx.x * kBS + threadIdx.x;
  if (i >= N) return;
  const long long o = (long long)blockIdx.y * ld + i;
  const float dv = den[o];
  d[o] = dv > 0.f ? num[o] / dv : 0.f;
}

__global__ void k_axpy(int N, long long ld, const float* __restrict__ x, float a, const float* __restrict__ d,
                       float* __restrict__ out) {
  const int i = blockIdx.x * kBS + threadIdx.x;
  if (i >= N) return;
  const long long o = (long long)blockIdx.y * ld + i;
  out[o] = x[o] + a * d[o];
}

__global__ void k_neg(long long n, const float* __restrict__ s, float* __restrict__ d) {
  const long long i = (long long)blockIdx.x * kBS + threadIdx.x;
  if (i < n) d[i] = -s[i];
}

__global__ void k_count_nonzero(const uint8_t* __restrict__ v, long long n, unsigned long long* __restrict__ out) {
  __shared__ unsigned int red[kBS / 32];
  unsigned int c = 0;
  for (long long i = (long long)blockIdx.x * kBS + threadIdx.x; i < n; i += (long long)gridDim.x * kBS) c += v[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kBS / 32; ++w) s += red[w];
    atomicAdd(out, s);
  }
}

dim3 vec_grid(int N) { return dim3((unsigned)((N + kBS - 1) / kBS), kNP); }

}  // namespace

int pcg_blocks(int N) { return std::max(1, std::min((N + kBS - 1) / kBS, kVecBlocks)); }

cudaError_t launch_reduce_partials(const double* partials, int n, double* out, cudaStream_t st) {
  { k_reduce<<<1, kBS, 0, st>>>(partials, n, out); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(int N, long long ld, const float* b, const float* M, const float* D, float* x,
                            double* partials, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_pcg_init<<<pcg_blocks(N), kBS, 0, st>>>(N, ld, 0, b, M, D, 1u, x, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_residual0(int N, long long ld, const float* b, const float* g, const float* M, const float* D,
                                 const float* x, float lambda, float* r, float* z, float* p, double* partials,
                                 cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_pcg_residual0<<<pcg_blocks(N), kBS, 0, st>>>(N, ld, 0, b, g, M, D, 1u, x, lambda, r, z, p, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_scalars(PcgScalars* sc, const double* partials, int n_partials, int stage, float break_rel2,
                               cudaStream_t st) {
  { k_pcg_scalars<<<1, kBS, 0, st>>>(sc, partials, n_partials, 0, stage, break_rel2); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(int N, long long ld, const PcgScalars* sc, const float* p, const float* g,
                              const float* M, const float* D, float* x, float* r, float* z, double* partials,
                              cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_pcg_update<<<pcg_blocks(N), kBS, 0, st>>>(N, ld, 0, sc, p, g, M, D, 1u, x, r, z, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_init_batch(int n, int N, long long ld, long long vs, const float* b, const float* M,
                                  const float* D, unsigned d_mask, float* x, double* partials, cudaStream_t st) {
  if (N <= 0 || n <= 0) return cudaSuccess;
  { k_pcg_init<<<dim3(pcg_blocks(N), n), kBS, 0, st>>>(N, ld, vs, b, M, D, d_mask, x, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_residual0_batch(int n, int N, long long ld, long long vs, const float* b, const float* g,
                                       const float* M, const float* D, unsigned d_mask, const float* x, float lambda,
                                       float* r, float* z, float* p, double* partials, cudaStream_t st) {
  if (N <= 0 || n <= 0) return cudaSuccess;
  { k_pcg_residual0<<<dim3(pcg_blocks(N), n), kBS, 0, st>>>(N, ld, vs, b, g, M, D, d_mask, x, lambda, r, z, p, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_update_batch(int n, int N, long long ld, long long vs, const PcgScalars* sc, const float* p,
                                    const float* g, const float* M, const float* D, unsigned d_mask, float* x,
                                    float* r, float* z, double* partials, cudaStream_t st) {
  if (N <= 0 || n <= 0) return cudaSuccess;
  { k_pcg_update<<<dim3(pcg_blocks(N), n), kBS, 0, st>>>(N, ld, vs, sc, p, g, M, D, d_mask, x, r, z, partials); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_pcg_scalars_batch(int n, PcgScalars* sc, const double* partials, int n_partials, int pstride,
                                     int stage, float break_rel2, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_pcg_scalars<<<dim3(1, n), kBS, 0, st>>>(sc, partials, n_partials, pstride, stage, break_rel2); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_combine_acc(int N, long long ld, const float* delta, const float* diag, float* num, float* den,
                               cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_combine_acc<<<vec_grid(N), kBS, 0, st>>>(N, ld, delta, diag, num, den); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_combine_finish(int N, long long ld, const float* num, const float* den, float* delta,
                                  cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_combine_finish<<<vec_grid(N), kBS, 0, st>>>(N, ld, num, den, delta); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_axpy_params(int N, long long ld, const float* x, float a, const float* d, float* out,
                               cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  { k_axpy<<<vec_grid(N), kBS, 0, st>>>(N, ld, x, a, d, out); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_neg_copy(long long n, const float* src, float* dst, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_neg<<<(unsigned)((n + kBS - 1) / kBS), kBS, 0, st>>>(n, src, dst); note_launch(); }
  return cudaGetLastError();
}

cudaError_t launch_count_nonzero_u8(const uint8_t* v, long long n, unsigned long long* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || n <= 0) return e;
  const long long blocks = std::min<long long>((n + kBS - 1) / kBS, 4096);
  { k_count_nonzero<<<(unsigned)blocks, kBS, 0, st>>>(v, n, out); note_launch(); }
  return cudaGetLastError();
}

}  // namespace gslm
